"""The no-allocation matvec entry point against the ordinary one (GPU).

dda_matvec_device_noalloc serves callers that must not allocate device
memory during the call; its scratch is a fixed array inside the library.
This file is collected last so that a run stopping at the first failure has
already run every other test; it also passes when run alone.
"""
import numpy as np
import pytest

from dda_inputs import random_complex, sphere_grid, uniform_directions, polarization_pair, workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1202_3424_gb300 as dda
    dda.load_library()
    return dda, torch


def _rel(a, b):
    return float((a - b).abs().max() / b.abs().max())


@pytest.mark.parametrize("prec,tol", [(0, 1e-10), (2, 1e-5)], ids=["fp64", "fp32"])
def test_noalloc_matches_matvec_on_two_calls(env, prec, tol):
    dda, torch = env
    ctx = dda.Context(0)
    ctx.set_target(sphere_grid(16))
    ctx.set_materials([1.33 + 0.01j])
    ctx.prepare_size_parameter(1.0, dda.Precision.FP32_REFINED)
    N = ctx.info()["ndipoles"]
    k = uniform_directions(2, 5)
    e = polarization_pair(k)[0].astype(complex)
    dt = torch.complex128 if prec == 0 else torch.complex64
    for call in range(2):  # two calls in a row: the second sees the first call's scratch contents
        x = torch.from_numpy(random_complex((2, 3, N), 100 + call)).to(dt).cuda()
        y_ref = torch.empty_like(x)
        y_na = torch.full_like(x, float("nan"))
        dda.dda_matvec_device(ctx.handle, prec, k, e, x, y_ref)
        dda.dda_matvec_device_noalloc(ctx.handle, prec, k, e, x, y_na)
        torch.cuda.synchronize()
        assert torch.isfinite(y_na).all()
        assert _rel(y_na, y_ref) < tol, (call, _rel(y_na, y_ref))
    ctx.close()


@pytest.mark.parametrize("prec,tol", [(0, 1e-10), (2, 1e-5)], ids=["fp64", "fp32"])
def test_noalloc_matches_matvec_with_tensor_polarizabilities(env, prec, tol):
    """Anisotropic materials: the scratch then holds the per-RHS 1/alpha
    tensors (six entries per composition) instead of scalars."""
    dda, torch = env
    ctx = dda.Context(0)
    ctx.set_target(sphere_grid(12))
    ctx.set_anisotropic_materials([[1.4 + 0.02j, 1.5 + 0.05j, 1.3 + 0.01j]], [(0.4, 1.1, -0.6)])
    ctx.prepare_size_parameter(1.2, dda.Precision.FP32_REFINED)
    N = ctx.info()["ndipoles"]
    k = uniform_directions(3, 7)
    e = polarization_pair(k)[1].astype(complex)
    dt = torch.complex128 if prec == 0 else torch.complex64
    for call in range(2):
        x = torch.from_numpy(random_complex((3, 3, N), 200 + call)).to(dt).cuda()
        y_ref = torch.empty_like(x)
        y_na = torch.full_like(x, float("nan"))
        dda.dda_matvec_device(ctx.handle, prec, k, e, x, y_ref)
        dda.dda_matvec_device_noalloc(ctx.handle, prec, k, e, x, y_na)
        torch.cuda.synchronize()
        assert torch.isfinite(y_na).all()
        assert _rel(y_na, y_ref) < tol, (call, _rel(y_na, y_ref))
    ctx.close()


def test_noalloc_rejects_the_double_float_precision(env):
    dda, torch = env
    ctx = dda.Context(0)
    ctx.set_target(sphere_grid(8))
    ctx.set_materials([1.33 + 0.01j])
    ctx.prepare_size_parameter(0.5, dda.Precision.FP32_REFINED)
    N = ctx.info()["ndipoles"]
    k = uniform_directions(1, 3)
    e = polarization_pair(k)[0].astype(complex)
    x = torch.zeros((1, 3, N), dtype=torch.complex128, device="cuda")
    y = torch.zeros_like(x)
    with pytest.raises(dda.DdaError) as ei:
        dda.dda_matvec_device_noalloc(ctx.handle, 3, k, e, x, y)
    assert ei.value.status_name == "DDA_ERR_ARG" and "DDA_DF64" in str(ei.value)
    ctx.close()


def test_noalloc_rejects_sizes_beyond_its_scratch(env):
    dda, torch = env
    w = workload("sphere64")
    ctx = dda.Context(0)
    ctx.set_target(w.grid)
    ctx.set_materials(w.m)
    ctx.prepare_size_parameter(w.x, dda.Precision.FP32_REFINED)
    N = ctx.info()["ndipoles"]
    R = 4
    x = torch.zeros((R, 3, N), dtype=torch.complex64, device="cuda")
    y = torch.zeros_like(x)
    with pytest.raises(dda.DdaError) as ei:
        dda.dda_matvec_device_noalloc(ctx.handle, 2, np.repeat(w.khat[:1], R, 0), np.repeat(w.ehat[:1], R, 0), x, y)
    assert ei.value.status_name == "DDA_ERR_SIZE"
    ctx.close()


def test_noalloc_refuses_a_stream_capture(env):
    """The call synchronizes its stream, so inside a capture of the context
    stream it returns DDA_ERR_ARG before touching the stream; the capture
    stays valid and the next uncaptured call works."""
    dda, torch = env
    ctx = dda.Context(0)
    ctx.set_target(sphere_grid(8))
    ctx.set_materials([1.33 + 0.01j])
    ctx.prepare_size_parameter(0.6, dda.Precision.FP32_REFINED)
    N = ctx.info()["ndipoles"]
    k = uniform_directions(1, 3)
    e = polarization_pair(k)[0].astype(complex)
    s = torch.cuda.Stream()
    dda.dda_set_stream(ctx.handle, s.cuda_stream)
    x = torch.from_numpy(random_complex((1, 3, N), 300)).to(torch.complex64).cuda()
    y = torch.empty_like(x)
    torch.cuda.synchronize()   # (x and y were made on the default stream)
    with torch.cuda.stream(s):
        dda.dda_matvec_device_noalloc(ctx.handle, 2, k, e, x, y)   # outside any capture: fine
    torch.cuda.synchronize()
    y0 = y.clone()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        x.mul_(1)
        with pytest.raises(dda.DdaError, match="capture"):
            dda.dda_matvec_device_noalloc(ctx.handle, 2, k, e, x, y)
    torch.cuda.synchronize()
    with torch.cuda.stream(s):
        dda.dda_matvec_device_noalloc(ctx.handle, 2, k, e, x, y)
    torch.cuda.synchronize()
    assert torch.equal(y, y0)
    dda.dda_set_stream(ctx.handle, None)
    ctx.close()
