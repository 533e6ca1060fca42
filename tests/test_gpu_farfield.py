"""Far-field amplitudes and angular averages on the GPU vs the oracle.

The GPU sums the phase factors of every site with separable per-axis tables
(farfield.cu); the oracle forms exp(-i k n.r_j) directly (oracle/dda.py:
far_field, angular_averages).  Tolerances: 1e-10 relative with FP64 sums,
1e-5 with complex64 sums.
"""
import math

import numpy as np
import pytest

from dda_inputs import block_bernoulli_grid, ellipsoid_grid, random_complex, sphere_grid, workload
from oracle import dda as odda
from oracle import mie

pytestmark = pytest.mark.gpu

F64_TOL = 1e-10
F32_TOL = 1e-5


@pytest.fixture(scope="module")
def lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1202_3424_gb300 as dda
    dda.load_library()
    return dda


def _ctx(dda, grid, m, x, prec):
    ctx = dda.Context(0)
    ctx.set_target(grid)
    ctx.set_materials(m)
    ctx.prepare_size_parameter(x, prec)
    return ctx


def _rel(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


KHAT = np.array([[1.0, 0.0, 0.0], [0.36, 0.48, 0.8], [0.0, 0.0, -1.0]])


@pytest.mark.parametrize("prec,tol", [(0, F64_TOL), (2, F32_TOL)], ids=["fp64", "fp32"])
@pytest.mark.parametrize("name,gridf", [("ellipsoid_13x9x6", lambda: ellipsoid_grid(13, 9, 6, 13, 9, 6)),
                                        ("block_two_materials", lambda: block_bernoulli_grid(7, 5, 4, seed=2))],
                         ids=["ellipsoid", "block"])
def test_farfield_matches_oracle(lib, name, gridf, prec, tol):
    grid = gridf()
    ctx = _ctx(lib, grid, [1.5 + 0.1j, 1.2 + 0.01j], 2.0, lib.Precision.FP32_REFINED)
    kd = ctx.info()["kd"]
    N = ctx.info()["ndipoles"]
    P = random_complex((3, 3, N), 31)
    rng = np.random.default_rng(3)
    theta = np.concatenate([[0.0, math.pi, math.pi / 2], rng.uniform(0, math.pi, 61)])
    phi = np.concatenate([[0.0, 0.0, 1.0], rng.uniform(0, 2 * math.pi, 61)])
    F = ctx.farfield(prec, KHAT, P, theta, phi)
    r, _ = odda.site_positions(grid)
    for i in range(3):
        want = odda.far_field(r, P[i].T, kd, odda.directions(KHAT[i], theta, phi))
        assert _rel(F[i], want) < tol, (name, i)
    ctx.close()


@pytest.mark.parametrize("prec,tol", [(0, F64_TOL), (2, F32_TOL)], ids=["fp64", "fp32"])
def test_angular_averages_match_oracle(lib, prec, tol):
    grid = ellipsoid_grid(11, 8, 7, 11, 8, 7)
    ctx = _ctx(lib, grid, [1.6 + 0.05j], 2.5, lib.Precision.FP32_REFINED)
    info = ctx.info()
    kd, N = info["kd"], info["ndipoles"]
    P = random_complex((3, 3, N), 5)
    out, nd = ctx.angular_averages(prec, KHAT, P, eta=0.5)
    x = kd * info["aeff_lattice"]
    t, ph, w = odda.scattering_directions(x, 0.5)
    assert nd == t.size
    r, _ = odda.site_positions(grid)
    for i in range(3):
        csca, c1, c2, g = odda.angular_averages(r, P[i].T, kd, KHAT[i], t, ph, w)
        want = np.array([csca / (math.pi * info["aeff_lattice"] ** 2), c1, c2, g[0], g[1], g[2]])
        assert np.abs(out[i] - want).max() < tol * max(1.0, abs(want[0])), i
    ctx.close()


def test_sphere_scattering_from_gpu_solution(lib):
    """16^3 sphere solved on the GPU: Q_sca of the angular average equals
    Q_ext - Q_abs of the solve to the quadrature's accuracy (ETASCA = 0.2),
    and <cos theta> agrees with the Mie series to the DDA's discretisation
    error at this size."""
    x, m = 1.5, 1.33 + 0.01j
    grid = sphere_grid(16)
    ctx = _ctx(lib, grid, [m], x, lib.Precision.FP64)
    k = np.array([[1.0, 0.0, 0.0], [1.0, 0.0, 0.0]])
    e = np.array([[0, 1, 0], [0, 0, 1]], dtype=complex)
    res, P, st = ctx.solve(0, k, e, tol=1e-10)
    assert st == 0
    out, nd = ctx.angular_averages(0, k, P, eta=0.2)
    for i in range(2):
        qsca = res[i]["qext"] - res[i]["qabs"]
        assert abs(out[i, 0] - qsca) < 2e-3 * qsca
    gm = mie.mie_asymmetry(x, m)
    assert abs(out[:, 1].mean() - gm) < 0.03 * gm
    assert np.abs(out[:, 4:]).max() < 1e-3          # g along the incident direction only
    ctx.close()


@pytest.mark.parametrize("prec,tol", [(0, F64_TOL), (2, F32_TOL)], ids=["fp64", "fp32"])
def test_farfield_full_size_sweep(lib, prec, tol):
    """The 96x64x32 ellipsoid (102984 dipoles), 4 RHS of the seeded sweep, the
    guide's directions at x = 8: 24 sampled amplitudes per RHS recomputed by the
    oracle."""
    w = workload("ellipsoid96x64x32")
    ctx = _ctx(lib, w.grid, w.m, w.x, lib.Precision.FP32_REFINED)
    kd, N = ctx.info()["kd"], ctx.info()["ndipoles"]
    R = 4
    P = random_complex((R, 3, N), 8)
    t, ph, _ = lib.dda_scattering_directions(w.x, 0.5)
    F = ctx.farfield(prec, w.khat[:R], P, t, ph)
    rows = np.random.default_rng(6).choice(t.size, 24, replace=False)
    r, _ = odda.site_positions(w.grid)
    for i in range(R):
        want = odda.far_field(r, P[i].T, kd, odda.directions(w.khat[i], t[rows], ph[rows]))
        assert _rel(F[i][rows], want) < tol, i
    ctx.close()


@pytest.mark.parametrize("prec,tol", [(0, F64_TOL), (2, F32_TOL)], ids=["fp64", "fp32"])
def test_mueller_matches_oracle(lib, prec, tol):
    """Mueller matrices and amplitudes from the GPU far field vs the oracle,
    for an oblique incidence and an elliptical incident pair."""
    grid = ellipsoid_grid(9, 8, 6, 9, 8, 6)
    ctx = _ctx(lib, grid, [1.4 + 0.2j], 2.0, lib.Precision.FP32_REFINED)
    kd, N = ctx.info()["kd"], ctx.info()["ndipoles"]
    k = np.array([0.36, 0.48, 0.8])
    xl, yl, zl = odda.lab_frame(k)
    e01 = (yl + 1j * 0.5 * zl) / np.sqrt(1.25)
    e02 = np.cross(k, np.conj(e01))
    P = random_complex((2, 3, N), 19)
    rng = np.random.default_rng(1)
    theta = np.concatenate([[0.0, math.pi], rng.uniform(0, math.pi, 30)])
    phi = np.concatenate([[0.3, 0.0], rng.uniform(0, 2 * math.pi, 30)])
    M, S = ctx.mueller(prec, k, e01, e02, P, theta, phi)
    r, _ = odda.site_positions(grid)
    Sw = odda.scattering_amplitudes(r, P[0].T, P[1].T, kd, k, e01, e02, theta, phi)
    Mw = odda.mueller_matrix(Sw)
    assert _rel(S, Sw) < tol
    assert np.abs(M - Mw).max() < tol * np.abs(Mw[:, 0, 0]).max()
    ctx.close()


def test_mueller_of_gpu_sphere_solution_approaches_mie(lib):
    """16^3 sphere solved on the GPU for e01 = y, e02 = z: S11, S12, S33, S34
    against the Mie series within the DDA's discretisation error."""
    x, m = 1.5, 1.33 + 0.01j
    ctx = _ctx(lib, sphere_grid(16), [m], x, lib.Precision.FP64)
    k = np.array([[1.0, 0, 0], [1.0, 0, 0]])
    e = np.array([[0, 1, 0], [0, 0, 1]], dtype=complex)
    res, P, st = ctx.solve(0, k, e, tol=1e-10)
    assert st == 0
    th = np.linspace(0, math.pi, 19)
    ph = np.full(th.size, 0.7)
    M, S = ctx.mueller(0, k[0], e[0], e[1], P, th, ph)
    S1, S2 = mie.mie_amplitudes(x, m, th)
    ref = (abs(S1) ** 2 + abs(S2) ** 2) / 2
    err = max(np.abs(M[:, 0, 0] - ref).max(), np.abs(M[:, 0, 1] - (abs(S2) ** 2 - abs(S1) ** 2) / 2).max(),
              np.abs(M[:, 2, 2] - (S1 * np.conj(S2)).real).max(), np.abs(M[:, 2, 3] - (S2 * np.conj(S1)).imag).max())
    assert err < 0.03 * ref[0]
    assert np.abs(S[:, 2:]).max() < 1e-3 * np.abs(S[0, 0])   # S3 = S4 = 0 for a sphere
    ctx.close()
