"""Near-field E (the guide's NRFLD = 1 calculation) on the GPU vs the oracle.

The GPU evaluates E_sca on the extended box as a zero-padded FFT convolution;
the oracle sums the dipole fields directly (oracle/dda.py: scattered_field,
oracle/pairwise.c: oracle_field_points).  Tolerances as for the matvec: 1e-10
relative (max |diff| / max |ref|) with the complex128 convolution, 1e-5 with
complex64.
"""
import numpy as np
import pytest

from dda_inputs import block_bernoulli_grid, ellipsoid_grid, random_complex, sphere_grid, workload
from oracle import dda as odda
from oracle import pairwise

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


def _dirs():
    k = np.array([[0.0, 0.6, 0.8], [1.0, 0.0, 0.0]])
    e = np.array([[1.0, 0.0, 0.0], [0.0, 0.6 + 0.8j, 0.0]], dtype=complex)
    return k, e


CASES = [
    ("block_two_materials", lambda: block_bernoulli_grid(5, 4, 3, seed=11), [1.6 + 0.3j, 1.2 + 0.05j], 1.1,
     (0.4, 0.6, 0.0, 0.5, 1.0, 0.3)),
    ("ellipsoid_ragged", lambda: ellipsoid_grid(9, 7, 6, 9, 7, 6), [1.5 + 0.1j], 1.4, (0.5, 0.5, 0.5, 0.5, 0.5, 0.5)),
    ("single_dipole", lambda: np.ones((1, 1, 1), np.uint8), [2.0 + 0.5j], 0.3, (3.0, 2.0, 1.0, 4.0, 2.0, 2.0)),
    ("no_extension", lambda: sphere_grid(8), [1.33 + 0.01j], 1.0, (0.0,) * 6),
]


@pytest.mark.parametrize("name,gridf,m,x,ext", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("prec,tol", [(0, F64_TOL), (2, F32_TOL)], ids=["fp64", "fp32"])
def test_nearfield_matches_oracle(lib, name, gridf, m, x, ext, prec, tol):
    grid = gridf()
    ctx = _ctx(lib, grid, m, x, lib.Precision.FP32_REFINED)
    kd = ctx.info()["kd"]
    N = ctx.info()["ndipoles"]
    k, e = _dirs()
    P = random_complex((2, 3, N), 17)
    Ei, Es, dims, off = ctx.nearfield(prec, k, e, P, ext)
    wdims, woff = odda.nearfield_box(grid.shape, ext)
    assert tuple(dims) == wdims and tuple(off) == woff
    r_src, _ = odda.site_positions(grid)
    pts = odda.nearfield_points(grid.shape, ext)
    for r in range(2):
        want = odda.scattered_field(r_src, P[r].T, pts, kd)
        assert _rel(Es[r].T, want) < tol, (name, r)
        einc = odda.incident_field(pts, kd, k[r], e[r] / np.linalg.norm(e[r]))
        assert _rel(Ei[r].T, einc) < 1e-12, (name, r)
    ctx.close()


def test_nearfield_of_gpu_solution_satisfies_dda_equations(lib):
    """The guide's check of a near-field run: P_j = alpha_j (E_inc,j + E_sca,j)
    at the target points, here with P from the GPU's own FP64 solve."""
    grid = block_bernoulli_grid(6, 5, 4, seed=5)
    m = [1.7 + 0.3j, 1.2 + 0.01j]
    ctx = _ctx(lib, grid, m, 1.2, lib.Precision.FP64)
    kd = ctx.info()["kd"]
    k, e = _dirs()
    res, P, _ = ctx.solve(0, k, e, tol=1e-11, maxit=500)
    assert all(r["status"] == 0 for r in res)
    ext = (0.5, 0.5, 1.0, 0.0, 0.25, 0.75)
    Ei, Es, dims, off = ctx.nearfield(0, k, e, P, ext)
    iz, iy, ix = np.nonzero(grid)
    box = ((iz + off[2]) * dims[1] + (iy + off[1])) * dims[0] + (ix + off[0])
    _, comp = odda.site_positions(grid)
    for r in range(2):
        beta = odda.ldr_inverse_polarizability((np.asarray(m) ** 2)[comp - 1], kd, k[r], e[r] / np.linalg.norm(e[r]))
        lhs = P[r].T
        rhs = (Ei[r][:, box] + Es[r][:, box]).T / beta[:, None]
        assert _rel(lhs, rhs) < 1e-8, r
    ctx.close()


@pytest.mark.parametrize("prec,tol", [(0, F64_TOL), (2, F32_TOL)], ids=["fp64", "fp32"])
def test_nearfield_full_size_point_samples(lib, prec, tol):
    """The 96x64x32 ellipsoid (102984 dipoles) extended by a quarter of its
    size on every side (a 144x96x48 box, 384x192x96 padded): 48 seeded box
    points, inside and outside the target, recomputed by the C oracle."""
    w = workload("ellipsoid96x64x32")
    ctx = _ctx(lib, w.grid, w.m, w.x, lib.Precision.FP32_REFINED)
    kd = ctx.info()["kd"]
    N = ctx.info()["ndipoles"]
    ext = (0.25,) * 6
    P = random_complex((1, 3, N), 23)
    _, Es, dims, off = ctx.nearfield(prec, w.khat[:1], w.ehat[:1], P, ext, want_inc=False)
    assert tuple(dims) == (144, 96, 48)
    pts = odda.nearfield_points(w.grid.shape, ext)
    rows = np.random.default_rng(4).choice(pts.shape[0], 48, replace=False)
    rows[:2] = [0, pts.shape[0] - 1]
    r_src, _ = odda.site_positions(w.grid)
    want = pairwise.scattered_field(r_src, P[0].T, pts[rows], kd)
    assert _rel(Es[0].T[rows], want) < tol
    ctx.close()


def test_nearfield_box_errors(lib):
    grid = sphere_grid(48)
    ctx = _ctx(lib, grid, [1.5 + 0.01j], 5.0, lib.Precision.FP32_REFINED)
    dims, off = ctx.nearfield_dims([0.5] * 6)
    assert dims == (96, 96, 96) and off == (24, 24, 24)   # the guide's ELLIPSOID_NEARFIELD volume
    with pytest.raises(lib.DdaError) as ei:
        ctx.nearfield_dims([3.0] * 6)                       # 336 points: above the largest padded length
    assert ei.value.status == 4
    with pytest.raises(lib.DdaError) as ei:
        ctx.nearfield_dims([-0.1, 0, 0, 0, 0, 0])
    assert ei.value.status == 1
    ctx.close()
