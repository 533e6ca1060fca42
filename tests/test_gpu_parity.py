"""GPU path vs the CPU oracle, element by element (needs a GB300).

Every comparison runs the CUDA library through its C ABI (ctypes binding)
on seeded inputs from dda_inputs, and the oracle on the same inputs.
Tolerances: 1e-10 relative (max |diff| / max |ref|) for complex128, 1e-5 for
complex64, as the hot-path specification states.
"""
import math

import numpy as np
import pytest

from dda_inputs import (block_bernoulli_grid, ellipsoid_grid, random_complex, sphere_grid, uniform_directions,
                        polarization_pair, workload)
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


def _site_beta(grid, m, kd, khat, ehat):
    r, comp = odda.site_positions(grid)
    eps = (np.asarray(m, dtype=complex) ** 2)[comp - 1]
    return r, odda.ldr_inverse_polarizability(eps, kd, khat, ehat)


def _rel(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


def _rel_elem(a, b, floor):
    """Largest error of any single element, relative to that element's own
    magnitude plus floor * max|b|.  An FFT convolution spreads its rounding
    error evenly over the output (about eps * log2(L) * max|b| per element),
    so elements far below floor * max|b| cannot be matched to the relative
    tolerance; every element above it is held to it on its own."""
    return float((np.abs(a - b) / (np.abs(b) + floor * np.abs(b).max())).max())


def _rhs_set(R, seed=20120214):
    k = uniform_directions(R, seed)
    e1, _ = polarization_pair(k)
    return k, e1.astype(complex)


MATVEC_CASES = [
    ("sphere16", lambda: sphere_grid(16), [1.33 + 0.01j], 1.0),
    ("block7x5x3_two_materials", lambda: block_bernoulli_grid(7, 5, 3, seed=3), [1.7 + 0.3j, 1.2 + 0.01j], 2.0),
    ("ellipsoid_ragged_13x9x6", lambda: ellipsoid_grid(13, 9, 6, 13, 9, 6), [2.0 + 1.0j], 1.5),
    ("single_dipole", lambda: np.ones((1, 1, 1), np.uint8), [1.5 + 0.1j], 0.3),
    ("line_of_dipoles_1x1x17", lambda: np.ones((17, 1, 1), np.uint8), [1.5 + 0.1j], 0.8),
    # 64x64 in x and y: the fused x+y slice passes run
    ("plate_25x25x3_slices", lambda: block_bernoulli_grid(25, 25, 3, seed=8), [1.4 + 0.2j, 1.9 + 0.05j], 2.2),
]


@pytest.mark.parametrize("name,gridf,m,x", MATVEC_CASES, ids=[c[0] for c in MATVEC_CASES])
@pytest.mark.parametrize("prec,tol", [(0, F64_TOL), (3, F64_TOL), (2, F32_TOL)], ids=["fp64", "df64", "fp32"])
def test_matvec_matches_pairwise_oracle(lib, name, gridf, m, x, prec, tol):
    grid = gridf()
    ctx = _ctx(lib, grid, m, x, lib.Precision.FP32_REFINED)
    kd = ctx.info()["kd"]
    R = 2
    khat, ehat = _rhs_set(R)
    N = ctx.info()["ndipoles"]
    X = random_complex((R, 3, N), 11)
    Y = ctx.matvec(prec, khat, ehat, X)
    for r in range(R):
        rr, beta = _site_beta(grid, m, kd, khat[r], ehat[r])
        want, _ = pairwise.matvec(rr, kd, beta, X[r].T)
        assert _rel(Y[r].T, want) < tol, (name, r)
        if prec != 2:   # FP64 and double-float: element by element above 1 % of the largest
            assert _rel_elem(Y[r].T, want, 1e-2) < tol, (name, r)
    ctx.close()


REG_Z_LENGTHS = (16, 32, 64, 128, 256, 512)  # z plans with at most 8 points per thread
Z_PLAN_VARIANTS = (128, 256)                  # lengths with a radix-16 plan (schedules 3, 4)
Z_IDS = ["zgroups", "zregs", "zregs_octant", "zregs_radix16", "zregs_octant_radix16"]


def _z_expected(zpass, Lz):
    if Lz not in REG_Z_LENGTHS:
        return 0
    return zpass if (zpass < 3 or Lz in Z_PLAN_VARIANTS) else zpass - 2


Z_CASES = MATVEC_CASES + [
    ("rod_z128_block_3x4x60", lambda: block_bernoulli_grid(3, 4, 60, seed=24), [1.5 + 0.1j, 1.25 + 0.02j], 2.0),
    ("rod_z256_ellipsoid_6x5x110", lambda: ellipsoid_grid(6, 5, 110, 6, 5, 110), [1.4 + 0.05j], 2.5),
]


@pytest.mark.parametrize("name,gridf,m,x", Z_CASES, ids=[c[0] for c in Z_CASES])
@pytest.mark.parametrize("zpass", [0, 1, 2, 3, 4], ids=Z_IDS)
def test_matvec_z_schedules_match_oracle(lib, name, gridf, m, x, zpass):
    """The complex64 z-pass schedules against the pairwise oracle.  Nine RHS
    span full blocks of RHS and a ragged one; a grid whose z plan has no
    register-resident schedule must fall back to schedule 0, and one with a
    single radix plan from 3, 4 to 1, 2."""
    grid = gridf()
    ctx = _ctx(lib, grid, m, x, lib.Precision.FP32_REFINED)
    info = ctx.info()
    ctx.set_schedule(zpass)
    R = 9
    assert ctx.get_schedule(R) == _z_expected(zpass, info["Lz"])
    kd = info["kd"]
    khat, ehat = _rhs_set(R)
    X = random_complex((R, 3, info["ndipoles"]), 12)
    Y = ctx.matvec(2, khat, ehat, X)
    for r in range(R):
        rr, beta = _site_beta(grid, m, kd, khat[r], ehat[r])
        want, _ = pairwise.matvec(rr, kd, beta, X[r].T)
        assert _rel(Y[r].T, want) < F32_TOL, (name, zpass, r)
    ctx.close()


@pytest.mark.parametrize("zpass", [0, 1, 2, 3, 4], ids=Z_IDS)
def test_matvec_long_z_columns_many_rhs(lib, zpass):
    """A 4x5x100 rod (256-point z transform, where the register schedules
    take 16 or, with octant columns, 4 RHS per block) with 18 RHS: full blocks
    of RHS and a ragged one, against the pairwise oracle."""
    grid = np.ones((100, 5, 4), np.uint8)
    m = [1.4 + 0.05j]
    ctx = _ctx(lib, grid, m, 2.0, lib.Precision.FP32_REFINED)
    info = ctx.info()
    assert info["Lz"] == 256
    ctx.set_schedule(zpass)
    R = 18
    khat, ehat = _rhs_set(R)
    X = random_complex((R, 3, info["ndipoles"]), 13)
    Y = ctx.matvec(2, khat, ehat, X)
    for r in range(R):
        rr, beta = _site_beta(grid, m, info["kd"], khat[r], ehat[r])
        want, _ = pairwise.matvec(rr, info["kd"], beta, X[r].T)
        assert _rel(Y[r].T, want) < F32_TOL, (zpass, r)
    ctx.close()


@pytest.mark.parametrize("zpass", [0, 1, 2, 3, 4], ids=Z_IDS)
def test_matvec_512_point_z_columns(lib, zpass):
    """A 3x2x200 rod (512-point z transform, one radix plan: schedules 3
    and 4 fall back to 1 and 2) with 18 RHS: a full block of 16 RHS and a
    ragged one, against the pairwise oracle."""
    grid = np.ones((200, 2, 3), np.uint8)
    m = [1.5 + 0.02j]
    ctx = _ctx(lib, grid, m, 2.5, lib.Precision.FP32_REFINED)
    info = ctx.info()
    assert info["Lz"] == 512
    ctx.set_schedule(zpass)
    R = 18
    khat, ehat = _rhs_set(R)
    X = random_complex((R, 3, info["ndipoles"]), 15)
    Y = ctx.matvec(2, khat, ehat, X)
    for r in range(R):
        rr, beta = _site_beta(grid, m, info["kd"], khat[r], ehat[r])
        want, _ = pairwise.matvec(rr, info["kd"], beta, X[r].T)
        assert _rel(Y[r].T, want) < F32_TOL, (zpass, r)
    ctx.close()


# Rows of the hot x lengths (Lx = 128, 192, 256, 512): full, ragged and
# two-material rows, every x-pass schedule (0 staged rows, 1 + V the
# warp-local rows with radix plan variant V; the last variant of 64, 128, 256
# and 512 points exchanges by warp shuffles).
X_CASES = [
    ("rows128_block_64x6x4", lambda: block_bernoulli_grid(64, 6, 4, seed=21), [1.6 + 0.1j, 1.3 + 0.02j], 2.0),
    ("rows192_ellipsoid_90x7x5", lambda: ellipsoid_grid(90, 7, 5, 90, 7, 5), [1.5 + 0.05j], 3.0),
    ("rows256_block_120x3x3", lambda: block_bernoulli_grid(120, 3, 3, seed=22), [1.4 + 0.2j, 2.0 + 0.5j], 2.5),
    ("rows512_rod_200x2x2", lambda: np.ones((2, 2, 200), np.uint8), [1.33 + 0.01j], 2.0),
    ("rows64_plate_25x25x3", MATVEC_CASES[5][1], MATVEC_CASES[5][2], MATVEC_CASES[5][3]),
    ("rows32_ellipsoid_ragged", MATVEC_CASES[2][1], MATVEC_CASES[2][2], MATVEC_CASES[2][3]),
]
X_VARIANTS = {64: 2, 128: 3, 192: 2, 256: 3, 512: 3}   # radix plan variants of the warp-local rows


@pytest.mark.parametrize("name,gridf,m,x", X_CASES, ids=[c[0] for c in X_CASES])
@pytest.mark.parametrize("xpass", [0, 1, 2, 3], ids=["xstaged", "xwarp_plan0", "xwarp_plan1", "xwarp_plan2"])
def test_matvec_x_schedules_match_oracle(lib, name, gridf, m, x, xpass):
    """The complex64 x-pass schedules against the pairwise oracle, isotropic
    and with tilted biaxial materials (the tensor 1/alpha of the x-inverse)."""
    grid = gridf()
    ctx = _ctx(lib, grid, m, x, lib.Precision.FP32_REFINED)
    info = ctx.info()
    ctx.set_xpass(xpass)
    R = 5
    nvar = X_VARIANTS.get(info["Lx"], 1)
    assert ctx.get_xpass(R) == (min(xpass, nvar),) * 2
    kd = info["kd"]
    khat, ehat = _rhs_set(R)
    X = random_complex((R, 3, info["ndipoles"]), 14)
    Y = ctx.matvec(2, khat, ehat, X)
    for r in range(R):
        rr, beta = _site_beta(grid, m, kd, khat[r], ehat[r])
        want, _ = pairwise.matvec(rr, kd, beta, X[r].T)
        assert _rel(Y[r].T, want) < F32_TOL, (name, xpass, r)
    # tensor polarizabilities: same schedule, against the oracle's tensor matvec
    m3 = [[mm * f for f in (1.0, 1.06, 0.94)] for mm in m]
    ang = [(0.3 + 0.2 * i, 1.0, -0.5) for i in range(len(m))]
    ctx.set_anisotropic_materials(m3, ang)
    ctx.prepare_size_parameter(x, lib.Precision.FP32_REFINED)
    ctx.set_xpass(xpass)
    Y = ctx.matvec(2, khat, ehat, X)
    rr, comp = odda.site_positions(grid)
    for r in (0, R - 1):
        bt = np.stack([odda.ldr_inverse_tensor(np.asarray(m3[c - 1]) ** 2, ang[c - 1], kd, khat[r], ehat[r])
                       for c in comp])
        # the C oracle sums the interaction part (scalar diagonal 0); the tensor diagonal is added here
        off, _ = pairwise.matvec(rr, kd, np.zeros(len(rr), complex), X[r].T)
        want = off + np.einsum("nab,nb->na", bt, X[r].T)
        assert _rel(Y[r].T, want) < F32_TOL, (name, xpass, "tensor", r)
    ctx.close()


@pytest.mark.parametrize("xpass", [0, 1, 2, 3], ids=["xstaged", "xwarp_plan0", "xwarp_plan1", "xwarp_plan2"])
def test_refined_solve_through_each_x_schedule(lib, xpass):
    """The BiCGstab updates fused into the x passes (gather and scatter modes
    1 and 2, with their reductions) under each x schedule: a FP32-refined
    solve of a 64x6x4 two-material block (128-point rows) reaches the FP64
    solution's efficiencies."""
    grid = block_bernoulli_grid(64, 6, 4, seed=23)
    m = [1.6 + 0.1j, 1.3 + 0.02j]
    ctx = _ctx(lib, grid, m, 2.0, lib.Precision.FP32_REFINED)
    k, e = _rhs_set(3)
    ref, _, st = ctx.solve(lib.Precision.FP64, k, e, want_P=False, tol=1e-10, maxit=2000)
    assert st == 0
    ctx.set_xpass(xpass)
    res, _, st = ctx.solve(lib.Precision.FP32_REFINED, k, e, want_P=False, tol=1e-6, maxit=2000)
    assert st == 0 and max(r["resid_rel"] for r in res) <= 1e-6
    q = np.array([[r["qext"], r["qabs"], r["qsca"]] for r in res])
    q0 = np.array([[r["qext"], r["qabs"], r["qsca"]] for r in ref])
    assert np.abs(q - q0).max() < 1e-5 * np.abs(q0).max(), (xpass, q, q0)
    ctx.close()


# Columns of the y lengths with two radix plans (Ly = 128, 192, 256)
Y_CASES = [
    ("cols128_block_5x64x3", lambda: block_bernoulli_grid(5, 64, 3, seed=26), [1.5 + 0.1j, 1.25 + 0.02j], 2.0),
    ("cols192_ellipsoid_7x90x5", lambda: ellipsoid_grid(7, 90, 5, 7, 90, 5), [1.45 + 0.05j], 3.0),
    ("cols256_block_3x120x3", lambda: block_bernoulli_grid(3, 120, 3, seed=27), [1.4 + 0.2j, 2.0 + 0.5j], 2.5),
    ("cols512_ellipsoid_2x230x2", lambda: ellipsoid_grid(2, 230, 2, 2, 230, 2), [1.33 + 0.01j], 2.0),
]


@pytest.mark.parametrize("name,gridf,m,x", Y_CASES, ids=[c[0] for c in Y_CASES])
@pytest.mark.parametrize("ypass", [0, 1], ids=["yplan0", "yplan1"])
def test_matvec_y_plans_match_oracle(lib, name, gridf, m, x, ypass):
    """Both radix plans of the complex64 y passes against the pairwise oracle
    (full, ragged and two-material columns)."""
    grid = gridf()
    ctx = _ctx(lib, grid, m, x, lib.Precision.FP32_REFINED)
    info = ctx.info()
    ctx.set_ypass(ypass)
    R = 5
    assert ctx.get_ypass(R) == ypass
    kd = info["kd"]
    khat, ehat = _rhs_set(R)
    X = random_complex((R, 3, info["ndipoles"]), 15)
    Y = ctx.matvec(2, khat, ehat, X)
    for r in range(R):
        rr, beta = _site_beta(grid, m, kd, khat[r], ehat[r])
        want, _ = pairwise.matvec(rr, kd, beta, X[r].T)
        assert _rel(Y[r].T, want) < F32_TOL, (name, ypass, r)
    with pytest.raises(lib.DdaError):
        ctx.set_ypass(2)
    ctx.close()


def test_refined_solve_through_the_second_y_plan(lib):
    """The solve's matvecs (fused BiCGstab updates) with the y plan 8 x 16."""
    grid = block_bernoulli_grid(5, 64, 3, seed=28)
    m = [1.6 + 0.1j, 1.3 + 0.02j]
    ctx = _ctx(lib, grid, m, 2.5, lib.Precision.FP32_REFINED)
    k, e = _rhs_set(3)
    ref, _, st = ctx.solve(lib.Precision.FP64, k, e, want_P=False, tol=1e-10, maxit=2000)
    assert st == 0
    ctx.set_ypass(1)
    res, _, st = ctx.solve(lib.Precision.FP32_REFINED, k, e, want_P=False, tol=1e-6, maxit=2000)
    assert st == 0 and max(r["resid_rel"] for r in res) <= 1e-6
    assert ctx.get_solve_schedule(3)["ypass"] == 1
    q = np.array([[r["qext"], r["qabs"], r["qsca"]] for r in res])
    q0 = np.array([[r["qext"], r["qabs"], r["qsca"]] for r in ref])
    assert np.abs(q - q0).max() < 1e-5 * np.abs(q0).max()
    ctx.close()


@pytest.mark.parametrize("zpass", [1, 2, 3, 4], ids=Z_IDS[1:])
def test_refined_solve_through_each_z_schedule(lib, zpass):
    """A FP32-refined solve of a 5x4x60 two-material rod (128-point z
    transform) under each register z schedule reaches the FP64 solution's
    efficiencies (the solve's matvecs carry the fused BiCGstab updates)."""
    grid = block_bernoulli_grid(5, 4, 60, seed=25)
    m = [1.6 + 0.1j, 1.3 + 0.02j]
    ctx = _ctx(lib, grid, m, 2.5, lib.Precision.FP32_REFINED)
    k, e = _rhs_set(3)
    ref, _, st = ctx.solve(lib.Precision.FP64, k, e, want_P=False, tol=1e-10, maxit=2000)
    assert st == 0
    ctx.set_schedule(zpass)
    res, _, st = ctx.solve(lib.Precision.FP32_REFINED, k, e, want_P=False, tol=1e-6, maxit=2000)
    assert st == 0 and max(r["resid_rel"] for r in res) <= 1e-6
    q = np.array([[r["qext"], r["qabs"], r["qsca"]] for r in res])
    q0 = np.array([[r["qext"], r["qabs"], r["qsca"]] for r in ref])
    assert np.abs(q - q0).max() < 1e-5 * np.abs(q0).max(), (zpass, q, q0)
    ctx.close()


def test_autotuned_schedule_reproduces_forced_one(lib):
    """The autotuner picks a z schedule and a slice-pass setting; the matvec
    it runs is bit-identical to forcing that choice."""
    w = workload("ellipsoid96x64x32")
    ctx = _ctx(lib, w.grid, w.m, w.x, lib.Precision.FP32_REFINED)
    R = 12
    ctx.set_schedule(-1)
    ctx.set_slice_passes(-1)
    zpick, spick = ctx.get_schedule(R, with_slices=True)
    xpick = ctx.get_xpass(R)
    ypick = ctx.get_ypass(R)
    assert zpick in (0, 1, 2, 3, 4) and spick in (0, 1) and all(v in (0, 1, 2, 3) for v in xpick) and ypick in (0, 1)
    X = random_complex((R, 3, ctx.info()["ndipoles"]), 4).astype(np.complex64)
    k, e = np.resize(w.khat, (R, 3)), np.resize(w.ehat, (R, 3))
    y_auto = ctx.matvec(2, k, e, X)
    ctx.set_schedule(zpick)
    ctx.set_slice_passes(spick)
    ctx.set_xpass(xpick)
    ctx.set_ypass(ypick)
    assert ctx.get_xpass(R) == xpick
    y_forced = ctx.matvec(2, k, e, X)
    assert np.array_equal(y_auto, y_forced)
    with pytest.raises(lib.DdaError):
        ctx.set_schedule(5)
    with pytest.raises(lib.DdaError):
        ctx.set_xpass(4)
    ctx.close()


def test_matvec_is_complex_symmetric(lib):
    grid = ellipsoid_grid(11, 7, 5, 11, 7, 5)
    ctx = _ctx(lib, grid, [1.6 + 0.2j], 1.2, lib.Precision.FP64)
    N = ctx.info()["ndipoles"]
    k, e = np.array([[0, 0, 1.0]]), np.array([[1.0, 0, 0]], complex)
    x = random_complex((1, 3, N), 1)
    y = random_complex((1, 3, N), 2)
    Ax = ctx.matvec(0, k, e, x)
    Ay = ctx.matvec(0, k, e, y)
    a, b = np.sum(x * Ay), np.sum(y * Ax)
    assert abs(a - b) < 1e-13 * abs(a)
    ctx.close()


@pytest.mark.parametrize("name", ["sphere64", "ellipsoid96x64x32", "block48x48x24"])
def test_matvec_row_samples_full_size(lib, name):
    """Full-size workloads: 48 seeded rows recomputed by the O(N) pairwise oracle."""
    w = workload(name)
    ctx = _ctx(lib, w.grid, w.m, w.x, lib.Precision.FP32_REFINED)
    kd = ctx.info()["kd"]
    N = ctx.info()["ndipoles"]
    R = min(2, w.nrhs)
    X = random_complex((R, 3, N), 5)
    rows = np.random.default_rng(9).choice(N, 48, replace=False)
    rows[:2] = [0, N - 1]
    want = []
    for r in range(R):
        rr, beta = _site_beta(w.grid, w.m, kd, w.khat[r], w.ehat[r])
        want.append(pairwise.matvec(rr, kd, beta, X[r].T, rows=rows)[0])
    for prec, tol, zpass, slices, xpass in ((0, F64_TOL, -1, 1, -1), (0, F64_TOL, -1, 0, -1), (3, F64_TOL, -1, 1, -1),
                                            (2, F32_TOL, 0, 1, 0), (2, F32_TOL, 1, 1, 0), (2, F32_TOL, 1, 0, 0),
                                            (2, F32_TOL, 2, 0, 0), (2, F32_TOL, 2, 0, 1), (2, F32_TOL, 1, 0, 2),
                                            (2, F32_TOL, 3, 0, 1), (2, F32_TOL, 4, 0, 2)):
        ctx.set_schedule(zpass)
        ctx.set_slice_passes(slices)
        ctx.set_xpass(xpass)
        Y = ctx.matvec(prec, w.khat[:R], w.ehat[:R], X)
        for r in range(R):
            assert _rel(Y[r].T[rows], want[r]) < tol, (name, prec, zpass, slices, xpass, r)
    ctx.close()


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "fp32_refined"])
def test_solve_with_and_without_slice_passes(lib, prec):
    """A 32^3 sphere (64^3 padded, where the fused x+y slice passes run) solved
    with them and with the five separate passes: both converge to the same
    efficiencies (the passes differ only in rounding)."""
    grid = sphere_grid(32)
    ctx = _ctx(lib, grid, [1.5 + 0.05j], 3.0, lib.Precision.FP32_REFINED)
    k, e = _rhs_set(3)
    out = []
    for slices in (1, 0):
        ctx.set_slice_passes(slices)
        res, P, st = ctx.solve(prec, k, e, tol=1e-8 if prec == 0 else 1e-5, maxit=800)
        assert st == 0, slices
        out.append((np.array([[r["qext"], r["qabs"], r["qsca"]] for r in res]), P))
    (qa, Pa), (qb, Pb) = out
    tol = 1e-7 if prec == 0 else 2e-5
    assert np.abs(qa - qb).max() < tol * np.abs(qa).max()
    assert _rel(Pa, Pb) < (1e-6 if prec == 0 else 1e-4)
    with pytest.raises(lib.DdaError):
        ctx.set_slice_passes(2)
    ctx.close()


@pytest.mark.parametrize("zpass", [0, 1, 2], ids=["zgroups", "zregs", "zregs_octant"])
def test_matvec_row_samples_sphere256(lib, zpass):
    """The 256^3 sphere (512^3 padded grid), complex64, every z schedule:
    32 seeded rows recomputed by the pairwise oracle, over 3 RHS."""
    w = workload("sphere256")
    ctx = _ctx(lib, w.grid, w.m, w.x, lib.Precision.FP32_REFINED)
    ctx.set_schedule(zpass)
    ctx.set_xpass(zpass % 2)   # the 512-point rows: staged and warp-local
    kd = ctx.info()["kd"]
    N = ctx.info()["ndipoles"]
    R = 3
    X = random_complex((R, 3, N), 6).astype(np.complex64)
    rows = np.random.default_rng(10).choice(N, 32, replace=False)
    rows[:2] = [0, N - 1]
    Y = ctx.matvec(2, w.khat[:R], w.ehat[:R], X)
    for r in range(R):
        rr, beta = _site_beta(w.grid, w.m, kd, w.khat[r], w.ehat[r])
        want, _ = pairwise.matvec(rr, kd, beta, X[r].T.astype(complex), rows=rows)
        assert _rel(Y[r].T[rows], want) < F32_TOL, (zpass, r)
    ctx.close()


def test_incident_field_matches_oracle(lib):
    grid = ellipsoid_grid(10, 8, 6, 10, 8, 6)
    ctx = _ctx(lib, grid, [1.33 + 0.01j], 2.0, lib.Precision.FP64)
    kd = ctx.info()["kd"]
    k, e = _rhs_set(3)
    E = ctx.incident_field(k, e)
    r, _ = odda.site_positions(grid)
    for i in range(3):
        assert _rel(E[i].T, odda.incident_field(r, kd, k[i], e[i])) < 1e-13
    ctx.close()


def _oracle_solution(grid, m, kd, khat, ehat):
    r, beta = _site_beta(grid, m, kd, khat, ehat)
    E = odda.incident_field(r, kd, khat, ehat)
    P = odda.solve_dense(odda.dense_matrix(r, kd, beta), E)
    aeff = odda.aeff_lattice(len(r))
    return P, odda.efficiencies(odda.cross_sections(kd, E, P, beta), aeff)


@pytest.mark.parametrize("prec,tol,qtol", [(0, 1e-12, 1e-10), (1, 1e-8, 1e-7), (2, 1e-5, 1e-4)],
                         ids=["fp64", "fp32_refined", "fp32"])
def test_solve_matches_dense_lu(lib, prec, tol, qtol):
    grid = block_bernoulli_grid(7, 6, 5, seed=20120514)
    m = [1.7 + 0.3j, 1.2 + 0.01j]
    ctx = _ctx(lib, grid, m, 1.6, lib.Precision.FP32_REFINED)
    kd = ctx.info()["kd"]
    k, e = _rhs_set(3)
    res, P, st = ctx.solve(prec, k, e, tol=tol, maxit=2000)
    assert st == 0, res
    for i in range(3):
        Po, qo = _oracle_solution(grid, m, kd, k[i], e[i])
        assert res[i]["resid_rel"] <= tol
        assert _rel(P[i].T, Po) < max(30 * tol, 1e-10)
        for a, b in zip((res[i]["qext"], res[i]["qabs"], res[i]["qsca"]), qo):
            assert abs(a - b) <= qtol * abs(b), (i, a, b)
    ctx.close()


def test_sphere16_solve_matches_oracle_bicgstab(lib):
    """c1 workload (2176 dipoles, 2 polarizations) at tight tolerance vs the
    oracle's BiCGstab over the C pairwise matvec."""
    w = workload("sphere16")
    ctx = _ctx(lib, w.grid, w.m, w.x, lib.Precision.FP64)
    kd = ctx.info()["kd"]
    res, P, st = ctx.solve(0, w.khat, w.ehat, tol=1e-11)
    assert st == 0
    r, _ = odda.site_positions(w.grid)
    aeff = odda.aeff_lattice(len(r))
    for i in range(2):
        _, beta = _site_beta(w.grid, w.m, kd, w.khat[i], w.ehat[i])
        E = odda.incident_field(r, kd, w.khat[i], w.ehat[i])
        mv = lambda v: pairwise.matvec(r, kd, beta, v.reshape(-1, 3))[0].ravel()  # noqa: E731
        Po, it, nmv, rel = odda.bicgstab(mv, E.ravel(), 1e-12, 500)
        Po = Po.reshape(-1, 3)
        qo = odda.efficiencies(odda.cross_sections(kd, E, Po, beta), aeff)
        assert _rel(P[i].T, Po) < 1e-9
        for a, b in zip((res[i]["qext"], res[i]["qabs"], res[i]["qsca"]), qo):
            assert abs(a - b) <= 1e-10 * abs(b)
    # the sphere is symmetric under y <-> z: both polarizations give the same Q
    assert abs(res[0]["qext"] - res[1]["qext"]) < 1e-9 * res[0]["qext"]
    ctx.close()


@pytest.mark.parametrize("k", [1, 3, 7])
def test_iteration_limit_returns_the_kth_bicgstab_iterate(lib, k):
    """A solve stopped by its iteration limit returns the oracle BiCGstab's
    k-th iterate: the update x += alpha p + omega s of the last iteration,
    which the GPU solve applies in the next iteration's first gather, is
    applied after the loop for a RHS that stops (c1 workload, FP64)."""
    w = workload("sphere16")
    ctx = _ctx(lib, w.grid, w.m, w.x, lib.Precision.FP64)
    kd = ctx.info()["kd"]
    res, P, st = ctx.solve(0, w.khat[:1], w.ehat[:1], tol=1e-14, maxit=k)
    assert res[0]["iters"] == k
    assert res[0]["status_name"] == "DDA_ERR_NOT_CONVERGED"
    r, _ = odda.site_positions(w.grid)
    _, beta = _site_beta(w.grid, w.m, kd, w.khat[0], w.ehat[0])
    E = odda.incident_field(r, kd, w.khat[0], w.ehat[0])
    mv = lambda v: pairwise.matvec(r, kd, beta, v.reshape(-1, 3))[0].ravel()  # noqa: E731
    Po, it, _, _ = odda.bicgstab(mv, E.ravel(), 1e-14, k)
    assert it == k
    assert _rel(P[0].T, Po.reshape(-1, 3)) < 1e-10
    ctx.close()


def test_batched_masked_solve_equals_single_solves(lib):
    grid = ellipsoid_grid(12, 10, 8, 12, 10, 8)
    m = [1.33 + 0.05j]
    ctx = _ctx(lib, grid, m, 2.5, lib.Precision.FP32_REFINED)
    k, e = _rhs_set(6)
    res_b, P_b, st = ctx.solve(1, k, e, tol=1e-6)
    assert st == 0
    iters = [r["iters"] for r in res_b]
    for i in (0, 3, 5):
        res_1, P_1, st1 = ctx.solve(1, k[i:i + 1], e[i:i + 1], tol=1e-6)
        assert st1 == 0
        assert res_1[0]["iters"] == iters[i]
        assert _rel(P_b[i], P_1[0]) < 1e-6
    ctx.close()


def test_graph_and_eager_agree(lib):
    grid = sphere_grid(10)
    ctx = _ctx(lib, grid, [1.5 + 0.02j], 1.5, lib.Precision.FP32_REFINED)
    k, e = _rhs_set(2)
    a, Pa, _ = ctx.solve(1, k, e, tol=1e-6, use_graph=True)
    b, Pb, _ = ctx.solve(1, k, e, tol=1e-6, use_graph=False)
    assert np.array_equal(Pa, Pb)
    assert [r["iters"] for r in a] == [r["iters"] for r in b]
    ctx.close()


def test_gradient_matches_oracle_adjoint_and_fd(lib):
    grid = block_bernoulli_grid(4, 3, 3, seed=20120514)
    m = [1.7 + 0.3j, 1.2 + 0.01j]
    x = 1.2
    ctx = _ctx(lib, grid, m, x, lib.Precision.FP64)
    kd = ctx.info()["kd"]
    k, e = np.array([[1.0, 0, 0]]), np.array([[0, 1.0, 0]], complex)
    gre, gim, P, (rf, ra) = ctx.grad_qabs(0, k, e, tol=1e-12)
    r, comp = odda.site_positions(grid)
    eps = (np.asarray(m) ** 2)[comp - 1]
    beta = odda.ldr_inverse_polarizability(eps, kd, k[0], e[0])
    A = odda.dense_matrix(r, kd, beta)
    Eo = odda.incident_field(r, kd, k[0], e[0])
    Po = odda.solve_dense(A, Eo)
    w = odda.absorption_weights(kd, beta)
    nu = odda.solve_dense(A, w[:, None] * np.conj(Po))
    aeff = odda.aeff_lattice(len(r))
    ore, oim = odda.qabs_gradient(kd, aeff, eps, k[0], e[0], Po, nu)
    assert _rel(gre, ore) < 1e-9 and _rel(gim, oim) < 1e-9
    ctx.close()


def test_failure_statuses(lib):
    ctx = lib.Context(0)
    with pytest.raises(lib.DdaError) as ei:
        ctx.set_target(np.zeros((3, 3, 3), np.uint8))
    assert ei.value.status_name == "DDA_ERR_ARG"
    with pytest.raises(lib.DdaError) as ei:
        ctx.set_target(np.ones((2, 2, 300), np.uint8))
    assert ei.value.status_name == "DDA_ERR_SIZE"
    ctx.set_target(sphere_grid(8))
    with pytest.raises(lib.DdaError) as ei:
        ctx.set_materials([complex("nan")])
    assert ei.value.status_name == "DDA_ERR_NONFINITE"
    ctx.set_materials([1.5 + 0.1j])
    with pytest.raises(lib.DdaError):
        ctx.solve(0, [[1, 0, 0]], [[0, 1, 0]])          # not prepared
    ctx.prepare_size_parameter(1.0, lib.Precision.FP64)
    with pytest.raises(lib.DdaError) as ei:
        ctx.solve(0, [[1, 0, 0]], [[1, 0, 0]])          # not transverse
    assert ei.value.status_name == "DDA_ERR_ARG"
    with pytest.raises(lib.DdaError):
        ctx.solve(1, [[1, 0, 0]], [[0, 1, 0]])          # FP32 not prepared
    res, P, st = ctx.solve(0, [[1, 0, 0]], [[0, 1, 0]], tol=1e-10, maxit=2)
    assert res[0]["status_name"] == "DDA_ERR_NOT_CONVERGED" and res[0]["iters"] <= 2
    ctx.close()


def test_launch_tracing_counts_and_leaves_results_unchanged(lib):
    import ctypes
    grid = sphere_grid(12)
    ctx = _ctx(lib, grid, [1.5 + 0.02j], 2.0, lib.Precision.FP32_REFINED)
    k, e = _rhs_set(2)
    plain, P0, _ = ctx.solve(1, k, e, tol=1e-6)
    L = lib.load_library()
    assert L.dda_profile_enable(ctx.handle, 1) == 0

    class Stat(ctypes.Structure):
        _fields_ = [("name", ctypes.c_char * 24), ("launches", ctypes.c_int64), ("total_ms", ctypes.c_double),
                    ("units", ctypes.c_double)]

    traced, P1, _ = ctx.solve(1, k, e, tol=1e-6)
    arr = (Stat * 32)()
    n = ctypes.c_int()
    L.dda_profile_read.argtypes = [ctypes.c_void_p, ctypes.POINTER(Stat), ctypes.c_int, ctypes.POINTER(ctypes.c_int)]
    assert L.dda_profile_read(ctx.handle, arr, 32, ctypes.byref(n)) == 0
    stats = {arr[i].name.decode(): (arr[i].launches, arr[i].total_ms, arr[i].units) for i in range(n.value)}
    L.dda_profile_enable(ctx.handle, 0)
    assert np.array_equal(P0, P1)
    it = max(r["iters"] for r in traced)
    zl, zms, zu = stats["z_conv_c64"]
    assert zl >= 2 * it and zl % 8 == 0          # 2 matvecs per iteration, blocks of 4 iterations
    assert zu == 2 * zl and zms > 0               # both RHS in every launch
    # one true-residual matvec per refinement step, in double-float arithmetic by default
    assert stats["z_conv_df"][0] == max(r["outer_iters"] for r in traced)
    for name in ("x_fwd_c64", "y_fwd_c64", "y_inv_c64", "x_inv_c64"):
        assert stats[name][0] == zl
    ctx.close()


def test_refinement_residual_double_float_equals_fp64(lib):
    """The complex64 modes check their true residual with a double-float
    matvec by default; native FP64 arithmetic gives the same answers."""
    grid = ellipsoid_grid(20, 16, 12, 20, 16, 12)
    ctx = _ctx(lib, grid, [1.5 + 0.02j], 3.0, lib.Precision.FP32_REFINED)
    k, e = _rhs_set(3)
    a, Pa, sa = ctx.solve(1, k, e, tol=1e-6)
    b, Pb, sb = ctx.solve(1, k, e, tol=1e-6, residual_fp64=True)
    assert sa == 0 and sb == 0
    for ra, rb in zip(a, b):
        assert ra["iters"] == rb["iters"] and ra["outer_iters"] == rb["outer_iters"]
        assert abs(ra["resid_rel"] - rb["resid_rel"]) <= 1e-6 * rb["resid_rel"]
        for q in ("qext", "qabs", "qsca"):
            assert abs(ra[q] - rb[q]) <= 1e-11 * abs(rb[q])
    assert np.abs(Pa - Pb).max() <= 1e-11 * np.abs(Pb).max()
    ctx.close()
