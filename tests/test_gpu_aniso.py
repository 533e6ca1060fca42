"""Anisotropic dielectric-frame polarizabilities on the GPU vs the oracle.

Each composition carries three principal refractive indices and the angles
(theta_DF, phi_DF, beta_DF) of its dielectric frame ("Composite Targets with
Anisotropic Constituents"); the diagonal blocks of A become the symmetric
tensors sum_j (1/alpha_j) e_j e_j^T (oracle/dda.py: dielectric_frame,
ldr_inverse_tensor) and C_abs takes its tensor form.  Tolerances as for the
isotropic path: 1e-10 relative with complex128, 1e-5 with complex64.
"""
import math

import numpy as np
import pytest

from dda_inputs import (block_bernoulli_grid, ellipsoid_grid, polarization_pair, random_complex, uniform_directions,
                        workload)
from oracle import dda as odda
from oracle import pairwise

pytestmark = pytest.mark.gpu

F64_TOL = 1e-10
F32_TOL = 1e-5

# two anisotropic materials: a uniaxial one tilted out of the Target Frame and
# a biaxial absorbing one with a general orientation
M3 = [[1.55 + 0.02j, 1.40 + 0.01j, 1.40 + 0.01j], [1.9 + 0.4j, 1.6 + 0.1j, 1.3 + 0.05j]]
ANGLES = [[0.6, 1.1, 0.0], [2.1, -0.7, 0.9]]


@pytest.fixture(scope="module")
def lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1202_3424_gb300 as dda
    dda.load_library()
    return dda


def _ctx(dda, grid, m3, angles, x, prec=1):
    ctx = dda.Context(0)
    ctx.set_target(grid)
    ctx.set_anisotropic_materials(m3, angles)
    ctx.prepare_size_parameter(x, prec)
    return ctx


def _site_tensors(grid, m3, angles, kd, khat, ehat):
    """Per-site 1/alpha tensors (N, 3, 3) from the oracle."""
    r, comp = odda.site_positions(grid)
    ncomp = int(comp.max())
    Bc = np.array([odda.ldr_inverse_tensor(np.asarray(m3[c], dtype=complex) ** 2, angles[c], kd, khat, ehat)
                   for c in range(ncomp)])
    return r, Bc[comp - 1]


def _rel(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


def _rhs_set(R, seed=7):
    k = uniform_directions(R, seed)
    e1, _ = polarization_pair(k)
    return k, e1.astype(complex)


CASES = [
    ("block_two_materials", lambda: block_bernoulli_grid(7, 5, 4, seed=6), M3, ANGLES, 1.6),
    ("ellipsoid_ragged", lambda: ellipsoid_grid(13, 9, 6, 13, 9, 6), M3[1:], ANGLES[1:], 1.2),
    ("single_dipole", lambda: np.ones((1, 1, 1), np.uint8), M3[1:], ANGLES[1:], 0.3),
    # 64x64 in x and y, where the isotropic matvec may take the slice passes
    ("plate_25x25x3", lambda: block_bernoulli_grid(25, 25, 3, seed=8), M3, ANGLES, 2.2),
]


@pytest.mark.parametrize("name,gridf,m3,angles,x", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("prec,tol", [(0, F64_TOL), (3, F64_TOL), (2, F32_TOL)], ids=["fp64", "df64", "fp32"])
def test_aniso_matvec_matches_oracle(lib, name, gridf, m3, angles, x, prec, tol):
    grid = gridf()
    ctx = _ctx(lib, grid, m3, angles, x)
    ctx.set_slice_passes(1)
    kd = ctx.info()["kd"]
    R = 3
    k, e = _rhs_set(R)
    X = random_complex((R, 3, ctx.info()["ndipoles"]), 21)
    Y = ctx.matvec(prec, k, e, X)
    for r in range(R):
        rr, B = _site_tensors(grid, m3, angles, kd, k[r], e[r])
        want = odda.pairwise_matvec(rr, kd, B, X[r].T)
        assert _rel(Y[r].T, want) < tol, (name, r)
    ctx.close()


@pytest.mark.parametrize("zpass", [0, 1, 2], ids=["zgroups", "zregs", "zregs_octant"])
def test_aniso_matvec_z_schedules_nine_rhs(lib, zpass):
    grid = block_bernoulli_grid(9, 8, 7, seed=12)
    ctx = _ctx(lib, grid, M3, ANGLES, 1.8)
    ctx.set_schedule(zpass)
    kd = ctx.info()["kd"]
    R = 9
    k, e = _rhs_set(R, 3)
    X = random_complex((R, 3, ctx.info()["ndipoles"]), 22)
    Y = ctx.matvec(2, k, e, X)
    for r in range(R):
        rr, B = _site_tensors(grid, M3, ANGLES, kd, k[r], e[r])
        assert _rel(Y[r].T, odda.pairwise_matvec(rr, kd, B, X[r].T)) < F32_TOL, (zpass, r)
    ctx.close()


def _oracle_solution(grid, m3, angles, kd, khat, ehat):
    r, B = _site_tensors(grid, m3, angles, kd, khat, ehat)
    E = odda.incident_field(r, kd, khat, ehat)
    P = odda.solve_dense(odda.dense_matrix(r, kd, B), E)
    return P, odda.efficiencies(odda.cross_sections(kd, E, P, B), odda.aeff_lattice(len(r)))


@pytest.mark.parametrize("prec,tol,qtol", [(0, 1e-12, 1e-10), (1, 1e-8, 1e-7), (2, 1e-5, 1e-4)],
                         ids=["fp64", "fp32_refined", "fp32"])
def test_aniso_solve_matches_dense_lu(lib, prec, tol, qtol):
    """BiCGstab with the fused tensor diagonal, the refinement residual and the
    tensor C_abs, against a dense LU solve of the oracle's matrix."""
    grid = block_bernoulli_grid(7, 6, 5, seed=31)
    ctx = _ctx(lib, grid, M3, ANGLES, 1.5)
    kd = ctx.info()["kd"]
    k, e = _rhs_set(3, 11)
    res, P, st = ctx.solve(prec, k, e, tol=tol, maxit=2000)
    assert st == 0, res
    for i in range(3):
        Po, qo = _oracle_solution(grid, M3, ANGLES, kd, k[i], e[i])
        assert _rel(P[i].T, Po) < max(30 * tol, 1e-10)
        for a, b in zip((res[i]["qext"], res[i]["qabs"], res[i]["qsca"]), qo):
            assert abs(a - b) <= qtol * abs(b), (i, a, b)
    ctx.close()


def test_aniso_equal_indices_reduce_to_isotropic(lib):
    """Three equal principal indices at any orientation: the same matvec and
    solve as dda_set_materials with that index."""
    grid = ellipsoid_grid(11, 9, 7, 11, 9, 7)
    m = 1.5 + 0.05j
    k, e = _rhs_set(2, 5)
    iso = lib.Context(0)
    iso.set_target(grid)
    iso.set_materials([m])
    iso.prepare_size_parameter(1.4, 0)
    ani = _ctx(lib, grid, [[m, m, m]], [[0.8, -1.9, 2.4]], 1.4, 0)
    X = random_complex((2, 3, iso.info()["ndipoles"]), 3)
    assert _rel(ani.matvec(0, k, e, X), iso.matvec(0, k, e, X)) < 1e-14
    ri, _, _ = iso.solve(0, k, e, tol=1e-11)
    ra, _, _ = ani.solve(0, k, e, tol=1e-11)
    for a, b in zip(ra, ri):
        for q in ("qext", "qabs", "qsca"):
            assert abs(a[q] - b[q]) < 1e-9 * abs(b[q]), q
    iso.close()
    ani.close()


def test_aniso_rotated_frame_equals_permuted_indices(lib):
    """theta_DF = pi/2 puts e_1 on y and e_2 on -x: the material (ma, mb, mc)
    at that orientation is the frame-aligned material (mb, ma, mc)."""
    grid = ellipsoid_grid(9, 7, 6, 9, 7, 6)
    ma, mb, mc = 1.7 + 0.2j, 1.3 + 0.02j, 1.5 + 0.1j
    k, e = _rhs_set(2, 9)
    rot = _ctx(lib, grid, [[ma, mb, mc]], [[math.pi / 2, 0.0, 0.0]], 1.3, 0)
    ali = _ctx(lib, grid, [[mb, ma, mc]], [[0.0, 0.0, 0.0]], 1.3, 0)
    X = random_complex((2, 3, rot.info()["ndipoles"]), 8)
    assert _rel(rot.matvec(0, k, e, X), ali.matvec(0, k, e, X)) < 1e-13
    r1, _, _ = rot.solve(0, k, e, tol=1e-11)
    r2, _, _ = ali.solve(0, k, e, tol=1e-11)
    for a, b in zip(r1, r2):
        assert abs(a["qabs"] - b["qabs"]) < 1e-9 * abs(b["qabs"])
    rot.close()
    ali.close()


@pytest.mark.parametrize("prec,tol", [(0, F64_TOL), (2, F32_TOL)], ids=["fp64", "fp32"])
def test_aniso_full_size_row_samples(lib, prec, tol):
    """The 96x64x32 ellipsoid (102984 dipoles) of a tilted biaxial material,
    2 RHS: 48 seeded rows, the interaction part by the C pairwise oracle
    (zero diagonal) plus the site's tensor block."""
    w = workload("ellipsoid96x64x32")
    m3, ang = [[1.33 + 0.01j, 1.45 + 0.02j, 1.25 + 0.005j]], [[0.4, 2.0, -1.1]]
    ctx = _ctx(lib, w.grid, m3, ang, w.x)
    kd, N = ctx.info()["kd"], ctx.info()["ndipoles"]
    R = 2
    X = random_complex((R, 3, N), 14)
    rows = np.random.default_rng(10).choice(N, 48, replace=False)
    rows[:2] = [0, N - 1]
    for zpass in (0, 1, 2):
        ctx.set_schedule(zpass)
        Y = ctx.matvec(prec, w.khat[:R], w.ehat[:R], X)
        for r in range(R):
            rr, B = _site_tensors(w.grid, m3, ang, kd, w.khat[r], w.ehat[r])
            off, _ = pairwise.matvec(rr, kd, np.zeros(N, complex), X[r].T, rows=rows)
            want = off + np.einsum("jab,jb->ja", B[rows], X[r].T[rows])
            assert _rel(Y[r].T[rows], want) < tol, (zpass, r)
    ctx.close()


def test_aniso_rejects_gradient_and_bad_input(lib):
    grid = block_bernoulli_grid(4, 4, 4, seed=1)
    ctx = _ctx(lib, grid, M3, ANGLES, 1.0, 0)
    k, e = _rhs_set(1)
    with pytest.raises(lib.DdaError) as ei:
        ctx.grad_qabs(0, k[0], e[0])
    assert ei.value.status == 1
    with pytest.raises(lib.DdaError) as ei:
        ctx.set_anisotropic_materials([[1.5, 1.0, 1.4]], [[0, 0, 0]])      # an index equal to the ambient one
    assert ei.value.status == 1
    with pytest.raises(lib.DdaError) as ei:
        ctx.set_anisotropic_materials([[1.5, 1.6, 1.4]], [[0, float("nan"), 0]])
    assert ei.value.status == 7
    ctx.close()
