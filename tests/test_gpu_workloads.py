"""Full-size synthetic workloads on the GPU, checked with properties the
oracle can evaluate at any size (needs a GB300).

- 3:2:1 ellipsoid, 128 RHS batched (FP32-refined): every RHS converges to a
  true FP64 residual <= 1e-5, and for sampled RHS the oracle's far-field
  quadrature of the GPU's P gives C_sca = C_ext - C_abs (optical theorem).
- two-material block, adjoint gradient vs central finite differences on 16
  seeded dipoles.
- 256^3 sphere, 16 RHS: Q vs the Mie series within the guide's "few percent".
- 64^3 sphere (both polarizations) and 16 RHS of the ellipsoid sweep: the
  production mode (complex64 matvec, FP64 refinement, tol 1e-5) against a
  plain FP64 solve to 1e-10, Q_ext, Q_abs and Q_sca per RHS to 1e-5
  relative.  (The FP64 path itself matches the oracle to 1e-10 in
  test_gpu_parity.py.)
"""
import math

import numpy as np
import pytest

from dda_inputs import SEED_COMPOSITION, workload
from oracle import dda as odda
from oracle import mie

pytestmark = pytest.mark.gpu


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


def test_ellipsoid_sweep_128_rhs_converges_and_conserves_energy(lib):
    w = workload("ellipsoid96x64x32")
    ctx = _ctx(lib, w.grid, w.m, w.x, lib.Precision.FP32_REFINED)
    kd = ctx.info()["kd"]
    res, P, st = ctx.solve(lib.Precision.FP32_REFINED, w.khat, w.ehat, tol=1e-5, maxit=3000)
    assert st == 0 and len(res) == 128
    assert max(r["resid_rel"] for r in res) <= 1e-5
    r, _ = odda.site_positions(w.grid)
    aeff = odda.aeff_lattice(len(r))
    for i in (0, 77):
        csca = odda.csca_quadrature(r, kd, P[i].T, ntheta=48, nphi=96)
        qsca = csca / (math.pi * aeff ** 2)
        assert abs(qsca - res[i]["qsca"]) < 2e-4 * res[i]["qext"], (i, qsca, res[i])
    ctx.close()


def test_block_gradient_matches_finite_differences(lib):
    w = workload("block48x48x24")
    grid = w.grid
    m = list(w.m)
    ctx = _ctx(lib, grid, m, w.x, lib.Precision.FP64)
    gre, gim, P, (rf, ra) = ctx.grad_qabs(lib.Precision.FP64, w.khat, w.ehat, tol=1e-12, maxit=3000)
    assert rf["status"] == 0 and ra["status"] == 0
    N = ctx.info()["ndipoles"]
    r, comp = odda.site_positions(grid)
    rng = np.random.default_rng(SEED_COMPOSITION)
    picks = rng.choice(N, 16, replace=False)
    flat = np.flatnonzero(grid.ravel())          # site j -> flat grid index (x-fastest scan)
    for j in picks:                                 # 16 dipoles x (Re, Im) x 2 sides = 64 extra solves
        eps = complex(m[comp[j] - 1]) ** 2
        for part, g in ((1.0, gre[j]), (1j, gim[j])):
            h = 1e-4 * abs(eps)
            q = []
            for sgn in (+1, -1):
                g3 = grid.copy().ravel()
                g3[flat[j]] = 3
                ctx.set_target(g3.reshape(grid.shape))
                ctx.set_materials(m + [np.sqrt(eps + sgn * part * h)])
                ctx.prepare_size_parameter(w.x, lib.Precision.FP64)
                rr, _, st = ctx.solve(lib.Precision.FP64, w.khat, w.ehat, want_P=False, tol=1e-12, maxit=3000)
                assert st == 0
                q.append(rr[0]["qabs"])
            fd = (q[0] - q[1]) / (2 * h)
            assert abs(fd - g) <= 1e-3 * abs(g) + 1e-10 * abs(rf["qabs"]), (j, part, fd, g)
    ctx.close()


def test_sphere256_matches_mie(lib):
    w = workload("sphere256")
    ctx = _ctx(lib, w.grid, w.m, w.x, lib.Precision.FP32_REFINED)
    res, _, st = ctx.solve(lib.Precision.FP32_REFINED, w.khat, w.ehat, want_P=False, tol=1e-5, maxit=3000)
    assert st == 0
    qm = mie.mie_efficiencies(w.x, w.m[0])
    qe = np.array([r["qext"] for r in res])
    qa = np.array([r["qabs"] for r in res])
    assert np.all(np.abs(qe - qm[0]) < 0.03 * qm[0]), (qe, qm)
    assert np.all(np.abs(qa - qm[1]) < 0.03 * qm[1]), (qa, qm)
    # a sphere: every direction and polarization sees the same Q up to lattice anisotropy
    assert qe.max() - qe.min() < 0.01 * qm[0]
    ctx.close()


Q_RTOL = 1e-5


def _q(res):
    return np.array([[r["qext"], r["qabs"], r["qsca"]] for r in res])


def _refined_vs_fp64(lib, w, nrhs):
    ctx = _ctx(lib, w.grid, w.m, w.x, lib.Precision.FP32_REFINED)
    k, e = w.khat[:nrhs], w.ehat[:nrhs]
    r32, _, st = ctx.solve(lib.Precision.FP32_REFINED, k, e, want_P=False, tol=1e-5, maxit=3000)
    assert st == 0 and max(r["resid_rel"] for r in r32) <= 1e-5
    r64, _, st = ctx.solve(lib.Precision.FP64, k, e, want_P=False, tol=1e-10, maxit=4000)
    assert st == 0 and max(r["resid_rel"] for r in r64) <= 1e-10
    ctx.close()
    q32, q64 = _q(r32), _q(r64)
    return np.abs(q32 - q64) / np.abs(q64)


def test_sphere64_refined_q_matches_fp64(lib):
    """The bench workload: both polarizations, every factor within 1e-5."""
    err = _refined_vs_fp64(lib, workload("sphere64"), 2)
    assert err.max() <= Q_RTOL, err


def test_ellipsoid_sweep_refined_q_matches_fp64(lib):
    """16 RHS of the 128-RHS sweep (seeded directions, both polarizations)."""
    err = _refined_vs_fp64(lib, workload("ellipsoid96x64x32"), 16)
    assert err.max() <= Q_RTOL, err
