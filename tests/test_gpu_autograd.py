"""QabsFn (torch.autograd) and solver options on the GPU vs the oracle."""
import numpy as np
import pytest

from dda_inputs import block_bernoulli_grid, ellipsoid_grid, uniform_directions, polarization_pair
from oracle import dda as odda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1202_3424_gb300 as dda
    from paper_1202_3424_gb300.autograd import DipoleTarget, QabsFn
    dda.load_library()
    return dda, torch, DipoleTarget, QabsFn


def _oracle_qabs_grad(occ, eps, x, khat, ehat):
    r, _ = odda.site_positions(occ.astype(np.uint8))
    N = len(r)
    aeff = odda.aeff_lattice(N)
    kd = x / aeff
    beta = odda.ldr_inverse_polarizability(eps, kd, khat, ehat)
    A = odda.dense_matrix(r, kd, beta)
    E = odda.incident_field(r, kd, khat, ehat)
    P = odda.solve_dense(A, E)
    q = odda.efficiencies(odda.cross_sections(kd, E, P, beta), aeff)[1]
    w = odda.absorption_weights(kd, beta)
    nu = odda.solve_dense(A, w[:, None] * np.conj(P))
    gre, gim = odda.qabs_gradient(kd, aeff, eps, khat, ehat, P, nu)
    return q, gre + 1j * gim


def test_qabsfn_matches_dense_oracle(env):
    dda, torch, DipoleTarget, QabsFn = env
    occ = ellipsoid_grid(5, 4, 4, 5, 4, 4).astype(bool)
    N = int(occ.sum())
    rng = np.random.default_rng(20120514)
    eps = (1.6 + 0.4 * rng.random(N)) + 1j * (0.05 + 0.3 * rng.random(N))   # every dipole its own material
    k, e = np.array([0.0, 0.6, 0.8]), np.array([1.0, 0.0, 0.0], complex)
    tgt = DipoleTarget(occ, 1.3, k, e, tol=1e-12)
    t = torch.tensor(eps, dtype=torch.complex128, requires_grad=True)
    q = QabsFn.apply(t, tgt)
    q.backward()
    qo, go = _oracle_qabs_grad(occ, eps, 1.3, k, e)
    assert abs(q.item() - qo) < 1e-10 * abs(qo)
    assert np.abs(t.grad.numpy() - go).max() < 1e-8 * np.abs(go).max()
    tgt.close()


def test_qabsfn_gradient_matches_finite_differences(env):
    dda, torch, DipoleTarget, QabsFn = env
    occ = block_bernoulli_grid(4, 4, 3, seed=5).astype(bool)
    N = int(occ.sum())
    eps = np.where(block_bernoulli_grid(4, 4, 3, seed=6).ravel() == 1, (1.7 + 0.3j) ** 2, (1.2 + 0.01j) ** 2)
    k, e = np.array([1.0, 0.0, 0.0]), np.array([0.0, 1.0, 0.0], complex)
    tgt = DipoleTarget(occ, 1.0, k, e, tol=1e-13)
    t = torch.tensor(eps, dtype=torch.complex128, requires_grad=True)
    QabsFn.apply(t, tgt).backward()
    g = t.grad.numpy()
    for j in (0, 17, N - 1):
        for d in (1.0, 1j):
            h = 1e-4
            ep, em = eps.copy(), eps.copy()
            ep[j] += d * h
            em[j] -= d * h
            fd = (tgt.qabs_and_grad(ep)[0] - tgt.qabs_and_grad(em)[0]) / (2 * h)
            want = g[j].real if d == 1.0 else g[j].imag
            assert abs(fd - want) < 1e-5 * np.abs(g).max(), (j, d, fd, want)
    tgt.close()


def test_warm_start_and_normal_equation_error(env):
    dda, torch, DipoleTarget, QabsFn = env
    grid = ellipsoid_grid(14, 12, 10, 14, 12, 10)
    ctx = dda.Context(0)
    ctx.set_target(grid)
    ctx.set_materials([1.5 + 0.05j])
    ctx.prepare_size_parameter(2.0, dda.Precision.FP32_REFINED)
    k = uniform_directions(2, 3)
    e = polarization_pair(k)[0].astype(complex)
    res, P, st = ctx.solve(0, k, e, tol=1e-10, normal_eq=True)
    assert st == 0
    for r in res:
        assert 0 <= r["resid_normal_eq"] < 1e-8         # eq. err_tol form, reported next to the residual
    # resuming from the solution needs no iterations and reproduces Q
    res2, P2, st2 = ctx.solve(0, k, e, tol=1e-8, x0=P)
    assert st2 == 0 and all(r["iters"] == 0 for r in res2)
    for a, b in zip(res, res2):
        assert abs(a["qext"] - b["qext"]) < 1e-9 * abs(a["qext"])
    # and a coarse FP32-refined start continued in FP64 converges to the tight answer
    res3, P3, _ = ctx.solve(1, k, e, tol=1e-4)
    res4, P4, st4 = ctx.solve(0, k, e, tol=1e-10, x0=P3)
    assert st4 == 0 and res4[0]["iters"] < res[0]["iters"]
    assert np.abs(P4 - P).max() < 1e-8 * np.abs(P).max()
    ctx.close()


def test_qabsfn_runs_the_adjoint_only_in_backward(env):
    """The forward pass is one solve; the adjoint solve (target.grad) runs
    when, and only when, the gradient is asked for."""
    dda, torch, DipoleTarget, QabsFn = env
    occ = ellipsoid_grid(6, 5, 4, 6, 5, 4).astype(bool)
    N = int(occ.sum())
    eps = np.full(N, 2.2 + 0.3j)
    tgt = DipoleTarget(occ, 1.1, [1.0, 0.0, 0.0], np.array([0.0, 0.0, 1.0], complex), tol=1e-12)
    calls = []
    grad = tgt.grad
    tgt.grad = lambda *a, **k: calls.append(1) or grad(*a, **k)
    q0 = QabsFn.apply(torch.tensor(eps), tgt)                      # no gradient wanted
    t = torch.tensor(eps, requires_grad=True)
    q1 = QabsFn.apply(t, tgt)
    assert calls == [] and abs(q0.item() - q1.item()) < 1e-12 * abs(q0.item())
    q1.backward()
    assert calls == [1] and torch.isfinite(t.grad).all()
    tgt.close()


def test_qabsfn_on_the_block_with_every_dipole_distinct(env):
    """The 48x48x24 two-material block with a seeded perturbation of every
    dipole's eps (55,296 distinct values, beyond any composition-code table):
    QabsFn's gradient against central finite differences on 16 seeded dipoles
    (h = 1e-4 |eps|, FP64 solves to 1e-12)."""
    dda, torch, DipoleTarget, QabsFn = env
    from dda_inputs import SEED_COMPOSITION, workload
    w = workload("block48x48x24")
    occ = w.grid > 0
    N = int(occ.sum())
    base = (np.asarray(w.m) ** 2)[w.grid[occ] - 1]
    rng = np.random.default_rng(SEED_COMPOSITION + 1)
    eps = base * (1.0 + 0.02 * (rng.random(N) - 0.5)) + 0.01j * rng.random(N)
    assert np.unique(eps).size == N
    tgt = DipoleTarget(occ, w.x, w.khat[0], w.ehat[0], tol=1e-12, maxit=3000)
    t = torch.tensor(eps, requires_grad=True)
    q = QabsFn.apply(t, tgt)
    q.backward()
    g = t.grad.numpy()
    picks = np.random.default_rng(SEED_COMPOSITION).choice(N, 16, replace=False)
    for j in picks:
        for d in (1.0, 1j):
            h = 1e-4 * abs(eps[j])
            ep, em = eps.copy(), eps.copy()
            ep[j] += d * h
            em[j] -= d * h
            fd = (tgt.qabs(ep)[0] - tgt.qabs(em)[0]) / (2 * h)
            want = g[j].real if d == 1.0 else g[j].imag
            assert abs(fd - want) <= 1e-3 * abs(want) + 1e-10 * abs(q.item()), (j, d, fd, want)
    tgt.close()


def test_site_materials_match_composition_codes(env):
    """Per-site materials given the values of a composition table reproduce
    the composition-code solve (same tables, other indexing)."""
    dda, torch, DipoleTarget, QabsFn = env
    grid = block_bernoulli_grid(9, 7, 5, seed=31)
    m = [1.7 + 0.3j, 1.2 + 0.01j]
    ctx = dda.Context(0)
    ctx.set_target(grid)
    ctx.set_materials(m)
    ctx.prepare_size_parameter(1.5, dda.Precision.FP32_REFINED)
    k = uniform_directions(3, 11)
    e = polarization_pair(k)[1].astype(complex)
    out = []
    for site in (False, True):
        if site:
            ctx.set_site_materials(np.asarray(m)[grid[grid > 0] - 1])
            ctx.prepare_size_parameter(1.5, dda.Precision.FP32_REFINED)
        for prec in (0, 1):
            res, P, st = ctx.solve(prec, k, e, tol=1e-9 if prec == 0 else 1e-6)
            assert st == 0
            out.append(np.array([[r["qext"], r["qabs"], r["qsca"]] for r in res]))
    assert np.abs(out[0] - out[2]).max() < 1e-12 * np.abs(out[0]).max()
    assert np.abs(out[1] - out[3]).max() < 1e-5 * np.abs(out[1]).max()
    # a new target ends the per-site mode: materials must be given again
    ctx.set_target(grid)
    with pytest.raises(dda.DdaError):
        ctx.prepare_size_parameter(1.5, dda.Precision.FP64)
    ctx.close()
