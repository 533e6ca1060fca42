"""Planted mistakes in the CPU oracle must each fail at least one pin.

Every mutation is applied with monkeypatch to the oracle only (CPU); the
pins are the functions of tests/test_oracle_pins.py.  A mutation that no pin
catches would mean that part of the oracle is not pinned.
"""
import inspect
import math
import textwrap

import numpy as np
import pytest

from oracle import dda, mie
import test_oracle_pins as pins

_orig_tensor = dda.interaction_tensor
_orig_ldr = dda.ldr_inverse_polarizability
_orig_xs = dda.cross_sections
_orig_einc = dda.incident_field
_orig_j = dda._sph_j012
_orig_grad = dda.qabs_gradient
_orig_sites = dda.site_positions
_orig_scat = dda.scattered_field
_orig_box = dda.nearfield_box
_orig_ff = dda.far_field
_orig_dirs = dda.scattering_directions
_orig_mueller = dda.mueller_matrix
_orig_frame = dda.dielectric_frame


def _mutant(fn, old, new):
    """fn recompiled from its source with one statement changed."""
    src = textwrap.dedent(inspect.getsource(fn))
    assert src.count(old) == 1, old
    ns = dict(vars(inspect.getmodule(fn)))
    exec(compile(src.replace(old, new), inspect.getsourcefile(fn), "exec"), ns)
    out = ns[fn.__name__]
    out.__name__ = f"{fn.__name__}: {new.strip()}"
    return out


def _tensor_sign(rvec, kd):            # (1 - ik rho) instead of (ik rho - 1)
    rvec = np.asarray(rvec, float)
    rho = np.linalg.norm(rvec, axis=-1)
    rh = rvec / rho[..., None]
    rr = rh[..., :, None] * rh[..., None, :]
    ph = np.exp(1j * kd * rho) / rho
    c2 = (1.0 - 1j * kd * rho) / rho ** 2
    return ph[..., None, None] * (kd * kd * (rr - np.eye(3)) + c2[..., None, None] * (3 * rr - np.eye(3)))


def _tensor_no_far(rvec, kd):          # dropped k^2 (rr - I) radiation term
    rvec = np.asarray(rvec, float)
    rho = np.linalg.norm(rvec, axis=-1)
    rh = rvec / rho[..., None]
    rr = rh[..., :, None] * rh[..., None, :]
    ph = np.exp(1j * kd * rho) / rho
    c2 = (1j * kd * rho - 1.0) / rho ** 2
    return ph[..., None, None] * (c2[..., None, None] * (3 * rr - np.eye(3)))


def _tensor_incoming(rvec, kd):        # exp(-ik rho): incoming instead of outgoing wave
    return np.conj(_orig_tensor(rvec, kd))


def _ldr_no_rr(eps, kd, khat, ehat):   # dropped radiative reaction
    return _orig_ldr(eps, kd, khat, ehat) + (2.0 / 3.0) * 1j * kd ** 3


def _xs_no_conj(kd, E, P, beta):       # Im(E . P) instead of Im(E^* . P)
    c = list(_orig_xs(kd, np.conj(E), P, beta))
    return c[0], c[1], c[0] - c[1]


def _xs_rr_sign(kd, E, P, beta):       # +(2/3)k^3 in C_abs
    cext, cabs, _ = _orig_xs(kd, E, P, beta)
    cabs += 4 * math.pi * kd * (4.0 / 3.0) * kd ** 3 * float(np.sum(np.abs(P) ** 2))
    return cext, cabs, cext - cabs


def _einc_backward(r, kd, khat, ehat):  # wave travelling along -khat
    return _orig_einc(r, kd, -np.asarray(khat, float), ehat)


def _j_sign(u):                         # wrong sign of the j2 Rhat Rhat term
    j0, j1, j2 = _orig_j(u)
    return j0, j1, -j2


def _grad_sign(kd, aeff, eps, khat, ehat, P, nu):   # dropped factor 2 on the adjoint term
    return _orig_grad(kd, aeff, eps, khat, ehat, P, 0.5 * nu)


def _sites_zyx(grid):                   # x and z swapped in the site positions
    r, c = _orig_sites(grid)
    return r[:, ::-1].copy(), c


def _scat_sign(r_src, P, r_pts, kd, chunk=256):   # +A P instead of -A P
    return -_orig_scat(r_src, P, r_pts, kd, chunk)


def _scat_self(r_src, P, r_pts, kd, chunk=256):   # a self term at target points (here + P_j)
    out = _orig_scat(r_src, P, r_pts, kd, chunk)
    for j, rv in enumerate(r_pts):
        hit = np.nonzero(np.all(r_src == rv, axis=1))[0]
        if hit.size:
            out[j] += P[hit[0]]
    return out


def _box_floor(shape_zyx, ext):                    # floor instead of nearest for the added layers
    nz, ny, nx = shape_zyx
    lo = [int(math.floor(ext[0] * nx)), int(math.floor(ext[2] * ny)), int(math.floor(ext[4] * nz))]
    hi = [int(math.floor(ext[1] * nx)), int(math.floor(ext[3] * ny)), int(math.floor(ext[5] * nz))]
    return (nx + lo[0] + hi[0], ny + lo[1] + hi[1], nz + lo[2] + hi[2]), tuple(lo)


def _ff_phase(r, P, kd, n, chunk=64):             # exp(+ik n.r): the far field of the wrong hemisphere
    return _orig_ff(r, P, kd, -n, chunk)


def _ff_no_projection(r, P, kd, n, chunk=64):     # I instead of (I - n n)
    P = np.asarray(P, dtype=np.complex128)
    return kd * kd * (np.exp(-1j * kd * (n @ r.T)) @ P)


def _dirs_uniform_weights(x, eta):                # equal weights on the forward-dense directions
    t, ph, w = _orig_dirs(x, eta)
    return t, ph, np.full_like(w, 4 * math.pi / w.size)


def _mueller_s34_sign(S):                          # S34 = Im(S1 S2^* + ...) instead of Im(S2 S1^* + ...)
    M = _orig_mueller(S)
    M[:, 2, 3] = -M[:, 2, 3]
    return M


def _frame_e3_sign(theta, phi, beta):             # left-handed third axis
    e1, e2, e3 = _orig_frame(theta, phi, beta)
    return e1, e2, -e3


def _xs_tensor_unconjugated(kd, E, P, beta):      # Im(P . beta P^*) instead of Im(P . beta^* P^*)
    b = np.asarray(beta)
    return _orig_xs(kd, E, P, np.conj(b) if b.ndim == 3 else b)


MUTATIONS = [
    ("interaction_tensor", _tensor_sign, [pins.two_dipole_error]),
    ("interaction_tensor", _tensor_no_far, [pins.two_dipole_error]),
    ("interaction_tensor", _tensor_incoming, [pins.two_dipole_error, pins.energy_balance_error]),
    ("ldr_inverse_polarizability", _ldr_no_rr, [pins.lossless_cabs]),
    ("cross_sections", _xs_no_conj, [pins.energy_balance_error, pins.forward_amplitude_error]),
    ("cross_sections", _xs_rr_sign, [pins.single_dipole_errors, pins.lossless_cabs]),
    ("incident_field", _einc_backward, [pins.forward_amplitude_error]),
    ("_sph_j012", _j_sign, [pins.pair_sum_vs_quadrature_error]),
    ("qabs_gradient", _grad_sign, [pins.adjoint_gradient_error]),
    ("site_positions", _sites_zyx, [pins.site_axes_error]),
    ("scattered_field", _scat_sign, [pins.nearfield_self_consistency_error, pins.nearfield_single_dipole_error]),
    ("scattered_field", _scat_self, [pins.nearfield_self_consistency_error]),
    ("nearfield_box", _box_floor, [pins.nearfield_box_error]),
    ("far_field", _ff_phase, [pins.dda_asymmetry_vs_mie_error]),
    ("far_field", _ff_no_projection, [pins.farfield_single_dipole_error]),
    ("scattering_directions", _dirs_uniform_weights, [pins.farfield_single_dipole_error]),
    ("mueller_matrix", _mueller_s34_sign, [pins.mueller_sphere_vs_mie_error]),
    ("dielectric_frame", _frame_e3_sign, [pins.dielectric_frame_error]),
    ("cross_sections", _xs_tensor_unconjugated, [pins.anisotropic_energy_balance_error]),
    ("bicgstab_l", _mutant(dda.bicgstab_l, "r[0] = r[0] - gp[ell] * r[ell]", "r[0] = r[0] + gp[ell] * r[ell]"),
     [pins.bicgstab_l2_mr_error]),
    ("bicgstab_l", _mutant(dda.bicgstab_l, "tau[i, j] = np.vdot(r[i], r[j]) / sigma[i]",
                           "tau[i, j] = np.dot(r[i], r[j]) / sigma[i]"), [pins.bicgstab_l2_mr_error]),
    ("bicgstab_l", _mutant(dda.bicgstab_l, "beta = alpha * rho1 / rho0", "beta = alpha * rho1 / abs(rho0)"),
     [pins.bicgstab_l1_vs_bicgstab_error, pins.bicgstab_l2_mr_error]),
    ("bicgstab_l", _mutant(dda.bicgstab_l, "x = x + gpp[j] * r[j]", "x = x - gpp[j] * r[j]"),
     [pins.bicgstab_l2_mr_error]),
    ("ldr_inverse_polarizability", _mutant(dda.ldr_inverse_polarizability, "(LDR_B1 + LDR_B2", "(-LDR_B1 + LDR_B2"),
     [pins.ldr_dispersion_error]),
    ("ldr_inverse_polarizability", _mutant(dda.ldr_inverse_polarizability, "+ LDR_B2 * eps +", "- LDR_B2 * eps +"),
     [pins.ldr_dispersion_error]),
    ("ldr_inverse_polarizability", _mutant(dda.ldr_inverse_polarizability, "LDR_B2 * eps +", "LDR_B2 +"),
     [pins.ldr_dispersion_error]),
    ("ldr_inverse_polarizability", _mutant(dda.ldr_inverse_polarizability, "+ LDR_B3 * eps * S)", "- LDR_B3 * eps * S)"),
     [pins.ldr_dispersion_error]),
    ("ldr_inverse_polarizability", _mutant(dda.ldr_inverse_polarizability, "LDR_B3 * eps * S)", "LDR_B3 * eps)"),
     [pins.ldr_dispersion_error]),
    ("ldr_inverse_polarizability", _mutant(dda.ldr_inverse_polarizability, "LDR_B3 * eps * S)", "LDR_B3 * S)"),
     [pins.ldr_dispersion_error]),
    ("ldr_inverse_polarizability", _mutant(dda.ldr_inverse_polarizability, "S = np.sum(khat ** 2 * np.abs(ehat) ** 2)",
                                           "S = np.sum((khat * ehat) ** 2)"), [pins.ldr_dispersion_error]),
    ("ldr_inverse_polarizability", _mutant(dda.ldr_inverse_polarizability, "S = np.sum(khat ** 2 * np.abs(ehat) ** 2)",
                                           "S = np.sum((khat * np.conj(ehat)) ** 2)"), [pins.ldr_dispersion_error]),
    ("ldr_inverse_polarizability", _mutant(dda.ldr_inverse_polarizability, "S = np.sum(khat ** 2 * np.abs(ehat) ** 2)",
                                           "S = np.sum(np.abs(khat * ehat))"), [pins.ldr_dispersion_error]),
    ("ldr_inverse_polarizability", _mutant(dda.ldr_inverse_polarizability, "* kd ** 2 -", "* kd ** 3 -"),
     [pins.ldr_dispersion_error]),
    ("ldr_inverse_polarizability", _mutant(dda.ldr_inverse_polarizability, "(eps + 2.0) / (eps - 1.0)",
                                           "(eps + 2.0) / (eps + 1.0)"), [pins.ldr_dispersion_error]),
    ("qmr_sym", _mutant(dda.qmr_sym, "alpha = (v @ w) / delta", "alpha = np.vdot(v, w) / delta"),
     [pins.qmr_complex_symmetric_error]),
    ("qmr_sym", _mutant(dda.qmr_sym, "gamma = beta_next * delta / delta_prev", "gamma = beta_next"),
     [pins.qmr_complex_symmetric_error]),
    ("qmr_sym", _mutant(dda.qmr_sym, "tau = -np.conj(s1) * h1 + c1 * alpha", "tau = -s1 * h1 + c1 * alpha"),
     [pins.qmr_complex_symmetric_error]),
    ("qmr_sym", _mutant(dda.qmr_sym, "eps = s2 * gamma", "eps = 0.0 * gamma"),
     [pins.qmr_minres_error, pins.qmr_complex_symmetric_error]),
]


@pytest.mark.parametrize("name,fn,checks", MUTATIONS, ids=[f"{m[0]}:{m[1].__name__}" for m in MUTATIONS])
def test_planted_mistake_is_caught(monkeypatch, name, fn, checks):
    monkeypatch.setattr(dda, name, fn)
    worst = max(check() for check in checks)
    assert worst > 1e-6, f"mutation {fn.__name__} of {name} not caught (error {worst})"


@pytest.mark.parametrize("name,delta", [("LDR_B1", 1e-4), ("LDR_B2", -1e-4), ("LDR_B3", 1e-4)])
def test_ldr_constant_drift_is_caught(monkeypatch, name, delta):
    """A constant off in its fifth significant digit no longer matches the
    coefficients that the lattice sum gives."""
    monkeypatch.setattr(dda, name, getattr(dda, name) + delta)
    b = pins.ldr_coefficients_from_lattice()
    assert np.abs(b - [dda.LDR_B1, dda.LDR_B2, dda.LDR_B3]).max() > 5e-5


def test_mie_planted_mistake_is_caught(monkeypatch, golden_dir):
    """A wrong refractive index reaching the coefficients fails the textbook example."""
    src = mie.mie_efficiencies

    def wrong(x, m):
        return src(x, complex(m).conjugate() * 1.1)

    monkeypatch.setattr(mie, "mie_efficiencies", wrong)
    with pytest.raises(AssertionError):
        pins.test_mie_textbook_example(golden_dir)
