"""Dipole lattice sums -- TEST INFRASTRUCTURE (see the package docstring).

The guide's LATTDR option ("Dipole Polarizabilities") takes its
polarizability from the lattice dispersion relation of Draine & Goodman
(1993).  Its defining property is a statement about an infinite cubic lattice
of identical polarizable points, not a formula: the lattice must carry a
transverse plane wave P_l = e exp(i q . r_l), with the wavevector q = m k khat
of the continuum of refractive index m, with no incident field.  The DDA
equations of such a lattice reduce to one condition at the origin,

    (1/alpha) e = T(q) e,    T(q) = sum_{l != 0} G(r_l) exp(i q . r_l),

where G(r) = (k^2 I + grad grad) exp(ikr)/r is the field of a unit dipole
(G = -A_jl off the diagonal of the DDA matrix).  LATTDR is the expansion of
that condition to second order in kd.  This module evaluates T(q) itself, so
that the oracle's closed form of 1/alpha can be checked against it.

T(q) does not converge as written (its terms fall as 1/r), so it is evaluated
by Ewald's method: the scalar Green function is split in Fourier space by the
Gaussian factor exp(-(p^2 - k^2)/(4 eta^2)) into a short-range part, summed
over lattice sites, and a smooth long-range part, summed over reciprocal
lattice vectors by Poisson's formula; the smooth part's value at the origin is
subtracted because the site l = 0 is excluded.  The result does not depend on
eta, which the pins check, and for a damped wavenumber (Im k > 0) it equals
the plain site sum, which converges absolutely there.  All sums are analytic
in k and q, so complex k, q and m are allowed.

Units: lattice units (d = 1), Gaussian units, as in oracle.dda.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erfc


def _integer_points(n: int) -> np.ndarray:
    """All integer 3-vectors with components in [-n, n], shape (P, 3) float."""
    g = np.arange(-n, n + 1, dtype=np.float64)
    return np.stack(np.meshgrid(g, g, g, indexing="ij"), axis=-1).reshape(-1, 3)


def short_range_radial(r, kd, eta: float):
    """phi_s(r) and its first two radial derivatives.

    phi_s = [exp(ikr) erfc(eta r + a) + exp(-ikr) erfc(eta r - a)] / (2r),
    a = ik/(2 eta): the part of exp(ikr)/r whose Fourier transform is
    4pi [1 - exp(-(p^2 - k^2)/(4 eta^2))] / (p^2 - k^2).  With
    F = 2 r phi_s and H = exp(ikr) erfc(eta r + a) - exp(-ikr) erfc(eta r - a):
    F' = ik H - (4 eta/sqrt(pi)) g,  H' = ik F,
    F'' = -k^2 F + (8 eta^3 r/sqrt(pi)) g,   g = exp(-eta^2 r^2 - a^2)
    (the Gaussian of erfc's derivative times the plane-wave factor; the ikr
    phases cancel in it).
    """
    r = np.asarray(r, dtype=np.float64)
    a = 1j * kd / (2.0 * eta)
    up, dn = np.exp(1j * kd * r) * erfc(eta * r + a), np.exp(-1j * kd * r) * erfc(eta * r - a)
    F, H = up + dn, up - dn
    g = np.exp(-(eta * r) ** 2 - a * a)
    F1 = 1j * kd * H - (4.0 * eta / math.sqrt(math.pi)) * g
    F2 = -kd * kd * F + (8.0 * eta ** 3 * r / math.sqrt(math.pi)) * g
    phi = F / (2.0 * r)
    d1 = F1 / (2.0 * r) - F / (2.0 * r * r)
    d2 = F2 / (2.0 * r) - F1 / (r * r) + F / r ** 3
    return phi, d1, d2


def long_range_origin(kd, eta: float):
    """c0 = phi_L(0) and the tensor [(k^2 + grad grad) phi_L](0) / I.

    phi_L = exp(ikr)/r - phi_s is smooth at the origin.  c0 follows from the
    O(r^0) terms of the two expansions: c0 = ik erfc(-a) + (2 eta/sqrt(pi))
    exp(k^2/(4 eta^2)).  phi_L is radial, phi_L = c0 + c2 r^2 + ..., so
    grad grad phi_L(0) = 2 c2 I, and (lap + k^2) phi_L = -4pi rho_eta with the
    Gaussian rho_eta(0) = exp(k^2/(4 eta^2)) eta^3 / pi^(3/2) fixes
    6 c2 + k^2 c0.  Returns (c0, k^2 c0 + 2 c2).
    """
    a = 1j * kd / (2.0 * eta)
    gk = np.exp(kd * kd / (4.0 * eta * eta))
    c0 = 1j * kd * erfc(-a) + (2.0 * eta / math.sqrt(math.pi)) * gk
    c2 = (-4.0 * eta ** 3 * gk / math.sqrt(math.pi) - kd * kd * c0) / 6.0
    return c0, kd * kd * c0 + 2.0 * c2


def dipole_lattice_sum(kd, q, eta: float = 1.2, n_real: int = 6, n_recip: int = 6) -> np.ndarray:
    """T(q) = sum_{l != 0} G(r_l) exp(i q . r_l) on the unit cubic lattice, (3, 3) complex.

    Ewald split (module docstring):
      sites       sum_{l != 0} [(k^2 + grad grad) phi_s](r_l) exp(i q . r_l),
                  with grad grad f(r) = f'' rr + (f'/r)(I - rr) for radial f;
      reciprocal  sum_G 4pi (k^2 I - p p) exp((k^2 - p.p)/(4 eta^2)) / (p.p - k^2),
                  p = q + G, G = 2 pi n (unit cell volume 1; p.p unconjugated);
      origin      minus [(k^2 + grad grad) phi_L](0) = (k^2 c0 + 2 c2) I.
    n_real and n_recip bound the two sums (|n_a| <= n); the defaults give
    about 1e-13 relative at |k|, |q| < 1 with eta = 1.2.
    """
    q = np.asarray(q, dtype=np.complex128)
    eye = np.eye(3)
    L = _integer_points(n_real)
    L = L[np.any(L != 0.0, axis=1)]
    r = np.linalg.norm(L, axis=1)
    rh = L / r[:, None]
    rr = rh[:, :, None] * rh[:, None, :]
    phi, d1, d2 = short_range_radial(r, kd, eta)
    Gs = (kd * kd * phi)[:, None, None] * eye + d2[:, None, None] * rr + (d1 / r)[:, None, None] * (eye - rr)
    T = np.einsum("l,lab->ab", np.exp(1j * (L @ q)), Gs)

    p = 2.0 * math.pi * _integer_points(n_recip) + q
    pp = np.sum(p * p, axis=1)
    w = 4.0 * math.pi * np.exp((kd * kd - pp) / (4.0 * eta * eta)) / (pp - kd * kd)
    T = T + np.einsum("l,lab->ab", w, kd * kd * eye[None] - p[:, :, None] * p[:, None, :])

    _, origin = long_range_origin(kd, eta)
    return T - origin * eye


def lattice_mode_inverse_polarizability(eps, kd: float, khat, ehat, **kw) -> complex:
    """The 1/alpha that lets the lattice carry the mode e exp(i m k khat . r):
    e^* . T(m k khat) . e for a unit e (the Rayleigh quotient of T; exact where
    e is an eigenvector of T, as for every transverse e when khat lies on a
    3- or 4-fold axis of the cube).  m = sqrt(eps) with Im m >= 0."""
    khat = np.asarray(khat, dtype=np.float64)
    ehat = np.asarray(ehat, dtype=np.complex128)
    m = np.sqrt(complex(eps))
    T = dipole_lattice_sum(kd, m * kd * khat, **kw)
    return complex(np.conj(ehat) @ T @ ehat)
