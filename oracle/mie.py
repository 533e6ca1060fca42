"""Mie-series efficiencies of a homogeneous sphere -- test infrastructure.

The guide validates DDSCAT against "exact values ... obtained with Mie
theory" (Fig. 1, "Applicability of the DDA").  This is an independent
implementation of the standard Lorenz-Mie coefficients (Bohren & Huffman
1983, ch. 4): the logarithmic derivative D_n(mx) by downward recurrence,
Riccati-Bessel functions psi_n, chi_n by upward recurrence, and

  a_n = [(D_n/m + n/x) psi_n - psi_{n-1}] / [(D_n/m + n/x) xi_n - xi_{n-1}]
  b_n = [(m D_n + n/x) psi_n - psi_{n-1}] / [(m D_n + n/x) xi_n - xi_{n-1}]
  Q_ext = (2/x^2) sum (2n+1) Re(a_n + b_n)
  Q_sca = (2/x^2) sum (2n+1) (|a_n|^2 + |b_n|^2)

Pinned by the Rayleigh limit, the lossless identity Q_ext = Q_sca, and the
large-sphere extinction limit Q_ext -> 2; the amplitude functions S1, S2 and
the asymmetry g by the optical theorem Q_ext = (4/x^2) Re S(0) and by
angular quadrature of the phase function.
"""
from __future__ import annotations

import math

import numpy as np


def mie_coefficients(x: float, m: complex):
    """(a_n, b_n), n = 1..nstop, by the recurrences described above."""
    m = complex(m)
    nstop = int(x + 4.0 * x ** (1.0 / 3.0) + 2.0)
    nmx = int(max(nstop, abs(m * x))) + 16
    mx = m * x
    D = np.zeros(nmx + 1, dtype=np.complex128)
    for n in range(nmx, 0, -1):
        D[n - 1] = n / mx - 1.0 / (D[n] + n / mx)
    psi_m1, psi_0 = math.cos(x), math.sin(x)
    chi_m1, chi_0 = -math.sin(x), math.cos(x)
    xi_prev = complex(psi_0, -chi_0)
    a = np.zeros(nstop, dtype=np.complex128)
    b = np.zeros(nstop, dtype=np.complex128)
    for n in range(1, nstop + 1):
        psi = (2 * n - 1) / x * psi_0 - psi_m1
        chi = (2 * n - 1) / x * chi_0 - chi_m1
        xi = complex(psi, -chi)
        ta = D[n] / m + n / x
        tb = m * D[n] + n / x
        a[n - 1] = (ta * psi - psi_0) / (ta * xi - xi_prev)
        b[n - 1] = (tb * psi - psi_0) / (tb * xi - xi_prev)
        psi_m1, psi_0 = psi_0, psi
        chi_m1, chi_0 = chi_0, chi
        xi_prev = xi
    return a, b


def mie_asymmetry(x: float, m: complex) -> float:
    """g = <cos theta> from the coefficients (Bohren & Huffman eq. 4.62):
    Q_sca g = (4/x^2) [sum n(n+2)/(n+1) Re(a_n a_{n+1}^* + b_n b_{n+1}^*)
                       + sum (2n+1)/(n(n+1)) Re(a_n b_n^*)]."""
    a, b = mie_coefficients(x, m)
    n = np.arange(1, a.size + 1, dtype=np.float64)
    qsca = 2.0 / x ** 2 * np.sum((2 * n + 1) * (np.abs(a) ** 2 + np.abs(b) ** 2))
    t1 = np.sum((n[:-1] * (n[:-1] + 2) / (n[:-1] + 1)) * (a[:-1] * np.conj(a[1:]) + b[:-1] * np.conj(b[1:])).real)
    t2 = np.sum(((2 * n + 1) / (n * (n + 1))) * (a * np.conj(b)).real)
    return float(4.0 / x ** 2 * (t1 + t2) / qsca)


def mie_amplitudes(x: float, m: complex, theta: np.ndarray):
    """Scattering amplitudes S1(theta), S2(theta) (Bohren & Huffman eq. 4.74)
    from the angular functions pi_n, tau_n by their upward recurrences."""
    a, b = mie_coefficients(x, m)
    mu = np.cos(np.asarray(theta, dtype=np.float64))
    S1 = np.zeros(mu.shape, dtype=np.complex128)
    S2 = np.zeros(mu.shape, dtype=np.complex128)
    pi_m1 = np.zeros_like(mu)
    pi_0 = np.ones_like(mu)
    for n in range(1, a.size + 1):
        tau = n * mu * pi_0 - (n + 1) * pi_m1
        f = (2 * n + 1) / (n * (n + 1))
        S1 += f * (a[n - 1] * pi_0 + b[n - 1] * tau)
        S2 += f * (a[n - 1] * tau + b[n - 1] * pi_0)
        pi_m1, pi_0 = pi_0, ((2 * n + 1) * mu * pi_0 - (n + 1) * pi_m1) / n
    return S1, S2


def mie_efficiencies(x: float, m: complex):
    """Return (Q_ext, Q_abs, Q_sca) for size parameter x and relative index m."""
    m = complex(m)
    nstop = int(x + 4.0 * x ** (1.0 / 3.0) + 2.0)
    nmx = int(max(nstop, abs(m * x))) + 16
    mx = m * x
    D = np.zeros(nmx + 1, dtype=np.complex128)
    for n in range(nmx, 0, -1):
        D[n - 1] = n / mx - 1.0 / (D[n] + n / mx)
    psi_m1, psi_0 = math.cos(x), math.sin(x)
    chi_m1, chi_0 = -math.sin(x), math.cos(x)
    xi_prev = complex(psi_0, -chi_0)
    qext = 0.0
    qsca = 0.0
    for n in range(1, nstop + 1):
        psi = (2 * n - 1) / x * psi_0 - psi_m1
        chi = (2 * n - 1) / x * chi_0 - chi_m1
        xi = complex(psi, -chi)
        ta = D[n] / m + n / x
        tb = m * D[n] + n / x
        an = (ta * psi - psi_0) / (ta * xi - xi_prev)
        bn = (tb * psi - psi_0) / (tb * xi - xi_prev)
        qext += (2 * n + 1) * (an + bn).real
        qsca += (2 * n + 1) * (abs(an) ** 2 + abs(bn) ** 2)
        psi_m1, psi_0 = psi_0, psi
        chi_m1, chi_0 = chi_0, chi
        xi_prev = xi
    qext *= 2.0 / x ** 2
    qsca *= 2.0 / x ** 2
    return qext, qext - qsca, qsca
