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
large-sphere extinction limit Q_ext -> 2.
"""
from __future__ import annotations

import math

import numpy as np


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
