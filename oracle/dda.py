"""FP64 numpy statement of the discrete dipole approximation (DDA).

Test infrastructure (see the package docstring).  Units: lattice units,
dipole spacing d = 1, incident amplitude |E0| = 1, Gaussian units, so
"kd" below is the dimensionless k*d.

The guide states the linear system A P = E ("Choice of Iterative
Algorithm", eq. AP=E) and names the formulae it uses (Draine 1988 for the
DDA equations and cross sections; Draine & Goodman 1993 for the LATTDR
polarizability; Goodman, Draine & Flatau 1990 for the FFT method) without
printing them.  The forms below are the published ones; each docstring says
which reading is taken and what pins it.
"""
from __future__ import annotations

import math

import numpy as np

# LATTDR coefficients of the lattice dispersion relation (Draine & Goodman
# 1993), cited by the guide in "Dipole Polarizabilities".  The guide does not
# print them.  Pinned by the relation's defining property: the second-order
# coefficient of the lattice sum of oracle.lattice, extrapolated to kd -> 0
# over several refractive indices and directions, is b1 + b2 eps + b3 eps S
# with these values to 1e-6.
LDR_B1 = -1.8915316
LDR_B2 = 0.1648469
LDR_B3 = -1.7700004


# ---------------------------------------------------------------- geometry --
def site_positions(grid: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """Occupied sites of a composition grid [nz, ny, nx] (x fastest).

    Returns (r, comp): r (N, 3) float64 dipole positions in lattice units,
    r = (ix-(nx-1)/2, iy-(ny-1)/2, iz-(nz-1)/2), ordered with x fastest, then
    y, then z (the order of a row-major scan of the grid); comp (N,) the
    composition code (1..ncomp) of each site.  Target Frame origin at the
    centre of the computational volume (ELLIPSOID section: origin at the
    centroid).
    """
    nz, ny, nx = grid.shape
    iz, iy, ix = np.nonzero(grid)           # row-major order == x fastest
    r = np.stack([ix - (nx - 1) / 2.0, iy - (ny - 1) / 2.0, iz - (nz - 1) / 2.0], axis=1)
    return r.astype(np.float64), grid[iz, iy, ix].astype(np.int64)


def aeff_lattice(ndipoles: int) -> float:
    """a_eff = (3V/4pi)^(1/3) with V = N d^3 (eq. for a_eff, "Applicability
    of the DDA"), in units of d."""
    return (3.0 * ndipoles / (4.0 * math.pi)) ** (1.0 / 3.0)


def kd_from_size_parameter(x: float, ndipoles: int) -> float:
    """k d from x = k a_eff (size-parameter equation)."""
    return x / aeff_lattice(ndipoles)


# ---------------------------------------------------------- polarizability --
def ldr_inverse_polarizability(eps, kd: float, khat, ehat) -> np.ndarray:
    """1/alpha for the LATTDR prescription (Draine & Goodman 1993).

    alpha_CM = (3/4pi) (eps-1)/(eps+2)          (Clausius-Mossotti, d = 1)
    1/alpha  = 1/alpha_CM + (b1 + b2 eps + b3 eps S) (kd)^2 - (2/3) i (kd)^3
    S        = sum_a khat_a^2 |ehat_a|^2         (ehat a unit vector)

    eps may be an array (one value per composition or per dipole).  Pinned by
    the defining property of the lattice dispersion relation: this 1/alpha
    equals e^* T(m k khat) e, the lattice sum of oracle.lattice, up to
    O((kd)^4), for every direction and polarization, real and complex.  For a
    real ehat, S = sum_a (khat_a ehat_a)^2, Draine & Goodman's form; for a
    complex one the lattice sum decides between the candidate extensions: on
    a 3-fold axis of the cube every transverse ehat (circular too) is a mode
    of the lattice with one eigenvalue, which the |ehat_a|^2 form reproduces
    and the unconjugated square (zero for circular ehat there) does not.  The
    -(2/3) i k^3 term is the radiative-reaction correction, also pinned by
    the N = 1 closed forms and the lossless invariant.
    """
    eps = np.asarray(eps, dtype=np.complex128)
    khat = np.asarray(khat, dtype=np.float64)
    ehat = np.asarray(ehat, dtype=np.complex128)
    S = np.sum(khat ** 2 * np.abs(ehat) ** 2)
    inv_acm = (4.0 * math.pi / 3.0) * (eps + 2.0) / (eps - 1.0)
    return inv_acm + (LDR_B1 + LDR_B2 * eps + LDR_B3 * eps * S) * kd ** 2 - (2.0 / 3.0) * 1j * kd ** 3


def dielectric_frame(theta: float, phi: float, beta: float):
    """Principal axes e1, e2, e3 of an anisotropic material in the Target
    Frame ("Composite Targets with Anisotropic Constituents"), from the
    rotation angles theta_DF, phi_DF, beta_DF, as the guide writes them:
      e1 =  x cos(th) + y sin(th) cos(ph) + z sin(th) sin(ph)
      e2 = -x sin(th) cos(be) + y [cos(th) cos(be) cos(ph) - sin(be) sin(ph)]
                              + z [cos(th) cos(be) sin(ph) + sin(be) cos(ph)]
      e3 =  x sin(th) sin(be) - y [cos(th) sin(be) cos(ph) + cos(be) sin(ph)]
                              - z [cos(th) sin(be) sin(ph) - cos(be) cos(ph)]"""
    ct, st, cp, sp, cb, sb = (math.cos(theta), math.sin(theta), math.cos(phi), math.sin(phi),
                              math.cos(beta), math.sin(beta))
    e1 = np.array([ct, st * cp, st * sp])
    e2 = np.array([-st * cb, ct * cb * cp - sb * sp, ct * cb * sp + sb * cp])
    e3 = np.array([st * sb, -(ct * sb * cp + cb * sp), -(ct * sb * sp - cb * cp)])
    return e1, e2, e3


def ldr_inverse_tensor(eps3, angles, kd: float, khat, ehat) -> np.ndarray:
    """1/alpha tensor (3, 3) of an anisotropic dipole: the LATTDR value of each
    principal dielectric constant eps3[j] (same S for all three), along the
    dielectric axes e_j: sum_j (1/alpha_j) e_j e_j^T (the guide's
    alpha^TF = R alpha^DF R^-1; the inverse has the same axes)."""
    ev = dielectric_frame(*angles)
    b = ldr_inverse_polarizability(np.asarray(eps3, dtype=np.complex128), kd, khat, ehat)
    return sum(b[j] * np.outer(ev[j], ev[j]) for j in range(3))


def ldr_inverse_polarizability_derivative(eps, kd: float, khat, ehat) -> np.ndarray:
    """d(1/alpha)/d(eps) of the LATTDR form above: -4pi/(eps-1)^2 + (b2 + b3 S) k^2."""
    eps = np.asarray(eps, dtype=np.complex128)
    S = np.sum(np.asarray(khat, float) ** 2 * np.abs(np.asarray(ehat, complex)) ** 2)
    return -4.0 * math.pi / (eps - 1.0) ** 2 + (LDR_B2 + LDR_B3 * S) * kd ** 2


# ------------------------------------------------------ interaction matrix --
def interaction_tensor(rvec, kd: float) -> np.ndarray:
    """Off-diagonal 3x3 block A_jl for displacement r = r_j - r_l != 0.

    A_jl = exp(ik rho)/rho [ k^2 (rr - I) + (ik rho - 1)/rho^2 (3 rr - I) ],
    rr = rhat rhat^T, rho = |r|, so that the field at j from dipole l is
    -A_jl P_l and the DDA equations read A P = E with A_jj = (1/alpha_j) I
    (Draine 1988, the form the guide cites under eq. AP=E).  Pinned by the
    two-dipole test against the textbook dipole field.  Vectorised over
    leading axes of rvec (..., 3).
    """
    rvec = np.asarray(rvec, dtype=np.float64)
    rho = np.linalg.norm(rvec, axis=-1)
    rh = rvec / rho[..., None]
    rr = rh[..., :, None] * rh[..., None, :]
    eye = np.eye(3)
    ph = np.exp(1j * kd * rho) / rho
    t1 = (kd * kd)[..., None, None] if np.ndim(kd) else kd * kd
    c2 = (1j * kd * rho - 1.0) / rho ** 2
    return ph[..., None, None] * (t1 * (rr - eye) + c2[..., None, None] * (3.0 * rr - eye))


def _diag_block(beta, j):
    """Diagonal block of dipole j: beta (N,) isotropic 1/alpha, or (N, 3, 3) tensors."""
    b = np.asarray(beta)
    return b[j] * np.eye(3) if b.ndim == 1 else b[j]


def dense_matrix(r: np.ndarray, kd: float, beta: np.ndarray) -> np.ndarray:
    """The full 3N x 3N matrix A, row/column index 3*j + a.

    beta (N,) holds 1/alpha_j for each dipole (isotropic diagonal blocks), or
    (N, 3, 3) the symmetric 1/alpha tensors of anisotropic dipoles.
    """
    n = r.shape[0]
    A = np.zeros((n, 3, n, 3), dtype=np.complex128)
    for j in range(n):
        d = r[j] - r
        d[j] = (1.0, 0.0, 0.0)                # placeholder, overwritten below
        blk = interaction_tensor(d, kd)       # (n, 3, 3)
        blk[j] = _diag_block(beta, j)
        A[j] = np.transpose(blk, (1, 0, 2))
    return A.reshape(3 * n, 3 * n)


def pairwise_matvec(r: np.ndarray, kd: float, beta: np.ndarray, P: np.ndarray,
                    rows: np.ndarray | None = None, chunk: int = 256) -> np.ndarray:
    """(A P)_j = beta_j P_j + sum_{l != j} A(r_j - r_l) P_l, the plain O(N^2) sum.

    P (N, 3) complex.  If ``rows`` is given only those output rows are formed
    (row sampling for large targets).  Returns (len(rows) or N, 3).
    """
    P = np.asarray(P, dtype=np.complex128)
    rows = np.arange(r.shape[0]) if rows is None else np.asarray(rows)
    out = np.empty((rows.size, 3), dtype=np.complex128)
    for s in range(0, rows.size, chunk):
        jj = rows[s:s + chunk]
        d = r[jj][:, None, :] - r[None, :, :]            # (c, N, 3)
        self_mask = np.zeros(d.shape[:2], dtype=bool)
        self_mask[np.arange(jj.size), jj] = True
        d[self_mask] = (1.0, 0.0, 0.0)
        blk = interaction_tensor(d, kd)                   # (c, N, 3, 3)
        blk[self_mask] = 0.0
        b = np.asarray(beta)
        diag = b[jj][:, None] * P[jj] if b.ndim == 1 else np.einsum("cab,cb->ca", b[jj], P[jj])
        out[s:s + chunk] = np.einsum("clab,lb->ca", blk, P) + diag
    return out


# ----------------------------------------------------------- incident field --
def incident_field(r: np.ndarray, kd: float, khat, ehat) -> np.ndarray:
    """E_inc,j = ehat exp(i kd khat . r_j)  (N, 3); phase origin at the lattice centre."""
    ph = np.exp(1j * kd * (r @ np.asarray(khat, dtype=np.float64)))
    return ph[:, None] * np.asarray(ehat, dtype=np.complex128)[None, :]


# ------------------------------------------------------------------ solvers --
def solve_dense(A: np.ndarray, E: np.ndarray) -> np.ndarray:
    """Direct solve of A P = E (LAPACK LU via numpy); E, P as (N, 3)."""
    return np.linalg.solve(A, E.reshape(-1)).reshape(-1, 3)


def bicgstab(matvec, b: np.ndarray, tol: float, maxit: int, x0=None):
    """Unpreconditioned BiCGstab (van der Vorst 1992) for complex A x = b.

    The guide's recommended solvers are BiCGstab variants (PBCGS2, PBCGST,
    "Choice of Iterative Algorithm").  Stops when ||b - A x|| <= tol ||b||
    (recurrence residual; the caller re-checks the true residual).  Vectors
    are flat complex arrays.  Returns (x, iterations, matvecs, relres).
    """
    b = np.asarray(b, dtype=np.complex128).ravel()
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.complex128).ravel()
    r = b - matvec(x) if x0 is not None else b.copy()
    nmv = 1 if x0 is not None else 0
    bnorm = np.linalg.norm(b)
    if bnorm == 0.0:
        return x, 0, nmv, 0.0
    rhat = r.copy()
    rho_old = alpha = omega = 1.0 + 0j
    v = np.zeros_like(b)
    p = np.zeros_like(b)
    relres = np.linalg.norm(r) / bnorm
    it = 0
    while relres > tol and it < maxit:
        rho = np.vdot(rhat, r)
        beta = (rho / rho_old) * (alpha / omega)
        p = r + beta * (p - omega * v)
        v = matvec(p)
        alpha = rho / np.vdot(rhat, v)
        s = r - alpha * v
        t = matvec(s)
        nmv += 2
        omega = np.vdot(t, s) / np.vdot(t, t)
        x = x + alpha * p + omega * s
        r = s - omega * t
        rho_old = rho
        it += 1
        relres = np.linalg.norm(r) / bnorm
    return x, it, nmv, relres


def bicgstab_l(matvec, b: np.ndarray, tol: float, maxit: int, ell: int = 2, x0=None, trace=None):
    """BiCGstab(l) (Sleijpen & Fokkema 1993; the guide's PBCGS2 is Botchev's
    ZBCG2 implementation of it, "Choice of Iterative Algorithm") for complex
    A x = b, unpreconditioned, shadow residual rt = r0.

    One iteration is l BiCG steps (2l matvecs) followed by a minimal-residual
    polynomial step of degree l over the residuals r_1..r_l, orthogonalized by
    modified Gram-Schmidt.  Inner products are Hermitian, (a, c) = c^H a.
    Stops when the recurrence residual ||r_0|| <= tol ||b||.  With a list as
    `trace`, each iteration appends (r_0 after the MR step, the orthogonalized
    r_1..r_l).  Returns (x, iterations, matvecs, relres).
    """
    b = np.asarray(b, dtype=np.complex128).ravel()
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.complex128).ravel()
    r = [b - matvec(x) if x0 is not None else b.copy()] + [None] * ell
    nmv = 1 if x0 is not None else 0
    bnorm = np.linalg.norm(b)
    if bnorm == 0.0:
        return x, 0, nmv, 0.0
    rt = r[0].copy()
    u = [np.zeros_like(b)] + [None] * ell
    rho0, alpha, omega = 1.0 + 0j, 0.0 + 0j, 1.0 + 0j
    relres = np.linalg.norm(r[0]) / bnorm
    it = 0
    while relres > tol and it < maxit:
        rho0 = -omega * rho0
        for j in range(ell):                       # BiCG part
            rho1 = np.vdot(rt, r[j])
            beta = alpha * rho1 / rho0
            rho0 = rho1
            for i in range(j + 1):
                u[i] = r[i] - beta * u[i]
            u[j + 1] = matvec(u[j])
            alpha = rho0 / np.vdot(rt, u[j + 1])
            for i in range(j + 1):
                r[i] = r[i] - alpha * u[i + 1]
            r[j + 1] = matvec(r[j])
            x = x + alpha * u[0]
            nmv += 2
        tau = np.zeros((ell + 1, ell + 1), dtype=np.complex128)   # MR part (modified Gram-Schmidt)
        sigma = np.zeros(ell + 1)
        gp = np.zeros(ell + 1, dtype=np.complex128)                # gamma'
        for j in range(1, ell + 1):
            for i in range(1, j):
                tau[i, j] = np.vdot(r[i], r[j]) / sigma[i]
                r[j] = r[j] - tau[i, j] * r[i]
            sigma[j] = np.vdot(r[j], r[j]).real
            gp[j] = np.vdot(r[j], r[0]) / sigma[j]
        g = np.zeros(ell + 1, dtype=np.complex128)                 # gamma
        g[ell] = gp[ell]
        omega = g[ell]
        for j in range(ell - 1, 0, -1):
            g[j] = gp[j] - sum(tau[j, i] * g[i] for i in range(j + 1, ell + 1))
        gpp = np.zeros(ell + 1, dtype=np.complex128)               # gamma''
        for j in range(1, ell):
            gpp[j] = g[j + 1] + sum(tau[j, i] * g[i + 1] for i in range(j + 1, ell))
        x = x + g[1] * r[0]
        r[0] = r[0] - gp[ell] * r[ell]
        u[0] = u[0] - g[ell] * u[ell]
        for j in range(1, ell):
            u[0] = u[0] - g[j] * u[j]
            x = x + gpp[j] * r[j]
            r[0] = r[0] - gp[j] * r[j]
        it += 1
        relres = np.linalg.norm(r[0]) / bnorm
        if trace is not None:
            trace.append([v.copy() for v in r])
    return x, it, nmv, relres


def qmr_sym(matvec, b: np.ndarray, tol: float, maxit: int, x0=None, trace=None):
    """Quasi-minimal residual method for complex symmetric A = A^T (Freund
    1992; the guide's QMRCCG option, "Choice of Iterative Algorithm"), one
    matvec per iteration, without look-ahead.

    Lanczos with the bilinear form v^T w (no conjugate): v_1 = r_0/|r_0|,
    delta_n = v_n^T v_n, alpha_n = v_n^T A v_n / delta_n,
    gamma_n = beta_n delta_n / delta_{n-1},
    v~_{n+1} = A v_n - alpha_n v_n - gamma_n v_{n-1}, beta_{n+1} = |v~_{n+1}|,
    so that A V_n = V_{n+1} H_n with H_n tridiagonal ((n+1) x n).  The iterate
    x_n = x_0 + V_n z_n minimizes |beta_1 e_1 - H_n z| (the quasi-residual),
    by complex Givens rotations of H_n updated one column at a time; the
    residual is updated alongside (r_n = r_{n-1} - t_n A p_n).  Stops when
    |r_n| <= tol |b|.  With a list as `trace`, each iteration appends
    (v_n, the quasi-residual |t~_{n+1}|).  Returns (x, iterations, matvecs, relres).
    """
    b = np.asarray(b, dtype=np.complex128).ravel()
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.complex128).ravel()
    r = b - matvec(x) if x0 is not None else b.copy()
    nmv = 1 if x0 is not None else 0
    bnorm = np.linalg.norm(b)
    if bnorm == 0.0:
        return x, 0, nmv, 0.0
    beta = np.linalg.norm(r)
    v_prev, v = np.zeros_like(b), r / beta
    delta_prev, delta = 1.0 + 0j, v @ v
    gamma = 0.0 + 0j
    p1, p2, ap1, ap2 = (np.zeros_like(b) for _ in range(4))   # p_{n-1}, p_{n-2}, A p_{n-1}, A p_{n-2}
    c1, s1, c2, s2 = 1.0, 0j, 1.0, 0j                          # rotations G_{n-1}, G_{n-2}
    tt = beta + 0j                                             # t~_n
    relres = beta / bnorm
    it = 0
    while relres > tol and it < maxit:
        w = matvec(v)
        nmv += 1
        alpha = (v @ w) / delta
        vt = w - alpha * v - gamma * v_prev
        beta_next = np.linalg.norm(vt)
        # new column of H: gamma (row n-1), alpha (row n), beta_next (row n+1)
        eps = s2 * gamma                                       # G_{n-2} on rows n-2, n-1
        h1 = c2 * gamma
        dlt = c1 * h1 + s1 * alpha                             # G_{n-1} on rows n-1, n
        tau = -np.conj(s1) * h1 + c1 * alpha
        if abs(tau) == 0.0:
            c, s = 0.0, 1.0 + 0j
        else:
            c = abs(tau) / np.hypot(abs(tau), beta_next)
            s = c * beta_next / np.conj(tau)
        rho = c * tau + s * beta_next
        t = c * tt                                             # x_n = x_{n-1} + t p_n
        tt = -np.conj(s) * tt
        p = (v - dlt * p1 - eps * p2) / rho
        ap = (w - dlt * ap1 - eps * ap2) / rho
        x = x + t * p
        r = r - t * ap
        p2, p1, ap2, ap1 = p1, p, ap1, ap
        c2, s2, c1, s1 = c1, s1, c, s
        it += 1
        relres = np.linalg.norm(r) / bnorm
        if trace is not None:
            trace.append((v.copy(), abs(tt)))
        if beta_next == 0.0:
            break
        v_prev, v = v, vt / beta_next
        delta_prev, delta = delta, v @ v
        gamma = beta_next * delta / delta_prev
    return x, it, nmv, relres


def normal_equation_error(matvec, P: np.ndarray, E: np.ndarray) -> float:
    """|A^H A P - A^H E| / |A^H E| (eq. err_tol).  Uses A^H x = conj(A conj(x)),
    valid because A = A^T."""
    P = np.asarray(P).ravel()
    E = np.asarray(E).ravel()
    ah = lambda v: np.conj(matvec(np.conj(v)))  # noqa: E731
    num = np.linalg.norm(ah(matvec(P)) - ah(E))
    return float(num / np.linalg.norm(ah(E)))


# ---------------------------------------------------------- cross sections --
def cross_sections(kd: float, E_inc: np.ndarray, P: np.ndarray, beta: np.ndarray):
    """(C_ext, C_abs, C_sca) in units of d^2 (Draine 1988 forms).

    C_ext = 4 pi k sum_j Im(E_inc,j^* . P_j)
    C_abs = 4 pi k sum_j [ Im(P_j . (1/alpha_j)^* P_j^*) - (2/3) k^3 |P_j|^2 ]
    C_sca = C_ext - C_abs  (the guide's printed output obeys Q_ext = Q_abs +
    Q_sca to all digits, App. "Sample output", and defines Q_ext that way in
    "What Does DDSCAT Calculate?").
    Pinned by the single-dipole closed forms and by the independent far-field
    C_sca of a converged solve.
    """
    k = kd
    cext = 4.0 * math.pi * k * float(np.sum(np.imag(np.conj(E_inc) * P)))
    p2 = np.sum(np.abs(P) ** 2, axis=1)
    b = np.asarray(beta)
    if b.ndim == 1:
        quad = np.imag(np.conj(b)) * p2
    else:  # Im(P . beta^* P^*) for the tensor blocks
        quad = np.imag(np.einsum("ja,jab,jb->j", P, np.conj(b), np.conj(P)))
    cabs = 4.0 * math.pi * k * float(np.sum(quad - (2.0 / 3.0) * k ** 3 * p2))
    return cext, cabs, cext - cabs


def efficiencies(C, aeff: float):
    """Q = C / (pi a_eff^2) ("What Does DDSCAT Calculate?")."""
    return tuple(c / (math.pi * aeff ** 2) for c in C)


def _sph_j012(u: np.ndarray):
    """Spherical Bessel j0, j1, j2.  For u < 1 the power series
    j_n(u) = u^n/(2n+1)!! sum_k (-u^2/2)^k / (k! (2n+3)(2n+5)...(2n+2k+1))
    (12 terms) avoids the cancellation of the closed forms."""
    u = np.asarray(u, dtype=np.float64)
    out = []
    small = u < 1.0
    us = u[small]
    ul = u[~small]
    s, c = np.sin(ul), np.cos(ul)
    closed = (s / ul, s / ul ** 2 - c / ul, (3 / ul ** 3 - 1 / ul) * s - 3 * c / ul ** 2)
    for n, dfact in ((0, 1.0), (1, 3.0), (2, 15.0)):
        j = np.empty_like(u)
        term = us ** n / dfact
        acc = term.copy()
        for k in range(1, 13):
            term = term * (-us * us / 2.0) / (k * (2 * n + 2 * k + 1))
            acc += term
        j[small] = acc
        j[~small] = closed[n]
        out.append(j)
    return tuple(out)


def csca_pair_sum(r: np.ndarray, kd: float, P: np.ndarray, chunk: int = 256) -> float:
    """Scattering cross section as an exact pair sum.

    dC_sca/dOmega = k^4 |sum_j (I - nn) P_j exp(-ik n.r_j)|^2; integrating
    over directions with  int (I - nn) exp(iu n.Rhat) dOmega
    = 4 pi [ (j0(u) - j1(u)/u) I + j2(u) Rhat Rhat ],  u = k|r_j - r_l|,
    gives C_sca = 4 pi k^4 sum_{j,l} P_j^* . [..] . P_l (self term 2/3 I).
    Pinned by ``csca_quadrature`` (direct angular integration).
    """
    k = kd
    P = np.asarray(P, dtype=np.complex128)
    n = r.shape[0]
    total = 0.0 + 0.0j
    for s in range(0, n, chunk):
        jj = np.arange(s, min(n, s + chunk))
        d = r[jj][:, None, :] - r[None, :, :]
        R = np.linalg.norm(d, axis=-1)
        u = k * R
        j0, j1, j2 = _sph_j012(u)
        with np.errstate(invalid="ignore", divide="ignore"):
            iso = np.where(u > 0, j0 - j1 / np.where(u > 0, u, 1.0), 2.0 / 3.0)
            Rh = d / np.where(R > 0, R, 1.0)[..., None]
        pl_dot = np.einsum("cla,la->cl", Rh, P)                  # Rhat . P_l
        pj_dot = np.einsum("cla,ca->cl", Rh, np.conj(P[jj]))     # P_j^* . Rhat
        pp = np.conj(P[jj]) @ P.T                                # P_j^* . P_l
        total += np.sum(iso * pp + j2 * pj_dot * pl_dot)
    return float(4.0 * math.pi * k ** 4 * total.real)


def csca_quadrature(r: np.ndarray, kd: float, P: np.ndarray, ntheta: int = 64, nphi: int = 128) -> float:
    """C_sca by direct angular quadrature of the far field: Gauss-Legendre in
    cos(theta) times the trapezoid rule in phi."""
    k = kd
    P = np.asarray(P, dtype=np.complex128)
    mu, w = np.polynomial.legendre.leggauss(ntheta)
    phi = np.arange(nphi) * (2 * math.pi / nphi)
    st = np.sqrt(1 - mu ** 2)
    n = np.stack([st[:, None] * np.cos(phi)[None, :], st[:, None] * np.sin(phi)[None, :],
                  np.broadcast_to(mu[:, None], (ntheta, nphi))], axis=-1).reshape(-1, 3)
    wt = np.repeat(w, nphi) * (2 * math.pi / nphi)
    total = 0.0
    for s in range(0, n.shape[0], 512):
        nn = n[s:s + 512]
        F = np.exp(-1j * k * (nn @ r.T)) @ P                    # (c, 3)
        F = F - nn * np.sum(nn * F, axis=1, keepdims=True)
        total += float(np.sum(wt[s:s + 512] * np.sum(np.abs(F) ** 2, axis=1)))
    return k ** 4 * total


# ----------------------------------------------------------------- adjoint --
def qabs_gradient(kd: float, aeff: float, eps_site: np.ndarray, khat, ehat,
                  P: np.ndarray, nu: np.ndarray):
    """dQ_abs/dRe(eps_j), dQ_abs/dIm(eps_j), treating each dipole's eps as
    independent (no counterpart in the guide; derived from the cross-section
    and polarizability forms above).

    With Q_abs = K sum_j w_j |P_j|^2, w_j = -Im beta_j - (2/3) k^3,
    K = 4 k / a_eff^2, beta' = d beta/d eps, and nu solving A nu = W P^*
    (A = A^T):
      dQ/dRe eps_j = K [ -|P_j|^2 Im beta'_j - 2 Re(beta'_j nu_j.P_j) ]
      dQ/dIm eps_j = K [ -|P_j|^2 Re beta'_j + 2 Im(beta'_j nu_j.P_j) ]
    Pinned by central finite differences of dense solves.
    """
    K = 4.0 * kd / aeff ** 2
    bp = ldr_inverse_polarizability_derivative(eps_site, kd, khat, ehat)
    p2 = np.sum(np.abs(P) ** 2, axis=1)
    nup = np.sum(nu * P, axis=1)
    g_re = K * (-p2 * bp.imag - 2.0 * (bp * nup).real)
    g_im = K * (-p2 * bp.real + 2.0 * (bp * nup).imag)
    return g_re, g_im


def absorption_weights(kd: float, beta: np.ndarray) -> np.ndarray:
    """w_j = -Im(1/alpha_j) - (2/3) k^3, so that C_abs = 4 pi k sum_j w_j |P_j|^2."""
    return -np.imag(beta) - (2.0 / 3.0) * kd ** 3


# --------------------------------------------------------------- near field --
def nearfield_box(shape_zyx, ext) -> tuple[tuple[int, int, int], tuple[int, int, int]]:
    """Extended computational volume of a near-field calculation ("Near-Field
    Calculations"; ddscat.par NRFLD = 1 with the six fractions r1..r6).

    The guide extends X1 <= x <= X2 to X1 - r1 Lx <= x <= X2 + r2 Lx (and
    likewise in y with r3, r4 and in z with r5, r6), Lx = X2 - X1.  Reading:
    the extended volume is a box of lattice points of the same spacing, with
    nint(r n) points added on each side of an axis of n points (its
    ELLIPSOID_NEARFIELD example, 48^3 extended by 0.5 on every side, is the
    96^3 volume the guide's timing line quotes).

    shape_zyx: target grid shape (nz, ny, nx); ext: (r1, ..., r6).
    Returns ((ex, ey, ez), (ox, oy, oz)): box extent in points and the box
    index of target point (0, 0, 0) (the points added on the low side).
    """
    nz, ny, nx = shape_zyx
    lo, hi = [], []
    for n, (ra, rb) in zip((nx, ny, nz), ((ext[0], ext[1]), (ext[2], ext[3]), (ext[4], ext[5]))):
        if ra < 0 or rb < 0:
            raise ValueError("near-field extension fractions must be non-negative")
        lo.append(int(math.floor(ra * n + 0.5)))
        hi.append(int(math.floor(rb * n + 0.5)))
    dims = (nx + lo[0] + hi[0], ny + lo[1] + hi[1], nz + lo[2] + hi[2])
    return dims, (lo[0], lo[1], lo[2])


def nearfield_points(shape_zyx, ext) -> np.ndarray:
    """Positions (Ne, 3) of every point of the extended box, x fastest, in
    the target's frame (origin at the centre of the target's own
    computational volume, as in site_positions)."""
    nz, ny, nx = shape_zyx
    (ex, ey, ez), (ox, oy, oz) = nearfield_box(shape_zyx, ext)
    iz, iy, ix = np.meshgrid(np.arange(ez), np.arange(ey), np.arange(ex), indexing="ij")
    return np.stack([(ix - ox - (nx - 1) / 2.0).ravel(), (iy - oy - (ny - 1) / 2.0).ravel(),
                     (iz - oz - (nz - 1) / 2.0).ravel()], axis=1).astype(np.float64)


def scattered_field(r_src: np.ndarray, P: np.ndarray, r_pts: np.ndarray, kd: float,
                    chunk: int = 256) -> np.ndarray:
    """E_sca at each point: the field of all dipoles P_l at r_src, except a
    dipole sitting on the point itself (the guide's E_sca "not including the
    dipole at j"): E_sca(r) = -sum_{l: r_l != r} A(r - r_l) P_l, with A the
    off-diagonal block of interaction_tensor.  Returns (Npts, 3)."""
    P = np.asarray(P, dtype=np.complex128)
    out = np.empty((r_pts.shape[0], 3), dtype=np.complex128)
    for s in range(0, r_pts.shape[0], chunk):
        d = r_pts[s:s + chunk][:, None, :] - r_src[None, :, :]      # (c, N, 3)
        same = np.all(d == 0.0, axis=-1)
        d[same] = (1.0, 0.0, 0.0)
        blk = interaction_tensor(d, kd)
        blk[same] = 0.0
        out[s:s + chunk] = -np.einsum("clab,lb->ca", blk, P)
    return out


def nearfield(grid: np.ndarray, P: np.ndarray, kd: float, khat, ehat, ext):
    """E_inc and E_sca at every point of the extended box (x fastest).

    P (N, 3): the target's polarization in site order.  Returns
    (dims, offset, E_inc (Ne, 3), E_sca (Ne, 3)); at a target point j an
    exact solution satisfies P_j = alpha_j (E_inc,j + E_sca,j).
    """
    dims, off = nearfield_box(grid.shape, ext)
    r_src, _ = site_positions(grid)
    r_pts = nearfield_points(grid.shape, ext)
    return dims, off, incident_field(r_pts, kd, khat, ehat), scattered_field(r_src, P, r_pts, kd)


# ---------------------------------------------------------------- far field --
def scattering_directions(x: float, eta: float):
    """The scattering directions and solid-angle weights of the guide's angular
    averages ("Selection of Scattering Angles", "Angular Averaging").

    theta values equally spaced in s(theta) = theta + theta/(theta + theta0),
    theta0 = 2 pi/(1 + x), from 0 to pi; their number N_theta = nint of the
    guide's expression in x and eta (reading: nearest integer, as for N_phi);
    N_phi(j) = 1 at theta = 0 and pi, else max(3, nint(4 pi sin(theta_j) /
    (theta_{j+1} - theta_{j-1}))), phi_jk = 2 pi (k - 1)/N_phi(j); weights
    Omega_jk from the guide's quadrature formulas.
    Returns (theta (D,), phi (D,), omega (D,)) in radians / steradians.
    """
    th0 = 2.0 * math.pi / (1.0 + x)
    nth_real = 1.0 + (2.0 * (3.0 + x) / eta) * (1.0 + 1.0 / (math.pi + th0)) / (1.0 + th0 / (math.pi + th0) ** 2)
    nth = int(math.floor(nth_real + 0.5))
    s = np.arange(nth) * math.pi / (nth - 1) * (1.0 + 1.0 / (math.pi + th0))
    th = ((s - 1.0 - th0) + np.sqrt((1.0 + th0 - s) ** 2 + 4.0 * th0 * s)) / 2.0
    th[0], th[-1] = 0.0, math.pi
    T, F, W = [], [], []
    for j in range(nth):
        if j == 0 or j == nth - 1:
            nphi = 1
        else:
            nphi = max(3, int(math.floor(4.0 * math.pi * math.sin(th[j]) / (th[j + 1] - th[j - 1]) + 0.5)))
        if j == 0:
            om = 2.0 * math.pi / nphi * (1.0 - (math.cos(th[0]) + math.cos(th[1])) / 2.0)
        elif j == nth - 1:
            om = 2.0 * math.pi / nphi * ((math.cos(th[j - 1]) + math.cos(th[j])) / 2.0 + 1.0)
        else:
            om = math.pi / nphi * (math.cos(th[j - 1]) - math.cos(th[j + 1]))
        for k in range(nphi):
            T.append(th[j])
            F.append(2.0 * math.pi * k / nphi)
            W.append(om)
    return np.array(T), np.array(F), np.array(W)


def lab_frame(khat):
    """Lab Frame of a right-hand side: x_L = khat, y_L = the first polarization
    basis vector normalize(z x khat) (x if khat is along z), z_L = x_L x y_L
    (for khat = x this is the guide's frame, with e01 = y_L, e02 = z_L)."""
    k = np.asarray(khat, dtype=np.float64)
    k = k / np.linalg.norm(k)
    y = np.cross([0.0, 0.0, 1.0], k)
    if np.linalg.norm(y) < 1e-8:
        y = np.array([1.0, 0.0, 0.0])
    y = y / np.linalg.norm(y)
    return k, y, np.cross(k, y)


def directions(khat, theta, phi) -> np.ndarray:
    """Unit vectors n = cos(theta) x_L + sin(theta) cos(phi) y_L + sin(theta) sin(phi) z_L, (D, 3)."""
    xl, yl, zl = lab_frame(khat)
    th = np.asarray(theta)[:, None]
    ph = np.asarray(phi)[:, None]
    return np.cos(th) * xl + np.sin(th) * np.cos(ph) * yl + np.sin(th) * np.sin(ph) * zl


def far_field(r: np.ndarray, P: np.ndarray, kd: float, n: np.ndarray, chunk: int = 64) -> np.ndarray:
    """Vector scattering amplitude F(n) = k^2 sum_j (I - n n) P_j exp(-i k n.r_j):
    the scattered field is E_sca -> exp(ikR)/R F(n) at distance R along n, so
    dC_sca/dOmega = |F|^2 for |E0| = 1 (the same far field as csca_quadrature).
    Returns (D, 3)."""
    P = np.asarray(P, dtype=np.complex128)
    out = np.empty((n.shape[0], 3), dtype=np.complex128)
    for s in range(0, n.shape[0], chunk):
        nn = n[s:s + chunk]
        ph = np.exp(-1j * kd * (nn @ r.T))            # (c, N)
        S = ph @ P                                      # (c, 3): sum_j P_j e^{-ik n.r_j}
        out[s:s + chunk] = kd * kd * (S - nn * np.sum(nn * S, axis=1, keepdims=True))
    return out


def angular_averages(r: np.ndarray, P: np.ndarray, kd: float, khat, theta, phi, omega):
    """C_sca, <cos theta>, <cos^2 theta> and the vector g in Lab Frame
    components, as the guide's weighted sums over scattering directions
    ("Angular Averaging": <f> = sum f dC/dOmega Omega / C_sca)."""
    n = directions(khat, theta, phi)
    F = far_field(r, P, kd, n)
    dC = np.sum(np.abs(F) ** 2, axis=1)
    w = dC * np.asarray(omega)
    csca = float(np.sum(w))
    c = np.cos(theta)
    g = np.array([np.sum(w * c), np.sum(w * np.sin(theta) * np.cos(phi)),
                  np.sum(w * np.sin(theta) * np.sin(phi))]) / csca
    return csca, float(g[0]), float(np.sum(w * c * c) / csca), g


def scattering_amplitudes(r: np.ndarray, P1: np.ndarray, P2: np.ndarray, kd: float, khat, e01, e02, theta, phi):
    """Amplitude scattering matrix (S1, S2, S3, S4) per direction ("Two
    Orthogonal Incident Polarizations (IORTH=2)"), from the polarizations P1,
    P2 (N, 3) induced by incident states e01, e02 (complex 3-vectors).

    f_ml = k (F_l . e_m) with e_1 = theta_hat, e_2 = phi_hat of the direction
    (F_l the far field of P_l, so that E_s . e_m = exp(ikr)/(kr) f_ml for a
    unit incident state l); with a = e01^*.y_L, b = e01^*.z_L, c = e02^*.y_L,
    d = e02^*.z_L the guide's relations give
      S1 = -i [f21 (b cos phi - a sin phi) + f22 (d cos phi - c sin phi)]
      S2 = -i [f11 (a cos phi + b sin phi) + f12 (c cos phi + d sin phi)]
      S3 =  i [f11 (b cos phi - a sin phi) + f12 (d cos phi - c sin phi)]
      S4 =  i [f21 (a cos phi + b sin phi) + f22 (c cos phi + d sin phi)].
    Returns (D, 4) complex (S1, S2, S3, S4)."""
    xl, yl, zl = lab_frame(khat)
    th = np.asarray(theta, dtype=np.float64)
    ph = np.asarray(phi, dtype=np.float64)
    n = directions(khat, th, ph)
    that = (-np.sin(th)[:, None] * xl + (np.cos(th) * np.cos(ph))[:, None] * yl
            + (np.cos(th) * np.sin(ph))[:, None] * zl)
    phat = -np.sin(ph)[:, None] * yl + np.cos(ph)[:, None] * zl
    F1 = far_field(r, P1, kd, n)
    F2 = far_field(r, P2, kd, n)
    f11 = kd * np.sum(F1 * that, axis=1)
    f21 = kd * np.sum(F1 * phat, axis=1)
    f12 = kd * np.sum(F2 * that, axis=1)
    f22 = kd * np.sum(F2 * phat, axis=1)
    e01 = np.conj(np.asarray(e01, dtype=np.complex128))
    e02 = np.conj(np.asarray(e02, dtype=np.complex128))
    a, b, c, d = e01 @ yl, e01 @ zl, e02 @ yl, e02 @ zl
    cp, sp = np.cos(ph), np.sin(ph)
    S1 = -1j * (f21 * (b * cp - a * sp) + f22 * (d * cp - c * sp))
    S2 = -1j * (f11 * (a * cp + b * sp) + f12 * (c * cp + d * sp))
    S3 = 1j * (f11 * (b * cp - a * sp) + f12 * (d * cp - c * sp))
    S4 = 1j * (f21 * (a * cp + b * sp) + f22 * (c * cp + d * sp))
    return np.stack([S1, S2, S3, S4], axis=1)


def mueller_matrix(S: np.ndarray) -> np.ndarray:
    """4x4 Mueller matrix per direction from (S1, S2, S3, S4) (D, 4): the
    Stokes-parameter transformation of Bohren & Huffman (1983, sec. 3.3), as
    the guide lists it.  Returns (D, 4, 4), element [i-1, j-1] = S_ij."""
    S1, S2, S3, S4 = (S[:, i] for i in range(4))
    a1, a2, a3, a4 = (np.abs(s) ** 2 for s in (S1, S2, S3, S4))
    M = np.empty((S.shape[0], 4, 4))
    M[:, 0, 0] = (a1 + a2 + a3 + a4) / 2
    M[:, 0, 1] = (a2 - a1 + a4 - a3) / 2
    M[:, 0, 2] = (S2 * np.conj(S3) + S1 * np.conj(S4)).real
    M[:, 0, 3] = (S2 * np.conj(S3) - S1 * np.conj(S4)).imag
    M[:, 1, 0] = (a2 - a1 + a3 - a4) / 2
    M[:, 1, 1] = (a1 + a2 - a3 - a4) / 2
    M[:, 1, 2] = (S2 * np.conj(S3) - S1 * np.conj(S4)).real
    M[:, 1, 3] = (S2 * np.conj(S3) + S1 * np.conj(S4)).imag
    M[:, 2, 0] = (S2 * np.conj(S4) + S1 * np.conj(S3)).real
    M[:, 2, 1] = (S2 * np.conj(S4) - S1 * np.conj(S3)).real
    M[:, 2, 2] = (S1 * np.conj(S2) + S3 * np.conj(S4)).real
    M[:, 2, 3] = (S2 * np.conj(S1) + S4 * np.conj(S3)).imag
    M[:, 3, 0] = (S4 * np.conj(S2) + S1 * np.conj(S3)).imag
    M[:, 3, 1] = (S4 * np.conj(S2) - S1 * np.conj(S3)).imag
    M[:, 3, 2] = (S1 * np.conj(S2) - S3 * np.conj(S4)).imag
    M[:, 3, 3] = (S1 * np.conj(S2) - S3 * np.conj(S4)).real
    return M
