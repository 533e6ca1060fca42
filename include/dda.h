/*
 * dda.h -- C ABI of the GB300 discrete-dipole-approximation (DDA) hot path.
 *
 * What it computes.  The DDSCAT 7.2 user guide (Draine & Flatau 2012) states
 * the scattering problem as the linear system  A P = E  (section "Choice of
 * Iterative Algorithm", eq. AP=E): E holds the incident field at the N
 * occupied lattice sites, P the unknown dipole moments, A is the 3N x 3N
 * complex-symmetric interaction matrix.  This library evaluates A.P as a
 * zero-padded 3-D FFT convolution (Goodman, Draine & Flatau 1990, the FFT
 * method the guide cites), solves A P = E with BiCGstab (the guide's
 * recommended solvers are BiCGstab variants, "Choice of Iterative
 * Algorithm") to the residual tolerance TOL (eq. err_tol and the TOL entry of
 * ddscat.par), and reduces P to the efficiency factors Q_ext, Q_abs, Q_sca
 * (section "What Does DDSCAT Calculate?").  Readings taken where the guide
 * is silent (LATTDR polarizability of Draine & Goodman 1993, Draine 1988
 * interaction tensor and cross sections):
 *   1/alpha = (4pi/3)(eps+2)/(eps-1) + (b1 + b2 eps + b3 eps S)(kd)^2 - (2/3) i (kd)^3,
 *   b1 = -1.8915316, b2 = 0.1648469, b3 = -1.7700004, S = sum_a khat_a^2 |e_a|^2
 *   (= sum_a (khat_a e_a)^2 for a real e; for a complex e the |e_a|^2 form is the
 *   one that keeps the lattice dispersion relation exact on the cube's 3-fold
 *   axes, where circular polarizations are lattice modes too),
 *   A_jl = e^{ik rho}/rho [k^2 (rr - I) + (ik rho - 1)/rho^2 (3 rr - I)]  (j != l),
 *   A_jj = (1/alpha_j) I  (anisotropic materials: the 1/alpha tensor of site j),
 *   C_ext = 4 pi k sum Im(E_inc^* . P),  C_abs = 4 pi k sum (-Im(1/alpha) - 2k^3/3)|P|^2
 *   (tensor form: Im(P . (1/alpha)^* P^*) - 2k^3/3 |P|^2),
 *   C_sca = C_ext - C_abs,  Q = C / (pi a_eff^2),  a_eff = (3N/4pi)^(1/3) d.
 *
 * Conventions.
 *  - Lattice units inside: dipole spacing d = 1; |E0| = 1; Gaussian units.
 *  - Target grid: uint8 composition code per lattice site, 0 = vacuum,
 *    1..ncomp = material, row-major with x fastest: comp[(iz*ny + iy)*nx + ix].
 *  - Site order: the N occupied sites in that same scan order.  Site j at
 *    r_j = (ix-(nx-1)/2, iy-(ny-1)/2, iz-(nz-1)/2): the Target Frame origin is
 *    the centre of the computational volume (also the incident phase origin).
 *  - Vectors (E, P, x, y): [R][3][N] complex numbers, each stored as two
 *    doubles (re, im) on the host API; R right-hand sides, component-major
 *    (all x components of RHS 0, then its y components, ...).
 *  - Directions khat: [R][3] real unit vectors in the Target Frame.
 *    Polarizations e: [R][3] complex (re, im pairs, 6 doubles per RHS),
 *    normalized, transverse to khat.
 *  - Ownership: the caller owns every host buffer it passes (read during the
 *    call only; never retained).  The context owns all device memory it
 *    allocates.  Device-pointer variants (suffix _device) read/write
 *    caller-owned device buffers and run on the context's stream.
 *  - Errors: every call returns a dda_status; on failure the message is
 *    available from dda_last_error(ctx) and no output buffer is written,
 *    except that dda_solve fills res[] (status per RHS) when it returns
 *    DDA_ERR_NOT_CONVERGED or DDA_ERR_BREAKDOWN.
 *  - Threads: a context is used by one host thread at a time.
 */
#ifndef DDA_GB300_H
#define DDA_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dda_ctx dda_ctx;

typedef enum {
    DDA_OK = 0,
    DDA_ERR_ARG = 1,            /* invalid argument or call order                          */
    DDA_ERR_CUDA = 2,           /* CUDA runtime error (message has the CUDA error string)  */
    DDA_ERR_OOM = 3,            /* device allocation failed                                */
    DDA_ERR_SIZE = 4,           /* lattice too large for the supported FFT lengths         */
    DDA_ERR_NOT_CONVERGED = 5,  /* some RHS did not reach tol within maxit                 */
    DDA_ERR_BREAKDOWN = 6,      /* BiCGstab breakdown (rho or <rhat,v> exactly zero)        */
    DDA_ERR_NONFINITE = 7       /* NaN/Inf in an input or in the iteration                 */
} dda_status;

typedef enum {
    DDA_FP64 = 0,         /* complex128 matvec and vectors, FP64 scalars                     */
    DDA_FP32_REFINED = 1, /* complex64 matvec in an FP64 iterative-refinement loop           */
    DDA_FP32 = 2,         /* complex64 matvec and vectors, FP64 scalars (no refinement)      */
    DDA_DF64 = 3          /* matvec entry points only: complex128 vectors, arithmetic in
                             double-float (pairs of FP32, ~44 significant bits); the
                             arithmetic of the complex64 modes' refinement residuals       */
} dda_precision;

typedef struct {
    double tol;        /* relative residual |E - A P| / |E| to reach (guide: TOL = 1e-5)     */
    int maxit;         /* max Krylov iterations per RHS, summed over refinement steps       */
    int use_graph;     /* 1: replay the iteration block as a captured CUDA graph            */
    double inner_tol;  /* FP32_REFINED: floor of the inner (FP32) relative tolerance        */
    int max_outer;     /* max refinement (outer) steps; <= 0 selects 8                       */
    int normal_eq;     /* 1: also report |A^H A P - A^H E| / |A^H E| (eq. err_tol)          */
    const double* x0;  /* nullable initial guess, [R][3][N] complex (warm start / resume)    */
    int residual_fp64; /* complex64 modes: 1 = true residuals E - A P with native FP64
                          arithmetic; 0 (default) = double-float arithmetic (FP32 pipes,
                          ~1e-12 relative accuracy, 6-8x faster on GB300)                  */
    int solver;        /* DDA_SOLVER_BICGSTAB (0, default): BiCGstab, 2 matvecs an iteration;
                          DDA_SOLVER_BICGSTAB2 (1): BiCGstab(2) (guide: PBCGS2, "Choice of
                          Iterative Algorithm"), 4 matvecs an iteration;
                          DDA_SOLVER_QMR (2): QMR for complex symmetric A (guide: QMRCCG;
                          Freund 1992), 1 matvec an iteration, no look-ahead             */
} dda_opts;

enum { DDA_SOLVER_BICGSTAB = 0, DDA_SOLVER_BICGSTAB2 = 1, DDA_SOLVER_QMR = 2 };

typedef struct {
    double qext, qabs, qsca;  /* efficiency factors                                         */
    double resid_rel;         /* true relative residual |E - A P|/|E| on FP64 vectors; its   *
                               * matvec is native FP64 for DDA_FP64, and for the complex64    *
                               * modes double-float (FP32 pairs, ~44 bits, within 1e-10 of   *
                               * FP64) unless dda_opts.residual_fp64 = 1 selects native FP64 */
    double resid_normal_eq;   /* eq. err_tol form, or -1 if not requested                    */
    int iters;                /* Krylov iterations, all refinement steps (BiCGstab: 2 matvecs
                                 each, BiCGstab(2): 4, QMR: 1)                              */
    int outer_iters;          /* refinement steps (1 for a converged plain solve)           */
    int matvecs;              /* A.x products applied to this RHS, all precisions           */
    dda_status status;        /* DDA_OK, DDA_ERR_NOT_CONVERGED, DDA_ERR_BREAKDOWN, ...      */
} dda_result;

typedef struct {
    int nx, ny, nz;        /* lattice                                                   */
    int Lx, Ly, Lz;        /* padded FFT lengths (>= 2n, 2^a 3^b)                       */
    int64_t ndipoles;      /* N occupied sites                                          */
    int ncomp;             /* compositions                                               */
    double aeff_lattice;   /* a_eff / d = (3N/4pi)^(1/3)                                 */
    double kd;             /* k d of the prepared wavelength (0 before dda_prepare)      */
    double x;              /* size parameter k a_eff                                     */
} dda_info;

/* Create a context on CUDA device `device`; allocates a stream.  */
dda_status dda_create(int device, dda_ctx** out);
/* Free all device memory, graphs and the stream owned by ctx. NULL is a no-op. */
dda_status dda_destroy(dda_ctx* ctx);
/* Message of the last failed call on ctx (owned by ctx, valid until the next call). */
const char* dda_last_error(const dda_ctx* ctx);
/* Run subsequent work on a caller stream (cudaStream_t passed as void*); NULL restores the ctx stream. */
dda_status dda_set_stream(dda_ctx* ctx, void* stream);

/* Target (guide: "Target Generation"; shape arrays IXYZ/ICOMP): nx*ny*nz
 * composition codes, copied in.  Invalidates any prepared wavelength.
 * DDA_ERR_ARG if no site is occupied or a code exceeds 255; DDA_ERR_SIZE if
 * some 2n exceeds the largest supported FFT length (512).                     */
dda_status dda_set_target(dda_ctx* ctx, int nx, int ny, int nz, const uint8_t* comp);
/* Materials (guide: "Dielectric Functions", ambient medium "Target in a
 * medium"): complex refractive index per composition (2*ncomp doubles) and the
 * real refractive index of the ambient medium.  Relative index m/m_ambient is
 * used.  DDA_ERR_ARG if ncomp < max code in the grid or m_ambient <= 0.        */
dda_status dda_set_materials(dda_ctx* ctx, int ncomp, const double* m_complex, double m_ambient);
/* Anisotropic materials (guide: "Composite Targets with Anisotropic
 * Constituents"; the per-site ICOMP(J,1-3) and THETADF, PHIDF, BETADF of the
 * anisotropic target types).  Composition c (1..ncomp) has the complex
 * refractive indices m_principal[6c..6c+5] (re, im of m_1, m_2, m_3) along the
 * principal axes e_1, e_2, e_3 of its dielectric tensor, and the dielectric
 * frame is rotated from the Target Frame by df_angles[3c..3c+2] = (theta_DF,
 * phi_DF, beta_DF) in radians: e_1 = (cos th, sin th cos ph, sin th sin ph),
 * e_2, e_3 as the guide gives them.  Each site's 1/alpha is then the
 * symmetric tensor sum_j (1/alpha_j) e_j e_j^T, 1/alpha_j the LATTDR value of
 * (m_j/m_ambient)^2 with the same propagation/polarization factor S for the
 * three.  Sites whose dielectric frames differ use different codes (up to
 * 255).  Replaces any isotropic materials (dda_set_materials switches back);
 * solves, matvecs, Q and the field calls then use the tensor diagonal, the
 * fused slice passes are skipped, and dda_grad_qabs returns DDA_ERR_ARG.
 * Errors as for dda_set_materials; DDA_ERR_NONFINITE for a non-finite angle. */
dda_status dda_set_anisotropic_materials(dda_ctx* ctx, int ncomp, const double* m_principal,
                                         const double* df_angles, double m_ambient);
/* Per-site materials (the guide's ICOMP per dipole, without the 255-code
 * limit): one complex refractive index for every occupied site of the
 * current target, m_site[2j], m_site[2j+1] for site j in the order of
 * dda_set_target (x fastest), and the ambient index.  Each site's 1/alpha is
 * the LATTDR value of its own (m_j/m_ambient)^2; the grid's composition
 * codes then only mark occupancy.  Solves, matvecs, Q, the gradient and the
 * field calls all apply; the fused slice passes are skipped.  Needs
 * dda_set_target (DDA_ERR_ARG otherwise); a later dda_set_target,
 * dda_set_materials or dda_set_anisotropic_materials ends the mode.  Errors
 * as for dda_set_materials, per site.                                          */
dda_status dda_set_site_materials(dda_ctx* ctx, const double* m_site, double m_ambient);
/* Wavelength and size (guide: WAVINI / AEFFINI, same physical units): sets
 * d = aeff/(3N/4pi)^(1/3), k = 2 pi m_ambient / lambda_vac, and builds the
 * transformed Green tensor for `precision` (FP64 tensor always; FP32 copy for
 * the FP32 modes).                                                             */
dda_status dda_prepare(dda_ctx* ctx, double lambda_vac, double aeff, dda_precision precision);
dda_status dda_get_info(const dda_ctx* ctx, dda_info* info);

/* Solve A P = E for R incident plane waves (direction khat[3R], polarization
 * e[6R]) and reduce Q.  P_out (nullable): [R][3][N] complex, caller-owned.
 * res: R entries.  Returns DDA_OK when every RHS converged, else the worst
 * per-RHS status.  precision must have been prepared (FP64 is always).       */
dda_status dda_solve(dda_ctx* ctx, dda_precision precision, int R, const double* khat, const double* e,
                     const dda_opts* opts, double* P_out, dda_result* res);
/* Same, P written to a caller device buffer of R*3*N double2 (complex128).  */
dda_status dda_solve_device(dda_ctx* ctx, dda_precision precision, int R, const double* khat, const double* e,
                            const dda_opts* opts, void* P_dev, dda_result* res);

/* One product y = A x for R RHS (A's diagonal depends on each RHS through S).
 * x, y: host [R][3][N] complex.  precision DDA_FP64, DDA_DF64 (needs an FP32
 * mode prepared), or DDA_FP32 (x rounded to complex64, result widened back).
 * For testing and timing.                                                      */
dda_status dda_matvec(dda_ctx* ctx, dda_precision precision, int R, const double* khat, const double* e,
                      const double* x, double* y);
/* Device variant: x, y device buffers of R*3*N complex elements of the
 * precision's type (double2 for DDA_FP64 and DDA_DF64, float2 for DDA_FP32).  */
dda_status dda_matvec_device(dda_ctx* ctx, dda_precision precision, int R, const double* khat, const double* e,
                             const void* x_dev, void* y_dev);

/* No-allocation variant of dda_matvec_device, for callers that must not
 * allocate device memory during the call: code whose device memory is all
 * reserved up front by its own allocator or memory pool (a cudaMalloc here
 * could fail or fragment that pool), and latency-critical loops that cannot
 * afford the implicit synchronization an allocation may cause.  There is no
 * counterpart in the paper; this is a deployment convenience.
 * Same arguments, layout and result as dda_matvec_device, for the
 * precisions DDA_FP64 and DDA_FP32 (DDA_DF64 and DDA_FP32_REFINED are
 * rejected with DDA_ERR_ARG); the context must
 * already be prepared (dda_prepare allocates; this call does not).  The
 * padded FFT work buffers and the 1/alpha table live in one fixed scratch
 * array of 64 MiB (67108864 bytes) that the library declares in device
 * memory: every GPU that loads the library holds it until the process exits.
 * Lattices or RHS counts whose scratch would exceed it are rejected with
 * DDA_ERR_SIZE (about 96 bytes per RHS for every site of the lattice
 * rounded up to half the padded FFT lengths, (Lx/2)(Ly/2)(Lz/2), for
 * complex64, twice that for complex128: the 64^3 lattice fits two complex64
 * RHS).  The first call on a device looks up the array's device address,
 * and so does the first call after that device's context was destroyed and
 * re-created (cudaDeviceReset): make that first call before any stream
 * capture.  All calls, from every context of the process, share the
 * one array and leave their data in it; no part of it needs to start at zero
 * (every buffer is written before it is read), but calls that overlap on the
 * GPU race on it, so do not run two of them concurrently on one device.
 * Synchronizes the context stream before returning, so it cannot be part of
 * a CUDA graph: called while the context stream is being captured it returns
 * DDA_ERR_ARG and leaves the capture untouched.                               */
dda_status dda_matvec_device_noalloc(dda_ctx* ctx, dda_precision precision, int R, const double* khat,
                                     const double* e, const void* x_dev, void* y_dev);

/* Incident field E_inc,j = e exp(i k khat.r_j) at every site, [R][3][N] complex (host). */
dda_status dda_incident_field(dda_ctx* ctx, int R, const double* khat, const double* e, double* E_out);

/* Near field ("Near-Field Calculations", NRFLD = 1; Flatau & Draine 2012):
 * E_inc and E_sca at every lattice point of the target's computational volume
 * extended by the fractions ext[0..5] = (r1, ..., r6): nint(r1 nx) points
 * are added below x and nint(r2 nx) above, likewise r3, r4 in y and r5, r6
 * in z (the guide's X1 - r1 Lx <= x <= X2 + r2 Lx, ...).  E_sca,j is the
 * field of the target's polarization P at point j, without the dipole at j
 * itself: E_sca,j = -sum_{l != j} A_jl P_l with A_jl the off-diagonal blocks
 * of the solve's matrix, so an exact solution satisfies
 * P_j = alpha_j (E_inc,j + E_sca,j) at target points.  Evaluated as the same
 * zero-padded FFT convolution as the matvec, on the extended box.
 * dda_nearfield_dims: box extent dims[3] (x, y, z points) and the box index
 * offset[3] of target point (0, 0, 0); DDA_ERR_SIZE if an extent exceeds the
 * largest padded length (256 points).  Needs dda_set_target.
 * dda_nearfield: P host [R][3][N] complex (the solve's P_out layout);
 * E_inc_out (nullable), E_sca_out host [R][3][Ne] complex, Ne = dims[0]
 * dims[1] dims[2], box points x fastest; phase origin as in dda_solve.
 * precision DDA_FP64 (complex128 convolution) or DDA_FP32 /
 * DDA_FP32_REFINED (complex64 convolution).  Needs dda_prepare.              */
dda_status dda_nearfield_dims(dda_ctx* ctx, const double* ext, int* dims, int* offset);
dda_status dda_nearfield(dda_ctx* ctx, dda_precision precision, int R, const double* khat, const double* e,
                         const double* P, const double* ext, double* E_inc_out, double* E_sca_out);

/* Far field ("Averaging over Scattering Directions", "Scattering by Finite
 * Targets: The Mueller Matrix").  Directions are given in each RHS's Lab
 * Frame: x_L = khat, y_L = normalize(z x khat) (x if khat is along z),
 * z_L = x_L x y_L, n = cos(theta) x_L + sin(theta) cos(phi) y_L +
 * sin(theta) sin(phi) z_L (for khat = x: the guide's frame with e01 = y).
 * dda_scattering_directions: the guide's directions for angular averages
 *   (theta equally spaced in s(theta) = theta + theta/(theta + theta0),
 *   theta0 = 2 pi/(1 + x), N_theta = nint of its expression in x and eta
 *   (ETASCA); nint(4 pi sin theta_j / (theta_{j+1} - theta_{j-1})), at least
 *   3, azimuths per interior theta) with their solid-angle weights omega
 *   (summing to 4 pi).  *count = number of directions; the arrays are filled
 *   only if capacity >= *count (call with capacity 0 to size them).  No
 *   context needed; DDA_ERR_ARG for non-positive x or eta.
 * dda_farfield: vector amplitudes F(n) = k^2 (I - n n) sum_j P_j
 *   exp(-i k n.r_j) (lattice units, |E0| = 1: the scattered field is
 *   exp(ikR)/R F, dC_sca/dOmega = |F|^2), for ndir directions (theta, phi in
 *   radians) and R RHS: P host [R][3][N] complex, F_out host [R][ndir][3]
 *   complex.  precision DDA_FP64 or a complex64 mode (complex64 sums, FP64
 *   block totals).  Needs dda_prepare.
 * dda_angular_averages: per RHS, out[6] = (Q_sca, <cos theta>, <cos^2 theta>,
 *   g_x, g_y, g_z): the guide's weighted sums over dda_scattering_directions
 *   (x = k a_eff of the prepared target, eta = ETASCA), Q_sca = C_sca/(pi
 *   a_eff^2), g the Lab Frame components of <n>.  *ndir_out (nullable) =
 *   directions used.                                                        */
/* dda_mueller: the guide's amplitude scattering matrix and 4x4 Mueller
 *   matrix ("Two Orthogonal Incident Polarizations (IORTH=2)") for one
 *   incident direction khat: P host [2][3][N] complex, the polarizations
 *   induced by the orthonormal incident states e01, e02 (complex 3-vectors,
 *   6 doubles each; the guide takes e02 = khat x e01^*).  Per direction:
 *   f_ml = k (F_l . e_m), e_1 = theta_hat, e_2 = phi_hat; S1..S4 from f_ml,
 *   a = e01^*.y_L, b = e01^*.z_L, c = e02^*.y_L, d = e02^*.z_L and phi; and
 *   S_ij from S1..S4 (Bohren & Huffman).  S_out [ndir][16] row-major S_11 ..
 *   S_44; amp_out (nullable) [ndir][4] complex S1..S4.                      */
dda_status dda_mueller(dda_ctx* ctx, dda_precision precision, const double* khat, const double* e01, const double* e02,
                       const double* P, int ndir, const double* theta, const double* phi, double* S_out,
                       double* amp_out);
dda_status dda_scattering_directions(double x, double eta, int capacity, double* theta, double* phi, double* omega,
                                     int* count);
dda_status dda_farfield(dda_ctx* ctx, dda_precision precision, int R, const double* khat, const double* P, int ndir,
                        const double* theta, const double* phi, double* F_out);
dda_status dda_angular_averages(dda_ctx* ctx, dda_precision precision, int R, const double* khat, const double* P,
                                double eta, double* out, int* ndir_out);

/* dQ_abs/dRe(eps_j) and dQ_abs/dIm(eps_j) for every dipole (each dipole's eps
 * treated as independent; forward values from the composition table), by an
 * adjoint solve A nu = W P^* that reuses the matvec because A = A^T.  One RHS.
 * The guide has no gradients; this is the project's differentiation pattern.
 * res[0] forward solve, res[1] adjoint solve.  P_out (nullable) [3][N].        */
dda_status dda_grad_qabs(dda_ctx* ctx, dda_precision precision, const double* khat, const double* e,
                         const dda_opts* opts, double* dq_dre_eps, double* dq_dim_eps, double* P_out,
                         dda_result* res);

/* Schedule autotuning.  Two choices about how a matvec runs are made by
 * measurement, per arithmetic type and RHS count:
 *  - the z pass (FFT along z, the 3x3 Fourier-space product, inverse FFT),
 *    for complex64 on grids whose z transform keeps at most 8 points per
 *    thread (Lz = 16, 32, 64, 128, 256 or 512):
 *      0  three component groups per column, spectra exchanged through
 *         shared memory;
 *      1  register-resident: one thread holds all three components of its
 *         points, and the loads of the next RHS are issued before the current
 *         one is transformed;
 *      2  as 1, with each block owning columns of the Green octant and
 *         transforming the four columns (+-kx, +-ky) that share them (a
 *         quarter of the Green staging; faster for few RHS);
 *      3, 4  as 1 and 2 with a radix-16 plan of the z transform (Lz = 128:
 *         8 x 16, Lz = 256: 16 x 16): one exchange per transform instead of
 *         two, 16 points per thread, no register prefetch of the next RHS;
 *  - the fused x+y slice passes: where the half-y spectrum of one z-slice,
 *    Lx x (Ly/2) points, fits in shared memory (Lx, Ly in 64..192 for
 *    complex64, 64 or 96 for complex128 and double-float), one block can
 *    transform a whole slice along x and y, so the x-transformed rows never
 *    go through HBM (3 kernels per matvec instead of 5);
 *  - the x passes (complex64 only): 0 stages each block's rows through
 *    shared memory around the transform; 1 + V holds each row in one warp
 *    (up to 32 lanes, read and scattered straight from and to global memory,
 *    warp barriers between the radix stages) with radix plan V: V = 0 is the
 *    staged plan, V = 1 (Lx = 128, 192, 256) a plan with fewer exchanges
 *    (radix 16, or more points per lane);
 *  - the y passes (complex64 only, Ly = 128, 192, 256): 0 the plan of the
 *    staged passes, 1 a radix plan with one exchange fewer (8 x 16,
 *    8 x 8 x 3, 16 x 16).
 * All choices compute the same product; results agree to rounding.  In
 * automatic mode the context times the available choices inside whole
 * matvecs on its own workspace the first time a matvec of a given type and
 * RHS count runs outside a stream capture (the z schedule with the slice
 * passes, then the x-forward, then the x-inverse schedule, each keeping the
 * fastest so far), and keeps the result (inside a capture an untimed choice
 * is used until then).
 * dda_set_schedule: zpass -1 automatic (the default), 0..4 forces that z
 *   schedule wherever it exists (3 and 4 fall back to 1 and 2 where the
 *   length has one plan, 1..4 to 0 where the register schedules do not exist).
 * dda_set_slice_passes: on -1 automatic, 0 always the separate passes (the
 *   default: measured on GB300 the slice passes are faster only for small
 *   grids outside a solve), 1 the slice passes wherever they are built.
 * dda_set_xpass: xfwd, xinv -1 automatic (the default), 0..3 forces that
 *   x-forward / x-inverse schedule: 0 rows staged through shared memory,
 *   1 + V the warp-local rows with radix plan variant V (Lx = 128, 256, 512:
 *   V = 0, 1, 2; Lx = 64, 192: V = 0, 1; else V = 0; the last variant of 64,
 *   128, 256 and 512 points exchanges by warp shuffles); a V beyond the
 *   length's variants falls back to its last one.
 * The setters clear the timings; any other value: DDA_ERR_ARG.
 * dda_get_schedule: the z schedule (and, if slices is not NULL, whether the
 *   slice passes run) of complex64 matvecs of R RHS on the current target,
 *   timing the candidates now if needed (this sizes the workspace for R).
 *   Needs dda_prepare with DDA_FP32_REFINED or DDA_FP32.
 * dda_get_xpass: likewise, the x-forward and x-inverse schedules of those
 *   matvecs.
 * dda_set_ypass: ypass -1 automatic (the default), 0 or 1 forces that y
 *   plan where it exists.  dda_get_ypass: the y plan of plain matvecs.
 * dda_get_solve_schedule: the z, x-forward, x-inverse and y schedules of the
 *   complex64 matvecs inside a solve of R RHS (those carry the fused BiCGstab
 *   updates and are tuned apart from plain matvecs, with the same candidates). */
dda_status dda_set_schedule(dda_ctx* ctx, int zpass);
dda_status dda_set_slice_passes(dda_ctx* ctx, int on);
dda_status dda_set_xpass(dda_ctx* ctx, int xfwd, int xinv);
dda_status dda_get_schedule(dda_ctx* ctx, int R, int* zpass, int* slices);
dda_status dda_get_xpass(dda_ctx* ctx, int R, int* xfwd, int* xinv);
dda_status dda_set_ypass(dda_ctx* ctx, int ypass);
dda_status dda_get_ypass(dda_ctx* ctx, int R, int* ypass);
dda_status dda_get_solve_schedule(dda_ctx* ctx, int R, int* zpass, int* xfwd, int* xinv, int* ypass);

/* Launch tracing (the guide's TIMEIT timing switch, per kernel kind rather than
 * per run): when on, every hot-path kernel launch is bracketed by CUDA events
 * on the stream it runs on -- also inside replayed CUDA graphs -- and its
 * duration is accumulated per kernel kind.  `units` sums the right-hand sides
 * each launch processed.  Enabling resets the counters.                        */
typedef struct {
    char name[24];      /* kernel kind, e.g. "z_conv_c64"                                */
    int64_t launches;
    double total_ms;
    double units;
} dda_kernel_stat;
dda_status dda_profile_enable(dda_ctx* ctx, int on);
/* Fills up to max_entries kinds that launched at least once; *n_entries = all such kinds. */
dda_status dda_profile_read(const dda_ctx* ctx, dda_kernel_stat* out, int max_entries, int* n_entries);

#ifdef __cplusplus
}
#endif
#endif /* DDA_GB300_H */
