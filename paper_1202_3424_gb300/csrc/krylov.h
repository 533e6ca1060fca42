// Launchers of the BiCGstab, reduction and physics kernels (krylov.cu).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace dda {

enum KStatus : int { KS_RUNNING = 0, KS_CONVERGED = 1, KS_BREAKDOWN = 2, KS_MAXIT = 3, KS_NONFINITE = 4, KS_IDLE = 5 };

// QMR scalars of one RHS (qmr.cu): Lanczos coefficients, the last two
// Givens rotations, the rotated right-hand side and this step's update.
struct QmrScalars {
    double2 delta, delta_prev;  // v_n^T v_n, v_{n-1}^T v_{n-1}
    double2 gamma, alpha;       // H(n-1, n), H(n, n)
    double2 s1, s2;             // rotations G_{n-1}, G_{n-2}: sines
    double c1, c2;              // ... and cosines
    double2 tt;                 // t~_n, the unrotated last entry of the right-hand side
    double2 t, rho, dlt, eps;   // x += t p_n,  p_n = (v_n - dlt p_{n-1} - eps p_{n-2}) / rho
    double inv_beta;            // 1 / |v~_{n+1}| (0: invariant subspace)
    int lanczos_breakdown;      // v_{n+1}^T v_{n+1} = 0
    double best;                // smallest |r| so far and its iteration (stagnation test)
    int best_iter;
};

// Per-RHS scalars of one Krylov solve, all FP64, kept on the device.
struct KState {
    double2 rho;    // <rhat, r> of the current residual
    double2 alpha;
    double2 omega;
    double2 beta;   // coefficient of the next search-direction update
    double2 gamma1; // BiCGstab(2): first minimal-residual coefficient (the second is omega)
    double bnorm;   // |b|
    double rnorm;   // recurrence residual |r|
    double tol_abs; // stop when rnorm <= tol_abs
    int iter;       // iterations completed in this solve
    int maxit;
    int status;     // KStatus
    int pending;    // BiCGstab: stopped with the last x update still to apply (KrylovOps::finish_x)
    QmrScalars q;   // QMR only
};

static constexpr int kMaxReduceBlocks = 1024;
int reduce_blocks(int64_t n);

template <typename C> struct KrylovOps {
    // (s_ may be null; BiCGstab passes its s vector, which starts as b)
    static cudaError_t init(int R, int64_t n, const C* b, C* x, C* r, C* rhat, C* p, C* v, C* s_, KState* st,
                            const double* tol_rel, const int* want, int* active, double2* part, unsigned* cnt,
                            cudaStream_t s);
    // x += alpha p + omega s for the RHS that stopped with that update pending
    static cudaError_t finish_x(int R, int64_t n, C* x, const C* p, const C* s_, const KState* st, cudaStream_t s);
    static cudaError_t to_inner(int R, int64_t n, const double2* r64, C* bin, const double* scale, const int* active,
                                cudaStream_t s);
    static cudaError_t accumulate(int R, int64_t n, double2* x64, const C* xin, const double* coef,
                                  const int* active, cudaStream_t s);
};

// BiCGstab(2) steps (bicgstab2.cu); the u updates and alpha reductions run
// inside the fused matvecs.
template <typename C> struct BiCGstab2Ops {
    static cudaError_t r0(int R, int64_t n, C* r0, const C* u1, C* x, const C* u0, const KState* st,
                          const int* active, cudaStream_t s);
    static cudaError_t rho(int R, int64_t n, const C* rt, const C* r1, KState* st, int* active, double2* part,
                           unsigned* cnt, cudaStream_t s);
    static cudaError_t r1(int R, int64_t n, C* r0, C* r1, C* u0, const C* u1, const C* u2, C* x,
                          const KState* st, const int* active, cudaStream_t s);
    static cudaError_t gram(int R, int64_t n, const C* r0, const C* r1, const C* r2, KState* st, int* active,
                            double2* part, unsigned* cnt, cudaStream_t s);
    static cudaError_t mr(int R, int64_t n, C* x, C* r0, const C* r1, const C* r2, C* u0, const C* u1, const C* u2,
                          const C* rt, KState* st, int* active, double2* part, unsigned* cnt, cudaStream_t s);
};

// QMR steps for complex symmetric A (qmr.cu): init after KrylovOps::init,
// then per iteration w = A v, alpha, the Lanczos step with the rotations,
// and the update of p, A p, x, r and v.
template <typename C> struct QmrOps {
    static cudaError_t init(int R, int64_t n, const C* r, C* v, C* v_prev, C* ap1, C* ap2, KState* st,
                            int* active, double2* part, unsigned* cnt, cudaStream_t s);
    static cudaError_t alpha(int R, int64_t n, const C* v, const C* w, KState* st, int* active, double2* part,
                             unsigned* cnt, cudaStream_t s);
    static cudaError_t lanczos(int R, int64_t n, const C* w, const C* v, C* v_prev, KState* st, int* active,
                               double2* part, unsigned* cnt, cudaStream_t s);
    static cudaError_t update(int R, int64_t n, const C* v, C* vt, const C* w, const C* p1, C* p2, const C* ap1,
                              C* ap2, C* x, C* r, KState* st, int* active, double2* part, unsigned* cnt,
                              cudaStream_t s);
};

cudaError_t launch_count_active(const int* active, int R, int* out, cudaStream_t s);
cudaError_t launch_residual(int R, int64_t n, const double2* a, const double2* b, double2* out_vec, double* out_norm2,
                            const int* active, double2* part, unsigned* cnt, cudaStream_t s);
cudaError_t launch_conj_diff(int R, int64_t n, const double2* a, const double2* b, double2* out, cudaStream_t s);
cudaError_t launch_c64_to_c128(int64_t n, const float2* s_, double2* d, cudaStream_t s);
cudaError_t launch_c128_to_c64v(int64_t n, const double2* s_, float2* d, cudaStream_t s);
struct Geom;
cudaError_t launch_einc(int R, int64_t N, const int* lat_of, const Geom& g, double kd, const double* khat,
                        const double2* e, double2* E, cudaStream_t s);
// E_inc at points lat_of[j] of an nx*ny-row lattice, phase origin at (cx, cy, cz) in its index space.
cudaError_t launch_einc_at(int R, int64_t N, const int* lat_of, int nx, int ny, double cx, double cy, double cz,
                           double kd, const double* khat, const double2* e, double2* E, cudaStream_t s);
// Near field: target sites into the extended-box vector; E_sca = -y in complex128.
template <typename C>
cudaError_t launch_scatter_sites(int R, int64_t N, int64_t Ne, const int* box_of, const double2* P, C* Pbox,
                                 cudaStream_t s);
template <typename C> cudaError_t launch_negate_c128(int64_t n, const C* y, double2* out, cudaStream_t s);
cudaError_t launch_qsums(int R, int64_t N, const double2* E, const double2* P, const uint8_t* comp_of, const double* w,
                         int w_stride, bool tensor, double2* sums, double2* part, unsigned* cnt, cudaStream_t s);
cudaError_t launch_adjoint_rhs(int64_t N, const double2* P, const uint8_t* comp_of, const double* w, double2* b,
                               cudaStream_t s);
cudaError_t launch_grad(int64_t N, const double2* P, const double2* nu, const uint8_t* comp_of, const double2* dbeta,
                        double K, double* g_re, double* g_im, cudaStream_t s);

}  // namespace dda
