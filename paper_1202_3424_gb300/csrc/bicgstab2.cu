// BiCGstab(2) vector kernels: the guide's PBCGS2 option ("Choice of Iterative
// Algorithm": Botchev's ZBCG2, BiCGstab(l) of Sleijpen & Fokkema 1993 with
// l = 2), one independent iteration per right-hand side.
//
// Vectors (complex64 or complex128, [R][3N]): r0, r1, r2, u0, u1, u2, x and
// the shadow residual rt = r0 at the start.  One iteration = two BiCG steps
// and a degree-2 minimal-residual step (4 matvecs):
//   j = 0:  u0 = r0 - beta u0;  u1 = A u0;  alpha = rho / <rt, u1>;
//           r0 -= alpha u1;  x += alpha u0;  r1 = A r0
//   j = 1:  rho' = <rt, r1>;  beta = alpha rho' / rho;  rho = rho';
//           u0 = r0 - beta u0;  u1 = r1 - beta u1;  u2 = A u1;  alpha = rho / <rt, u2>;
//           r0 -= alpha u1;  r1 -= alpha u2;  x += alpha u0;  r2 = A r1
// The u1 and u2 matvecs are the fused BiCGstab matvec (internal.h,
// FusedKrylov mode 1), whose gather forms p <- r + beta (p - omega v) and
// whose scatter forms alpha = rho / <rhat, A p>: between the BiCG steps the
// state holds -beta in `beta` and 0 in `omega`, so that gather is u <- r - beta u.
//   MR:     tau = <r1, r2>/s1, r2' = r2 - tau r1, s_j = |r_j'|^2, g'_j = <r_j', r0>/s_j,
//           g2 = g'2 = omega, g1 = g'1 - tau g2;
//           x += g1 r0 + g2 r1;  r0 -= g'1 r1 + g'2 r2';  u0 -= g1 u1 + g2 u2
//           (with r2' written out, r0 -= g1 r1 + g2 r2: the three updates share g1, g2)
//   next:   rho' = <rt, r0>;  beta = alpha rho' / (-omega rho);  rho = rho'
// (<a, b> = a^H b).  The Gram entries of r0, r1, r2 come from one reduction,
// so r2' is never formed.  Scalars are FP64 in KState; the last block of each
// reduction updates them on the device (graph-replayable, per-RHS masks).
#include <math.h>

#include "internal.h"
#include "krylov.h"
#include "krylov_dev.cuh"
#include "profiler.h"

namespace dda {

namespace {

constexpr int kThreads = 256;

#define RHS_LOOP_SETUP(active)                                          \
    const int r = blockIdx.y;                                           \
    if (active != nullptr && active[r] == 0) return;                    \
    const int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;  \
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;             \
    const int64_t off = (int64_t)r * n;

__device__ __forceinline__ void stop(KState& s, int* active, int r, int status) {
    s.status = status;
    active[r] = 0;
}

// r0 -= alpha u1;  x += alpha u0
template <typename C>
__global__ void __launch_bounds__(kThreads)
    k_b2_r0(int64_t n, C* __restrict__ r0, const C* __restrict__ u1, C* __restrict__ x, const C* __restrict__ u0,
            const KState* __restrict__ st, const int* __restrict__ active) {
    RHS_LOOP_SETUP(active)
    const C alpha = from2<C>(st[r].alpha);
    for (int64_t i = i0; i < n; i += stride) {
        r0[off + i] = csub(r0[off + i], cmul(alpha, u1[off + i]));
        x[off + i] = cadd(x[off + i], cmul(alpha, u0[off + i]));
    }
}

// rho' = <rt, r1>;  beta = alpha rho' / rho (stored as -beta);  rho = rho'
template <typename C>
__global__ void __launch_bounds__(kThreads)
    k_b2_rho(int64_t n, const C* __restrict__ rt, const C* __restrict__ r1, KState* __restrict__ st,
             int* __restrict__ active, double2* __restrict__ part, unsigned* __restrict__ cnt) {
    RHS_LOOP_SETUP(active)
    DotAcc<C> d[1];
    for (int64_t i = i0; i < n; i += stride) d[0].add_cdot(rt[off + i], r1[off + i]);
    double2 acc[1];
    block_totals<C, 1>(d, acc);
    if (last_block_total_reduced<1>(acc, part + (int64_t)r * gridDim.x, cnt + r) && threadIdx.x == 0) {
        KState& s = st[r];
        if (!finite2(acc[0])) stop(s, active, r, KS_NONFINITE);
        else if (s.rho.x == 0.0 && s.rho.y == 0.0) stop(s, active, r, KS_BREAKDOWN);
        else {
            const double2 b = cmul(s.alpha, zdiv(acc[0], s.rho));
            s.beta = make_double2(-b.x, -b.y);
            s.omega = make_double2(0.0, 0.0);  // (the solve's first iteration starts with omega = 1)
            s.rho = acc[0];
        }
    }
}

// u0 = r0 - beta u0 (the state holds -beta);  r0 -= alpha u1;  r1 -= alpha u2;  x += alpha u0
template <typename C>
__global__ void __launch_bounds__(kThreads)
    k_b2_r1(int64_t n, C* __restrict__ r0, C* __restrict__ r1, C* __restrict__ u0, const C* __restrict__ u1,
            const C* __restrict__ u2, C* __restrict__ x, const KState* __restrict__ st,
            const int* __restrict__ active) {
    RHS_LOOP_SETUP(active)
    const C alpha = from2<C>(st[r].alpha), mbeta = from2<C>(st[r].beta);
    for (int64_t i = i0; i < n; i += stride) {
        const C a = r0[off + i];
        const C u = cadd(a, cmul(mbeta, u0[off + i]));
        u0[off + i] = u;
        r0[off + i] = csub(a, cmul(alpha, u1[off + i]));
        r1[off + i] = csub(r1[off + i], cmul(alpha, u2[off + i]));
        x[off + i] = cadd(x[off + i], cmul(alpha, u));
    }
}

// Gram entries |r1|^2, <r1, r2>, |r2|^2, <r1, r0>, <r2, r0> -> the MR coefficients and omega.
template <typename C>
__global__ void __launch_bounds__(kThreads)
    k_b2_gram(int64_t n, const C* __restrict__ r0, const C* __restrict__ r1, const C* __restrict__ r2,
              KState* __restrict__ st, int* __restrict__ active, double2* __restrict__ part,
              unsigned* __restrict__ cnt) {
    RHS_LOOP_SETUP(active)
    DotAcc<C> d[5];
    for (int64_t i = i0; i < n; i += stride) {
        const C a = r0[off + i], b = r1[off + i], c = r2[off + i];
        d[0].add_norm2(b);
        d[1].add_cdot(b, c);
        d[2].add_norm2(c);
        d[3].add_cdot(b, a);
        d[4].add_cdot(c, a);
    }
    double2 acc[5];
    block_totals<C, 5>(d, acc);
    if (last_block_total_reduced<5>(acc, part + (int64_t)r * gridDim.x * 5, cnt + r) && threadIdx.x == 0) {
        KState& s = st[r];
        const double s1 = acc[0].x;
        bool ok = true;
        for (int k = 0; k < 5; ++k) ok = ok && finite2(acc[k]);
        if (!ok) {
            stop(s, active, r, KS_NONFINITE);
        } else if (!(s1 > 0.0)) {
            stop(s, active, r, KS_BREAKDOWN);
        } else {
            const double2 tau = make_double2(acc[1].x / s1, acc[1].y / s1);
            const double s2 = acc[2].x - (acc[1].x * acc[1].x + acc[1].y * acc[1].y) / s1;
            if (!(s2 > 0.0)) {
                stop(s, active, r, KS_BREAKDOWN);
            } else {
                const double2 g1p = make_double2(acc[3].x / s1, acc[3].y / s1);
                // <r2', r0> = <r2, r0> - conj(tau) <r1, r0>
                const double2 ctau = make_double2(tau.x, -tau.y);
                const double2 n2 = csub(acc[4], cmul(ctau, acc[3]));
                const double2 g2p = make_double2(n2.x / s2, n2.y / s2);
                s.omega = g2p;                         // gamma_2 = gamma'_2 = gamma''_1
                s.gamma1 = csub(g1p, cmul(tau, g2p));  // gamma_1
            }
        }
    }
}

// x += g1 r0 + g2 r1;  r0 -= g1 r1 + g2 r2;  u0 -= g1 u1 + g2 u2  (g2 = omega);
// rho' = <rt, r0>, |r0|^2; convergence; beta of the next iteration (stored
// as -beta, with omega = 0, for the next u0 gather).
template <typename C>
__global__ void __launch_bounds__(kThreads)
    k_b2_mr(int64_t n, C* __restrict__ x, C* __restrict__ r0, const C* __restrict__ r1, const C* __restrict__ r2,
            C* __restrict__ u0, const C* __restrict__ u1, const C* __restrict__ u2, const C* __restrict__ rt,
            KState* __restrict__ st, int* __restrict__ active, double2* __restrict__ part,
            unsigned* __restrict__ cnt) {
    RHS_LOOP_SETUP(active)
    const C g1 = from2<C>(st[r].gamma1), g2 = from2<C>(st[r].omega);
    DotAcc<C> d[2];
    for (int64_t i = i0; i < n; i += stride) {
        const C a = r0[off + i], b = r1[off + i];
        x[off + i] = cadd(x[off + i], cadd(cmul(g1, a), cmul(g2, b)));
        const C rn = csub(a, cadd(cmul(g1, b), cmul(g2, r2[off + i])));
        r0[off + i] = rn;
        u0[off + i] = csub(u0[off + i], cadd(cmul(g1, u1[off + i]), cmul(g2, u2[off + i])));
        d[0].add_cdot(rt[off + i], rn);
        d[1].add_norm2(rn);
    }
    double2 acc[2];
    block_totals<C, 2>(d, acc);
    if (last_block_total_reduced<2>(acc, part + (int64_t)r * gridDim.x * 2, cnt + r) && threadIdx.x == 0) {
        KState& s = st[r];
        const double rn = sqrt(acc[1].x);
        s.rnorm = rn;
        s.iter += 1;
        if (!isfinite(rn) || !finite2(acc[0])) {
            stop(s, active, r, KS_NONFINITE);
        } else if (rn <= s.tol_abs) {
            stop(s, active, r, KS_CONVERGED);
        } else if (s.iter >= s.maxit) {
            stop(s, active, r, KS_MAXIT);
        } else if ((acc[0].x == 0.0 && acc[0].y == 0.0) || (s.omega.x == 0.0 && s.omega.y == 0.0) ||
                   (s.rho.x == 0.0 && s.rho.y == 0.0)) {
            stop(s, active, r, KS_BREAKDOWN);
        } else {
            // beta = alpha rho' / (-omega rho), stored negated
            s.beta = cmul(s.alpha, zdiv(acc[0], cmul(s.omega, s.rho)));
            s.omega = make_double2(0.0, 0.0);
            s.rho = acc[0];
        }
    }
}

#undef RHS_LOOP_SETUP

constexpr KernelKind kind_of(int bytes) { return bytes == 8 ? KK_KRYLOV_C64 : KK_KRYLOV_C128; }

}  // namespace

template <typename C>
cudaError_t BiCGstab2Ops<C>::r0(int R, int64_t n, C* r0_, const C* u1, C* x, const C* u0_, const KState* st,
                                const int* active, cudaStream_t s) {
    PROF_BEGIN(s);
    k_b2_r0<C><<<dim3(reduce_blocks(n), R), kThreads, 0, s>>>(n, r0_, u1, x, u0_, st, active);
    PROF_END(kind_of(sizeof(C)), R, s);
    return cudaGetLastError();
}

template <typename C>
cudaError_t BiCGstab2Ops<C>::rho(int R, int64_t n, const C* rt, const C* r1, KState* st, int* active,
                                 double2* part, unsigned* cnt, cudaStream_t s) {
    PROF_BEGIN(s);
    k_b2_rho<C><<<dim3(reduce_blocks(n), R), kThreads, 0, s>>>(n, rt, r1, st, active, part, cnt);
    PROF_END(kind_of(sizeof(C)), R, s);
    return cudaGetLastError();
}

template <typename C>
cudaError_t BiCGstab2Ops<C>::r1(int R, int64_t n, C* r0_, C* r1_, C* u0_, const C* u1_, const C* u2,
                                C* x, const KState* st, const int* active, cudaStream_t s) {
    PROF_BEGIN(s);
    k_b2_r1<C><<<dim3(reduce_blocks(n), R), kThreads, 0, s>>>(n, r0_, r1_, u0_, u1_, u2, x, st, active);
    PROF_END(kind_of(sizeof(C)), R, s);
    return cudaGetLastError();
}

template <typename C>
cudaError_t BiCGstab2Ops<C>::gram(int R, int64_t n, const C* r0_, const C* r1_, const C* r2, KState* st,
                                  int* active, double2* part, unsigned* cnt, cudaStream_t s) {
    PROF_BEGIN(s);
    k_b2_gram<C><<<dim3(reduce_blocks(n), R), kThreads, 0, s>>>(n, r0_, r1_, r2, st, active, part, cnt);
    PROF_END(kind_of(sizeof(C)), R, s);
    return cudaGetLastError();
}

template <typename C>
cudaError_t BiCGstab2Ops<C>::mr(int R, int64_t n, C* x, C* r0_, const C* r1_, const C* r2, C* u0_, const C* u1_,
                                const C* u2, const C* rt, KState* st, int* active, double2* part, unsigned* cnt,
                                cudaStream_t s) {
    PROF_BEGIN(s);
    k_b2_mr<C><<<dim3(reduce_blocks(n), R), kThreads, 0, s>>>(n, x, r0_, r1_, r2, u0_, u1_, u2, rt, st, active,
                                                               part, cnt);
    PROF_END(kind_of(sizeof(C)), R, s);
    return cudaGetLastError();
}

template struct BiCGstab2Ops<float2>;
template struct BiCGstab2Ops<double2>;

}  // namespace dda
