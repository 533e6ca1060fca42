// QMR for complex symmetric A = A^T (Freund 1992; the guide's QMRCCG option,
// "Choice of Iterative Algorithm"), one matvec per iteration and RHS, without
// look-ahead.
//
// Lanczos with the bilinear form v^T w (no conjugate):
//   w = A v_n;  alpha = v_n^T w / delta_n;
//   v~ = w - alpha v_n - gamma_n v_{n-1};  beta' = |v~|;  v_{n+1} = v~ / beta';
//   delta_{n+1} = v_{n+1}^T v_{n+1};  gamma_{n+1} = beta' delta_{n+1} / delta_n,
// so A V_n = V_{n+1} H_n with H_n tridiagonal.  x_n = x_0 + V_n z_n minimizes
// the quasi-residual |beta_1 e_1 - H_n z|: the new column (gamma, alpha,
// beta') of H goes through the last two Givens rotations, a new rotation
// zeroes beta', and
//   p_n = (v_n - dlt p_{n-1} - eps p_{n-2}) / rho,  A p_n likewise from w,
//   x += t p_n,  r -= t A p_n   (t = c t~, t~ <- -conj(s) t~).
// Per iteration: the matvec, then three kernels (alpha; the Lanczos vector
// with the rotations; the updates with |r| and the convergence test).
// Without look-ahead the bilinear Lanczos process loses accuracy when
// v^T v becomes small against |v|^2 = 1, which complex64 vectors meet much
// earlier than complex128 ones; a solve whose |r| has not reached a new
// minimum for kQmrStall iterations stops (status MAXIT), so that the
// refinement loop restarts it from the true residual.
// Scalars are FP64 in KState::q; the last block of each reduction updates
// them on the device (graph-replayable, per-RHS masks).  Vectors rotate
// through two slots each (v, p, A p), so the host swaps pointers every
// iteration and a graph of an even number of iterations replays.
#include <math.h>

#include "internal.h"
#include "krylov.h"
#include "krylov_dev.cuh"
#include "profiler.h"

namespace dda {

namespace {

constexpr int kThreads = 256;
constexpr int kQmrStall = 40;

#define QMR_LOOP_SETUP(active)                                          \
    const int r = blockIdx.y;                                           \
    if (active != nullptr && active[r] == 0) return;                    \
    const int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;  \
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;             \
    const int64_t off = (int64_t)r * n;

// += a^T b (bilinear: no conjugate)
template <typename C> __device__ __forceinline__ void add_bdot(DotAcc<C>& d, C a, C b) {
    d.re += a.x * b.x - a.y * b.y;
    d.im += a.x * b.y + a.y * b.x;
}

__device__ __forceinline__ double2 dscale(double2 a, double f) { return make_double2(a.x * f, a.y * f); }
__device__ __forceinline__ double2 dconj(double2 a) { return make_double2(a.x, -a.y); }
__device__ __forceinline__ bool dzero(double2 a) { return a.x == 0.0 && a.y == 0.0; }

__device__ __forceinline__ void stop(KState& s, int* active, int r, int status) {
    s.status = status;
    active[r] = 0;
}

// v = r / |r|; v_prev = A p_{-1} = A p_0 = 0 (p slots were zeroed by k_init); delta = v^T v.
template <typename C>
__global__ void __launch_bounds__(kThreads)
    k_qmr_init(int64_t n, const C* __restrict__ r_, C* __restrict__ v, C* __restrict__ v_prev, C* __restrict__ ap1,
               C* __restrict__ ap2, KState* __restrict__ st, int* __restrict__ active, double2* __restrict__ part,
               unsigned* __restrict__ cnt) {
    QMR_LOOP_SETUP(active)
    using T = typename real_of<C>::type;
    const T f = (T)(1.0 / st[r].bnorm);
    DotAcc<C> d[1];
    for (int64_t i = i0; i < n; i += stride) {
        const C vi = cscale(r_[off + i], f);
        v[off + i] = vi;
        v_prev[off + i] = czero<C>();
        ap1[off + i] = czero<C>();
        ap2[off + i] = czero<C>();
        add_bdot(d[0], vi, vi);
    }
    double2 acc[1];
    block_totals<C, 1>(d, acc);
    if (last_block_total_reduced<1>(acc, part + (int64_t)r * gridDim.x, cnt + r) && threadIdx.x == 0) {
        KState& s = st[r];
        QmrScalars& q = s.q;
        q.delta = acc[0];
        q.delta_prev = make_double2(1.0, 0.0);
        q.gamma = q.alpha = make_double2(0.0, 0.0);
        q.s1 = q.s2 = make_double2(0.0, 0.0);
        q.c1 = q.c2 = 1.0;
        q.tt = make_double2(s.bnorm, 0.0);
        q.inv_beta = 0.0;
        q.lanczos_breakdown = 0;
        q.best = s.bnorm;
        q.best_iter = 0;
        if (!finite2(acc[0])) stop(s, active, r, KS_NONFINITE);
        else if (dzero(acc[0])) stop(s, active, r, KS_BREAKDOWN);
    }
}

// alpha = v^T w / delta
template <typename C>
__global__ void __launch_bounds__(kThreads)
    k_qmr_alpha(int64_t n, const C* __restrict__ v, const C* __restrict__ w, KState* __restrict__ st,
                int* __restrict__ active, double2* __restrict__ part, unsigned* __restrict__ cnt) {
    QMR_LOOP_SETUP(active)
    DotAcc<C> d[1];
    for (int64_t i = i0; i < n; i += stride) add_bdot(d[0], v[off + i], w[off + i]);
    double2 acc[1];
    block_totals<C, 1>(d, acc);
    if (last_block_total_reduced<1>(acc, part + (int64_t)r * gridDim.x, cnt + r) && threadIdx.x == 0) {
        KState& s = st[r];
        if (!finite2(acc[0])) stop(s, active, r, KS_NONFINITE);
        else s.q.alpha = zdiv(acc[0], s.q.delta);
    }
}

// v~ = w - alpha v - gamma v_prev (into the v_prev slot); |v~|^2, v~^T v~;
// the new column of H through the rotations; the next Lanczos scalars.
template <typename C>
__global__ void __launch_bounds__(kThreads)
    k_qmr_lanczos(int64_t n, const C* __restrict__ w, const C* __restrict__ v, C* __restrict__ v_prev,
                  KState* __restrict__ st, int* __restrict__ active, double2* __restrict__ part,
                  unsigned* __restrict__ cnt) {
    QMR_LOOP_SETUP(active)
    const C alpha = from2<C>(st[r].q.alpha), gamma = from2<C>(st[r].q.gamma);
    DotAcc<C> d[2];
    for (int64_t i = i0; i < n; i += stride) {
        const C vt = csub(csub(w[off + i], cmul(alpha, v[off + i])), cmul(gamma, v_prev[off + i]));
        v_prev[off + i] = vt;
        d[0].add_norm2(vt);
        add_bdot(d[1], vt, vt);
    }
    double2 acc[2];
    block_totals<C, 2>(d, acc);
    if (last_block_total_reduced<2>(acc, part + (int64_t)r * gridDim.x * 2, cnt + r) && threadIdx.x == 0) {
        KState& s = st[r];
        QmrScalars& q = s.q;
        if (!finite2(acc[0]) || !finite2(acc[1])) {
            stop(s, active, r, KS_NONFINITE);
            return;
        }
        const double bn = sqrt(acc[0].x);
        const double2 eps = cmul(q.s2, q.gamma);  // G_{n-2} on rows n-2, n-1
        const double2 h1 = dscale(q.gamma, q.c2);
        const double2 dlt = cadd(dscale(h1, q.c1), cmul(q.s1, q.alpha));  // G_{n-1} on rows n-1, n
        const double2 tau = csub(dscale(q.alpha, q.c1), cmul(dconj(q.s1), h1));
        const double at = hypot(tau.x, tau.y);
        double c;
        double2 sn;
        if (at == 0.0) {
            c = 0.0;
            sn = make_double2(1.0, 0.0);
        } else {
            c = at / hypot(at, bn);
            sn = dscale(zdiv(make_double2(bn, 0.0), dconj(tau)), c);
        }
        const double2 rho = cadd(dscale(tau, c), dscale(sn, bn));
        q.t = dscale(q.tt, c);
        q.tt = cmul(make_double2(-sn.x, sn.y), q.tt);  // -conj(s) t~
        q.rho = rho;
        q.dlt = dlt;
        q.eps = eps;
        q.c2 = q.c1;
        q.s2 = q.s1;
        q.c1 = c;
        q.s1 = sn;
        if (dzero(rho)) {
            stop(s, active, r, KS_BREAKDOWN);
        } else if (bn > 0.0) {
            const double2 dn = dscale(acc[1], 1.0 / (bn * bn));  // v_{n+1}^T v_{n+1}
            q.gamma = cmul(make_double2(bn, 0.0), zdiv(dn, q.delta));
            q.delta_prev = q.delta;
            q.delta = dn;
            q.inv_beta = 1.0 / bn;
            q.lanczos_breakdown = dzero(dn);
        } else {
            q.inv_beta = 0.0;  // invariant subspace: this step's iterate is exact
        }
    }
}

// p = (v - dlt p1 - eps p2) / rho into p2;  A p likewise from w into ap2;
// x += t p;  r -= t A p;  v_next = v~ / beta' in place;  |r|^2 and the test.
template <typename C>
__global__ void __launch_bounds__(kThreads)
    k_qmr_update(int64_t n, const C* __restrict__ v, C* __restrict__ vt, const C* __restrict__ w,
                 const C* __restrict__ p1, C* __restrict__ p2, const C* __restrict__ ap1, C* __restrict__ ap2,
                 C* __restrict__ x, C* __restrict__ r_, KState* __restrict__ st, int* __restrict__ active,
                 double2* __restrict__ part, unsigned* __restrict__ cnt) {
    QMR_LOOP_SETUP(active)
    using T = typename real_of<C>::type;
    const QmrScalars& qs = st[r].q;
    const double2 ir = zdiv(make_double2(1.0, 0.0), qs.rho);
    const C irho = from2<C>(ir), dlt = from2<C>(qs.dlt), eps = from2<C>(qs.eps), t = from2<C>(qs.t);
    const T ib = (T)qs.inv_beta;
    DotAcc<C> d[1];
    for (int64_t i = i0; i < n; i += stride) {
        const C p = cmul(irho, csub(csub(v[off + i], cmul(dlt, p1[off + i])), cmul(eps, p2[off + i])));
        const C ap = cmul(irho, csub(csub(w[off + i], cmul(dlt, ap1[off + i])), cmul(eps, ap2[off + i])));
        p2[off + i] = p;
        ap2[off + i] = ap;
        x[off + i] = cadd(x[off + i], cmul(t, p));
        const C rn = csub(r_[off + i], cmul(t, ap));
        r_[off + i] = rn;
        vt[off + i] = cscale(vt[off + i], ib);
        d[0].add_norm2(rn);
    }
    double2 acc[1];
    block_totals<C, 1>(d, acc);
    if (last_block_total_reduced<1>(acc, part + (int64_t)r * gridDim.x, cnt + r) && threadIdx.x == 0) {
        KState& s = st[r];
        const double rn = sqrt(acc[0].x);
        s.rnorm = rn;
        s.iter += 1;
        if (rn < s.q.best) {
            s.q.best = rn;
            s.q.best_iter = s.iter;
        }
        if (!isfinite(rn)) stop(s, active, r, KS_NONFINITE);
        else if (rn <= s.tol_abs) stop(s, active, r, KS_CONVERGED);
        else if (s.iter >= s.maxit || s.iter - s.q.best_iter >= kQmrStall) stop(s, active, r, KS_MAXIT);
        else if (s.q.inv_beta == 0.0 || s.q.lanczos_breakdown) stop(s, active, r, KS_BREAKDOWN);
    }
}

#undef QMR_LOOP_SETUP

constexpr KernelKind kind_of(int bytes) { return bytes == 8 ? KK_KRYLOV_C64 : KK_KRYLOV_C128; }

}  // namespace

template <typename C>
cudaError_t QmrOps<C>::init(int R, int64_t n, const C* r, C* v, C* v_prev, C* ap1, C* ap2, KState* st, int* active,
                            double2* part, unsigned* cnt, cudaStream_t s) {
    PROF_BEGIN(s);
    k_qmr_init<C><<<dim3(reduce_blocks(n), R), kThreads, 0, s>>>(n, r, v, v_prev, ap1, ap2, st, active, part, cnt);
    PROF_END(kind_of(sizeof(C)), R, s);
    return cudaGetLastError();
}

template <typename C>
cudaError_t QmrOps<C>::alpha(int R, int64_t n, const C* v, const C* w, KState* st, int* active, double2* part,
                             unsigned* cnt, cudaStream_t s) {
    PROF_BEGIN(s);
    k_qmr_alpha<C><<<dim3(reduce_blocks(n), R), kThreads, 0, s>>>(n, v, w, st, active, part, cnt);
    PROF_END(kind_of(sizeof(C)), R, s);
    return cudaGetLastError();
}

template <typename C>
cudaError_t QmrOps<C>::lanczos(int R, int64_t n, const C* w, const C* v, C* v_prev, KState* st, int* active,
                               double2* part, unsigned* cnt, cudaStream_t s) {
    PROF_BEGIN(s);
    k_qmr_lanczos<C><<<dim3(reduce_blocks(n), R), kThreads, 0, s>>>(n, w, v, v_prev, st, active, part, cnt);
    PROF_END(kind_of(sizeof(C)), R, s);
    return cudaGetLastError();
}

template <typename C>
cudaError_t QmrOps<C>::update(int R, int64_t n, const C* v, C* vt, const C* w, const C* p1, C* p2, const C* ap1,
                              C* ap2, C* x, C* r, KState* st, int* active, double2* part, unsigned* cnt,
                              cudaStream_t s) {
    PROF_BEGIN(s);
    k_qmr_update<C><<<dim3(reduce_blocks(n), R), kThreads, 0, s>>>(n, v, vt, w, p1, p2, ap1, ap2, x, r, st, active,
                                                                    part, cnt);
    PROF_END(kind_of(sizeof(C)), R, s);
    return cudaGetLastError();
}

template struct QmrOps<float2>;
template struct QmrOps<double2>;

}  // namespace dda
