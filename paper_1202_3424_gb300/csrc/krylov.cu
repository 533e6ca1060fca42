// BiCGstab vector kernels, FP64 reductions, incident field, cross-section
// sums and the adjoint-gradient kernels of the DDA solve.
//
// Solver: unpreconditioned BiCGstab (van der Vorst 1992), the family of the
// guide's recommended PBCGS2/PBCGST ("Choice of Iterative Algorithm"), for
// complex A x = b, one independent iteration per right-hand side:
//   p = r + beta (p - omega v);  v = A p;  alpha = rho / <rhat, v>;
//   s = r - alpha v;  t = A s;  omega = <t, s> / <t, t>;
//   x += alpha p + omega s;  r = s - omega t;  rho' = <rhat, r>;
//   beta = (rho'/rho)(alpha/omega).
// In the solve these updates ride in the matvec passes (internal.h,
// FusedKrylov): the gather of the first matvec forms the previous
// iteration's r and x and the new p, the second matvec's scatter sums
// <t, s>, <t, t>, <s, s>, <rhat, s>, <rhat, t>, from which |r'|^2 =
// <s, s> - |<t, s>|^2 / <t, t> and rho' = <rhat, s> - omega <rhat, t>
// (krylov_dev.cuh: finalize_omega_rho); k_finish_x applies the last x
// update of a RHS that stopped.
// Vectors are complex64 or complex128; every scalar (rho, alpha, omega,
// beta, norms) is FP64.  The iteration's sums are written as partials by the
// x-inverse blocks and summed per RHS, in a fixed order, by k_fused_finalize
// (krylov_dev.cuh), which also updates the scalars; the reductions of this
// file (initial rho, norms, Q sums) write one FP64 partial per block and the
// last block of each (atomic ticket) sums them.  Either way the scalars stay
// on the device, so an iteration needs no host round trip and can be
// replayed as a CUDA graph.  A RHS whose `active` flag is 0 is skipped by
// every kernel (per-RHS convergence masking).
#include <math.h>

#include "internal.h"
#include "krylov.h"
#include "krylov_dev.cuh"
#include "profiler.h"

namespace dda {

static constexpr int kThreads = 256;

#define RHS_PROLOGUE(active)                                    \
    const int r = blockIdx.y;                                   \
    if (active != nullptr && active[r] == 0) return;            \
    const int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; \
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;

// ---- inner-solve kernels ---------------------------------------------------------
// x = 0, r = rhat = b (and s = b when given), p = v = 0;  |b|^2 -> scalars.
template <typename C>
__global__ void __launch_bounds__(kThreads)
    k_init(int64_t n, const C* __restrict__ b, C* __restrict__ x, C* __restrict__ r_, C* __restrict__ rhat,
           C* __restrict__ p, C* __restrict__ v, C* __restrict__ s_, KState* __restrict__ st,
           const double* __restrict__ tol_rel, const int* __restrict__ want, int* __restrict__ active,
           double2* __restrict__ part, unsigned* __restrict__ cnt) {
    const int r = blockIdx.y;
    const int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x, stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t off = (int64_t)r * n;
    DotAcc<C> d[1];
    for (int64_t i = i0; i < n; i += stride) {
        const C bi = b[off + i];
        x[off + i] = czero<C>();
        r_[off + i] = bi;
        rhat[off + i] = bi;
        p[off + i] = czero<C>();
        v[off + i] = czero<C>();
        if (s_ != nullptr) s_[off + i] = bi;
        d[0].add_norm2(bi);
    }
    double2 acc[1];
    block_totals<C, 1>(d, acc);
    if (last_block_total_reduced<1>(acc, part + (int64_t)r * gridDim.x, cnt + r) && threadIdx.x == 0) {
        KState& s = st[r];  // (in place: a copy of the whole state costs registers)
        const double bn = sqrt(acc[0].x);
        s.bnorm = bn;
        s.rnorm = bn;
        s.rho = make_double2(acc[0].x, 0.0);
        s.alpha = s.omega = make_double2(1.0, 0.0);
        s.beta = make_double2(0.0, 0.0);
        s.iter = 0;
        s.tol_abs = tol_rel[r] * bn;
        int run = (want == nullptr || want[r] != 0);
        if (!isfinite(bn)) {
            s.status = KS_NONFINITE;
            run = 0;
        } else if (bn <= s.tol_abs || bn == 0.0) {
            s.status = KS_CONVERGED;
            run = 0;
        } else {
            s.status = run ? KS_RUNNING : KS_IDLE;
        }
        active[r] = run;
    }
}

// x += alpha p + omega s for each RHS whose BiCGstab iteration stopped with
// that update pending (finalize_omega_rho); the others are left alone.
template <typename C>
__global__ void __launch_bounds__(kThreads)
    k_finish_x(int64_t n, C* __restrict__ x, const C* __restrict__ p, const C* __restrict__ s_,
               const KState* __restrict__ st) {
    const int r = blockIdx.y;
    if (!st[r].pending) return;
    const C alpha = from2<C>(st[r].alpha), omega = from2<C>(st[r].omega);
    const int64_t off = (int64_t)r * n;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        x[off + i] = cadd(x[off + i], cadd(cmul(alpha, p[off + i]), cmul(omega, s_[off + i])));
}

__global__ void k_count_active(const int* __restrict__ active, int R, int* __restrict__ out) {
    int c = 0;
    for (int r = threadIdx.x; r < R; r += blockDim.x) c += active[r] != 0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if (threadIdx.x == 0) *out = c;
}

// ---- refinement kernels (FP64 outer vectors) -------------------------------------
// out[r] = sum |v|^2 (or |a - b|^2 into r64 = a - b when b != nullptr)
__global__ void __launch_bounds__(kThreads)
    k_residual(int64_t n, const double2* __restrict__ a, const double2* __restrict__ b, double2* __restrict__ out_vec,
               double* __restrict__ out_norm2, const int* __restrict__ active, double2* __restrict__ part,
               unsigned* __restrict__ cnt) {
    RHS_PROLOGUE(active)
    const int64_t off = (int64_t)r * n;
    double2 acc[1] = {make_double2(0.0, 0.0)};
    for (int64_t i = i0; i < n; i += stride) {
        double2 d = a[off + i];
        if (b != nullptr) d = csub(d, b[off + i]);
        if (out_vec != nullptr) out_vec[off + i] = d;
        acc[0].x += d.x * d.x + d.y * d.y;
    }
    if (last_block_total<1>(acc, part + (int64_t)r * gridDim.x, cnt + r) && threadIdx.x == 0) out_norm2[r] = acc[0].x;
}

// bin = (C)(scale[r] * r64)
template <typename C>
__global__ void __launch_bounds__(kThreads)
    k_to_inner(int64_t n, const double2* __restrict__ r64, C* __restrict__ bin, const double* __restrict__ scale,
               const int* __restrict__ active) {
    RHS_PROLOGUE(active)
    const double sc = scale[r];
    const int64_t off = (int64_t)r * n;
    for (int64_t i = i0; i < n; i += stride) bin[off + i] = from2<C>(cscale(r64[off + i], sc));
}

// x64 += coef[r] * xin
template <typename C>
__global__ void __launch_bounds__(kThreads)
    k_accumulate(int64_t n, double2* __restrict__ x64, const C* __restrict__ xin, const double* __restrict__ coef,
                 const int* __restrict__ active) {
    RHS_PROLOGUE(active)
    const double cf = coef[r];
    const int64_t off = (int64_t)r * n;
    for (int64_t i = i0; i < n; i += stride) {
        const C v = xin[off + i];
        double2 xv = x64[off + i];
        xv.x += cf * (double)v.x;
        xv.y += cf * (double)v.y;
        x64[off + i] = xv;
    }
}

// out = conj(a - b) (b nullable)
__global__ void __launch_bounds__(kThreads)
    k_conj_diff(int64_t n, const double2* __restrict__ a, const double2* __restrict__ b, double2* __restrict__ out) {
    const int r = blockIdx.y;
    const int64_t off = (int64_t)r * n;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double2 d = a[off + i];
        if (b != nullptr) d = csub(d, b[off + i]);
        out[off + i] = make_double2(d.x, -d.y);
    }
}

template <typename D, typename S>
__global__ void k_convert(int64_t n, const S* __restrict__ s, D* __restrict__ d) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        d[i] = ccast<D>(s[i]);
}

// ---- physics kernels -------------------------------------------------------------
// E_inc,j = e exp(i kd khat . r_j), r_j at half-integer offsets about the
// centre of the caller's box (cx, cy, cz); lat_of indexes the extended lattice.
__global__ void __launch_bounds__(kThreads)
    k_einc(int64_t N, const int* __restrict__ lat_of, int nx, int ny, double cx, double cy, double cz, double kd,
           const double* __restrict__ khat, const double2* __restrict__ e, double2* __restrict__ E) {
    const int r = blockIdx.y;
    const double kx = khat[3 * r], ky = khat[3 * r + 1], kz = khat[3 * r + 2];
    const double2 ex = e[3 * r], ey = e[3 * r + 1], ez = e[3 * r + 2];
    double2* Er = E + (int64_t)r * 3 * N;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < N; j += (int64_t)gridDim.x * blockDim.x) {
        const int lat = lat_of[j];
        const int ix = lat % nx, iy = (lat / nx) % ny, iz = lat / (nx * ny);
        const double ph = kd * (kx * (ix - cx) + ky * (iy - cy) + kz * (iz - cz));
        double sn, cs;
        sincos(ph, &sn, &cs);
        const double2 f = make_double2(cs, sn);
        Er[j] = cmul(ex, f);
        Er[N + j] = cmul(ey, f);
        Er[2 * N + j] = cmul(ez, f);
    }
}

// sums[r] = ( sum_j Im(E_j^* . P_j),  sum_j w(comp_j) |P_j|^2 ), or with
// tensor weights (anisotropic 1/alpha tensors B) the quadratic form
// sum_j Im(P_j . B^* P_j^*) - (2/3) k^3 |P_j|^2 written with six real weights
// per composition: w0..w2 |P_a|^2 + w3 Re(P_x P_y^*) + w4 Re(P_x P_z^*) + w5 Re(P_y P_z^*).
__global__ void __launch_bounds__(kThreads)
    k_qsums(int64_t N, const double2* __restrict__ E, const double2* __restrict__ P, const uint8_t* __restrict__ comp_of,
            const double* __restrict__ w, int w_stride, bool tensor, double2* __restrict__ sums,
            double2* __restrict__ part, unsigned* __restrict__ cnt) {
    const int r = blockIdx.y;
    const double2* Er = E + (int64_t)r * 3 * N;
    const double2* Pr = P + (int64_t)r * 3 * N;
    const double* wr = w + (int64_t)r * w_stride;
    double2 acc[1] = {make_double2(0.0, 0.0)};
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < N; j += (int64_t)gridDim.x * blockDim.x) {
        double im = 0.0, p2 = 0.0;
        double2 pv[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const double2 ev = Er[c * N + j];
            pv[c] = Pr[c * N + j];
            im += ev.x * pv[c].y - ev.y * pv[c].x;
            p2 += pv[c].x * pv[c].x + pv[c].y * pv[c].y;
        }
        acc[0].x += im;
        if (tensor) {
            const double* wt = wr + table_index(comp_of, j) * 6;
            double q = 0.0;
#pragma unroll
            for (int c = 0; c < 3; ++c) q += wt[c] * (pv[c].x * pv[c].x + pv[c].y * pv[c].y);
            q += wt[3] * (pv[0].x * pv[1].x + pv[0].y * pv[1].y) + wt[4] * (pv[0].x * pv[2].x + pv[0].y * pv[2].y) +
                 wt[5] * (pv[1].x * pv[2].x + pv[1].y * pv[2].y);
            acc[0].y += q;
        } else {
            acc[0].y += wr[table_index(comp_of, j)] * p2;
        }
    }
    if (last_block_total<1>(acc, part + (int64_t)r * gridDim.x, cnt + r) && threadIdx.x == 0) sums[r] = acc[0];
}

// b_j = w(comp_j) conj(P_j)  (adjoint right-hand side W P^*)
__global__ void __launch_bounds__(kThreads)
    k_adjoint_rhs(int64_t N, const double2* __restrict__ P, const uint8_t* __restrict__ comp_of,
                  const double* __restrict__ w, double2* __restrict__ b) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < N; j += (int64_t)gridDim.x * blockDim.x) {
        const double wj = w[table_index(comp_of, j)];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const double2 pv = P[c * N + j];
            b[c * N + j] = make_double2(wj * pv.x, -wj * pv.y);
        }
    }
}

// dQ/dRe eps_j = K[-|P|^2 Im b' - 2 Re(b' nu.P)],  dQ/dIm eps_j = K[-|P|^2 Re b' + 2 Im(b' nu.P)]
__global__ void __launch_bounds__(kThreads)
    k_grad(int64_t N, const double2* __restrict__ P, const double2* __restrict__ nu, const uint8_t* __restrict__ comp_of,
           const double2* __restrict__ dbeta, double K, double* __restrict__ g_re, double* __restrict__ g_im) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < N; j += (int64_t)gridDim.x * blockDim.x) {
        double p2 = 0.0;
        double2 nup = make_double2(0.0, 0.0);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const double2 pv = P[c * N + j], nv = nu[c * N + j];
            p2 += pv.x * pv.x + pv.y * pv.y;
            nup = cadd(nup, cmul(nv, pv));
        }
        const double2 bp = dbeta[table_index(comp_of, j)];
        const double2 q = cmul(bp, nup);
        g_re[j] = K * (-p2 * bp.y - 2.0 * q.x);
        g_im[j] = K * (-p2 * bp.x + 2.0 * q.y);
    }
}

// ---- host launchers --------------------------------------------------------------
int reduce_blocks(int64_t n) {
    int64_t b = (n + kThreads * 4 - 1) / (kThreads * 4);
    if (b > kMaxReduceBlocks) b = kMaxReduceBlocks;
    return (int)(b < 1 ? 1 : b);
}

template <typename C>
cudaError_t KrylovOps<C>::init(int R, int64_t n, const C* b, C* x, C* r, C* rhat, C* p, C* v, C* s_, KState* st,
                               const double* tol_rel, const int* want, int* active, double2* part, unsigned* cnt,
                               cudaStream_t s) {
    PROF_BEGIN(s);
    k_init<C><<<dim3(reduce_blocks(n), R), kThreads, 0, s>>>(n, b, x, r, rhat, p, v, s_, st, tol_rel, want, active,
                                                              part, cnt);
    PROF_END((sizeof(C) == 8 ? KK_KRYLOV_C64 : KK_KRYLOV_C128), R, s);
    return cudaGetLastError();
}
template <typename C>
cudaError_t KrylovOps<C>::finish_x(int R, int64_t n, C* x, const C* p, const C* s_, const KState* st,
                                   cudaStream_t s) {
    PROF_BEGIN(s);
    k_finish_x<C><<<dim3(reduce_blocks(n), R), kThreads, 0, s>>>(n, x, p, s_, st);
    PROF_END((sizeof(C) == 8 ? KK_KRYLOV_C64 : KK_KRYLOV_C128), R, s);
    return cudaGetLastError();
}
template <typename C>
cudaError_t KrylovOps<C>::to_inner(int R, int64_t n, const double2* r64, C* bin, const double* scale,
                                   const int* active, cudaStream_t s) {
    PROF_BEGIN(s);
    k_to_inner<C><<<dim3(reduce_blocks(n), R), kThreads, 0, s>>>(n, r64, bin, scale, active);
    PROF_END(KK_REFINE, R, s);
    return cudaGetLastError();
}
template <typename C>
cudaError_t KrylovOps<C>::accumulate(int R, int64_t n, double2* x64, const C* xin, const double* coef,
                                     const int* active, cudaStream_t s) {
    PROF_BEGIN(s);
    k_accumulate<C><<<dim3(reduce_blocks(n), R), kThreads, 0, s>>>(n, x64, xin, coef, active);
    PROF_END(KK_REFINE, R, s);
    return cudaGetLastError();
}
template struct KrylovOps<float2>;
template struct KrylovOps<double2>;

cudaError_t launch_count_active(const int* active, int R, int* out, cudaStream_t s) {
    PROF_BEGIN(s);
    k_count_active<<<1, 32, 0, s>>>(active, R, out);
    PROF_END(KK_OTHER, 1, s);
    return cudaGetLastError();
}
cudaError_t launch_residual(int R, int64_t n, const double2* a, const double2* b, double2* out_vec, double* out_norm2,
                            const int* active, double2* part, unsigned* cnt, cudaStream_t s) {
    PROF_BEGIN(s);
    k_residual<<<dim3(reduce_blocks(n), R), kThreads, 0, s>>>(n, a, b, out_vec, out_norm2, active, part, cnt);
    PROF_END(KK_REFINE, R, s);
    return cudaGetLastError();
}
cudaError_t launch_conj_diff(int R, int64_t n, const double2* a, const double2* b, double2* out, cudaStream_t s) {
    PROF_BEGIN(s);
    k_conj_diff<<<dim3(reduce_blocks(n), R), kThreads, 0, s>>>(n, a, b, out);
    PROF_END(KK_REFINE, R, s);
    return cudaGetLastError();
}
cudaError_t launch_c64_to_c128(int64_t n, const float2* s_, double2* d, cudaStream_t s) {
    PROF_BEGIN(s);
    k_convert<double2, float2><<<reduce_blocks(n), kThreads, 0, s>>>(n, s_, d);
    PROF_END(KK_REFINE, 1, s);
    return cudaGetLastError();
}
cudaError_t launch_c128_to_c64v(int64_t n, const double2* s_, float2* d, cudaStream_t s) {
    PROF_BEGIN(s);
    k_convert<float2, double2><<<reduce_blocks(n), kThreads, 0, s>>>(n, s_, d);
    PROF_END(KK_REFINE, 1, s);
    return cudaGetLastError();
}
cudaError_t launch_einc(int R, int64_t N, const int* lat_of, const Geom& g, double kd, const double* khat,
                        const double2* e, double2* E, cudaStream_t s) {
    return launch_einc_at(R, N, lat_of, g.nx, g.ny, 0.5 * (g.ox - 1), 0.5 * (g.oy - 1), 0.5 * (g.oz - 1), kd, khat,
                          e, E, s);
}
cudaError_t launch_einc_at(int R, int64_t N, const int* lat_of, int nx, int ny, double cx, double cy, double cz,
                           double kd, const double* khat, const double2* e, double2* E, cudaStream_t s) {
    PROF_BEGIN(s);
    k_einc<<<dim3(reduce_blocks(N), R), kThreads, 0, s>>>(N, lat_of, nx, ny, cx, cy, cz, kd, khat, e, E);
    PROF_END(KK_EINC, R, s);
    return cudaGetLastError();
}

// ---- near field ----------------------------------------------------------------
// Pbox[r][c][box_of[j]] = P[r][c][j] for the N target sites (Pbox zeroed first).
template <typename C>
__global__ void __launch_bounds__(kThreads)
    k_scatter_sites(int64_t N, int64_t Ne, const int* __restrict__ box_of, const double2* __restrict__ P,
                    C* __restrict__ Pbox) {
    const int r = blockIdx.y;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < N; j += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = box_of[j];
#pragma unroll
        for (int c = 0; c < 3; ++c)
            Pbox[((int64_t)r * 3 + c) * Ne + b] = ccast<C>(P[((int64_t)r * 3 + c) * N + j]);
    }
}
// out = -(double) y  (E_sca = -sum_l A P_l)
template <typename C>
__global__ void __launch_bounds__(kThreads) k_negate_c128(int64_t n, const C* __restrict__ y, double2* __restrict__ out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double2 v = ccast<double2>(y[i]);
        out[i] = make_double2(-v.x, -v.y);
    }
}
template <typename C>
cudaError_t launch_scatter_sites(int R, int64_t N, int64_t Ne, const int* box_of, const double2* P, C* Pbox,
                                 cudaStream_t s) {
    PROF_BEGIN(s);
    k_scatter_sites<C><<<dim3(reduce_blocks(N), R), kThreads, 0, s>>>(N, Ne, box_of, P, Pbox);
    PROF_END(KK_OTHER, R, s);
    return cudaGetLastError();
}
template <typename C> cudaError_t launch_negate_c128(int64_t n, const C* y, double2* out, cudaStream_t s) {
    PROF_BEGIN(s);
    k_negate_c128<C><<<reduce_blocks(n), kThreads, 0, s>>>(n, y, out);
    PROF_END(KK_OTHER, 1, s);
    return cudaGetLastError();
}
template cudaError_t launch_scatter_sites<float2>(int, int64_t, int64_t, const int*, const double2*, float2*,
                                                  cudaStream_t);
template cudaError_t launch_scatter_sites<double2>(int, int64_t, int64_t, const int*, const double2*, double2*,
                                                   cudaStream_t);
template cudaError_t launch_negate_c128<float2>(int64_t, const float2*, double2*, cudaStream_t);
template cudaError_t launch_negate_c128<double2>(int64_t, const double2*, double2*, cudaStream_t);
cudaError_t launch_qsums(int R, int64_t N, const double2* E, const double2* P, const uint8_t* comp_of, const double* w,
                         int w_stride, bool tensor, double2* sums, double2* part, unsigned* cnt, cudaStream_t s) {
    PROF_BEGIN(s);
    k_qsums<<<dim3(reduce_blocks(N), R), kThreads, 0, s>>>(N, E, P, comp_of, w, w_stride, tensor, sums, part, cnt);
    PROF_END(KK_QSUMS, R, s);
    return cudaGetLastError();
}
cudaError_t launch_adjoint_rhs(int64_t N, const double2* P, const uint8_t* comp_of, const double* w, double2* b,
                               cudaStream_t s) {
    PROF_BEGIN(s);
    k_adjoint_rhs<<<reduce_blocks(N), kThreads, 0, s>>>(N, P, comp_of, w, b);
    PROF_END(KK_OTHER, 1, s);
    return cudaGetLastError();
}
cudaError_t launch_grad(int64_t N, const double2* P, const double2* nu, const uint8_t* comp_of, const double2* dbeta,
                        double K, double* g_re, double* g_im, cudaStream_t s) {
    PROF_BEGIN(s);
    k_grad<<<reduce_blocks(N), kThreads, 0, s>>>(N, P, nu, comp_of, dbeta, K, g_re, g_im);
    PROF_END(KK_OTHER, 1, s);
    return cudaGetLastError();
}

}  // namespace dda
