// Device-side pieces of the BiCGstab solve shared by the Krylov kernels and
// the matvec passes that fuse Krylov updates into their gather/scatter:
// dot-product accumulators, block and last-block reductions (FP64 totals
// per right-hand side, with an atomic ticket so that the last block to
// finish updates the per-RHS scalars on the device), the partial sums of the
// fused passes and the per-RHS kernel that sums them (k_fused_finalize), and
// the scalar updates.
#pragma once

#include <math.h>

#include "common.cuh"
#include "krylov.h"

namespace dda {

// ---- reductions ------------------------------------------------------------------
// Block sum of ND complex partials.  Warp-level sums run in the precision of
// the partials (float for complex64 vectors: FP64 shuffles and adds run at
// ~1/60 of the FP32 rate here); the per-warp results are summed in FP64.
template <typename R, int ND>
__device__ __forceinline__ void block_reduce(R (&vx)[ND], R (&vy)[ND], double2 (&out)[ND]) {
    __shared__ double2 sh[32 * ND];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int d = 0; d < ND; ++d)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            vx[d] += __shfl_xor_sync(0xffffffffu, vx[d], o);
            vy[d] += __shfl_xor_sync(0xffffffffu, vy[d], o);
        }
    __syncthreads();
    if (lane == 0)
#pragma unroll
        for (int d = 0; d < ND; ++d) sh[warp * ND + d] = make_double2((double)vx[d], (double)vy[d]);
    __syncthreads();
#pragma unroll
    for (int d = 0; d < ND; ++d) out[d] = make_double2(0.0, 0.0);
    if (threadIdx.x == 0)
        for (int w = 0; w < nw; ++w)
#pragma unroll
            for (int d = 0; d < ND; ++d) {
                out[d].x += sh[w * ND + d].x;
                out[d].y += sh[w * ND + d].y;
            }
}

template <int ND>
__device__ __forceinline__ void block_reduce(double2 (&v)[ND]) {
    double vx[ND], vy[ND];
#pragma unroll
    for (int d = 0; d < ND; ++d) {
        vx[d] = v[d].x;
        vy[d] = v[d].y;
    }
    block_reduce<double, ND>(vx, vy, v);
}

// Ticket of the last-block reduction: an acquire-release add at GPU scope.
// The release publishes the partials this thread stored before it; the
// acquire (of the block that draws the last ticket) makes every block's
// partials visible to that block, whose other threads read them after a
// barrier, so no sequentially consistent fence (__threadfence) is needed.
__device__ __forceinline__ unsigned ticket_acq_rel(unsigned* counter) {
    unsigned t;
    asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], 1;" : "=r"(t) : "l"(counter) : "memory");
    return t;
}

// Store this block's partial sums (block totals already in thread 0's v[])
// as partial `bid` of `nblocks`; the last block to arrive gets the grand
// totals in thread 0's v[] and returns true (in every thread of that block).
template <int ND>
__device__ __forceinline__ bool last_block_combine(double2 (&v)[ND], double2* partials, unsigned* counter, int bid,
                                                   int nblocks) {
    __shared__ bool is_last;
    if (threadIdx.x == 0) {
#pragma unroll
        for (int d = 0; d < ND; ++d) partials[bid * ND + d] = v[d];
        is_last = (ticket_acq_rel(counter) == (unsigned)nblocks - 1);
    }
    __syncthreads();
    if (!is_last) return false;
    // the partials are read UN per thread at a time, all loads issued before
    // the first add: this block's combine is the launch's serial tail, and a
    // loop with one load per trip waits one L2 latency per trip (the sums
    // keep their order: partial b0 + k * blockDim.x is added k-th)
    constexpr int UN = ND <= 2 ? 8 : (ND <= 4 ? 4 : 2);
    double2 s[ND];
#pragma unroll
    for (int d = 0; d < ND; ++d) s[d] = make_double2(0.0, 0.0);
    for (int b0 = threadIdx.x; b0 < nblocks; b0 += UN * blockDim.x) {
        double2 q[UN][ND];
#pragma unroll
        for (int k = 0; k < UN; ++k) {
            const int b = b0 + k * blockDim.x;
#pragma unroll
            for (int d = 0; d < ND; ++d) q[k][d] = b < nblocks ? __ldcg(&partials[b * ND + d]) : make_double2(0.0, 0.0);
        }
#pragma unroll
        for (int k = 0; k < UN; ++k)
#pragma unroll
            for (int d = 0; d < ND; ++d) {
                s[d].x += q[k][d].x;
                s[d].y += q[k][d].y;
            }
    }
    block_reduce<ND>(s);
#pragma unroll
    for (int d = 0; d < ND; ++d) v[d] = s[d];
    if (threadIdx.x == 0) *counter = 0u;
    return true;
}

// One partial per block of a 1-D grid over the RHS's elements.
template <int ND>
__device__ __forceinline__ bool last_block_total_reduced(double2 (&v)[ND], double2* partials, unsigned* counter) {
    return last_block_combine<ND>(v, partials, counter, blockIdx.x, gridDim.x);
}

// Same, starting from per-thread FP64 partials.
template <int ND>
__device__ __forceinline__ bool last_block_total(double2 (&v)[ND], double2* partials, unsigned* counter) {
    block_reduce<ND>(v);
    return last_block_total_reduced<ND>(v, partials, counter);
}

__device__ __forceinline__ bool finite2(double2 a) { return isfinite(a.x) && isfinite(a.y); }

// Per-thread dot-product accumulator in the vector precision; the block
// reduction sums warps in that precision and warp totals in FP64.  A thread
// sees a few elements per RHS (see reduce_blocks), so FP32 partial sums keep
// ~1e-6 relative accuracy, ample for the Krylov scalars of the inner solve.
template <typename C> struct DotAcc {
    using T = typename real_of<C>::type;
    T re = 0, im = 0;
    __device__ __forceinline__ void add_cdot(C a, C b) {  // += conj(a) * b
        re += a.x * b.x + a.y * b.y;
        im += a.x * b.y - a.y * b.x;
    }
    __device__ __forceinline__ void add_norm2(C a) { re += a.x * a.x + a.y * a.y; }
    __device__ __forceinline__ void add_norms(C a, C b) {  // re += |a|^2, im += |b|^2
        re += a.x * a.x + a.y * a.y;
        im += b.x * b.x + b.y * b.y;
    }
};

// Block totals of ND accumulators (result valid in thread 0).
template <typename C, int ND>
__device__ __forceinline__ void block_totals(DotAcc<C> (&a)[ND], double2 (&out)[ND]) {
    using T = typename real_of<C>::type;
    T vx[ND], vy[ND];
#pragma unroll
    for (int d = 0; d < ND; ++d) {
        vx[d] = a[d].re;
        vy[d] = a[d].im;
    }
    block_reduce<T, ND>(vx, vy, out);
}

__device__ __forceinline__ double2 zdiv(double2 a, double2 b) {
    const double d = b.x * b.x + b.y * b.y;
    return make_double2((a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d);
}

template <typename C> __device__ __forceinline__ C from2(double2 a) {
    C r;
    r.x = (typename real_of<C>::type)a.x;
    r.y = (typename real_of<C>::type)a.y;
    return r;
}

// The finalizers update the fields they own in place: a copy of the whole
// per-RHS state would take its registers in every kernel that inlines them.

// a / b with one division (FP64 divisions take ~550 cycles here, and the
// finalizers run in the serial tail of a launch)
__device__ __forceinline__ double2 zdiv1(double2 a, double2 b) {
    const double id = 1.0 / (b.x * b.x + b.y * b.y);
    return make_double2((a.x * b.x + a.y * b.y) * id, (a.y * b.x - a.x * b.y) * id);
}

// sigma = <rhat, v>  ->  alpha = rho / sigma (breakdown if sigma == 0)
__device__ __forceinline__ void finalize_alpha(KState* st, int* active, int r, double2 sig) {
    KState& s = st[r];
    if (!finite2(sig)) {
        s.status = KS_NONFINITE;
        active[r] = 0;
    } else if (sig.x == 0.0 && sig.y == 0.0) {
        s.status = KS_BREAKDOWN;
        active[r] = 0;
    } else {
        s.alpha = zdiv1(s.rho, sig);
    }
}

// The end of a BiCGstab iteration, from sums over the new t = A s:
//   omega = <t, s> / <t, t>            (0 when t = 0: then s = 0)
//   r'    = s - omega t                (formed by the next x-forward gather)
//   |r'|^2 = <s, s> - |<t, s>|^2 / <t, t>
//   rho'  = <rhat, r'> = <rhat, s> - omega <rhat, t>
//   beta  = (rho' / rho) (alpha / omega)
// then the stopping tests of the iteration (converged, iteration limit,
// breakdown rho' = 0 or omega = 0).  A RHS that stops here still owes its
// x the update alpha p + omega s (pending: KrylovOps::finish_x applies it);
// one that goes on gets it, with r', in the next x-forward gather.
__device__ __forceinline__ void finalize_omega_rho(KState* st, int* active, int r, double2 ts, double tt, double ss,
                                                   double2 rs, double2 rt) {
    KState& s = st[r];
    if (!finite2(ts) || !isfinite(tt) || !isfinite(ss) || !finite2(rs) || !finite2(rt)) {
        s.status = KS_NONFINITE;
        active[r] = 0;
        return;
    }
    // (the FP64 divisions are the long steps of this serial code: the two
    // below are independent, 1/|rho omega|^2 being tt^2 / (|rho|^2 |ts|^2))
    const double its2 = 1.0 / ((s.rho.x * s.rho.x + s.rho.y * s.rho.y) * (ts.x * ts.x + ts.y * ts.y));
    const double itt = tt > 0.0 ? 1.0 / tt : 0.0;
    const double2 om = make_double2(ts.x * itt, ts.y * itt);
    const double rn2 = ss - (ts.x * ts.x + ts.y * ts.y) * itt;
    const double rn = sqrt(rn2 > 0.0 ? rn2 : 0.0);
    const double2 rho1 = make_double2(rs.x - (om.x * rt.x - om.y * rt.y), rs.y - (om.x * rt.y + om.y * rt.x));
    s.omega = om;
    s.rnorm = rn;
    s.iter += 1;
    int status = KS_RUNNING;
    if (rn <= s.tol_abs) status = KS_CONVERGED;
    else if (s.iter >= s.maxit) status = KS_MAXIT;
    else if ((rho1.x == 0.0 && rho1.y == 0.0) || (om.x == 0.0 && om.y == 0.0)) status = KS_BREAKDOWN;
    if (status != KS_RUNNING) {
        s.status = status;
        s.pending = 1;
        active[r] = 0;
    } else {
        // (rho'/rho)(alpha/omega) = rho' alpha conj(rho omega) / |rho omega|^2
        const double2 ro = cmul(s.rho, om);
        const double2 num = cmul(cmul(rho1, s.alpha), make_double2(ro.x, -ro.y));
        const double sc = its2 * tt * tt;
        s.beta = make_double2(num.x * sc, num.y * sc);
        s.rho = rho1;
    }
}

// The sums of the second BiCGstab scatter at one site (t = A s there):
// <t, s>, (<t, t>, <s, s>), <rhat, s>, <rhat, t>.
template <typename C> __device__ __forceinline__ void fused_dots_t(DotAcc<C> (&d)[4], C t, C s, C rh) {
    d[0].add_cdot(t, s);
    d[1].add_norms(t, s);
    d[2].add_cdot(rh, s);
    d[3].add_cdot(rh, t);
}
// Sums per block of the fused x-inverse passes: 1 (MODE 1: sigma) or 4
// (MODE 2: the five sums of fused_dots_t) complex values.
template <int MODE> __host__ __device__ constexpr int fused_sums() { return MODE == 1 ? 1 : 4; }

// The fused x-inverse passes end by writing block totals, which
// k_fused_finalize (the next launch) sums before it updates the scalars.  (A
// last-block combine inside the pass -- an atomic ticket every block waits
// for, then one block summing thousands of partials and running the FP64
// finalizer -- held the pass up to twice as long on the 64^3 sphere.)
//
// FP64 arithmetic runs at 1/64 of the FP32 rate here (a warp-wide add issues
// every 16 cycles per SM, and takes 64 cycles), so for complex64 vectors the
// sums above the warp level are double-float (dfl, FP32 pairs with ~48-bit
// mantissas): a block total is stored as four floats (hi, lo of the real and
// of the imaginary part) in the slot of one double2, and only the final
// total is converted to FP64 for the scalar updates.  Complex128 vectors keep
// FP64 sums throughout.

// Block totals in double-float, valid in thread 0 (complex64 partials).
template <int ND>
__device__ __forceinline__ void block_totals_df(DotAcc<float2> (&a)[ND], dfl (&out)[2 * ND]) {
    __shared__ float sh[32][2 * ND];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    float v[2 * ND];
#pragma unroll
    for (int d = 0; d < ND; ++d) {
        v[2 * d] = a[d].re;
        v[2 * d + 1] = a[d].im;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int k = 0; k < 2 * ND; ++k) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
    __syncthreads();  // (the shared array may still be read by a previous call)
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < 2 * ND; ++k) sh[warp][k] = v[k];
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < 2 * ND; ++k) out[k] = dfl(0.f, 0.f);
        for (int w = 0; w < nw; ++w)
#pragma unroll
            for (int k = 0; k < 2 * ND; ++k) out[k] = out[k] + dfl(sh[w][k], 0.f);
    }
}

// End of a fused x-inverse pass (grid: blocks x, components y, RHS z): the
// block writes its totals as partial blockIdx.y * gridDim.x + blockIdx.x of
// the RHS (ND slots of 16 bytes) and is done.
template <typename C, int MODE>
__device__ __forceinline__ void fused_partials(DotAcc<C> (&d)[4], double2* part, int r, int part_stride) {
    constexpr int ND = fused_sums<MODE>();
    DotAcc<C> dd[ND];
#pragma unroll
    for (int k = 0; k < ND; ++k) dd[k] = d[k];
    double2* pr = part + (int64_t)r * part_stride + (int64_t)(blockIdx.y * gridDim.x + blockIdx.x) * ND;
    if constexpr (sizeof(C) == 8) {
        dfl acc[2 * ND];
        block_totals_df<ND>(dd, acc);
        if (threadIdx.x == 0) {
            float4* pf = reinterpret_cast<float4*>(pr);
#pragma unroll
            for (int k = 0; k < ND; ++k) pf[k] = make_float4(acc[2 * k].hi, acc[2 * k].lo, acc[2 * k + 1].hi, acc[2 * k + 1].lo);
        }
    } else {
        double2 acc[ND];
        block_totals<C, ND>(dd, acc);
        if (threadIdx.x == 0)
#pragma unroll
            for (int k = 0; k < ND; ++k) pr[k] = acc[k];
    }
}

// One block per RHS: the nb partials of a fused x-inverse pass, summed in a
// fixed order (so graph replays reproduce them bit for bit), then the
// scalars (finalize_alpha, finalize_omega_rho).
constexpr int kFinThreads = 256;
__device__ __forceinline__ dfl shfl_xor_dfl(dfl a, int o) {
    return dfl(__shfl_xor_sync(0xffffffffu, a.hi, o), __shfl_xor_sync(0xffffffffu, a.lo, o));
}
template <typename C, int MODE>
__global__ void __launch_bounds__(kFinThreads)
    k_fused_finalize(const double2* __restrict__ part, int part_stride, int nb, KState* __restrict__ st,
                     int* __restrict__ active) {
    constexpr int ND = fused_sums<MODE>();
    const int r = blockIdx.x;
    if (active != nullptr && active[r] == 0) return;
    const double2* pr = part + (int64_t)r * part_stride;
    double2 tot[ND];
    if constexpr (sizeof(C) == 8) {
        // double-float sums: per thread over its partials, then lanes, then warps
        constexpr int UN = 4;
        const float4* pf = reinterpret_cast<const float4*>(pr);
        dfl v[2 * ND];
#pragma unroll
        for (int k = 0; k < 2 * ND; ++k) v[k] = dfl(0.f, 0.f);
        for (int b0 = threadIdx.x; b0 < nb; b0 += UN * kFinThreads) {
            float4 q[UN][ND];
#pragma unroll
            for (int u = 0; u < UN; ++u) {
                const int b = b0 + u * kFinThreads;
#pragma unroll
                for (int d = 0; d < ND; ++d) q[u][d] = b < nb ? pf[(int64_t)b * ND + d] : make_float4(0.f, 0.f, 0.f, 0.f);
            }
#pragma unroll
            for (int u = 0; u < UN; ++u)
#pragma unroll
                for (int d = 0; d < ND; ++d) {
                    v[2 * d] = v[2 * d] + dfl(q[u][d].x, q[u][d].y);
                    v[2 * d + 1] = v[2 * d + 1] + dfl(q[u][d].z, q[u][d].w);
                }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
#pragma unroll
            for (int k = 0; k < 2 * ND; ++k) v[k] = v[k] + shfl_xor_dfl(v[k], o);
        constexpr int NW = kFinThreads / 32;
        __shared__ dfl sh[NW][2 * ND];
        const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
        if (lane == 0)
#pragma unroll
            for (int k = 0; k < 2 * ND; ++k) sh[w][k] = v[k];
        __syncthreads();
        if (w != 0) return;
        // warp 0 combines the NW warp totals with a shuffle tree as well
#pragma unroll
        for (int k = 0; k < 2 * ND; ++k) v[k] = lane < NW ? sh[lane][k] : dfl(0.f, 0.f);
#pragma unroll
        for (int o = NW / 2; o > 0; o >>= 1)
#pragma unroll
            for (int k = 0; k < 2 * ND; ++k) v[k] = v[k] + shfl_xor_dfl(v[k], o);
        if (lane != 0) return;
#pragma unroll
        for (int d = 0; d < ND; ++d) tot[d] = make_double2((double)v[2 * d], (double)v[2 * d + 1]);
    } else {
        double2 s[ND];
#pragma unroll
        for (int d = 0; d < ND; ++d) s[d] = make_double2(0.0, 0.0);
        for (int b = threadIdx.x; b < nb; b += kFinThreads)
#pragma unroll
            for (int d = 0; d < ND; ++d) {
                const double2 q = pr[(int64_t)b * ND + d];
                s[d].x += q.x;
                s[d].y += q.y;
            }
        block_reduce<ND>(s);
        if (threadIdx.x != 0) return;
#pragma unroll
        for (int d = 0; d < ND; ++d) tot[d] = s[d];
    }
    if constexpr (MODE == 1) finalize_alpha(st, active, r, tot[0]);
    else finalize_omega_rho(st, active, r, tot[0], tot[1].x, tot[1].y, tot[2], tot[3]);
}

// Per-RHS scalars of the fused x-forward gathers (see FwdVecs).
template <typename C> struct GatherScalars {
    C a, b, c;
    bool first;
};
template <int MODE, typename C> __device__ __forceinline__ GatherScalars<C> gather_scalars(const KState* st, int r) {
    GatherScalars<C> g{czero<C>(), czero<C>(), czero<C>(), false};
    if constexpr (MODE == 1) {
        g.a = from2<C>(st[r].beta);
        g.b = from2<C>(st[r].omega);
    } else if constexpr (MODE == 2) {
        g.a = from2<C>(st[r].alpha);
    } else if constexpr (MODE == 3) {
        g.first = st[r].iter == 0;
        g.a = from2<C>(st[r].alpha);
        g.b = from2<C>(st[r].omega);
        g.c = from2<C>(st[r].beta);
    }
    return g;
}
// MODE 3 at one site, the previous iteration's end and this one's start:
//   r <- s - omega t,  x <- x + alpha p + omega s,  p <- r + beta (p - omega v)
// (the first iteration of a solve has no previous one: r <- s = b, x stays 0,
// and beta = 0 with p = v = 0 from the initialization)
template <typename C> struct Upd3 {
    C r, x, p;
};
template <typename C>
__device__ __forceinline__ Upd3<C> upd3(C sv, C tv, C pv, C vv, C xv, const GatherScalars<C>& g) {
    Upd3<C> u;
    u.r = g.first ? sv : csub(sv, cmul(g.b, tv));
    u.x = g.first ? xv : cadd(xv, cadd(cmul(g.a, pv), cmul(g.b, sv)));
    u.p = cadd(u.r, cmul(g.c, csub(pv, cmul(g.b, vv))));
    return u;
}

// Vectors of the fused x-forward gathers: r is read by modes 1 and 2 and
// written by mode 3, which also reads s, t and updates x.
template <typename C> struct FwdVecs {
    C* r;
    const C* v;
    const C* s;
    const C* t;
    C* x;
    const KState* st;
};
// The value an x-forward pass gathers at site s (off: the RHS and component
// row of the site vectors) and, for MODE 3, the r and x it writes back.
template <typename C> struct Gathered {
    C val, r, x;
};
template <int MODE, typename C>
__device__ __forceinline__ Gathered<C> fused_gather(const C* __restrict__ xs, const FwdVecs<C>& f, int64_t off,
                                                    int64_t s, const GatherScalars<C>& g) {
    Gathered<C> o;
    if constexpr (MODE == 0) {
        o.val = xs[s];
    } else if constexpr (MODE == 1) {
        o.val = cadd(f.r[off + s], cmul(g.a, csub(xs[s], cmul(g.b, f.v[off + s]))));
    } else if constexpr (MODE == 2) {
        o.val = csub(f.r[off + s], cmul(g.a, f.v[off + s]));
    } else {
        const Upd3<C> u = upd3(f.s[off + s], f.t[off + s], xs[s], f.v[off + s], f.x[off + s], g);
        o.val = u.p;
        o.r = u.r;
        o.x = u.x;
    }
    return o;
}
// Its stores: the gathered vector back to X (modes 1-3), and r and x (MODE 3).
template <int MODE, typename C>
__device__ __forceinline__ void fused_store(C* __restrict__ xs, const FwdVecs<C>& f, int64_t off, int64_t s,
                                            const Gathered<C>& o) {
    if constexpr (MODE != 0) xs[s] = o.val;
    if constexpr (MODE == 3) {
        f.r[off + s] = o.r;
        f.x[off + s] = o.x;
    }
}

}  // namespace dda
