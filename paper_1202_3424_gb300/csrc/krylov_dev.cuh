// Device-side pieces of the BiCGstab solve shared by the Krylov kernels and
// the matvec passes that fuse Krylov updates into their gather/scatter:
// dot-product accumulators, block and last-block reductions (FP64 totals
// per right-hand side, with an atomic ticket so that the last block to
// finish updates the per-RHS scalars on the device), and the scalar updates.
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
    constexpr int UN = ND <= 2 ? 8 : 2;
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
        s.alpha = zdiv(s.rho, sig);
    }
}

// omega = <t, s> / <t, t>  (0 when t = 0: then s = 0 and the update converges)
__device__ __forceinline__ void finalize_omega(KState* st, int* active, int r, double2 ts, double tt) {
    KState& s = st[r];
    if (!finite2(ts) || !isfinite(tt)) {
        s.status = KS_NONFINITE;
        active[r] = 0;
    } else {
        s.omega = tt > 0.0 ? make_double2(ts.x / tt, ts.y / tt) : make_double2(0.0, 0.0);
    }
}

}  // namespace dda
