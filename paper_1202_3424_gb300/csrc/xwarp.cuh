// x passes of the FFT-convolution matvec with warp-local pencils (complex64).
//
// The x passes transform rows of the padded lattice, which are contiguous in
// both of their buffers: the rows (z, y < ny) of U [nz][Ly][Lx] (RowMap in
// matvec_impl.cuh), and the compact site vectors,
// where the occupied sites of one lattice row have consecutive indices.  So a
// row can be held by NT <= 32 consecutive lanes of one warp and read and
// written straight from and to global memory in the layout of the first and
// last radix stage (lane u holds positions u + q NT + j L/R, which are
// consecutive across the lanes): the loads and the scatter coalesce without
// staging the rows in shared memory, and the exchanges between radix stages
// need only warp barriers.  Each pencil has its own exchange plane; the
// exchange after stage S stores and loads position pos at the slot
// pos ^ ((pos >> K) & 15), with K chosen per exchange by the shared-memory
// bank model (paper_1202_3424_gb300/bank_model.py, --warp) so that both the
// stride patterns of the stores and the consecutive loads keep every bank to
// one word per wavefront.
//
// Radix plans: variant 0 is the plan of the staged x passes; variant 1, where
// it exists, trades registers for fewer exchanges (radix 16 or 32, or radix 8
// with more points per lane); the last variant of 64, 128, 256 and 512 points
// is a two-stage plan whose exchange runs by warp shuffles.  The context
// times the variants inside whole matvecs and keeps the fastest (see
// pick_schedule in abi.cu).
#pragma once

#include "fft.cuh"
#include "krylov_dev.cuh"

namespace dda {

template <int L, int V> struct XwPlan;
template <> struct XwPlan<16, 0> : PlanDef<16, 4, 4, 4> {};
template <> struct XwPlan<32, 0> : PlanDef<32, 4, 4, 8> {};
template <> struct XwPlan<48, 0> : PlanDef<48, 4, 4, 4, 3> {};
template <> struct XwPlan<64, 0> : PlanDef<64, 8, 8, 8> {};
template <> struct XwPlan<96, 0> : PlanDef<96, 8, 4, 4, 3, 2> {};
template <> struct XwPlan<128, 0> : PlanDef<128, 16, 4, 4, 8> {};
template <> struct XwPlan<128, 1> : PlanDef<128, 8, 8, 16> {};
template <> struct XwPlan<192, 0> : PlanDef<192, 16, 4, 4, 4, 3> {};
template <> struct XwPlan<192, 1> : PlanDef<192, 8, 8, 8, 3> {};
template <> struct XwPlan<256, 0> : PlanDef<256, 32, 4, 8, 8> {};
template <> struct XwPlan<256, 1> : PlanDef<256, 16, 16, 16> {};
template <> struct XwPlan<384, 0> : PlanDef<384, 32, 4, 4, 4, 3, 2> {};
template <> struct XwPlan<512, 0> : PlanDef<512, 32, 8, 8, 8> {};
template <> struct XwPlan<512, 1> : PlanDef<512, 16, 32, 16> {};
// Warp-shuffle variants: the two-stage plans (8 x 8, 8 x 16, 16 x 16,
// 32 x 16) with their one exchange done by shuffles between the pencil's
// lanes (shfl_transpose in fft.cuh) instead of the shared-memory plane.
template <class B> struct ShflPlan : B {
    static constexpr bool kShuffle = true;
};
template <> struct XwPlan<64, 1> : ShflPlan<PlanDef<64, 8, 8, 8>> {};
template <> struct XwPlan<128, 2> : ShflPlan<PlanDef<128, 8, 8, 16>> {};
template <> struct XwPlan<256, 2> : ShflPlan<PlanDef<256, 16, 16, 16>> {};
template <> struct XwPlan<512, 2> : ShflPlan<PlanDef<512, 16, 32, 16>> {};

template <class PL, class = void> struct xw_shfl : std::false_type {};
template <class PL> struct xw_shfl<PL, std::void_t<decltype(PL::kShuffle)>> : std::bool_constant<PL::kShuffle> {};

// Number of plan variants per length.
__host__ __device__ constexpr int xw_variants(int L) {
    return (L == 128 || L == 256 || L == 512) ? 3 : ((L == 64 || L == 192) ? 2 : 1);
}

// Exchange-plane swizzle key K of the exchange after stage S (0: none).
__host__ __device__ constexpr int warp_swizzle_key(int L, int NT, int DIR, int S) {
    // (table of bank_model.py --warp)
    if (L == 16 && NT == 4 && DIR == -1 && S == 0) return 1;
    if (L == 16 && NT == 4 && DIR == 1 && S == 0) return 1;
    if (L == 32 && NT == 4 && DIR == -1 && S == 0) return 1;
    if (L == 32 && NT == 4 && DIR == 1 && S == 0) return 2;
    if (L == 48 && NT == 4 && DIR == -1 && S == 0) return 1;
    if (L == 64 && NT == 8 && DIR == -1 && S == 0) return 3;
    if (L == 64 && NT == 8 && DIR == 1 && S == 0) return 3;
    if (L == 96 && NT == 8 && DIR == -1 && S == 0) return 2;
    if (L == 96 && NT == 8 && DIR == -1 && S == 1) return 2;
    if (L == 96 && NT == 8 && DIR == 1 && S == 0) return 1;
    if (L == 96 && NT == 8 && DIR == 1 && S == 2) return 3;
    if (L == 128 && NT == 8 && DIR == -1 && S == 0) return 3;
    if (L == 128 && NT == 8 && DIR == 1 && S == 0) return 4;
    if (L == 128 && NT == 16 && DIR == -1 && S == 0) return 2;
    if (L == 128 && NT == 16 && DIR == -1 && S == 1) return 2;
    if (L == 128 && NT == 16 && DIR == 1 && S == 0) return 3;
    if (L == 128 && NT == 16 && DIR == 1 && S == 1) return 2;
    if (L == 192 && NT == 8 && DIR == -1 && S == 0) return 3;
    if (L == 192 && NT == 8 && DIR == 1 && S == 1) return 2;
    if (L == 192 && NT == 16 && DIR == -1 && S == 0) return 2;
    if (L == 192 && NT == 16 && DIR == -1 && S == 1) return 2;
    if (L == 192 && NT == 16 && DIR == 1 && S == 2) return 3;
    if (L == 256 && NT == 16 && DIR == -1 && S == 0) return 4;
    if (L == 256 && NT == 16 && DIR == 1 && S == 0) return 4;
    if (L == 256 && NT == 32 && DIR == -1 && S == 0) return 2;
    if (L == 256 && NT == 32 && DIR == -1 && S == 1) return 3;
    if (L == 256 && NT == 32 && DIR == 1 && S == 0) return 3;
    if (L == 256 && NT == 32 && DIR == 1 && S == 1) return 3;
    if (L == 384 && NT == 32 && DIR == -1 && S == 0) return 2;
    if (L == 384 && NT == 32 && DIR == -1 && S == 1) return 2;
    if (L == 384 && NT == 32 && DIR == 1 && S == 0) return 1;
    if (L == 384 && NT == 32 && DIR == 1 && S == 3) return 3;
    if (L == 512 && NT == 16 && DIR == -1 && S == 0) return 5;
    if (L == 512 && NT == 16 && DIR == 1 && S == 0) return 4;
    if (L == 512 && NT == 32 && DIR == -1 && S == 0) return 3;
    if (L == 512 && NT == 32 && DIR == -1 && S == 1) return 3;
    if (L == 512 && NT == 32 && DIR == 1 && S == 0) return 3;
    if (L == 512 && NT == 32 && DIR == 1 && S == 1) return 3;
    return 0;
}
// Plane padding (elements) per pencil width: with NT < 16 several pencils
// share a half-warp, and the padding puts their planes on different banks.
__host__ __device__ constexpr int warp_plane_pad(int NT) {
    // (table of bank_model.py --warp)
    if (NT == 4) return 8;
    if (NT == 8) return 8;
    if (NT == 16) return 0;
    if (NT == 32) return 0;
    return 0;
}

template <class PL> struct WarpSwz {
    static constexpr bool kShuffle = false;
    template <int DIR, int S> __device__ __forceinline__ static int map(int pos) {
        constexpr int K = warp_swizzle_key(PL::L, PL::NT, DIR, S);
        if constexpr (K == 0) return pos;
        else return pos ^ ((pos >> K) & 15);
    }
};

// Block sizes: the x-forward runs 256 threads; the x-inverse 128, so that
// the block reduction of its fused BiCGstab dot products waits for 4 warps,
// not 8 (the barrier stall of the 256-thread blocks was the second largest).
constexpr int kXwThreads = 256;
constexpr int kXwiThreads = 128;
template <class PL> __host__ __device__ constexpr int xw_rows() { return kXwThreads / PL::NT; }
template <class PL> __host__ __device__ constexpr int xwi_rows() { return kXwiThreads / PL::NT; }
// (the shuffle variants need no exchange plane)
template <class PL> __host__ __device__ constexpr int xw_plane() {
    return xw_shfl<PL>::value ? 0 : PL::L + warp_plane_pad(PL::NT);
}
template <class PL> using XwExchange = std::conditional_t<xw_shfl<PL>::value, ShflExchange, WarpSwz<PL>>;
// exchange planes of the block's rows, then the twiddle table
template <class PL> __host__ __device__ constexpr size_t xw_smem() {
    return ((size_t)xw_rows<PL>() * xw_plane<PL>() + (PL::L <= 256 ? PL::L : 0)) * sizeof(float2);
}
// register budgets (blocks per SM): 64 per thread up to 8 points per lane,
// then 85, then 128; the inverse keeps its diagonal operands in registers and
// takes the larger budget above 12 points per lane
template <class PL> __host__ __device__ constexpr int xwf_min_blocks() { return PL::E <= 8 ? 4 : (PL::E <= 16 ? 3 : 2); }
template <class PL> __host__ __device__ constexpr int xwi_min_blocks() {
    return PL::E <= 8 ? 8 : (PL::E <= 12 ? 6 : (PL::E <= 16 ? 4 : 2));
}
// the second BiCGstab scatter (MODE 2) keeps rhat and five sums besides: the
// next larger budget (85 registers at 8 points per lane, 102 at 12)
template <class PL, int MODE> __host__ __device__ constexpr int xwi_mode_min_blocks() {
    return MODE != 2 ? xwi_min_blocks<PL>() : (PL::E <= 8 ? 6 : (PL::E <= 12 ? 5 : xwi_min_blocks<PL>()));
}

// Up to 256 points the block copies the twiddle table to shared memory
// (after its global loads are issued): the stage twiddles of different lanes
// then cost shared wavefronts, not one L1 request per cache line they touch
// (measured: 192-point rows 2-5 % faster).  The 512-point rows read the
// table from global memory: there the block barrier of the copy cost 15 %.
template <int L> __host__ __device__ constexpr bool xw_shared_twiddles() { return L <= 256; }
template <int L> __device__ __forceinline__ const float2* stage_twiddles(float2* tws, const float2* __restrict__ tw) {
    if constexpr (!xw_shared_twiddles<L>()) {
        return tw;
    } else {
        for (int e = threadIdx.x; e < L; e += kXwThreads) tws[e] = tw[e];
        __syncthreads();
        return tws;
    }
}

// ---- x-forward: gather + row FFT, warp-local pencils -------------------------------
// Same result as k_xfwd: rows (iy, iz) of the padded-to-LX/2 lattice, sites
// x < LX/2 gathered through the lattice -> site map; MODE 1-3 form the
// BiCGstab update in the gather and write it back (fused_gather).
template <int LX, int V, int MODE>
__global__ void __launch_bounds__(kXwThreads, xwf_min_blocks<XwPlan<LX, V>>())
    k_xfwd_w(float2* __restrict__ X, float2* __restrict__ U, RowMap rm, const int* __restrict__ site_of, int nrows,
             int64_t N, const float2* __restrict__ tw, const int* __restrict__ active, FwdVecs<float2> fv) {
    using C = float2;
    using PL = XwPlan<LX, V>;
    constexpr int NT = PL::NT, E = PL::E, NX = LX / 2, RPB = xw_rows<PL>(), PS = xw_plane<PL>();
    constexpr int R0 = stage_radix<PL, -1>(0), NB0 = E / R0, JN = R0 / 2;  // half-zero first stage
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int c = blockIdx.y, r = blockIdx.z;
    if (active != nullptr && active[r] == 0) return;
    const int p = threadIdx.x / NT, u = threadIdx.x % NT;
    const int row = blockIdx.x * RPB + p;
    const bool ok = row < nrows;
    C* plane = reinterpret_cast<C*>(smem_raw) + p * PS;
    const int64_t off = ((int64_t)r * 3 + c) * N;
    C* xs = X + off;
    const GatherScalars<C> gs = gather_scalars<MODE, C>(fv.st, r);
    // site indices of the first stage's inputs (positions < LX/2), then the
    // values: all loads of the lane are in flight before the first is used
    int sidx[NB0 * JN];
#pragma unroll
    for (int q = 0; q < NB0; ++q)
#pragma unroll
        for (int j = 0; j < JN; ++j)
            sidx[q * JN + j] = ok ? site_of[(int64_t)row * NX + u + q * NT + j * (LX / R0)] : -1;
    // the twiddle table goes to shared memory while loads are in flight: in
    // the fused modes, which use their gathered values at once (the update is
    // stored), behind the site-index loads, so that the copy's block barrier
    // does not wait for the slowest warp's gathers; in MODE 0 behind the
    // gathers themselves
    const C* tws = tw;
    if constexpr (MODE != 0) tws = stage_twiddles<LX>(reinterpret_cast<C*>(smem_raw) + RPB * PS, tw);
    C v[E];
    Gathered<C> gv[MODE == 3 ? NB0 * JN : 1];  // (MODE 3 keeps r and x for the stores)
#pragma unroll
    for (int q = 0; q < NB0; ++q)
#pragma unroll
        for (int j = 0; j < JN; ++j) {
            const int s = sidx[q * JN + j];
            Gathered<C> o;
            o.val = czero<C>();
            if (s >= 0) o = fused_gather<MODE>(xs, fv, off, s, gs);
            v[q * R0 + j] = o.val;
            if constexpr (MODE == 3) gv[q * JN + j] = o;
        }
    if constexpr (MODE != 0) {
#pragma unroll
        for (int q = 0; q < NB0; ++q)
#pragma unroll
            for (int j = 0; j < JN; ++j) {
                const int s = sidx[q * JN + j];
                if (s < 0) continue;
                Gathered<C> o;
                if constexpr (MODE == 3) o = gv[q * JN + j];
                else o.val = v[q * R0 + j];
                fused_store<MODE>(xs, fv, off, s, o);
            }
    }
    if constexpr (MODE == 0) tws = stage_twiddles<LX>(reinterpret_cast<C*>(smem_raw) + RPB * PS, tw);
    auto ld = [&](int pos) { return plane[pos]; };
    auto stf = [&](int pos, C val) { plane[pos] = val; };
    fft_stages<C, PL, -1, 0, decltype(ld), decltype(stf), true, XwExchange<PL>>(v, u, tws, ld, stf, true);
    C* out = U + rm.at(r, c, ok ? row : 0, LX);
    for_each_out<PL, -1, false>(u, [&](int idx, int pos) {
        if (ok) out[pos] = v[idx];
    });
}

// ---- x-inverse: row IFFT + diagonal + scatter, warp-local pencils --------------
// Same result as k_xinv (Y = conv + (1/alpha) X at the occupied sites, the
// DIAG kinds, and the fused BiCGstab reductions of MODE 1 and 2).
template <int LX, int V, int MODE, int DIAG>
__global__ void __launch_bounds__(kXwiThreads, (xwi_mode_min_blocks<XwPlan<LX, V>, MODE>()))
    k_xinv_w(const float2* __restrict__ U, RowMap rm, float2* __restrict__ Y, const float2* __restrict__ X,
             const int* __restrict__ site_of, const uint8_t* __restrict__ comp_of, const float2* __restrict__ beta,
             int beta_stride, const int* __restrict__ rows, int nrows, int64_t N, const float2* __restrict__ tw,
             int* __restrict__ active,
             const float2* __restrict__ krhat, KState* __restrict__ st, double2* __restrict__ part,
             unsigned* __restrict__ cnt, int part_stride) {
    using C = float2;
    using PL = XwPlan<LX, V>;
    constexpr int NT = PL::NT, E = PL::E, NX = LX / 2, RPB = xwi_rows<PL>(), PS = xw_plane<PL>();
    constexpr int R0 = stage_radix<PL, +1>(0), NB0 = E / R0;
    constexpr int RL = stage_radix<PL, +1>(PL::NS - 1), NBL = E / RL, MN = RL / 2, NO = NBL * MN;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int c = blockIdx.y, r = blockIdx.z;
    if (active != nullptr && active[r] == 0) return;
    const int p = threadIdx.x / NT, u = threadIdx.x % NT;
    // row list entry blockIdx.x * RPB + p (rows: the rows with sites, else all)
    const int li = blockIdx.x * RPB + p;
    const bool ok = li < nrows;
    const int row = ok ? (rows != nullptr ? rows[li] : li) : 0;
    C* plane = reinterpret_cast<C*>(smem_raw) + p * PS;
    const int64_t off = ((int64_t)r * 3 + c) * N;
    const C* xs = X + off;
    C* ys = Y + off;
    constexpr bool TENSOR = DIAG == kDiagTensor;
    const C* br = beta + (int64_t)r * beta_stride + (TENSOR ? c * (beta_stride / 3) : 0);
    const C* in = U + rm.at(r, c, ok ? row : 0, LX);
    // the row in the first stage's layout, then the site indices of the
    // lattice-half outputs and (up to 12 points per lane) the diagonal
    // operands: their latency is hidden by the transform
    C v[E];
#pragma unroll
    for (int q = 0; q < NB0; ++q)
#pragma unroll
        for (int j = 0; j < R0; ++j) v[q * R0 + j] = ok ? in[u + q * NT + j * (LX / R0)] : czero<C>();
    int sidx[NO];
#pragma unroll
    for (int q = 0; q < NBL; ++q)
#pragma unroll
        for (int m = 0; m < MN; ++m)
            sidx[q * MN + m] = ok ? site_of[(int64_t)row * NX + u + q * NT + m * (LX / RL)] : -1;
    // (with 16 or more points per lane the transform needs those registers:
    // the operands are then loaded after it)
    constexpr bool kHoist = E <= 12;
    C xv[NO], bv[NO];
    C kh[MODE != 0 ? NO : 1];
    auto load_operands = [&]() {
#pragma unroll
        for (int k = 0; k < NO; ++k) {
            const int s = sidx[k];
            xv[k] = czero<C>();
            bv[k] = czero<C>();
            if constexpr (MODE != 0) kh[k] = czero<C>();
            if (s >= 0) {
                xv[k] = xs[s];
                bv[k] = diag_entry<DIAG>(br, comp_of, s, c);
                if constexpr (MODE != 0) kh[k] = krhat[off + s];
            }
        }
    };
    if constexpr (kHoist) load_operands();
    auto ld = [&](int pos) { return plane[pos]; };
    auto stf = [&](int pos, C val) { plane[pos] = val; };
    fft_stages<C, PL, +1, 0, decltype(ld), decltype(stf), true, XwExchange<PL>>(v, u, tw, ld, stf, false);
    if constexpr (!kHoist) load_operands();
    DotAcc<C> d[4];
#pragma unroll
    for (int q = 0; q < NBL; ++q)
#pragma unroll
        for (int m = 0; m < MN; ++m) {
            const int k = q * MN + m, s = sidx[k];
            if (s >= 0) {
                C yv = cadd(v[q * RL + m], cmul(bv[k], xv[k]));
                if constexpr (TENSOR) {  // the two off-diagonal entries of row c
                    const C* bb = br + comp_of[s] * 3;
                    const int c1 = c == 0 ? 1 : 0, c2 = c == 2 ? 1 : 2;
                    const C* xr = X + (int64_t)r * 3 * N;
                    yv = cadd(yv, cadd(cmul(bb[c1], xr[c1 * N + s]), cmul(bb[c2], xr[c2 * N + s])));
                }
                ys[s] = yv;
                if constexpr (MODE == 1) d[0].add_cdot(kh[k], yv);
                if constexpr (MODE == 2) fused_dots_t(d, yv, xv[k], kh[k]);
            }
        }
    if constexpr (MODE != 0) fused_partials<C, MODE>(d, part, r, part_stride);
}

}  // namespace dda
