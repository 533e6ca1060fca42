// FFT-convolution matvec of the DDA (Goodman, Draine & Flatau 1990; the
// method behind the guide's eq. AP=E solves, "Choice of FFT Algorithm"):
//
//   (A P)_j = (1/alpha_j) P_j + sum_{l != j} A(r_j - r_l) P_l
//
// The off-diagonal sum is a discrete convolution of P (on the nx*ny*nz
// lattice, zero on vacuum sites) with the six components of the symmetric
// tensor A(r).  Zero-padding every axis to L >= 2n turns it into a circular
// convolution, evaluated as IFFT(Ghat . FFT(P)) restricted to the lattice.
//
// Pass structure (one kernel each, per RHS and component unless noted):
//   x-fwd   gather P from the compact site vector, FFT rows along x (input
//           half zero)           -> rows (z, y < ny) of U [nz][Ly][Lx]
//   y-fwd   FFT along y (input half zero), in place     -> U [nz][Ly][Lx]
//   z-conv  for each (kx,ky) column, all three components: FFT along z
//           (input half zero), multiply by the symmetric 3x3 Ghat in
//           registers, inverse FFT along z, keep z < nz  -> U2 in place
//   y-inv   inverse FFT along y, keep y < ny, in place  -> rows (z, y < ny) of U
//   x-inv   inverse FFT along x, keep x < nx, add (1/alpha) P, scatter to
//           the compact site vector
// Ghat is stored as one octant (k <= L/2 on each axis) of the transformed
// kernel: each component is even or odd under each axis reflection, so
// Ghat(L-k) = +/- Ghat(k).  The 1/(Lx Ly Lz) of the inverse transform is
// folded into Ghat.
//
// This header holds the implementation; one translation unit per arithmetic
// type (matvec_f32.cu, matvec_f64.cu, matvec_df.cu) instantiates it, so that
// the three compile in parallel.
#pragma once

#include <cstdio>
#include <mutex>
#include <type_traits>
#include <unordered_map>

#include "fft.cuh"
#include "internal.h"
#include "krylov_dev.cuh"
#include "profiler.h"
#include "xwarp.cuh"

namespace dda {

// ---- tile sizes ------------------------------------------------------------
// x passes stage TP rows through shared memory (TP+1 stride); strided passes
// take TP adjacent pencils (coalesced across them); the z pass takes TP
// adjacent columns for each of 3 component groups.  ES is the element size
// in bytes.  For complex64 every x and strided tile is at least 16 wide:
// 128-byte row segments in global memory, and (per the shared-memory bank
// model in bank_model.py) no bank conflicts in the exchanges and transposes
// of a (TP+1)-strided x plane, where 4- and 8-wide tiles cost 1.8-1.9x the
// ideal wavefronts.  To fit 16 rows of 512 points in 512 threads the x
// passes then run that length with 32 threads of 16 points.
template <int L, int ES> struct XPlan : Plan<L> {};
template <> struct XPlan<512, 8> : PlanDef<512, 32, 8, 8, 8> {};
template <int L, int ES> __host__ __device__ constexpr int tp_x() {
    constexpr int nt = XPlan<L, ES>::NT;
    const int tp = (256 / nt) > 64 ? 64 : (256 / nt);
    return (ES == 8 && tp < 16) ? 16 : tp;
}
// x-inverse blocks per SM the register budget must allow: at least 1024
// threads (the hoisted scatter operands otherwise take 128 registers and a
// 512-thread block would run alone on its SM)
template <int L, int ES> __host__ __device__ constexpr int xinv_min_blocks() {
    constexpr int threads = tp_x<L, ES>() * XPlan<L, ES>::NT;
    return threads >= 1024 ? 1 : 1024 / threads;
}
// z pass: 3*TP*NT threads per block, TP adjacent columns, and enough blocks
// per SM (registers capped by the launch bound) to hide the latency of the
// strided column loads: measured on GB300, three 384-thread blocks per SM
// were 40 % faster than two on the 192x128x64 grid.  (Blocks of 768 threads
// with 128-byte shared-memory rows, a variant with one warp per pencil and
// staged tiles, and a row swizzle were all measured slower.)
template <int L, typename T> __host__ __device__ constexpr int tp_z() {
    constexpr int nt = ZPlan<L>::NT;
    int tp = nt >= 32 ? 256 / nt : 128 / nt;
    tp = tp > 32 ? 32 : (tp < 4 ? 4 : tp);
    // spectra [3][padded rows] and Green tensor [6][L/2+1] per column, and
    // the twiddle table [L], within 216 KB
    while (tp > 1) {
        const size_t rows = sizeof(cx<T>) == 8 ? exchange_rows8(L, nt, tp) : L;
        if (((size_t)3 * rows + (size_t)6 * (L / 2 + 1)) * tp + L <= 216 * 1024 / sizeof(cx<T>)) break;
        tp /= 2;
    }
    return tp;
}
// (complex128 z passes are FP64-ALU-bound and keep their registers; the
// double-float ones take two 384-thread blocks per SM where their registers
// fit 85 without spilling: the power-of-two lengths up to 128)
template <int L, typename T> __host__ __device__ constexpr int zconv_min_blocks() {
    constexpr int threads = 3 * tp_z<L, T>() * ZPlan<L>::NT;
    if constexpr (std::is_same<T, dfl>::value) return (threads == 384 && (L == 64 || L == 128)) ? 2 : 1;
    return (sizeof(T) == 4 && 2048 / threads >= 3) ? 3 : 1;
}
// Row stride (complex elements) of the z pass's shared-memory planes.
// (Padding rows narrower than 128 bytes by two elements was measured slower
// on the 128^3 grid: it removes the conflicts of stride-4 row patterns but
// creates them for consecutive rows.)
template <int L, typename T> __host__ __device__ constexpr int sp_z() {
    return tp_z<L, T>();
}
template <int L, typename T> __host__ __device__ constexpr int zconv_rows() {
    return exchange_rows<L, ZPlan<L>::NT, sp_z<L, T>(), sizeof(cx<T>)>();
}
template <int L, typename T> __host__ __device__ constexpr size_t zconv_smem() {
    return (((size_t)3 * zconv_rows<L, T>() + (size_t)6 * (L / 2 + 1)) * sp_z<L, T>() + L) * sizeof(cx<T>);
}

// ---- x-forward: gather + row FFT ---------------------------------------------
// Rows (iy, iz) of the padded-to-L/2 lattice; lattice sites x < LX/2.
// MODE 0 gathers X.  With the BiCGstab updates fused into the gather
// (per-RHS scalars from st), the gathered vector is formed on the fly and
// written back to X:  MODE 1  X = p <- r + beta (p - omega v);
//                      MODE 2  X = s <- r - alpha v;
//                      MODE 3  X = p <- r' + beta (p - omega v) with
//                              r' = s - omega t and x += alpha p + omega s
//                              (fused_gather in krylov_dev.cuh).
template <typename T, int LX, int MODE>
__global__ void __launch_bounds__(tp_x<LX, sizeof(cx<T>)>() * XPlan<LX, sizeof(cx<T>)>::NT)
    k_xfwd(cx<T>* __restrict__ X, cx<T>* __restrict__ U, RowMap rm, const int* __restrict__ site_of, int nrows,
           int64_t N, const cx<T>* __restrict__ tw, const int* __restrict__ active, FwdVecs<cx<T>> fv) {
    using C = cx<T>;
    using PL = XPlan<LX, sizeof(cx<T>)>;
    constexpr int TP = tp_x<LX, sizeof(cx<T>)>(), SP = TP + 1, NX = LX / 2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* buf = reinterpret_cast<C*>(smem_raw);
    const int c = blockIdx.y, r = blockIdx.z;
    if (active != nullptr && active[r] == 0) return;
    const int row0 = blockIdx.x * TP;
    const int64_t off = ((int64_t)r * 3 + c) * N;
    C* xs = X + off;
    const GatherScalars<C> gs = gather_scalars<MODE, C>(fv.st, r);
    // The gather runs in three unrolled phases (site indices, then values,
    // then shared-memory stores) so that every load of a thread is in flight
    // at once: the site -> value chain is two dependent memory latencies.
    constexpr int NTH = TP * PL::NT, NG = (TP * NX + NTH - 1) / NTH;
    int sidx[NG];
#pragma unroll
    for (int i = 0; i < NG; ++i) {
        const int e = threadIdx.x + i * NTH, t = e / NX, ix = e - t * NX, row = row0 + t;
        sidx[i] = (e < TP * NX && row < nrows) ? site_of[(int64_t)row * NX + ix] : -1;
    }
    Gathered<C> val[NG];
#pragma unroll
    for (int i = 0; i < NG; ++i) {
        const int s = sidx[i];
        val[i].val = czero<C>();
        if (s >= 0) val[i] = fused_gather<MODE>(xs, fv, off, s, gs);
    }
#pragma unroll
    for (int i = 0; i < NG; ++i) {
        const int e = threadIdx.x + i * NTH, t = e / NX, ix = e - t * NX;
        if (e < TP * NX) buf[ix * SP + t] = val[i].val;
        if (sidx[i] >= 0) fused_store<MODE>(xs, fv, off, sidx[i], val[i]);
    }
    __syncthreads();
    const int t = threadIdx.x % TP, u = threadIdx.x / TP;
    C* bt = buf + t;
    C v[PL::E];
    auto first = [&](int pos) { return bt[pos * SP]; };
    auto ld = [&](int pos) { return bt[pos * SP]; };
    auto stf = [&](int pos, C val) { bt[pos * SP] = val; };
    pencil_fft<C, PL, -1, true>(v, u, tw, first, ld, stf);
    __syncthreads();
    for_each_out<PL, -1, false>(u, [&](int idx, int pos) { bt[pos * SP] = v[idx]; });
    __syncthreads();
    constexpr int NO = (TP * LX + NTH - 1) / NTH;
#pragma unroll
    for (int i = 0; i < NO; ++i) {
        const int e = threadIdx.x + i * NTH, t2 = e / LX, x = e - t2 * LX, row = row0 + t2;
        if (e < TP * LX && row < nrows) U[rm.at(r, c, row, LX) + x] = buf[x * SP + t2];
    }
}

// ---- x-inverse: row IFFT + diagonal + scatter -----------------------------------
// Y = conv + (1/alpha) X at the occupied sites.  DIAG says how a site finds
// its 1/alpha (each kind its own instantiation, so that the common one keeps
// its registers and its load chain):
//   kDiagComp    the scalar of its composition code;
//   kDiagTensor  row c of its composition's tensor, times all three
//                components of X (layout in PadWork::beta_tensor);
//   kDiagSite    the scalar of site s itself, entry s + 1 (per-site materials).  Fused BiCGstab reductions
// (partial sums per block, summed per RHS by k_fused_finalize):
//   MODE 1  Y = v:  sigma = <rhat, v>                    ->  alpha = rho / sigma
//   MODE 2  Y = t:  <t, s>, <t, t>, <s, s>, <rhat, s>,
//                   <rhat, t> with X = s                 ->  finalize_omega_rho
template <typename T, int LX, int MODE, int DIAG>
__global__ void __launch_bounds__(tp_x<LX, sizeof(cx<T>)>() * XPlan<LX, sizeof(cx<T>)>::NT,
                                   xinv_min_blocks<LX, sizeof(cx<T>)>())
    k_xinv(const cx<T>* __restrict__ U, RowMap rm, cx<T>* __restrict__ Y, const cx<T>* __restrict__ X,
           const int* __restrict__ site_of, const uint8_t* __restrict__ comp_of, const cx<T>* __restrict__ beta,
           int beta_stride, const int* __restrict__ rows, int nrows, int64_t N, const cx<T>* __restrict__ tw,
           int* __restrict__ active,
           const cx<T>* __restrict__ krhat, KState* __restrict__ st, double2* __restrict__ part,
           unsigned* __restrict__ cnt, int part_stride) {
    using C = cx<T>;
    using PL = XPlan<LX, sizeof(cx<T>)>;
    constexpr int TP = tp_x<LX, sizeof(cx<T>)>(), SP = TP + 1, NX = LX / 2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* buf = reinterpret_cast<C*>(smem_raw);
    const int c = blockIdx.y, r = blockIdx.z;
    if (active != nullptr && active[r] == 0) return;
    // list entries row0 .. row0 + TP - 1 (rows: the rows with sites, else all)
    const int row0 = blockIdx.x * TP;
    auto row_of = [&](int t2) {
        const int li = row0 + t2;
        return li < nrows ? (rows != nullptr ? rows[li] : li) : -1;
    };
    const int64_t off = ((int64_t)r * 3 + c) * N;
    const C* xs = X + off;
    C* ys = Y + off;
    constexpr bool TENSOR = DIAG == kDiagTensor;
    const C* br = beta + (int64_t)r * beta_stride + (TENSOR ? c * (beta_stride / 3) : 0);
    // All global loads are issued up front: the rows to transform, then the
    // site indices and, behind them, the operands of the diagonal term, whose
    // latency the transform hides.
    constexpr int NTH = TP * PL::NT, NI = (TP * LX + NTH - 1) / NTH, NG = (TP * NX + NTH - 1) / NTH;
    int sidx[NG];
    {
        C rin[NI];
#pragma unroll
        for (int i = 0; i < NI; ++i) {
            const int e = threadIdx.x + i * NTH, t2 = e / LX, x = e - t2 * LX, row = e < TP * LX ? row_of(t2) : -1;
            rin[i] = row >= 0 ? U[rm.at(r, c, row, LX) + x] : czero<C>();
        }
#pragma unroll
        for (int i = 0; i < NG; ++i) {
            const int e = threadIdx.x + i * NTH, t2 = e / NX, ix = e - t2 * NX, row = e < TP * NX ? row_of(t2) : -1;
            sidx[i] = row >= 0 ? site_of[(int64_t)row * NX + ix] : -1;
        }
#pragma unroll
        for (int i = 0; i < NI; ++i) {
            const int e = threadIdx.x + i * NTH, t2 = e / LX, x = e - t2 * LX;
            if (e < TP * LX) buf[x * SP + t2] = rin[i];
        }
    }
    // (with 16 points per thread the transform needs those registers: the
    // operands are then loaded after it)
    constexpr bool kHoist = PL::E <= 12;
    C xv[NG], bv[NG];
    C kh[MODE != 0 ? NG : 1];
    auto load_operands = [&]() {
#pragma unroll
        for (int i = 0; i < NG; ++i) {
            const int s = sidx[i];
            xv[i] = czero<C>();
            bv[i] = czero<C>();
            if constexpr (MODE != 0) kh[i] = czero<C>();
            if (s >= 0) {
                xv[i] = xs[s];
                bv[i] = diag_entry<DIAG>(br, comp_of, s, c);
                if constexpr (MODE != 0) kh[i] = krhat[off + s];
            }
        }
    };
    if constexpr (kHoist) load_operands();
    __syncthreads();
    const int t = threadIdx.x % TP, u = threadIdx.x / TP;
    C* bt = buf + t;
    C v[PL::E];
    auto first = [&](int pos) { return bt[pos * SP]; };
    auto ld = [&](int pos) { return bt[pos * SP]; };
    auto stf = [&](int pos, C val) { bt[pos * SP] = val; };
    pencil_fft<C, PL, +1, false>(v, u, tw, first, ld, stf);
    __syncthreads();
    for_each_out<PL, +1, true>(u, [&](int idx, int pos) { bt[pos * SP] = v[idx]; });
    if constexpr (!kHoist) load_operands();
    __syncthreads();
    DotAcc<C> d[4];
#pragma unroll
    for (int i = 0; i < NG; ++i) {
        const int e = threadIdx.x + i * NTH, t2 = e / NX, ix = e - t2 * NX;
        const int s = sidx[i];
        if (s >= 0) {
            C yv = cadd(buf[ix * SP + t2], cmul(bv[i], xv[i]));
            if constexpr (TENSOR) {  // the two off-diagonal entries of row c
                const C* bb = br + comp_of[s] * 3;
                const int c1 = c == 0 ? 1 : 0, c2 = c == 2 ? 1 : 2;
                const C* xr = X + (int64_t)r * 3 * N;
                yv = cadd(yv, cadd(cmul(bb[c1], xr[c1 * N + s]), cmul(bb[c2], xr[c2 * N + s])));
            }
            ys[s] = yv;
            if constexpr (MODE == 1) d[0].add_cdot(kh[i], yv);
            if constexpr (MODE == 2) fused_dots_t(d, yv, xv[i], kh[i]);
        }
    }
    if constexpr (MODE != 0) fused_partials<C, MODE>(d, part, r, part_stride);
}

// ---- strided pencils (y passes; y and z passes of the Green tensor) -----------
// Pencil (b, w): points at src + b*src_bstride + w + pos*pt_stride; outputs
// to dst likewise.  MODE 0: forward with input positions >= L/2 zero;
// MODE 1: inverse keeping positions < L/2; MODE 2: full forward transform.
// TP pencils adjacent in w per block, so loads and stores coalesce across w.
// Radix plan variant V = 1 (complex64 y passes, tuned like the other passes):
// 128 = 8 x 16, 192 = 8 x 8 x 3, 256 = 16 x 16, 512 = 32 x 16, one exchange
// fewer than the plan of V = 0 at twice (512: four times) the points per thread.  A half-warp always
// covers 16 adjacent pencils at one position, so any position pattern of
// the exchanges is free of bank conflicts.
template <int L, int V> struct SPlan : Plan<L> {};
template <> struct SPlan<128, 1> : PlanDef<128, 8, 8, 16> {};
template <> struct SPlan<192, 1> : PlanDef<192, 8, 8, 8, 3> {};
template <> struct SPlan<256, 1> : PlanDef<256, 16, 16, 16> {};
template <> struct SPlan<512, 1> : PlanDef<512, 16, 32, 16> {};
__host__ __device__ constexpr int s_variants(int L) {
    return (L == 128 || L == 192 || L == 256 || L == 512) ? 2 : 1;
}
template <class PL, int ES> __host__ __device__ constexpr int tp_sp() {
    const int tp = (256 / PL::NT) > 32 ? 32 : ((256 / PL::NT) < 8 ? 8 : (256 / PL::NT));
    return (ES == 8 && tp < 16) ? 16 : tp;
}
template <typename T, int L, int MODE, int V>
__device__ __forceinline__ void strided_body(const cx<T>* src, cx<T>* dst, int64_t pt_stride, int width,
                                             int64_t src_bstride, int64_t dst_bstride, int batches_per_rhs,
                                             const cx<T>* __restrict__ tw, const int* __restrict__ active) {
    using C = cx<T>;
    using PL = SPlan<L, V>;
    constexpr int TP = tp_sp<PL, sizeof(cx<T>)>();
    constexpr int DIR = MODE == 1 ? +1 : -1;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* buf = reinterpret_cast<C*>(smem_raw);
    const int b = blockIdx.y;
    if (active != nullptr && active[b / batches_per_rhs] == 0) return;
    const int t = threadIdx.x % TP, u = threadIdx.x / TP;
    const int w = blockIdx.x * TP + t;
    const bool valid = w < width;
    const C* s = src + (int64_t)b * src_bstride + (valid ? w : 0);
    C* d = dst + (int64_t)b * dst_bstride + (valid ? w : 0);
    C* bt = buf + t;
    C v[PL::E];
    auto first = [&](int pos) { return valid ? s[pos * pt_stride] : czero<C>(); };
    auto ld = [&](int pos) { return bt[exchange_row<L, PL::NT, TP, sizeof(C)>(pos) * TP]; };
    auto st = [&](int pos, C val) { bt[exchange_row<L, PL::NT, TP, sizeof(C)>(pos) * TP] = val; };
    pencil_fft<C, PL, DIR, MODE == 0>(v, u, tw, first, ld, st);
    for_each_out<PL, DIR, MODE == 1>(u, [&](int idx, int pos) {
        if (valid) d[pos * pt_stride] = v[idx];
    });
}
template <typename T, int L, int MODE, int V = 0>
__global__ void __launch_bounds__(tp_sp<SPlan<L, V>, sizeof(cx<T>)>() * SPlan<L, V>::NT)
    k_strided(const cx<T>* src, cx<T>* dst, int64_t pt_stride, int width, int64_t src_bstride, int64_t dst_bstride,
              int batches_per_rhs, const cx<T>* __restrict__ tw, const int* __restrict__ active) {
    strided_body<T, L, MODE, V>(src, dst, pt_stride, width, src_bstride, dst_bstride, batches_per_rhs, tw, active);
}
// The complex64 512-point y passes with the 32 x 16 plan, capped at 80
// registers for three 256-thread blocks per SM (the inverse took 90 and ran
// two: 8.98 -> 8.39 ms on the 256^3 sphere).  The same cap slowed the 128- and
// 192-point passes by 11-14 %, so they keep k_strided.
template <typename T, int L, int MODE, int V = 0>
__global__ void __launch_bounds__(tp_sp<SPlan<L, V>, sizeof(cx<T>)>() * SPlan<L, V>::NT, 3)
    k_strided3(const cx<T>* src, cx<T>* dst, int64_t pt_stride, int width, int64_t src_bstride,
               int64_t dst_bstride, int batches_per_rhs, const cx<T>* __restrict__ tw, const int* __restrict__ active) {
    strided_body<T, L, MODE, V>(src, dst, pt_stride, width, src_bstride, dst_bstride, batches_per_rhs, tw, active);
}
template <typename T, int L, int V> __host__ __device__ constexpr bool strided_capped() {
    return sizeof(cx<T>) == 8 && L == 512 && V == 1;
}

// ---- z pass with the Fourier-space product ------------------------------------
// One block owns TP adjacent (kx) columns at one ky and up to RB right-hand
// sides.  It first stages the Green-tensor entries of its columns in shared
// memory -- kz <= LZ/2 of the octant, with the x and y reflection signs
// already applied -- and reuses them for every RHS.  Per RHS its threads form
// three groups, one per Cartesian component c: group c transforms P_c along z
// (input half zero), writes the spectrum to its shared-memory plane, and
// after a barrier forms row c of the symmetric product
//   Y_c(k) = sum_b Ghat_cb(k) P_b(k)
// for the points it holds, then inverse-transforms Y_c and keeps z < LZ/2.
template <typename T, int LZ, int RB>
__global__ void __launch_bounds__(3 * tp_z<LZ, T>() * ZPlan<LZ>::NT, zconv_min_blocks<LZ, T>())
    k_zconv(cx<T>* __restrict__ U2, const cx<T>* __restrict__ gh, int R, int Lx, int Ly,
            const cx<T>* __restrict__ tw, const int* __restrict__ active) {
    using C = cx<T>;
    using PL = ZPlan<LZ>;
    constexpr int TP = tp_z<LZ, T>(), SP = sp_z<LZ, T>(), NT = PL::NT, NZ = LZ / 2, HZ = LZ / 2 + 1;
    static_assert((TP * NT) % 32 == 0, "component groups must be whole warps");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* buf = reinterpret_cast<C*>(smem_raw);   // spectra [3][ROWS][SP]
    constexpr int ROWS = zconv_rows<LZ, T>();  // padded rows of a spectra plane
    C* gs = buf + 3 * ROWS * SP;               // Green tensor [6][HZ][SP]
    C* tws = gs + 6 * HZ * SP;                 // twiddle table [LZ]
    const int ky = blockIdx.y;
    const int r0 = blockIdx.z * RB;
    const int hx = Lx / 2 + 1, hy = Ly / 2 + 1;
    const int64_t cs = (int64_t)HZ * hy * hx;
    {
        const int kyo = ky <= Ly / 2 ? ky : Ly - ky;
        const bool fy = ky > Ly / 2;
        for (int e = threadIdx.x; e < 6 * HZ * TP; e += blockDim.x) {
            const int tt = e % TP, kz = (e / TP) % HZ, cc = e / (TP * HZ);
            const int kx = blockIdx.x * TP + tt;
            C g = czero<C>();
            if (kx < Lx) {
                const bool fx = kx > Lx / 2;
                const int kxo = fx ? Lx - kx : kx;
                g = gh[cc * cs + ((int64_t)kz * hy + kyo) * hx + kxo];
                // xy is odd in x and y, xz odd in x, yz odd in y (z handled at use)
                const bool flip = (cc == 1 && fx != fy) || (cc == 2 && fx) || (cc == 4 && fy);
                if (flip) g = cscale(g, T(-1));
            }
            gs[(cc * HZ + kz) * SP + tt] = g;
        }
        for (int e = threadIdx.x; e < LZ; e += blockDim.x) tws[e] = tw[e];
    }
    const int t = threadIdx.x % TP;
    const int rest = threadIdx.x / TP;
    const int u = rest % NT, c = rest / NT;
    const int kx = blockIdx.x * TP + t;
    const bool valid = kx < Lx;
    const int64_t plane = (int64_t)Ly * Lx;
    // row c of the symmetric tensor: components (xx,xy,xz,yy,yz,zz); entries
    // that are odd in z change sign for kz > LZ/2
    const int i0 = c == 0 ? 0 : (c == 1 ? 1 : 2);
    const int i1 = c == 0 ? 1 : (c == 1 ? 3 : 4);
    const int i2 = c == 0 ? 2 : (c == 1 ? 4 : 5);
    const bool z0 = (i0 == 2 || i0 == 4), z1 = (i1 == 2 || i1 == 4), z2 = (i2 == 2 || i2 == 4);
    const C* g0 = gs + i0 * HZ * SP + t;
    const C* g1 = gs + i1 * HZ * SP + t;
    const C* g2 = gs + i2 * HZ * SP + t;
    C* sb = buf + c * (ROWS * SP) + t;
    const C* pb = buf + t;
    auto row = [](int pos) { return exchange_row<LZ, NT, SP, sizeof(C)>(pos); };
    auto ld = [&](int pos) { return sb[row(pos) * SP]; };
    auto st = [&](int pos, C val) { sb[row(pos) * SP] = val; };
#pragma unroll 1
    for (int rr = 0; rr < RB; ++rr) {
        const int r = r0 + rr;
        if (r >= R) break;
        if (active != nullptr && active[r] == 0) continue;  // uniform across the block
        C* bc = U2 + ((int64_t)r * 3 + c) * NZ * plane + (int64_t)ky * Lx + (valid ? kx : 0);
        C v[PL::E];
        auto first = [&](int pos) { return valid ? bc[pos * plane] : czero<C>(); };
        __syncthreads();  // Green tile staged / previous RHS done with the spectra
        pencil_fft<C, PL, -1, true>(v, u, tws, first, ld, st);
        __syncthreads();
        for_each_out<PL, -1, false>(u, [&](int idx, int pos) { sb[row(pos) * SP] = v[idx]; });
        __syncthreads();
        for_each_out<PL, -1, false>(u, [&](int idx, int kz) {
            const bool fz = kz > LZ / 2;
            const int kzo = fz ? LZ - kz : kz;
            C a0 = g0[kzo * SP], a1 = g1[kzo * SP], a2 = g2[kzo * SP];
            if (fz) {
                if (z0) a0 = cscale(a0, T(-1));
                if (z1) a1 = cscale(a1, T(-1));
                if (z2) a2 = cscale(a2, T(-1));
            }
            const int kr = row(kz);
            const C pa = pb[kr * SP], pbv = pb[(ROWS + kr) * SP], pc = pb[(2 * ROWS + kr) * SP];
            v[idx] = cdot3(a0, pa, a1, pbv, a2, pc);
        });
        pencil_fft_regs<C, PL, +1>(v, u, tws, ld, st);
        for_each_out<PL, +1, true>(u, [&](int idx, int pos) {
            if (valid) bc[pos * plane] = v[idx];
        });
    }
}

// ---- z pass, register-resident schedule (complex64) ----------------------------
// Same product as k_zconv, but each thread keeps all three components of its
// points in registers: per RHS it transforms P_x, P_y, P_z of its column in
// lockstep (one exchange plane per component, so each stage's twiddles and
// barriers serve all three), forms the 3x3 product in registers (no spectra
// round trip through shared memory), and inverse-transforms.  The global loads of the next RHS are issued before
// the current one is transformed, so one block keeps its column's loads in
// flight while computing.  Shared traffic per point is about half that of
// k_zconv; the price is ~128 registers per thread, so the plan must keep
// L/NT <= 8 points per thread -- or, with radix-16 plan variants (one
// exchange per transform where the plain plan needs two), 16 points per
// thread and no register prefetch of the next RHS.
// Column mapping: a block takes TP adjacent columns kx at one ky and stages
// their Green entries with the signs of the odd components (xy in x and y,
// xz in x, yz in y) folded in; k_zconv_oct below maps octant columns instead.
template <int L, int V> struct ZrPlan : Plan<L> {};
template <> struct ZrPlan<128, 1> : PlanDef<128, 8, 8, 16> {};
template <> struct ZrPlan<256, 1> : PlanDef<256, 16, 16, 16> {};
__host__ __device__ constexpr int zr_variants(int L) { return (L == 128 || L == 256) ? 2 : 1; }
template <int L> __host__ __device__ constexpr bool zreg_ok() { return Plan<L>::E <= 8; }
template <class PL> __host__ __device__ constexpr int tp_zr() {
    int tp = 128 / PL::NT;
    return tp > 32 ? 32 : (tp < 4 ? 4 : tp);
}
template <class PL> __host__ __device__ constexpr int zreg_threads() { return tp_zr<PL>() * PL::NT; }
// 128 registers per thread: 512 / threads blocks per SM; the 16-point
// variants (whose ~100 KB of shared memory allows 2 blocks per SM anyway)
// take the registers of 2 blocks
template <class PL> __host__ __device__ constexpr int zreg_min_blocks() {
    return PL::E > 8 ? 2 : (512 / zreg_threads<PL>() < 1 ? 1 : 512 / zreg_threads<PL>());
}
template <class PL, typename T> __host__ __device__ constexpr int zreg_rows() {
    return exchange_rows<PL::L, PL::NT, tp_zr<PL>(), sizeof(cx<T>)>();
}
template <class PL, typename T> __host__ __device__ constexpr size_t zreg_smem() {
    return (((size_t)3 * zreg_rows<PL, T>() + (size_t)6 * (PL::L / 2 + 1)) * tp_zr<PL>() + PL::L) * sizeof(cx<T>);
}
// k_zconv_oct: one more Green column per tile
template <class PL, typename T> __host__ __device__ constexpr size_t zoct_smem() {
    return zreg_smem<PL, T>() + (size_t)6 * (PL::L / 2 + 1) * sizeof(cx<T>);
}
// the loads of the next RHS are prefetched into registers up to 8 points per thread
template <class PL> __host__ __device__ constexpr bool zreg_prefetch() { return PL::E <= 8; }

template <typename T, int LZ, int RB, int V = 0>
__global__ void __launch_bounds__(zreg_threads<ZrPlan<LZ, V>>(), zreg_min_blocks<ZrPlan<LZ, V>>())
    k_zconv_reg(cx<T>* __restrict__ U2, const cx<T>* __restrict__ gh, int R, int Lx, int Ly,
                const cx<T>* __restrict__ tw, const int* __restrict__ active) {
    using C = cx<T>;
    using PL = ZrPlan<LZ, V>;
    constexpr int TP = tp_zr<PL>(), NT = PL::NT, NZ = LZ / 2, HZ = LZ / 2 + 1, E = PL::E;
    constexpr int R0 = stage_radix<PL, -1>(0), NB0 = E / R0, JN = R0 / 2;  // half-zero first stage
    constexpr bool PF = zreg_prefetch<PL>();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* buf = reinterpret_cast<C*>(smem_raw);  // exchange planes [3][ROWS][TP]
    constexpr int ROWS = zreg_rows<PL, T>();  // padded rows of an exchange plane
    C* gs = buf + 3 * ROWS * TP;              // Green tensor [6][HZ][TP]
    C* tws = gs + 6 * HZ * TP;                // twiddle table [LZ]
    const int ky = blockIdx.y;
    const int r0 = blockIdx.z * RB;
    const int hx = Lx / 2 + 1, hy = Ly / 2 + 1;
    const int64_t cs = (int64_t)HZ * hy * hx;
    const int t = threadIdx.x % TP, u = threadIdx.x / TP;
    const int kx = blockIdx.x * TP + t;
    const bool valid = kx < Lx;
    const int64_t plane = (int64_t)Ly * Lx;
    C* bt = buf + t;
    const C* gt = gs + t;
    auto ld = [&](int p, int pos) { return bt[(p * ROWS + exchange_row<LZ, NT, TP, sizeof(C)>(pos)) * TP]; };
    auto st = [&](int p, int pos, C val) { bt[(p * ROWS + exchange_row<LZ, NT, TP, sizeof(C)>(pos)) * TP] = val; };
    const int rend = min(R, r0 + RB);
    auto next_active = [&](int r) {  // uniform across the block
        while (r < rend && active != nullptr && active[r] == 0) ++r;
        return r;
    };
    auto column = [&](int r, int c) {
        return U2 + ((int64_t)r * 3 + c) * NZ * plane + (int64_t)ky * Lx + (valid ? kx : 0);
    };
    C nxt[3][PF ? NB0 * JN : 1];  // first-stage inputs of the next RHS
    auto load_first = [&](int r, auto&& put) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const C* bc = column(r, c);
#pragma unroll
            for (int q = 0; q < NB0; ++q)
#pragma unroll
                for (int j = 0; j < JN; ++j)
                    put(c, q, j, valid ? __ldcs(bc + (int64_t)(u + q * NT + j * (LZ / R0)) * plane) : czero<C>());
        }
    };
    auto prefetch = [&](int r) {
        if constexpr (PF) load_first(r, [&](int c, int q, int j, C x) { nxt[c][q * JN + j] = x; });
    };
    // the first RHS's loads are in flight while the Green tensor is staged
    int r = next_active(r0);
    if (r < rend) prefetch(r);
    {
        const int kyo = ky <= Ly / 2 ? ky : Ly - ky;
        const bool fy = ky > Ly / 2;
        if constexpr (LZ >= 512) {  // (the 512-point plan has no registers to spare)
            for (int e = threadIdx.x; e < 6 * HZ * TP; e += blockDim.x) {
                const int tt = e % TP, kz = (e / TP) % HZ, cc = e / (TP * HZ);
                const int kxs = blockIdx.x * TP + tt;
                C g = czero<C>();
                if (kxs < Lx) {
                    const bool fx = kxs > Lx / 2;
                    const int kxo = fx ? Lx - kxs : kxs;
                    g = gh[cc * cs + ((int64_t)kz * hy + kyo) * hx + kxo];
                    // xy is odd in x and y, xz odd in x, yz odd in y (z handled at use)
                    const bool flip = (cc == 1 && fx != fy) || (cc == 2 && fx) || (cc == 4 && fy);
                    if (flip) g = cscale(g, T(-1));
                }
                gs[(cc * HZ + kz) * TP + tt] = g;
            }
        } else {
            // 4 independent loads per thread in flight: the tile's latency is
            // a fixed cost of every block
            constexpr int NS = 6 * HZ * TP, UN = 4;
            for (int e0 = threadIdx.x; e0 < NS; e0 += UN * blockDim.x) {
                C gv[UN];
#pragma unroll
                for (int q = 0; q < UN; ++q) {
                    const int e = e0 + q * blockDim.x;
                    const int tt = e % TP, kz = (e / TP) % HZ, cc = e / (TP * HZ);
                    const int kxs = blockIdx.x * TP + tt;
                    const int kxo = kxs > Lx / 2 ? Lx - kxs : kxs;
                    gv[q] = (e < NS && kxs < Lx) ? gh[cc * cs + ((int64_t)kz * hy + kyo) * hx + kxo] : czero<C>();
                }
#pragma unroll
                for (int q = 0; q < UN; ++q) {
                    const int e = e0 + q * blockDim.x;
                    if (e >= NS) continue;
                    const int tt = e % TP, cc = e / (TP * HZ);
                    const bool fx = blockIdx.x * TP + tt > Lx / 2;
                    // xy is odd in x and y, xz odd in x, yz odd in y (z handled at use)
                    const bool flip = (cc == 1 && fx != fy) || (cc == 2 && fx) || (cc == 4 && fy);
                    gs[e] = flip ? cscale(gv[q], T(-1)) : gv[q];
                }
            }
        }
        // twiddles from shared memory: the per-stage loads of the six
        // transforms per RHS then wait on shared, not L1, latency
        for (int e = threadIdx.x; e < LZ; e += blockDim.x) tws[e] = tw[e];
    }
#pragma unroll 1
    while (r < rend) {
        C vc[3][E];
        if constexpr (PF) {
#pragma unroll
            for (int c = 0; c < 3; ++c)
#pragma unroll
                for (int q = 0; q < NB0; ++q)
#pragma unroll
                    for (int j = 0; j < JN; ++j) vc[c][q * R0 + j] = nxt[c][q * JN + j];
        } else {
            load_first(r, [&](int c, int q, int j, C x) { vc[c][q * R0 + j] = x; });
        }
        const int rn = next_active(r + 1);
        if (rn < rend) prefetch(rn);
        // (each transform's first exchange opens with a barrier, which also
        // orders it after the previous transform's last reads of the planes)
        fft_stages_np<C, PL, -1, 0, 3>(vc, u, tws, ld, st, true);
        for_each_out<PL, -1, false>(u, [&](int idx, int kz) {
            const bool fz = kz > LZ / 2;
            const int kzo = fz ? LZ - kz : kz;
            const C* g = gt + kzo * TP;
            const C gxx = g[0], gyy = g[3 * HZ * TP], gzz = g[5 * HZ * TP];
            C gxy = g[HZ * TP], gxz = g[2 * HZ * TP], gyz = g[4 * HZ * TP];
            if (fz) {  // xz and yz are odd in z
                gxz = cscale(gxz, T(-1));
                gyz = cscale(gyz, T(-1));
            }
            const C px = vc[0][idx], py = vc[1][idx], pz = vc[2][idx];
            vc[0][idx] = cdot3(gxx, px, gxy, py, gxz, pz);
            vc[1][idx] = cdot3(gxy, px, gyy, py, gyz, pz);
            vc[2][idx] = cdot3(gxz, px, gyz, py, gzz, pz);
        });
        fft_stages_np<C, PL, +1, 0, 3>(vc, u, tws, ld, st, false);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            C* bc = column(r, c);
            for_each_out<PL, +1, true>(u, [&](int idx, int pos) {
                if (valid) __stcs(bc + (int64_t)pos * plane, vc[c][idx]);
            });
        }
        r = rn;
    }
}

// ---- z pass, register-resident schedule over octant columns (complex64) --------
// As k_zconv_reg, but a block owns TP columns of the Green octant at one kyo
// and transforms the (up to four) columns (+-kx, +-ky) that share them, so a
// staged Green tile serves 4 columns per RHS; the x and y signs of the odd
// components are applied at use.  Block a covers kx in [a, a+TP) directly and
// the mirrored columns Lx - kxo, kxo in (a, a+TP], in ascending order (thread
// t takes kxo = a + TP - t), so both loads are aligned rows of TP columns and
// every column 0..Lx-1 has one owner (the self-mirrored Lx/2 is a mirrored
// one of the last block); the tile therefore holds TP + 1 Green columns.
template <typename T, int LZ, int RB, int V = 0>
__global__ void __launch_bounds__(zreg_threads<ZrPlan<LZ, V>>(), zreg_min_blocks<ZrPlan<LZ, V>>())
    k_zconv_oct(cx<T>* __restrict__ U2, const cx<T>* __restrict__ gh, int R, int Lx, int Ly,
                const cx<T>* __restrict__ tw, const int* __restrict__ active) {
    using C = cx<T>;
    using PL = ZrPlan<LZ, V>;
    constexpr int TP = tp_zr<PL>(), NT = PL::NT, NZ = LZ / 2, HZ = LZ / 2 + 1, E = PL::E;
    constexpr int R0 = stage_radix<PL, -1>(0), NB0 = E / R0, JN = R0 / 2;  // half-zero first stage
    constexpr bool PF = zreg_prefetch<PL>();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* buf = reinterpret_cast<C*>(smem_raw);  // exchange planes [3][ROWS][TP]
    constexpr int ROWS = zreg_rows<PL, T>();  // padded rows of an exchange plane
    constexpr int TG = TP + 1;                // Green columns a .. a+TP
    C* gs = buf + 3 * ROWS * TP;              // Green tensor [6][HZ][TG]
    C* tws = gs + 6 * HZ * TG;                // twiddle table [LZ]
    const int hx = Lx / 2 + 1, hy = Ly / 2 + 1;
    const int64_t cs = (int64_t)HZ * hy * hx;
    const int t = threadIdx.x % TP, u = threadIdx.x / TP;
    const int a = blockIdx.x * TP, kyo = blockIdx.y;
    const int r0 = blockIdx.z * RB;
    // sign variants v = fx + 2 fy: octant column kxo = fx ? a + TP - t : a + t,
    // kx = fx ? Lx - kxo : kxo, ky = fy ? Ly - kyo : kyo.  kyo = 0 and Ly/2
    // have no distinct -ky (uniform per block).  (The odd components vanish
    // at kx = Lx/2, so its sign does not matter.)
    const int nv = (kyo == 0 || 2 * kyo == Ly) ? 2 : 4;
    auto octx = [&](int v) { return (v & 1) ? a + TP - t : a + t; };
    auto col_valid = [&](int v) {
        const int kxo = octx(v);
        return (v & 1) ? kxo <= Lx / 2 : kxo < Lx / 2;
    };
    const int64_t plane = (int64_t)Ly * Lx;
    C* bt = buf + t;
    auto ld = [&](int p, int pos) { return bt[(p * ROWS + exchange_row<LZ, NT, TP, sizeof(C)>(pos)) * TP]; };
    auto st = [&](int p, int pos, C val) { bt[(p * ROWS + exchange_row<LZ, NT, TP, sizeof(C)>(pos)) * TP] = val; };
    const int rend = min(R, r0 + RB);
    auto next_active = [&](int r) {  // uniform across the block
        while (r < rend && active != nullptr && active[r] == 0) ++r;
        return r;
    };
    auto column = [&](int r, int c, int v) {
        const int kx = (v & 1) ? Lx - octx(v) : octx(v), ky = (v >> 1) ? Ly - kyo : kyo;
        return U2 + ((int64_t)r * 3 + c) * NZ * plane + (int64_t)ky * Lx + (col_valid(v) ? kx : 0);
    };
    C nxt[3][PF ? NB0 * JN : 1];  // first-stage inputs of the next column
    auto load_first = [&](int r, int v, auto&& put) {
        const bool valid = col_valid(v);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const C* bc = column(r, c, v);
#pragma unroll
            for (int q = 0; q < NB0; ++q)
#pragma unroll
                for (int j = 0; j < JN; ++j)
                    put(c, q, j, valid ? __ldcs(bc + (int64_t)(u + q * NT + j * (LZ / R0)) * plane) : czero<C>());
        }
    };
    auto prefetch = [&](int r, int v) {
        if constexpr (PF) load_first(r, v, [&](int c, int q, int j, C x) { nxt[c][q * JN + j] = x; });
    };
    // the first column's loads are in flight while the Green tensor is staged
    int r = next_active(r0), v = 0;
    if (r < rend) prefetch(r, v);
    {
        // (8 independent loads per thread in flight: the tile is read once
        // per block, so its latency is the fixed cost of a launch)
        constexpr int NS = 6 * HZ * TG, UN = 8;
        for (int e0 = threadIdx.x; e0 < NS; e0 += UN * blockDim.x) {
            C gv[UN];
#pragma unroll
            for (int q = 0; q < UN; ++q) {
                const int e = e0 + q * blockDim.x;
                const int tt = e % TG, kz = (e / TG) % HZ, cc = e / (TG * HZ);
                gv[q] = (e < NS && a + tt < hx) ? gh[cc * cs + ((int64_t)kz * hy + kyo) * hx + a + tt] : czero<C>();
            }
#pragma unroll
            for (int q = 0; q < UN; ++q)
                if (e0 + q * blockDim.x < NS) gs[e0 + q * blockDim.x] = gv[q];
        }
        // twiddles from shared memory: the per-stage loads of the six
        // transforms per RHS then wait on shared, not L1, latency
        for (int e = threadIdx.x; e < LZ; e += blockDim.x) tws[e] = tw[e];
    }
#pragma unroll 1
    while (r < rend) {
        C vc[3][E];
        if constexpr (PF) {
#pragma unroll
            for (int c = 0; c < 3; ++c)
#pragma unroll
                for (int q = 0; q < NB0; ++q)
#pragma unroll
                    for (int j = 0; j < JN; ++j) vc[c][q * R0 + j] = nxt[c][q * JN + j];
        } else {
            load_first(r, v, [&](int c, int q, int j, C x) { vc[c][q * R0 + j] = x; });
        }
        int rn = r, vn = v + 1;
        if (vn >= nv) {
            rn = next_active(r + 1);
            vn = 0;
        }
        if (rn < rend) prefetch(rn, vn);
        const bool fx = v & 1, fy = v >> 1, valid = col_valid(v);
        // (each transform's first exchange opens with a barrier, which also
        // orders it after the previous transform's last reads of the planes)
        fft_stages_np<C, PL, -1, 0, 3>(vc, u, tws, ld, st, true);
        for_each_out<PL, -1, false>(u, [&](int idx, int kz) {
            const bool fz = kz > LZ / 2;
            const int kzo = fz ? LZ - kz : kz;
            const C* g = gs + (fx ? TP - t : t) + kzo * TG;
            const C gxx = g[0], gyy = g[3 * HZ * TG], gzz = g[5 * HZ * TG];
            C gxy = g[HZ * TG], gxz = g[2 * HZ * TG], gyz = g[4 * HZ * TG];
            if (fx != fy) gxy = cscale(gxy, T(-1));
            if (fx != fz) gxz = cscale(gxz, T(-1));
            if (fy != fz) gyz = cscale(gyz, T(-1));
            const C px = vc[0][idx], py = vc[1][idx], pz = vc[2][idx];
            vc[0][idx] = cdot3(gxx, px, gxy, py, gxz, pz);
            vc[1][idx] = cdot3(gxy, px, gyy, py, gyz, pz);
            vc[2][idx] = cdot3(gxz, px, gyz, py, gzz, pz);
        });
        fft_stages_np<C, PL, +1, 0, 3>(vc, u, tws, ld, st, false);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            C* bc = column(r, c, v);
            for_each_out<PL, +1, true>(u, [&](int idx, int pos) {
                if (valid) __stcs(bc + (int64_t)pos * plane, vc[c][idx]);
            });
        }
        r = rn;
        v = vn;
    }
}

// In-place forward FFT of dense rows of length LX (Green tensor x pass).
template <int LX>
__global__ void __launch_bounds__(tp_x<LX, 16>() * Plan<LX>::NT)
    k_xfull(double2* __restrict__ data, int64_t nrows, const double2* __restrict__ tw) {
    using C = double2;
    using PL = Plan<LX>;
    constexpr int TP = tp_x<LX, 16>(), SP = TP + 1;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* buf = reinterpret_cast<C*>(smem_raw);
    const int64_t row0 = (int64_t)blockIdx.x * TP;
    for (int e = threadIdx.x; e < TP * LX; e += blockDim.x) {
        const int t2 = e / LX, x = e - t2 * LX;
        const int64_t row = row0 + t2;
        buf[x * SP + t2] = row < nrows ? data[row * LX + x] : czero<C>();
    }
    __syncthreads();
    const int t = threadIdx.x % TP, u = threadIdx.x / TP;
    C* bt = buf + t;
    C v[PL::E];
    auto first = [&](int pos) { return bt[pos * SP]; };
    auto ld = [&](int pos) { return bt[pos * SP]; };
    auto st = [&](int pos, C val) { bt[pos * SP] = val; };
    pencil_fft<C, PL, -1, false>(v, u, tw, first, ld, st);
    __syncthreads();
    for_each_out<PL, -1, false>(u, [&](int idx, int pos) { bt[pos * SP] = v[idx]; });
    __syncthreads();
    for (int e = threadIdx.x; e < TP * LX; e += blockDim.x) {
        const int t2 = e / LX, x = e - t2 * LX;
        const int64_t row = row0 + t2;
        if (row < nrows) data[row * LX + x] = buf[x * SP + t2];
    }
}

// ---- host launchers -------------------------------------------------------------
// Give a kernel the maximum shared-memory carveout and, above 48 KB, the
// dynamic shared-memory size it needs -- once per kernel
// (so that only launches happen while a stream is being captured).
template <typename K> static inline cudaError_t allow_smem(K kernel, size_t bytes) {
    static std::mutex mu;
    static std::unordered_map<const void*, size_t> done;
    std::lock_guard<std::mutex> lock(mu);
    auto it = done.find((const void*)kernel);
    if (it != done.end() && it->second >= bytes) return cudaSuccess;
    // prefer shared memory over L1 so that several FFT blocks fit on an SM
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                                         (int)cudaSharedmemCarveoutMaxShared);
    if (e == cudaSuccess && bytes > 48 * 1024)
        e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess) done[(const void*)kernel] = bytes;
    return e;
}

static inline unsigned grid1d(int64_t n, int threads) {
    int64_t b = (n + threads - 1) / threads;
    if (b > 152 * 32) b = 152 * 32;
    return (unsigned)(b < 1 ? 1 : b);
}

#define DDA_DISPATCH_L(LVAL, FN, ...)                       \
    switch (LVAL) {                                         \
        case 16: return FN<16>(__VA_ARGS__);                \
        case 32: return FN<32>(__VA_ARGS__);                \
        case 48: return FN<48>(__VA_ARGS__);                \
        case 64: return FN<64>(__VA_ARGS__);                \
        case 96: return FN<96>(__VA_ARGS__);                \
        case 128: return FN<128>(__VA_ARGS__);              \
        case 192: return FN<192>(__VA_ARGS__);              \
        case 256: return FN<256>(__VA_ARGS__);              \
        case 384: return FN<384>(__VA_ARGS__);              \
        case 512: return FN<512>(__VA_ARGS__);              \
        default: return cudaErrorInvalidValue;              \
    }

// The x passes' rows inside the y-transformed buffer (see RowMap).
static inline RowMap row_map(const Geom& g) {
    return RowMap{g.ny, g.Ly, (int64_t)g.nz * g.Ly * g.Lx};
}

// The x-forward gathers' vectors of a fused matvec.
template <typename T> static inline FwdVecs<cx<T>> fwd_vecs(const FusedKrylov<T>& fk) {
    return FwdVecs<cx<T>>{fk.r, fk.v, fk.s, fk.t, fk.x, fk.st};
}
// The x-inverse scatter of mode 3 is that of mode 1 (v = A p, sigma).
static inline int inverse_mode(int mode) { return mode == 3 ? 1 : mode; }

// After a fused x-inverse pass of nb blocks per RHS: sum its partials and
// update the scalars (k_fused_finalize; traced as Krylov work).
template <typename T>
static inline cudaError_t fused_finalize(int mode, int R, int nb, const FusedKrylov<T>& fk, int* active,
                                         cudaStream_t st) {
    mode = inverse_mode(mode);
    if (mode == 0) return cudaSuccess;
    PROF_BEGIN(st);
    if (mode == 1) k_fused_finalize<cx<T>, 1><<<R, kFinThreads, 0, st>>>(fk.part, fk.part_stride, nb, fk.st, active);
    else k_fused_finalize<cx<T>, 2><<<R, kFinThreads, 0, st>>>(fk.part, fk.part_stride, nb, fk.st, active);
    PROF_END(sizeof(T) == 4 ? KK_KRYLOV_C64 : KK_KRYLOV_C128, R, st);
    return cudaGetLastError();
}

template <typename T> struct LaunchX {
    // double-float matvecs run only the plain passes (no fused Krylov modes)
    static constexpr bool kDouble = std::is_same<T, dfl>::value;
    static constexpr int koff = sizeof(T) == 4 ? 0 : (kDouble ? (KK_XFWD_DF - KK_XFWD_C64) : (KK_XFWD_C128 - KK_XFWD_C64));
    // warp-local x passes (xwarp.cuh, complex64): xvar = 1 + plan variant
    static constexpr bool kWarpX = sizeof(T) == 4 && !kDouble;
    template <int LX, int V>
    static cudaError_t fwd_w(const Geom& g, int R, cx<T>* x, cx<T>* u1, const int* site_of, const cx<T>* tw,
                             const int* active, const FusedKrylov<T>& fk, cudaStream_t st) {
        if constexpr (kWarpX) {
            using PL = XwPlan<LX, V>;
            const size_t sm = xw_smem<PL>();
            const int nrows = g.ny * g.nz;
            dim3 grid((nrows + xw_rows<PL>() - 1) / xw_rows<PL>(), 3, R);
            auto go = [&](auto kern) -> cudaError_t {
                cudaError_t e = allow_smem(kern, sm);
                if (e != cudaSuccess) return e;
                PROF_BEGIN(st);
                kern<<<grid, kXwThreads, sm, st>>>(x, u1, row_map(g), site_of, nrows, g.N, tw, active, fwd_vecs(fk));
                PROF_END(KK_XFWD_C64, R, st);
                return cudaGetLastError();
            };
            if (fk.mode == 1) return go(k_xfwd_w<LX, V, 1>);
            if (fk.mode == 2) return go(k_xfwd_w<LX, V, 2>);
            if (fk.mode == 3) return go(k_xfwd_w<LX, V, 3>);
            return go(k_xfwd_w<LX, V, 0>);
        }
        return cudaErrorInvalidValue;
    }
    template <int LX, int V, int DIAG>
    static cudaError_t inv_w(const Geom& g, int R, const cx<T>* u1, cx<T>* y, const cx<T>* x, const DevTarget& tg,
                             const cx<T>* beta, int beta_stride, const cx<T>* tw, int* active,
                             const FusedKrylov<T>& fk, cudaStream_t st) {
        if constexpr (kWarpX) {
            using PL = XwPlan<LX, V>;
            const size_t sm = (size_t)xwi_rows<PL>() * xw_plane<PL>() * sizeof(float2);
            const int nrows = tg.rows != nullptr ? tg.nrows : g.ny * g.nz;
            dim3 grid((nrows + xwi_rows<PL>() - 1) / xwi_rows<PL>(), 3, R);
            auto go = [&](auto kern) -> cudaError_t {
                cudaError_t e = allow_smem(kern, sm);
                if (e != cudaSuccess) return e;
                PROF_BEGIN(st);
                kern<<<grid, kXwiThreads, sm, st>>>(u1, row_map(g), y, x, tg.site_of, tg.comp_of, beta, beta_stride,
                                                    tg.rows, nrows, g.N, tw, active, fk.rhat, fk.st, fk.part, fk.cnt,
                                                    fk.part_stride);
                PROF_END(KK_XINV_C64, R, st);
                if ((e = cudaGetLastError()) != cudaSuccess) return e;
                return fused_finalize<T>(fk.mode, R, (int)(grid.x * grid.y), fk, active, st);
            };
            const int mode = inverse_mode(fk.mode);
            if (mode == 1) return go(k_xinv_w<LX, V, 1, DIAG>);
            if (mode == 2) return go(k_xinv_w<LX, V, 2, DIAG>);
            return go(k_xinv_w<LX, V, 0, DIAG>);
        }
        return cudaErrorInvalidValue;
    }
    template <int LX> static int xvariants() { return kWarpX ? 1 + xw_variants(LX) : 1; }
    // f(integral_constant<V>) for plan variant v of the warp-local rows (the
    // last variant where v is larger)
    template <int LX, int V = 0, class F> static cudaError_t by_xvariant(int v, F&& f) {
        if constexpr (V + 1 < xw_variants(LX)) {
            if (v > V) return by_xvariant<LX, V + 1>(v, f);
        }
        return f(std::integral_constant<int, V>{});
    }
    template <int LX>
    static cudaError_t fwd(const Geom& g, int R, cx<T>* x, cx<T>* u1, const int* site_of, const cx<T>* tw,
                           const int* active, const FusedKrylov<T>& fk, int xvar, cudaStream_t st) {
        if constexpr (kWarpX) {
            if (xvar >= 1)
                return by_xvariant<LX>(xvar - 1, [&](auto v) {
                    return fwd_w<LX, decltype(v)::value>(g, R, x, u1, site_of, tw, active, fk, st);
                });
        }
        constexpr int TP = tp_x<LX, sizeof(cx<T>)>(), NTH = TP * XPlan<LX, sizeof(cx<T>)>::NT;
        const size_t sm = (size_t)LX * (TP + 1) * sizeof(cx<T>);
        const int nrows = g.ny * g.nz;
        dim3 grid((nrows + TP - 1) / TP, 3, R);
        cudaError_t e = cudaSuccess;
        PROF_BEGIN(st);
        auto go = [&](auto kern) -> cudaError_t {
            cudaError_t ke = allow_smem(kern, sm);
            if (ke == cudaSuccess) kern<<<grid, NTH, sm, st>>>(x, u1, row_map(g), site_of, nrows, g.N, tw, active,
                                                               fwd_vecs(fk));
            return ke;
        };
        if (fk.mode == 0 || kDouble) {
            e = go(k_xfwd<T, LX, 0>);
        } else if constexpr (!kDouble) {
            if (fk.mode == 1) e = go(k_xfwd<T, LX, 1>);
            else if (fk.mode == 2) e = go(k_xfwd<T, LX, 2>);
            else e = go(k_xfwd<T, LX, 3>);
        }
        if (e != cudaSuccess) return e;
        PROF_END(KK_XFWD_C64 + koff, R, st);
        return cudaGetLastError();
    }
    template <int LX, int MODE, int DIAG>
    static cudaError_t inv_mode(const Geom& g, int R, const cx<T>* u1, cx<T>* y, const cx<T>* x, const DevTarget& tg,
                                const cx<T>* beta, int beta_stride, const cx<T>* tw, int* active,
                                const FusedKrylov<T>& fk, cudaStream_t st) {
        constexpr int TP = tp_x<LX, sizeof(cx<T>)>(), NTH = TP * XPlan<LX, sizeof(cx<T>)>::NT;
        const size_t sm = (size_t)LX * (TP + 1) * sizeof(cx<T>);
        const int nrows = tg.rows != nullptr ? tg.nrows : g.ny * g.nz;
        dim3 grid((nrows + TP - 1) / TP, 3, R);
        cudaError_t e;
        if ((e = allow_smem(k_xinv<T, LX, MODE, DIAG>, sm)) != cudaSuccess) return e;
        if constexpr (MODE == 0)
            k_xinv<T, LX, 0, DIAG><<<grid, NTH, sm, st>>>(u1, row_map(g), y, x, tg.site_of, tg.comp_of, beta,
                                                         beta_stride, tg.rows, nrows, g.N, tw, active, nullptr,
                                                         nullptr, nullptr, nullptr, 0);
        else
            k_xinv<T, LX, MODE, DIAG><<<grid, NTH, sm, st>>>(u1, row_map(g), y, x, tg.site_of, tg.comp_of, beta,
                                                            beta_stride, tg.rows, nrows, g.N, tw, active, fk.rhat,
                                                            fk.st, fk.part, fk.cnt, fk.part_stride);
        return cudaGetLastError();
    }
    // blocks per RHS of the staged x-inverse pass (the partials of its fused sums)
    template <int LX> static int inv_blocks(const Geom& g, const DevTarget& tg) {
        constexpr int TP = tp_x<LX, sizeof(cx<T>)>();
        const int nrows = tg.rows != nullptr ? tg.nrows : g.ny * g.nz;
        return (nrows + TP - 1) / TP * 3;
    }
    template <int LX>
    static cudaError_t inv(const Geom& g, int R, const cx<T>* u1, cx<T>* y, const cx<T>* x, const DevTarget& tg,
                           const cx<T>* beta, int beta_stride, bool tensor, const cx<T>* tw, int* active,
                           const FusedKrylov<T>& fk, int xvar, cudaStream_t st) {
        // the kind of diagonal: tensor table, composition codes, or per-site
        // materials (no composition array)
        const int diag = tensor ? kDiagTensor : (tg.comp_of ? kDiagComp : kDiagSite);
        auto by_diag = [&](auto launch) -> cudaError_t {
            if (diag == kDiagTensor) return launch(std::integral_constant<int, kDiagTensor>{});
            if (diag == kDiagSite) return launch(std::integral_constant<int, kDiagSite>{});
            return launch(std::integral_constant<int, kDiagComp>{});
        };
        if constexpr (kWarpX) {
            if (xvar >= 1)
                return by_xvariant<LX>(xvar - 1, [&](auto v) {
                    return by_diag([&](auto d) {
                        return inv_w<LX, decltype(v)::value, decltype(d)::value>(g, R, u1, y, x, tg, beta,
                                                                                 beta_stride, tw, active, fk, st);
                    });
                });
        }
        auto run = [&](auto mode) {
            constexpr int M = decltype(mode)::value;
            return by_diag([&](auto d) {
                return inv_mode<LX, M, decltype(d)::value>(g, R, u1, y, x, tg, beta, beta_stride, tw, active, fk, st);
            });
        };
        cudaError_t e = cudaSuccess;
        PROF_BEGIN(st);
        if (fk.mode == 0 || kDouble) {
            e = run(std::integral_constant<int, 0>{});
        } else if constexpr (!kDouble) {
            e = inverse_mode(fk.mode) == 1 ? run(std::integral_constant<int, 1>{})
                                            : run(std::integral_constant<int, 2>{});
        }
        if (e != cudaSuccess) return e;
        PROF_END(KK_XINV_C64 + koff, R, st);
        if (fk.mode == 0 || kDouble) return cudaSuccess;
        return fused_finalize<T>(fk.mode, R, inv_blocks<LX>(g, tg), fk, active, st);
    }
    template <int MODE, int L, int V = 0>
    static cudaError_t strided_mode(const cx<T>* src, cx<T>* dst, int64_t pt_stride, int width, int64_t sb,
                                    int64_t db, int batches, int per_rhs, const cx<T>* tw, const int* active,
                                    cudaStream_t st, int kind, double units) {
        using PL = SPlan<L, V>;
        constexpr int TP = tp_sp<PL, sizeof(cx<T>)>(), NTH = TP * PL::NT;
        const size_t sm = (size_t)exchange_rows<L, PL::NT, TP, sizeof(cx<T>)>() * TP * sizeof(cx<T>);
        auto kern = [] {
            if constexpr (strided_capped<T, L, V>()) return k_strided3<T, L, MODE, V>;
            else return k_strided<T, L, MODE, V>;
        }();
        cudaError_t e = allow_smem(kern, sm);
        if (e != cudaSuccess) return e;
        dim3 grid((width + TP - 1) / TP, batches, 1);
        PROF_BEGIN(st);
        kern<<<grid, NTH, sm, st>>>(src, dst, pt_stride, width, sb, db, per_rhs, tw, active);
        PROF_END(kind, units, st);
        return cudaGetLastError();
    }
    // yvar 1: radix plan variant 1 where it exists (complex64 y passes only)
    template <int L> static int yvariants() { return (sizeof(T) == 4 && !kDouble) ? s_variants(L) : 1; }
    template <int L>
    static cudaError_t strided(int mode, const cx<T>* src, cx<T>* dst, int64_t pt_stride, int width, int64_t sb,
                               int64_t db, int batches, int per_rhs, const cx<T>* tw, const int* active,
                               cudaStream_t st, int kind, double units, int yvar = 0) {
        if constexpr (sizeof(T) == 4 && !kDouble && s_variants(L) > 1) {
            if (yvar == 1 && mode == 0)
                return strided_mode<0, L, 1>(src, dst, pt_stride, width, sb, db, batches, per_rhs, tw, active, st, kind,
                                             units);
            if (yvar == 1 && mode == 1)
                return strided_mode<1, L, 1>(src, dst, pt_stride, width, sb, db, batches, per_rhs, tw, active, st, kind,
                                             units);
        }
        if (mode == 0)
            return strided_mode<0, L>(src, dst, pt_stride, width, sb, db, batches, per_rhs, tw, active, st, kind, units);
        if (mode == 1)
            return strided_mode<1, L>(src, dst, pt_stride, width, sb, db, batches, per_rhs, tw, active, st, kind, units);
        return strided_mode<2, L>(src, dst, pt_stride, width, sb, db, batches, per_rhs, tw, active, st, kind, units);
    }
    template <int LZ>
    static cudaError_t zconv(const Geom& g, int R, cx<T>* u2, const cx<T>* gh, const cx<T>* tw, const int* active,
                             int zvar, cudaStream_t st) {
        // several RHS per block reuse the staged Green tensor
        constexpr int RB = 8;
        const bool multi = R > 1;
        const int rb = multi ? RB : 1;
        cudaError_t e;
        if constexpr (sizeof(T) == 4 && zreg_ok<LZ>()) {
            // 1, 2: register-resident, by columns or octant columns, plan 0;
            // 3, 4: the same with radix plan variant 1 (zr_variants)
            if (zvar >= 1 && zvar <= 4) {
                auto sched = [&](auto var) -> cudaError_t {
                    constexpr int V = decltype(var)::value;
                    using PL = ZrPlan<LZ, V>;
                    // a staged Green tile serves RB column-RHS: RBZ RHS of one
                    // column, or of the (up to) 4 columns of an octant column
                    // (long columns: the tile is ~2 RHS of loads, so it serves 16)
                    // (one RHS per octant block for the radix-16 variant -- twice
                    // the blocks at 2 RHS -- was measured slower: the staging of
                    // the Green tile then costs more than the warps gain)
                    constexpr int TP = tp_zr<PL>(), RBZ = LZ >= 256 ? 16 : 8, RBO = RBZ / 4;
                    const bool oct = zvar == 2 || zvar == 4;
                    const size_t sm = oct ? zoct_smem<PL, T>() : zreg_smem<PL, T>();
                    const int rbz = !multi ? 1 : (oct ? RBO : RBZ);
                    dim3 grid(oct ? (g.Lx / 2 + TP - 1) / TP : (g.Lx + TP - 1) / TP, oct ? g.Ly / 2 + 1 : g.Ly,
                              (R + rbz - 1) / rbz);
                    auto go = [&](auto kern) -> cudaError_t {
                        cudaError_t ke = allow_smem(kern, sm);
                        if (ke != cudaSuccess) return ke;
                        PROF_BEGIN(st);
                        kern<<<grid, zreg_threads<PL>(), sm, st>>>(u2, gh, R, g.Lx, g.Ly, tw, active);
                        PROF_END(KK_ZCONV_C64 + koff, R, st);
                        return cudaGetLastError();
                    };
                    if (!multi) return oct ? go(k_zconv_oct<T, LZ, 1, V>) : go(k_zconv_reg<T, LZ, 1, V>);
                    return oct ? go(k_zconv_oct<T, LZ, RBO, V>) : go(k_zconv_reg<T, LZ, RBZ, V>);
                };
                if (zvar >= 3) {
                    if constexpr (zr_variants(LZ) > 1) return sched(std::integral_constant<int, 1>{});
                    return cudaErrorInvalidValue;
                }
                return sched(std::integral_constant<int, 0>{});
            }
        }
        constexpr int TP = tp_z<LZ, T>(), NTH = 3 * TP * ZPlan<LZ>::NT;
        const size_t sm = zconv_smem<LZ, T>();
        e = multi ? allow_smem(k_zconv<T, LZ, RB>, sm) : allow_smem(k_zconv<T, LZ, 1>, sm);
        if (e != cudaSuccess) return e;
        dim3 grid((g.Lx + TP - 1) / TP, g.Ly, (R + rb - 1) / rb);
        PROF_BEGIN(st);
        if (multi)
            k_zconv<T, LZ, RB><<<grid, NTH, sm, st>>>(u2, gh, R, g.Lx, g.Ly, tw, active);
        else
            k_zconv<T, LZ, 1><<<grid, NTH, sm, st>>>(u2, gh, R, g.Lx, g.Ly, tw, active);
        PROF_END(KK_ZCONV_C64 + koff, R, st);
        return cudaGetLastError();
    }
    template <int LZ> static int zvariants() {
        return (sizeof(T) == 4 && zreg_ok<LZ>()) ? 1 + 2 * zr_variants(LZ) : 1;
    }
};

// The lattice seen by the kernels is padded with vacuum to exactly L/2 sites
// per axis (g.nx == g.Lx/2, ...), see dda_set_target.  With fk.mode != 0 the
// x passes also carry the fused BiCGstab updates (see k_xfwd, k_xinv).
template <typename T>
cudaError_t launch_matvec_fused(const Geom& g, int R, cx<T>* x, cx<T>* y, const PadWork<T>& w, const DevTarget& tg,
                                const cx<T>* beta, int beta_stride, const cx<T>* ghat, const Twiddles<T>& tw,
                                int* active, const FusedKrylov<T>& fk, cudaStream_t st) {
    using LX = LaunchX<T>;
    if (g.nx * 2 != g.Lx || g.ny * 2 != g.Ly || g.nz * 2 != g.Lz) return cudaErrorInvalidValue;
    cudaError_t e;
    auto fwdx = [&]() -> cudaError_t {
        DDA_DISPATCH_L(g.Lx, LX::template fwd, g, R, x, w.u2, tg.site_of, tw.x, active, fk, w.xfwd, st);
    };
    auto ys = [&](int mode, const cx<T>* s, cx<T>* d, int64_t sb, int64_t db) -> cudaError_t {
        DDA_DISPATCH_L(g.Ly, LX::template strided, mode, s, d, (int64_t)g.Lx, g.Lx, sb, db, R * 3 * g.nz, 3 * g.nz,
                       tw.y, active, st, (mode == 0 ? KK_YFWD_C64 : KK_YINV_C64) + LX::koff, (double)R, w.yvar);
    };
    auto zc = [&]() -> cudaError_t {
        DDA_DISPATCH_L(g.Lz, LX::template zconv, g, R, w.u2, ghat, tw.z, active, w.zvar, st);
    };
    auto invx = [&]() -> cudaError_t {
        DDA_DISPATCH_L(g.Lx, LX::template inv, g, R, w.u2, y, x, tg, beta, beta_stride, w.beta_tensor, tw.x, active,
                       fk, w.xinv, st);
    };
    if (w.slices && !w.beta_tensor && slice_passes<T>(g)) {
        if ((e = launch_slice_fwd<T>(g, R, x, w.u2, tg.site_of, tw, active, fk, st)) != cudaSuccess) return e;
        if ((e = zc()) != cudaSuccess) return e;
        return launch_slice_inv<T>(g, R, w.u2, y, x, tg, beta, beta_stride, tw, active, fk, st);
    }
    // (both y passes in place on u2: see RowMap)
    const int64_t plane = (int64_t)g.Ly * g.Lx;
    if ((e = fwdx()) != cudaSuccess) return e;
    if ((e = ys(0, w.u2, w.u2, plane, plane)) != cudaSuccess) return e;
    if ((e = zc()) != cudaSuccess) return e;
    if ((e = ys(1, w.u2, w.u2, plane, plane)) != cudaSuccess) return e;
    return invx();
}

template <typename T> int zconv_schedules(const Geom& g) {
    switch (g.Lz) {
        case 16: return LaunchX<T>::template zvariants<16>();
        case 32: return LaunchX<T>::template zvariants<32>();
        case 48: return LaunchX<T>::template zvariants<48>();
        case 64: return LaunchX<T>::template zvariants<64>();
        case 96: return LaunchX<T>::template zvariants<96>();
        case 128: return LaunchX<T>::template zvariants<128>();
        case 192: return LaunchX<T>::template zvariants<192>();
        case 256: return LaunchX<T>::template zvariants<256>();
        case 384: return LaunchX<T>::template zvariants<384>();
        case 512: return LaunchX<T>::template zvariants<512>();
        default: return 0;
    }
}

// Number of x-pass schedules: 0 staged rows (k_xfwd, k_xinv); for complex64
// also 1 + V, the warp-local passes with radix plan variant V (xwarp.cuh).
template <typename T> int xpass_schedules(const Geom& g) {
    switch (g.Lx) {
        case 16: return LaunchX<T>::template xvariants<16>();
        case 32: return LaunchX<T>::template xvariants<32>();
        case 48: return LaunchX<T>::template xvariants<48>();
        case 64: return LaunchX<T>::template xvariants<64>();
        case 96: return LaunchX<T>::template xvariants<96>();
        case 128: return LaunchX<T>::template xvariants<128>();
        case 192: return LaunchX<T>::template xvariants<192>();
        case 256: return LaunchX<T>::template xvariants<256>();
        case 384: return LaunchX<T>::template xvariants<384>();
        case 512: return LaunchX<T>::template xvariants<512>();
        default: return 1;
    }
}

// Number of y-pass schedules: radix plan variants of the strided y passes
// (complex64: 2 for Ly = 128, 192, 256; else 1).
template <typename T> int ypass_schedules(const Geom& g) {
    switch (g.Ly) {
        case 128: return LaunchX<T>::template yvariants<128>();
        case 192: return LaunchX<T>::template yvariants<192>();
        case 256: return LaunchX<T>::template yvariants<256>();
        case 512: return LaunchX<T>::template yvariants<512>();
        default: return 1;
    }
}

template <typename T>
cudaError_t launch_zconv(const Geom& g, int R, cx<T>* u2, const cx<T>* ghat, const cx<T>* twz, const int* active,
                         int zvar, cudaStream_t st) {
    DDA_DISPATCH_L(g.Lz, LaunchX<T>::template zconv, g, R, u2, ghat, twz, active, zvar, st);
}

template <typename T>
cudaError_t launch_matvec(const Geom& g, int R, const cx<T>* x, cx<T>* y, const PadWork<T>& w, const DevTarget& tg,
                          const cx<T>* beta, int beta_stride, const cx<T>* ghat, const Twiddles<T>& tw,
                          const int* active, cudaStream_t st) {
    FusedKrylov<T> plain{};
    // mode 0 neither writes x nor clears active flags
    return launch_matvec_fused<T>(g, R, const_cast<cx<T>*>(x), y, w, tg, beta, beta_stride, ghat, tw,
                                  const_cast<int*>(active), plain, st);
}

}  // namespace dda
