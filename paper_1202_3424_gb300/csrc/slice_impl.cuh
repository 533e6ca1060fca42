// Fused x and y passes of the FFT-convolution matvec, one z-slice per block.
//
// The separate passes (matvec_impl.cuh) move every x-transformed row through
// HBM between the x and the y transforms (U1, 2M points per component).  For
// grids whose half-y spectrum of one z-slice, (Lx) x (Ly/2) points, fits in
// shared memory, one block can own a whole slice of one component of one
// right-hand side instead:
//
//   forward  k_xyfwd   gather the slice's sites (with the fused BiCGstab
//                      update of MODE 1/2), FFT every row along x (input half
//                      zero), then FFT every column along y (input half zero)
//                      and write the slice of U2 [nz][Ly][Lx]
//   inverse  k_yxinv   inverse FFT of every column of the U2 slice along y
//                      (keep y < Ly/2), inverse FFT of every row along x (keep
//                      x < Lx/2), add (1/alpha) X and scatter, with the fused
//                      BiCGstab dot products of MODE 1/2
//
// so that U1 never exists.  Traffic per RHS and component: P and Y once, U2
// once in each direction (the z pass is unchanged).  The slice plane is held
// column-major, element (x, y) at x*SPY + y with an odd SPY, so that both the
// column transforms (consecutive x across threads) and the row transforms
// (consecutive y across threads) touch distinct banks.
#pragma once

#include "matvec_impl.cuh"

namespace dda {

template <int LX, int LY, int ES> struct SliceCfg {
    static constexpr int NTH = 512;
    using PX = Plan<LX>;
    using PY = Plan<LY>;
    static constexpr int NX = LX / 2, NY = LY / 2;
    static constexpr int TPR = NTH / PX::NT;                            // rows per x round
    static constexpr int ROWS = ((NY + TPR - 1) / TPR) * TPR;           // rows the rounds touch
    static constexpr int SPY = ROWS | 1;                                // odd column stride
    static constexpr int TPC = NTH / PY::NT;                            // columns per y tile
    static constexpr int CROWS = exchange_rows<LY, PY::NT, TPC, ES>();  // column exchange rows
    static constexpr size_t smem = ((size_t)LX * SPY + (size_t)CROWS * TPC) * ES;
};

// Grids whose slice kernels are built: lengths 64-192 on both axes for
// complex64, 64 and 96 for 16-byte elements, and only where the plane fits.
template <int LX, int LY, int ES> __host__ __device__ constexpr bool slice_built() {
    constexpr bool lx = ES == 8 ? (LX == 64 || LX == 96 || LX == 128 || LX == 192) : (LX == 64 || LX == 96);
    constexpr bool ly = ES == 8 ? (LY == 64 || LY == 96 || LY == 128 || LY == 192) : (LY == 64 || LY == 96);
    return lx && ly && SliceCfg<LX, LY, ES>::smem <= 200 * 1024;
}

// ---- forward: gather, x transform of the rows, y transform of the columns ------
template <typename T, int LX, int LY, int MODE>
__global__ void __launch_bounds__(SliceCfg<LX, LY, sizeof(cx<T>)>::NTH)
    k_xyfwd(cx<T>* __restrict__ X, cx<T>* __restrict__ U2, const int* __restrict__ site_of, int64_t N,
            const cx<T>* __restrict__ twx, const cx<T>* __restrict__ twy, const int* __restrict__ active,
            FwdVecs<cx<T>> fv) {
    using C = cx<T>;
    using CF = SliceCfg<LX, LY, sizeof(C)>;
    using PX = typename CF::PX;
    using PY = typename CF::PY;
    constexpr int NTH = CF::NTH, NX = CF::NX, NY = CF::NY, SPY = CF::SPY, TPR = CF::TPR, TPC = CF::TPC;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* plane = reinterpret_cast<C*>(smem_raw);  // [LX][SPY]
    C* colbuf = plane + LX * SPY;               // [CROWS][TPC]
    const int z = blockIdx.x, c = blockIdx.y, r = blockIdx.z, nz = gridDim.x;
    if (active != nullptr && active[r] == 0) return;
    const int64_t off = ((int64_t)r * 3 + c) * N;
    C* xs = X + off;
    const GatherScalars<C> gs = gather_scalars<MODE, C>(fv.st, r);
    // gather the slice's sites: site indices first, then values (two
    // dependent latencies, every load of a thread in flight at once)
    constexpr int NG = (NY * NX + NTH - 1) / NTH;
    {
        const int* so = site_of + (int64_t)z * NY * NX;
        int sidx[NG];
#pragma unroll
        for (int i = 0; i < NG; ++i) {
            const int e = threadIdx.x + i * NTH;
            sidx[i] = e < NY * NX ? so[e] : -1;
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
            const int e = threadIdx.x + i * NTH;
            if (e < NY * NX) plane[(e % NX) * SPY + e / NX] = val[i].val;
            if (sidx[i] >= 0) fused_store<MODE>(xs, fv, off, sidx[i], val[i]);
        }
    }
    __syncthreads();
    // x transform of every row y < NY (input x >= NX zero), in place
    {
        const int t = threadIdx.x % TPR, u = threadIdx.x / TPR;
        for (int y0 = 0; y0 < NY; y0 += TPR) {
            C* bt = plane + y0 + t;
            auto first = [&](int pos) { return bt[pos * SPY]; };
            auto ld = [&](int pos) { return bt[pos * SPY]; };
            auto stf = [&](int pos, C val) { bt[pos * SPY] = val; };
            C v[PX::E];
            pencil_fft<C, PX, -1, true>(v, u, twx, first, ld, stf);
            __syncthreads();
            for_each_out<PX, -1, false>(u, [&](int idx, int pos) { bt[pos * SPY] = v[idx]; });
            __syncthreads();
        }
    }
    // y transform of every column kx (input y >= NY zero) -> U2 slice
    {
        C* dst = U2 + (((int64_t)r * 3 + c) * nz + z) * (int64_t)LY * LX;
        const int t = threadIdx.x % TPC, u = threadIdx.x / TPC;
        C* bt = colbuf + t;
        auto ld = [&](int pos) { return bt[exchange_row<LY, PY::NT, TPC, sizeof(C)>(pos) * TPC]; };
        auto stf = [&](int pos, C val) { bt[exchange_row<LY, PY::NT, TPC, sizeof(C)>(pos) * TPC] = val; };
        for (int kx0 = 0; kx0 < LX; kx0 += TPC) {
            const int kx = kx0 + t;
            const bool valid = kx < LX;
            const C* col = plane + (valid ? kx : 0) * SPY;
            auto first = [&](int pos) { return col[pos]; };
            C v[PY::E];
            // (each tile's first exchange opens with a barrier, after the
            // previous tile's last reads of the column buffer)
            pencil_fft<C, PY, -1, true>(v, u, twy, first, ld, stf);
            for_each_out<PY, -1, false>(u, [&](int idx, int pos) {
                if (valid) dst[(int64_t)pos * LX + kx] = v[idx];
            });
        }
    }
}

// ---- inverse: y transform of the columns, x transform of the rows, scatter -----
template <typename T, int LX, int LY, int MODE>
__global__ void __launch_bounds__(SliceCfg<LX, LY, sizeof(cx<T>)>::NTH)
    k_yxinv(const cx<T>* __restrict__ U2, cx<T>* __restrict__ Y, const cx<T>* __restrict__ X,
            const int* __restrict__ site_of, const uint8_t* __restrict__ comp_of, const cx<T>* __restrict__ beta,
            int beta_stride, int64_t N, const cx<T>* __restrict__ twx, const cx<T>* __restrict__ twy,
            int* __restrict__ active, const cx<T>* __restrict__ krhat, KState* __restrict__ st,
            double2* __restrict__ part, unsigned* __restrict__ cnt, int part_stride) {
    using C = cx<T>;
    using CF = SliceCfg<LX, LY, sizeof(C)>;
    using PX = typename CF::PX;
    using PY = typename CF::PY;
    constexpr int NTH = CF::NTH, NX = CF::NX, NY = CF::NY, SPY = CF::SPY, TPR = CF::TPR, TPC = CF::TPC;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* plane = reinterpret_cast<C*>(smem_raw);  // [LX][SPY]
    C* colbuf = plane + LX * SPY;               // [CROWS][TPC]
    const int z = blockIdx.x, c = blockIdx.y, r = blockIdx.z, nz = gridDim.x;
    if (active != nullptr && active[r] == 0) return;
    // inverse y transform of every column kx, keep y < NY; the loads of the
    // next tile of columns are issued before the current one is transformed
    {
        const C* src = U2 + (((int64_t)r * 3 + c) * nz + z) * (int64_t)LY * LX;
        const int t = threadIdx.x % TPC, u = threadIdx.x / TPC;
        C* bt = colbuf + t;
        auto ld = [&](int pos) { return bt[exchange_row<LY, PY::NT, TPC, sizeof(C)>(pos) * TPC]; };
        auto stf = [&](int pos, C val) { bt[exchange_row<LY, PY::NT, TPC, sizeof(C)>(pos) * TPC] = val; };
        constexpr int R0 = stage_radix<PY, +1>(0), NB0 = PY::E / R0;
        C nxt[PY::E];
        auto prefetch = [&](int kx0) {
            const int kx = kx0 + t;
            const bool valid = kx < LX;
#pragma unroll
            for (int q = 0; q < NB0; ++q)
#pragma unroll
                for (int j = 0; j < R0; ++j)
                    nxt[q * R0 + j] = valid ? src[(int64_t)(u + q * PY::NT + j * (LY / R0)) * LX + kx] : czero<C>();
        };
        prefetch(0);
        for (int kx0 = 0; kx0 < LX; kx0 += TPC) {
            const int kx = kx0 + t;
            const bool valid = kx < LX;
            C v[PY::E];
#pragma unroll
            for (int i = 0; i < PY::E; ++i) v[i] = nxt[i];
            if (kx0 + TPC < LX) prefetch(kx0 + TPC);
            pencil_fft_regs<C, PY, +1>(v, u, twy, ld, stf);
            for_each_out<PY, +1, true>(u, [&](int idx, int y) {
                if (valid) plane[kx * SPY + y] = v[idx];
            });
        }
    }
    // the scatter's site indices and operands, loaded while the rows transform
    const int64_t off = ((int64_t)r * 3 + c) * N;
    const C* xs = X + off;
    C* ys = Y + off;
    const C* br = beta + (int64_t)r * beta_stride;
    const int* so = site_of + (int64_t)z * NY * NX;
    constexpr int NG = (NY * NX + NTH - 1) / NTH;
    int sidx[NG];
#pragma unroll
    for (int i = 0; i < NG; ++i) {
        const int e = threadIdx.x + i * NTH;
        sidx[i] = e < NY * NX ? so[e] : -1;
    }
    // (the 1/alpha lookup, a small L1-resident table, stays in the scatter;
    // with more than 8 sites per thread X is loaded there too, the registers
    // being needed by the row transforms)
    constexpr bool kHoistX = NG <= 8;
    C xv[NG];
    if constexpr (kHoistX) {
#pragma unroll
        for (int i = 0; i < NG; ++i) xv[i] = sidx[i] >= 0 ? xs[sidx[i]] : czero<C>();
    }
    __syncthreads();
    // inverse x transform of every row y < NY, in place, keep x < NX
    {
        const int t = threadIdx.x % TPR, u = threadIdx.x / TPR;
        for (int y0 = 0; y0 < NY; y0 += TPR) {
            C* bt = plane + y0 + t;
            auto first = [&](int pos) { return bt[pos * SPY]; };
            auto ld = [&](int pos) { return bt[pos * SPY]; };
            auto stf = [&](int pos, C val) { bt[pos * SPY] = val; };
            C v[PX::E];
            pencil_fft<C, PX, +1, false>(v, u, twx, first, ld, stf);
            __syncthreads();
            for_each_out<PX, +1, true>(u, [&](int idx, int pos) { bt[pos * SPY] = v[idx]; });
            __syncthreads();
        }
    }
    // diagonal term, scatter, fused Krylov dot products
    DotAcc<C> d[4];
#pragma unroll
    for (int i = 0; i < NG; ++i) {
        const int e = threadIdx.x + i * NTH, s = sidx[i];
        if constexpr (!kHoistX) xv[i] = s >= 0 ? xs[s] : czero<C>();
        if (s >= 0) {
            const C yv = cadd(plane[(e % NX) * SPY + e / NX], cmul(br[comp_of[s]], xv[i]));
            ys[s] = yv;
            if constexpr (MODE == 1) d[0].add_cdot(krhat[off + s], yv);
            if constexpr (MODE == 2) fused_dots_t(d, yv, xv[i], krhat[off + s]);
        }
    }
    if constexpr (MODE != 0) fused_partials<C, MODE>(d, part, r, part_stride);
}

// ---- launchers ---------------------------------------------------------------------
template <typename T> struct LaunchSlice {
    static constexpr bool kDouble = std::is_same<T, dfl>::value;
    template <int LX, int LY>
    static cudaError_t fwd(const Geom& g, int R, cx<T>* x, cx<T>* u2, const int* site_of, const cx<T>* twx,
                           const cx<T>* twy, const int* active, const FusedKrylov<T>& fk, cudaStream_t st, int kind) {
        using CF = SliceCfg<LX, LY, sizeof(cx<T>)>;
        if constexpr (!slice_built<LX, LY, sizeof(cx<T>)>()) {
            return cudaErrorInvalidValue;
        } else {
            dim3 grid(g.nz, 3, R);
            cudaError_t e;
            PROF_BEGIN(st);
            auto go = [&](auto kern) -> cudaError_t {
                cudaError_t ke = allow_smem(kern, CF::smem);
                if (ke == cudaSuccess)
                    kern<<<grid, CF::NTH, CF::smem, st>>>(x, u2, site_of, g.N, twx, twy, active, fwd_vecs(fk));
                return ke;
            };
            e = cudaSuccess;
            if (fk.mode == 0 || kDouble) {
                e = go(k_xyfwd<T, LX, LY, 0>);
            } else if constexpr (!kDouble) {
                if (fk.mode == 1) e = go(k_xyfwd<T, LX, LY, 1>);
                else if (fk.mode == 2) e = go(k_xyfwd<T, LX, LY, 2>);
                else e = go(k_xyfwd<T, LX, LY, 3>);
            }
            if (e != cudaSuccess) return e;
            PROF_END(kind, R, st);
            return cudaGetLastError();
        }
    }
    template <int LX, int LY>
    static cudaError_t inv(const Geom& g, int R, const cx<T>* u2, cx<T>* y, const cx<T>* x, const DevTarget& tg,
                           const cx<T>* beta, int beta_stride, const cx<T>* twx, const cx<T>* twy, int* active,
                           const FusedKrylov<T>& fk, cudaStream_t st, int kind) {
        using CF = SliceCfg<LX, LY, sizeof(cx<T>)>;
        if constexpr (!slice_built<LX, LY, sizeof(cx<T>)>()) {
            return cudaErrorInvalidValue;
        } else {
            dim3 grid(g.nz, 3, R);
            cudaError_t e;
            PROF_BEGIN(st);
            if (fk.mode == 0 || kDouble) {
                if ((e = allow_smem(k_yxinv<T, LX, LY, 0>, CF::smem)) != cudaSuccess) return e;
                k_yxinv<T, LX, LY, 0><<<grid, CF::NTH, CF::smem, st>>>(u2, y, x, tg.site_of, tg.comp_of, beta,
                                                                      beta_stride, g.N, twx, twy, active, nullptr,
                                                                      nullptr, nullptr, nullptr, 0);
            } else if constexpr (!kDouble) {
                if (inverse_mode(fk.mode) == 1) {
                    if ((e = allow_smem(k_yxinv<T, LX, LY, 1>, CF::smem)) != cudaSuccess) return e;
                    k_yxinv<T, LX, LY, 1><<<grid, CF::NTH, CF::smem, st>>>(u2, y, x, tg.site_of, tg.comp_of, beta,
                                                                          beta_stride, g.N, twx, twy, active,
                                                                          fk.rhat, fk.st, fk.part, fk.cnt,
                                                                          fk.part_stride);
                } else {
                    if ((e = allow_smem(k_yxinv<T, LX, LY, 2>, CF::smem)) != cudaSuccess) return e;
                    k_yxinv<T, LX, LY, 2><<<grid, CF::NTH, CF::smem, st>>>(u2, y, x, tg.site_of, tg.comp_of, beta,
                                                                          beta_stride, g.N, twx, twy, active,
                                                                          fk.rhat, fk.st, fk.part, fk.cnt,
                                                                          fk.part_stride);
                }
            }
            PROF_END(kind, R, st);
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
            if (fk.mode == 0 || kDouble) return cudaSuccess;
            return fused_finalize<T>(fk.mode, R, (int)(grid.x * grid.y), fk, active, st);
        }
    }
};

}  // namespace dda
