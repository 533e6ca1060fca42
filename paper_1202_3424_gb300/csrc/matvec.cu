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
//           half zero)                                  -> U1 [nz][ny][Lx]
//   y-fwd   FFT along y (input half zero)               -> U2 [nz][Ly][Lx]
//   z-conv  for each (kx,ky) column, all three components: FFT along z
//           (input half zero), multiply by the symmetric 3x3 Ghat in
//           registers, inverse FFT along z, keep z < nz  -> U2 in place
//   y-inv   inverse FFT along y, keep y < ny            -> U1
//   x-inv   inverse FFT along x, keep x < nx, add (1/alpha) P, scatter to
//           the compact site vector
// Ghat is stored as one octant (k <= L/2 on each axis) of the transformed
// kernel: each component is even or odd under each axis reflection, so
// Ghat(L-k) = +/- Ghat(k).  The 1/(Lx Ly Lz) of the inverse transform is
// folded into Ghat.
#include <cstdio>
#include <mutex>
#include <unordered_map>

#include "fft.cuh"
#include "internal.h"
#include "profiler.h"

namespace dda {

// ---- tile sizes ------------------------------------------------------------
// x passes stage TP rows through shared memory (TP+1 stride); strided passes
// take TP adjacent pencils (coalesced across them); the z pass takes TP
// adjacent columns for each of 3 component groups.
template <int L> __host__ __device__ constexpr int tp_x() {
    return (256 / Plan<L>::NT) > 64 ? 64 : (256 / Plan<L>::NT);
}
template <int L> __host__ __device__ constexpr int tp_s() {
    return (256 / Plan<L>::NT) > 32 ? 32 : ((256 / Plan<L>::NT) < 8 ? 8 : (256 / Plan<L>::NT));
}
// z pass: 3*TP*NT threads per block; TP adjacent columns.  (Blocks of 768
// threads with 128-byte shared-memory rows were measured slower than two
// blocks of 384 per SM on the 128^3 grid.)
template <int L, typename T> __host__ __device__ constexpr int tp_z() {
    return (128 / Plan<L>::NT) > 32 ? 32 : ((128 / Plan<L>::NT) < 4 ? 4 : (128 / Plan<L>::NT));
}

// ---- x-forward: gather + row FFT ---------------------------------------------
// Rows (iy, iz) of the padded-to-L/2 lattice; lattice sites x < LX/2.
template <typename T, int LX>
__global__ void __launch_bounds__(tp_x<LX>() * Plan<LX>::NT)
    k_xfwd(const cx<T>* __restrict__ X, cx<T>* __restrict__ U1, const int* __restrict__ site_of, int nrows,
           int64_t N, const cx<T>* __restrict__ tw, const int* __restrict__ active) {
    using C = cx<T>;
    using PL = Plan<LX>;
    constexpr int TP = tp_x<LX>(), SP = TP + 1, NX = LX / 2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* buf = reinterpret_cast<C*>(smem_raw);
    const int c = blockIdx.y, r = blockIdx.z;
    if (active != nullptr && active[r] == 0) return;
    const int row0 = blockIdx.x * TP;
    const C* xs = X + ((int64_t)r * 3 + c) * N;
    for (int e = threadIdx.x; e < TP * NX; e += blockDim.x) {
        const int t = e / NX, ix = e - t * NX, row = row0 + t;
        C val = czero<C>();
        if (row < nrows) {
            const int s = site_of[(int64_t)row * NX + ix];
            if (s >= 0) val = xs[s];
        }
        buf[ix * SP + t] = val;
    }
    __syncthreads();
    const int t = threadIdx.x % TP, u = threadIdx.x / TP;
    C* bt = buf + t;
    C v[PL::E];
    auto first = [&](int pos) { return bt[pos * SP]; };
    auto ld = [&](int pos) { return bt[pos * SP]; };
    auto st = [&](int pos, C val) { bt[pos * SP] = val; };
    pencil_fft<C, PL, -1, true>(v, u, tw, first, ld, st);
    __syncthreads();
    for_each_out<PL, -1, false>(u, [&](int idx, int pos) { bt[pos * SP] = v[idx]; });
    __syncthreads();
    C* out = U1 + ((int64_t)r * 3 + c) * (int64_t)nrows * LX;
    for (int e = threadIdx.x; e < TP * LX; e += blockDim.x) {
        const int t2 = e / LX, x = e - t2 * LX, row = row0 + t2;
        if (row < nrows) out[(int64_t)row * LX + x] = buf[x * SP + t2];
    }
}

// ---- x-inverse: row IFFT + diagonal + scatter -----------------------------------
template <typename T, int LX>
__global__ void __launch_bounds__(tp_x<LX>() * Plan<LX>::NT)
    k_xinv(const cx<T>* __restrict__ U1, cx<T>* __restrict__ Y, const cx<T>* __restrict__ X,
           const int* __restrict__ site_of, const uint8_t* __restrict__ comp_of, const cx<T>* __restrict__ beta,
           int beta_stride, int nrows, int64_t N, const cx<T>* __restrict__ tw, const int* __restrict__ active) {
    using C = cx<T>;
    using PL = Plan<LX>;
    constexpr int TP = tp_x<LX>(), SP = TP + 1, NX = LX / 2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* buf = reinterpret_cast<C*>(smem_raw);
    const int c = blockIdx.y, r = blockIdx.z;
    if (active != nullptr && active[r] == 0) return;
    const int row0 = blockIdx.x * TP;
    const C* in = U1 + ((int64_t)r * 3 + c) * (int64_t)nrows * LX;
    for (int e = threadIdx.x; e < TP * LX; e += blockDim.x) {
        const int t2 = e / LX, x = e - t2 * LX, row = row0 + t2;
        buf[x * SP + t2] = row < nrows ? in[(int64_t)row * LX + x] : czero<C>();
    }
    __syncthreads();
    const int t = threadIdx.x % TP, u = threadIdx.x / TP;
    C* bt = buf + t;
    C v[PL::E];
    auto first = [&](int pos) { return bt[pos * SP]; };
    auto ld = [&](int pos) { return bt[pos * SP]; };
    auto st = [&](int pos, C val) { bt[pos * SP] = val; };
    pencil_fft<C, PL, +1, false>(v, u, tw, first, ld, st);
    __syncthreads();
    for_each_out<PL, +1, true>(u, [&](int idx, int pos) { bt[pos * SP] = v[idx]; });
    __syncthreads();
    const C* xs = X + ((int64_t)r * 3 + c) * N;
    C* ys = Y + ((int64_t)r * 3 + c) * N;
    const C* br = beta + (int64_t)r * beta_stride;
    for (int e = threadIdx.x; e < TP * NX; e += blockDim.x) {
        const int t2 = e / NX, ix = e - t2 * NX, row = row0 + t2;
        if (row < nrows) {
            const int s = site_of[(int64_t)row * NX + ix];
            if (s >= 0) ys[s] = cadd(buf[ix * SP + t2], cmul(br[comp_of[s]], xs[s]));
        }
    }
}

// ---- strided pencils (y passes; y and z passes of the Green tensor) -----------
// Pencil (b, w): points at src + b*src_bstride + w + pos*pt_stride; outputs
// to dst likewise.  MODE 0: forward with input positions >= L/2 zero;
// MODE 1: inverse keeping positions < L/2; MODE 2: full forward transform.
// TP pencils adjacent in w per block, so loads and stores coalesce across w.
template <typename T, int L, int MODE>
__global__ void __launch_bounds__(tp_s<L>() * Plan<L>::NT)
    k_strided(const cx<T>* src, cx<T>* dst, int64_t pt_stride, int width, int64_t src_bstride, int64_t dst_bstride,
              int batches_per_rhs, const cx<T>* __restrict__ tw, const int* __restrict__ active) {
    using C = cx<T>;
    using PL = Plan<L>;
    constexpr int TP = tp_s<L>();
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
    auto ld = [&](int pos) { return bt[pos * TP]; };
    auto st = [&](int pos, C val) { bt[pos * TP] = val; };
    pencil_fft<C, PL, DIR, MODE == 0>(v, u, tw, first, ld, st);
    for_each_out<PL, DIR, MODE == 1>(u, [&](int idx, int pos) {
        if (valid) d[pos * pt_stride] = v[idx];
    });
}

// ---- z pass with the Fourier-space product ------------------------------------
// One block owns TP adjacent (kx) columns at one ky for one RHS; its threads
// form three groups, one per Cartesian component c.  Group c transforms P_c
// along z (input half zero), writes the spectrum to its shared-memory plane,
// and after a barrier forms row c of the symmetric product
//   Y_c(k) = sum_b Ghat_cb(k) P_b(k)
// for the points it holds, then inverse-transforms Y_c and keeps z < LZ/2.
template <typename T, int LZ>
__global__ void __launch_bounds__(3 * tp_z<LZ, T>() * Plan<LZ>::NT)
    k_zconv(cx<T>* __restrict__ U2, const cx<T>* __restrict__ gh, int Lx, int Ly, const cx<T>* __restrict__ tw,
            const int* __restrict__ active) {
    using C = cx<T>;
    using PL = Plan<LZ>;
    constexpr int TP = tp_z<LZ, T>(), NT = PL::NT, NZ = LZ / 2;
    static_assert((TP * NT) % 32 == 0, "component groups must be whole warps");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* buf = reinterpret_cast<C*>(smem_raw);  // [3][LZ][TP]
    const int ky = blockIdx.y, r = blockIdx.z;
    if (active != nullptr && active[r] == 0) return;
    const int t = threadIdx.x % TP;
    const int rest = threadIdx.x / TP;
    const int u = rest % NT, c = rest / NT;
    const int kx = blockIdx.x * TP + t;
    const bool valid = kx < Lx;
    const int64_t plane = (int64_t)Ly * Lx;
    C* bc = U2 + ((int64_t)r * 3 + c) * NZ * plane + (int64_t)ky * Lx + (valid ? kx : 0);
    C* sb = buf + c * (LZ * TP) + t;
    auto ld = [&](int pos) { return sb[pos * TP]; };
    auto st = [&](int pos, C val) { sb[pos * TP] = val; };
    C v[PL::E];
    auto first = [&](int pos) { return valid ? bc[pos * plane] : czero<C>(); };
    pencil_fft<C, PL, -1, true>(v, u, tw, first, ld, st);
    __syncthreads();
    for_each_out<PL, -1, false>(u, [&](int idx, int pos) { sb[pos * TP] = v[idx]; });
    __syncthreads();
    // row c of the octant-stored symmetric tensor: components (xx,xy,xz,yy,yz,zz)
    const int i0 = c == 0 ? 0 : (c == 1 ? 1 : 2);
    const int i1 = c == 0 ? 1 : (c == 1 ? 3 : 4);
    const int i2 = c == 0 ? 2 : (c == 1 ? 4 : 5);
    const int hx = Lx / 2 + 1, hy = Ly / 2 + 1, hz = LZ / 2 + 1;
    const int kxv = valid ? kx : 0;
    const int kxo = kxv <= Lx / 2 ? kxv : Lx - kxv;
    const int kyo = ky <= Ly / 2 ? ky : Ly - ky;
    const bool fx = kxv > Lx / 2, fy = ky > Ly / 2;
    const int64_t cs = (int64_t)hz * hy * hx;
    const C* g0 = gh + (int64_t)kyo * hx + kxo;
    const C* p0b = buf + t;
    for_each_out<PL, -1, false>(u, [&](int idx, int kz) {
        const bool fz = kz > LZ / 2;
        const int kzo = fz ? LZ - kz : kz;
        const C* g = g0 + (int64_t)kzo * hy * hx;
        // odd components flip sign under a reflection of one of their two axes
        const bool sxy = fx != fy, sxz = fx != fz, syz = fy != fz;
        C a0 = g[i0 * cs], a1 = g[i1 * cs], a2 = g[i2 * cs];
        if (c == 0) { if (sxy) a1 = cscale(a1, T(-1)); if (sxz) a2 = cscale(a2, T(-1)); }
        if (c == 1) { if (sxy) a0 = cscale(a0, T(-1)); if (syz) a2 = cscale(a2, T(-1)); }
        if (c == 2) { if (sxz) a0 = cscale(a0, T(-1)); if (syz) a1 = cscale(a1, T(-1)); }
        const C pa = p0b[kz * TP], pb = p0b[LZ * TP + kz * TP], pc = p0b[2 * LZ * TP + kz * TP];
        v[idx] = cadd(cadd(cmul(a0, pa), cmul(a1, pb)), cmul(a2, pc));
    });
    pencil_fft_regs<C, PL, +1>(v, u, tw, ld, st);
    for_each_out<PL, +1, true>(u, [&](int idx, int pos) {
        if (valid) bc[pos * plane] = v[idx];
    });
}

// ---- Green tensor on the padded grid ------------------------------------------
// Displacement along an axis for padded index i: i for i < n, i - L for
// i > L - n, none otherwise (those entries, and r = 0, are zero).
__device__ __forceinline__ bool pad_disp(int i, int n, int L, int& d) {
    if (i < n) { d = i; return true; }
    if (i > L - n) { d = i - L; return true; }
    return false;
}

// A(r) = exp(ik rho)/rho [k^2 (rr - I) + (ik rho - 1)/rho^2 (3 rr - I)]
// (Draine 1988 off-diagonal block, lattice units), components xx,xy,xz,yy,yz,zz.
__global__ void k_green(double2* __restrict__ g, int nx, int ny, int nz, int Lx, int Ly, int Lz, double kd) {
    const int64_t total = (int64_t)Lx * Ly * Lz;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int ix = (int)(idx % Lx);
        const int iy = (int)((idx / Lx) % Ly);
        const int iz = (int)(idx / ((int64_t)Lx * Ly));
        int dx, dy, dz;
        double2 a[6];
#pragma unroll
        for (int c = 0; c < 6; ++c) a[c] = make_double2(0.0, 0.0);
        if (pad_disp(ix, nx, Lx, dx) && pad_disp(iy, ny, Ly, dy) && pad_disp(iz, nz, Lz, dz) &&
            (dx | dy | dz) != 0) {
            const double rho2 = (double)dx * dx + (double)dy * dy + (double)dz * dz;
            const double rho = sqrt(rho2);
            const double rh[3] = {dx / rho, dy / rho, dz / rho};
            double sn, cs;
            sincos(kd * rho, &sn, &cs);
            const double2 ph = make_double2(cs / rho, sn / rho);             // exp(ik rho)/rho
            const double2 c1 = make_double2(kd * kd * ph.x, kd * kd * ph.y);  // k^2 ph
            const double2 t = make_double2(-1.0 / rho2, kd / rho);           // (ik rho - 1)/rho^2
            const double2 c2 = cmul(ph, t);
            const int ia[6] = {0, 0, 0, 1, 1, 2}, ib[6] = {0, 1, 2, 1, 2, 2};
#pragma unroll
            for (int c = 0; c < 6; ++c) {
                const double rr = rh[ia[c]] * rh[ib[c]];
                const double dl = ia[c] == ib[c] ? 1.0 : 0.0;
                const double f1 = rr - dl, f2 = 3.0 * rr - dl;
                a[c] = make_double2(c1.x * f1 + c2.x * f2, c1.y * f1 + c2.y * f2);
            }
        }
#pragma unroll
        for (int c = 0; c < 6; ++c) g[c * total + idx] = a[c];
    }
}

// In-place forward FFT of dense rows of length LX (Green tensor x pass).
template <int LX>
__global__ void __launch_bounds__(tp_x<LX>() * Plan<LX>::NT)
    k_xfull(double2* __restrict__ data, int64_t nrows, const double2* __restrict__ tw) {
    using C = double2;
    using PL = Plan<LX>;
    constexpr int TP = tp_x<LX>(), SP = TP + 1;
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

__global__ void k_octant(const double2* __restrict__ g, double2* __restrict__ gh, int Lx, int Ly, int Lz,
                         double scale) {
    const int hx = Lx / 2 + 1, hy = Ly / 2 + 1, hz = Lz / 2 + 1;
    const int64_t per = (int64_t)hx * hy * hz, total = 6 * per;
    const int64_t full = (int64_t)Lx * Ly * Lz;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(idx / per);
        const int64_t rem = idx - c * per;
        const int kx = (int)(rem % hx), ky = (int)((rem / hx) % hy), kz = (int)(rem / ((int64_t)hx * hy));
        const double2 v = g[c * full + ((int64_t)kz * Ly + ky) * Lx + kx];
        gh[idx] = make_double2(v.x * scale, v.y * scale);
    }
}

__global__ void k_c128_to_c64(const double2* __restrict__ s, float2* __restrict__ d, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        d[i] = make_float2((float)s[i].x, (float)s[i].y);
}

// ---- host launchers -------------------------------------------------------------
int pick_fft_length(int n) {
    for (int L : kSupportedLengths)
        if (L >= 2 * n) return L;
    return 0;
}

// Give a kernel the maximum shared-memory carveout and, above 48 KB, the
// dynamic shared-memory size it needs -- once per kernel
// (so that only launches happen while a stream is being captured).
template <typename K> static cudaError_t allow_smem(K kernel, size_t bytes) {
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

static unsigned grid1d(int64_t n, int threads) {
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

template <typename T> struct LaunchX {
    static constexpr int koff = sizeof(T) == 4 ? 0 : (KK_XFWD_C128 - KK_XFWD_C64);
    template <int LX>
    static cudaError_t fwd(const Geom& g, int R, const cx<T>* x, cx<T>* u1, const int* site_of, const cx<T>* tw,
                           const int* active, cudaStream_t st) {
        constexpr int TP = tp_x<LX>(), NTH = TP * Plan<LX>::NT;
        const size_t sm = (size_t)LX * (TP + 1) * sizeof(cx<T>);
        cudaError_t e = allow_smem(k_xfwd<T, LX>, sm);
        if (e != cudaSuccess) return e;
        const int nrows = g.ny * g.nz;
        dim3 grid((nrows + TP - 1) / TP, 3, R);
        PROF_BEGIN(st);
        k_xfwd<T, LX><<<grid, NTH, sm, st>>>(x, u1, site_of, nrows, g.N, tw, active);
        PROF_END(KK_XFWD_C64 + koff, R, st);
        return cudaGetLastError();
    }
    template <int LX>
    static cudaError_t inv(const Geom& g, int R, const cx<T>* u1, cx<T>* y, const cx<T>* x, const DevTarget& tg,
                           const cx<T>* beta, int beta_stride, const cx<T>* tw, const int* active, cudaStream_t st) {
        constexpr int TP = tp_x<LX>(), NTH = TP * Plan<LX>::NT;
        const size_t sm = (size_t)LX * (TP + 1) * sizeof(cx<T>);
        cudaError_t e = allow_smem(k_xinv<T, LX>, sm);
        if (e != cudaSuccess) return e;
        const int nrows = g.ny * g.nz;
        dim3 grid((nrows + TP - 1) / TP, 3, R);
        PROF_BEGIN(st);
        k_xinv<T, LX><<<grid, NTH, sm, st>>>(u1, y, x, tg.site_of, tg.comp_of, beta, beta_stride, nrows, g.N, tw,
                                            active);
        PROF_END(KK_XINV_C64 + koff, R, st);
        return cudaGetLastError();
    }
    template <int MODE, int L>
    static cudaError_t strided_mode(const cx<T>* src, cx<T>* dst, int64_t pt_stride, int width, int64_t sb,
                                    int64_t db, int batches, int per_rhs, const cx<T>* tw, const int* active,
                                    cudaStream_t st, int kind, double units) {
        constexpr int TP = tp_s<L>(), NTH = TP * Plan<L>::NT;
        const size_t sm = (size_t)L * TP * sizeof(cx<T>);
        cudaError_t e = allow_smem(k_strided<T, L, MODE>, sm);
        if (e != cudaSuccess) return e;
        dim3 grid((width + TP - 1) / TP, batches, 1);
        PROF_BEGIN(st);
        k_strided<T, L, MODE><<<grid, NTH, sm, st>>>(src, dst, pt_stride, width, sb, db, per_rhs, tw, active);
        PROF_END(kind, units, st);
        return cudaGetLastError();
    }
    template <int L>
    static cudaError_t strided(int mode, const cx<T>* src, cx<T>* dst, int64_t pt_stride, int width, int64_t sb,
                               int64_t db, int batches, int per_rhs, const cx<T>* tw, const int* active,
                               cudaStream_t st, int kind, double units) {
        if (mode == 0)
            return strided_mode<0, L>(src, dst, pt_stride, width, sb, db, batches, per_rhs, tw, active, st, kind, units);
        if (mode == 1)
            return strided_mode<1, L>(src, dst, pt_stride, width, sb, db, batches, per_rhs, tw, active, st, kind, units);
        return strided_mode<2, L>(src, dst, pt_stride, width, sb, db, batches, per_rhs, tw, active, st, kind, units);
    }
    template <int LZ>
    static cudaError_t zconv(const Geom& g, int R, cx<T>* u2, const cx<T>* gh, const cx<T>* tw, const int* active,
                             cudaStream_t st) {
        constexpr int TP = tp_z<LZ, T>(), NTH = 3 * TP * Plan<LZ>::NT;
        const size_t sm = (size_t)3 * LZ * TP * sizeof(cx<T>);
        cudaError_t e = allow_smem(k_zconv<T, LZ>, sm);
        if (e != cudaSuccess) return e;
        dim3 grid((g.Lx + TP - 1) / TP, g.Ly, R);
        PROF_BEGIN(st);
        k_zconv<T, LZ><<<grid, NTH, sm, st>>>(u2, gh, g.Lx, g.Ly, tw, active);
        PROF_END(KK_ZCONV_C64 + koff, R, st);
        return cudaGetLastError();
    }
};

template <int LX> static cudaError_t launch_xfull(double2* data, int64_t nrows, const double2* tw, cudaStream_t st) {
    constexpr int TP = tp_x<LX>(), NTH = TP * Plan<LX>::NT;
    const size_t sm = (size_t)LX * (TP + 1) * sizeof(double2);
    cudaError_t e = allow_smem(k_xfull<LX>, sm);
    if (e != cudaSuccess) return e;
    PROF_BEGIN(st);
    k_xfull<LX><<<(unsigned)((nrows + TP - 1) / TP), NTH, sm, st>>>(data, nrows, tw);
    PROF_END(KK_GREEN, 1.0, st);
    return cudaGetLastError();
}

// The lattice seen by the kernels is padded with vacuum to exactly L/2 sites
// per axis (g.nx == g.Lx/2, ...), see dda_set_target.
template <typename T>
cudaError_t launch_matvec(const Geom& g, int R, const cx<T>* x, cx<T>* y, const PadWork<T>& w, const DevTarget& tg,
                          const cx<T>* beta, int beta_stride, const cx<T>* ghat, const Twiddles<T>& tw,
                          const int* active, cudaStream_t st) {
    using LX = LaunchX<T>;
    if (g.nx * 2 != g.Lx || g.ny * 2 != g.Ly || g.nz * 2 != g.Lz) return cudaErrorInvalidValue;
    cudaError_t e;
    auto fwdx = [&]() -> cudaError_t { DDA_DISPATCH_L(g.Lx, LX::template fwd, g, R, x, w.u1, tg.site_of, tw.x, active, st); };
    auto ys = [&](int mode, const cx<T>* s, cx<T>* d, int64_t sb, int64_t db) -> cudaError_t {
        DDA_DISPATCH_L(g.Ly, LX::template strided, mode, s, d, (int64_t)g.Lx, g.Lx, sb, db, R * 3 * g.nz, 3 * g.nz,
                       tw.y, active, st, (mode == 0 ? KK_YFWD_C64 : KK_YINV_C64) + LX::koff, (double)R);
    };
    auto zc = [&]() -> cudaError_t { DDA_DISPATCH_L(g.Lz, LX::template zconv, g, R, w.u2, ghat, tw.z, active, st); };
    auto invx = [&]() -> cudaError_t {
        DDA_DISPATCH_L(g.Lx, LX::template inv, g, R, w.u1, y, x, tg, beta, beta_stride, tw.x, active, st);
    };
    if ((e = fwdx()) != cudaSuccess) return e;
    if ((e = ys(0, w.u1, w.u2, (int64_t)g.ny * g.Lx, (int64_t)g.Ly * g.Lx)) != cudaSuccess) return e;
    if ((e = zc()) != cudaSuccess) return e;
    if ((e = ys(1, w.u2, w.u1, (int64_t)g.Ly * g.Lx, (int64_t)g.ny * g.Lx)) != cudaSuccess) return e;
    return invx();
}

template cudaError_t launch_matvec<float>(const Geom&, int, const float2*, float2*, const PadWork<float>&,
                                          const DevTarget&, const float2*, int, const float2*, const Twiddles<float>&,
                                          const int*, cudaStream_t);
template cudaError_t launch_matvec<double>(const Geom&, int, const double2*, double2*, const PadWork<double>&,
                                           const DevTarget&, const double2*, int, const double2*,
                                           const Twiddles<double>&, const int*, cudaStream_t);

cudaError_t launch_green_fft(const Geom& g, double kd, double2* scratch, double2* ghat64, const Twiddles<double>& tw,
                             cudaStream_t st) {
    const int64_t full = (int64_t)g.Lx * g.Ly * g.Lz;
    PROF_BEGIN(st);
    k_green<<<grid1d(full, 256), 256, 0, st>>>(scratch, g.nx, g.ny, g.nz, g.Lx, g.Ly, g.Lz, kd);
    PROF_END(KK_GREEN, 1.0, st);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    auto xf = [&]() -> cudaError_t { DDA_DISPATCH_L(g.Lx, launch_xfull, scratch, 6 * (int64_t)g.Lz * g.Ly, tw.x, st); };
    if ((e = xf()) != cudaSuccess) return e;
    using LX = LaunchX<double>;
    auto yf = [&]() -> cudaError_t {
        DDA_DISPATCH_L(g.Ly, LX::template strided, 2, scratch, scratch, (int64_t)g.Lx, g.Lx, (int64_t)g.Ly * g.Lx,
                       (int64_t)g.Ly * g.Lx, 6 * g.Lz, 1, tw.y, nullptr, st, KK_GREEN, 1.0);
    };
    if ((e = yf()) != cudaSuccess) return e;
    auto zf = [&]() -> cudaError_t {
        DDA_DISPATCH_L(g.Lz, LX::template strided, 2, scratch, scratch, (int64_t)g.Ly * g.Lx, g.Ly * g.Lx, full, full,
                       6, 1, tw.z, nullptr, st, KK_GREEN, 1.0);
    };
    if ((e = zf()) != cudaSuccess) return e;
    const int64_t oct = 6 * (int64_t)g.hx() * g.hy() * g.hz();
    PROF_BEGIN(st);
    k_octant<<<grid1d(oct, 256), 256, 0, st>>>(scratch, ghat64, g.Lx, g.Ly, g.Lz, 1.0 / (double)full);
    PROF_END(KK_GREEN, 1.0, st);
    return cudaGetLastError();
}

cudaError_t launch_convert_c128_to_c64(const double2* src, float2* dst, int64_t n, cudaStream_t st) {
    k_c128_to_c64<<<grid1d(n, 256), 256, 0, st>>>(src, dst, n);
    return cudaGetLastError();
}

}  // namespace dda
