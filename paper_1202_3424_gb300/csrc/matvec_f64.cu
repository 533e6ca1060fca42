// complex128 instantiation of the matvec passes, the Green-tensor build and shared host helpers.
#include "matvec_impl.cuh"

namespace dda {

template int zconv_schedules<double>(const Geom&);
template int xpass_schedules<double>(const Geom&);
template int ypass_schedules<double>(const Geom&);
template cudaError_t launch_zconv<double>(const Geom&, int, double2*, const double2*, const double2*, const int*, int, cudaStream_t);
template cudaError_t launch_matvec<double>(const Geom&, int, const double2*, double2*, const PadWork<double>&,
                                           const DevTarget&, const double2*, int, const double2*,
                                           const Twiddles<double>&, const int*, cudaStream_t);
template cudaError_t launch_matvec_fused<double>(const Geom&, int, double2*, double2*, const PadWork<double>&,
                                                 const DevTarget&, const double2*, int, const double2*,
                                                 const Twiddles<double>&, int*, const FusedKrylov<double>&,
                                                 cudaStream_t);

int pick_fft_length(int n) {
    for (int L : kSupportedLengths)
        if (L >= 2 * n) return L;
    return 0;
}

// Blocks of one RHS in the x-inverse pass (partial-sum slots per RHS): the
// most among the staged tilings of complex64 and 16-byte elements and the
// warp-local blocks of every plan variant.
template <int L, int V = 0> static int min_xwi_rows() {
    int tp = xwi_rows<XwPlan<L, V>>();
    if constexpr (V + 1 < xw_variants(L)) {
        const int rest = min_xwi_rows<L, V + 1>();
        tp = rest < tp ? rest : tp;
    }
    return tp;
}
template <int L> static int min_tp_x() {
    int tp = tp_x<L, 8>() < tp_x<L, 16>() ? tp_x<L, 8>() : tp_x<L, 16>();
    return min_xwi_rows<L>() < tp ? min_xwi_rows<L>() : tp;
}
int xinv_blocks_per_rhs(const Geom& g) {
    const int nrows = g.ny * g.nz;
    int tp = 1;
    switch (g.Lx) {
        case 16: tp = min_tp_x<16>(); break;
        case 32: tp = min_tp_x<32>(); break;
        case 48: tp = min_tp_x<48>(); break;
        case 64: tp = min_tp_x<64>(); break;
        case 96: tp = min_tp_x<96>(); break;
        case 128: tp = min_tp_x<128>(); break;
        case 192: tp = min_tp_x<192>(); break;
        case 256: tp = min_tp_x<256>(); break;
        case 384: tp = min_tp_x<384>(); break;
        case 512: tp = min_tp_x<512>(); break;
        default: tp = 1;
    }
    return 3 * ((nrows + tp - 1) / tp);
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

template <typename D, typename S>
__global__ void k_cconvert(const S* __restrict__ s, D* __restrict__ d, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        d[i] = ccast<D>(s[i]);
}

template <int LX> static cudaError_t launch_xfull(double2* data, int64_t nrows, const double2* tw, cudaStream_t st) {
    constexpr int TP = tp_x<LX, 16>(), NTH = TP * Plan<LX>::NT;
    const size_t sm = (size_t)LX * (TP + 1) * sizeof(double2);
    cudaError_t e = allow_smem(k_xfull<LX>, sm);
    if (e != cudaSuccess) return e;
    PROF_BEGIN(st);
    k_xfull<LX><<<(unsigned)((nrows + TP - 1) / TP), NTH, sm, st>>>(data, nrows, tw);
    PROF_END(KK_GREEN, 1.0, st);
    return cudaGetLastError();
}

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

cudaError_t launch_convert_c128_to_df(const double2* src, cdfl* dst, int64_t n, cudaStream_t st) {
    k_cconvert<cdfl, double2><<<grid1d(n, 256), 256, 0, st>>>(src, dst, n);
    return cudaGetLastError();
}

cudaError_t launch_convert_df_to_c128(const cdfl* src, double2* dst, int64_t n, cudaStream_t st) {
    k_cconvert<double2, cdfl><<<grid1d(n, 256), 256, 0, st>>>(src, dst, n);
    return cudaGetLastError();
}

cudaError_t launch_convert_c128_to_c64(const double2* src, float2* dst, int64_t n, cudaStream_t st) {
    k_c128_to_c64<<<grid1d(n, 256), 256, 0, st>>>(src, dst, n);
    return cudaGetLastError();
}



}  // namespace dda
