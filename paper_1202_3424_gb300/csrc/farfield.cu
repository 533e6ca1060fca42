// Far-field vector amplitudes of the dipole array ("Averaging over Scattering
// Directions", "Scattering by Finite Targets: The Mueller Matrix"):
//
//   F_r(n_d) = k^2 (I - n_d n_d) sum_j P_{r,j} exp(-i k n_d . r_j)
//
// for every right-hand side r and scattering direction n_d (the scattered
// field is exp(ikR)/R F at distance R along n_d, so dC_sca/dOmega = |F|^2).
// The sites lie on a lattice, so the phase factors separate,
// exp(-ik n.r) = ex(ix) ey(iy) ez(iz), with one table per axis and direction
// (FP64 on the host, rounded to the arithmetic type).  One block sums over
// all sites for TD directions of one RHS: each thread accumulates its share
// of the sites in registers, then the block reduces (warp sums in the
// arithmetic type, warp totals in FP64).
#include <cuda_runtime.h>

#include <algorithm>

#include "farfield.h"
#include "krylov_dev.cuh"
#include "profiler.h"

namespace dda {

namespace {

constexpr int kFFThreads = 256;
constexpr int kTD = 8;  // directions per block

template <typename C>
__global__ void __launch_bounds__(kFFThreads)
    k_farfield(int64_t N, const unsigned* __restrict__ site_xyz, const C* __restrict__ P, int ndir, int tab_len,
               const C* __restrict__ tabs, const double* __restrict__ dirs, double kd, double2* __restrict__ F) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* tab = reinterpret_cast<C*>(smem_raw);  // [kTD][tab_len]: the ex | ey | ez tables of the tile
    const int r = blockIdx.y;
    const int d0 = blockIdx.x * kTD;
    const int nd = min(kTD, ndir - d0);
    const int64_t tr = (int64_t)r * ndir;
    for (int e = threadIdx.x; e < kTD * tab_len; e += blockDim.x) {
        const int td = e / tab_len, i = e - td * tab_len;
        tab[e] = td < nd ? tabs[(tr + d0 + td) * tab_len + i] : czero<C>();
    }
    __syncthreads();
    const C* Pr = P + (int64_t)r * 3 * N;
    DotAcc<C> acc[kTD * 3];  // re/im partial sums of sum_j P_j phase_j
    for (int64_t j = (int64_t)blockIdx.z * blockDim.x + threadIdx.x; j < N; j += (int64_t)gridDim.z * blockDim.x) {
        const unsigned xyz = site_xyz[j];
        const int ix = xyz & 1023u, iy = (xyz >> 10) & 1023u, iz = xyz >> 20;
        const C p0 = Pr[j], p1 = Pr[N + j], p2 = Pr[2 * N + j];
#pragma unroll
        for (int td = 0; td < kTD; ++td) {
            const C* tt = tab + td * tab_len;
            const C ph = cmul(cmul(tt[ix], tt[tab_len / 3 + iy]), tt[2 * (tab_len / 3) + iz]);
            const C a = cmul(p0, ph), b = cmul(p1, ph), c = cmul(p2, ph);
            acc[td * 3 + 0].re += a.x;
            acc[td * 3 + 0].im += a.y;
            acc[td * 3 + 1].re += b.x;
            acc[td * 3 + 1].im += b.y;
            acc[td * 3 + 2].re += c.x;
            acc[td * 3 + 2].im += c.y;
        }
    }
    double2 tot[kTD * 3];
    block_totals<C, kTD * 3>(acc, tot);
    if (threadIdx.x == 0) {
        for (int td = 0; td < nd; ++td) {
            const double* n = dirs + (tr + d0 + td) * 3;
            double2 s[3];
            for (int a = 0; a < 3; ++a) s[a] = tot[td * 3 + a];
            // (I - n n) s, times k^2; partial sums of the site chunks add atomically
            const double2 ns = make_double2(n[0] * s[0].x + n[1] * s[1].x + n[2] * s[2].x,
                                            n[0] * s[0].y + n[1] * s[1].y + n[2] * s[2].y);
            double2* out = F + (tr + d0 + td) * 3;
            const double k2 = kd * kd;
            for (int a = 0; a < 3; ++a) {
                atomicAdd(&out[a].x, k2 * (s[a].x - n[a] * ns.x));
                atomicAdd(&out[a].y, k2 * (s[a].y - n[a] * ns.y));
            }
        }
    }
}

// tabs[(q*3 + a)*Lm + i] = exp(-i kd n_a (i - c_a)) for direction q, axis a (FP64 sincos)
template <typename C>
__global__ void k_phase_tables(int64_t nq, int Lm, double cx, double cy, double cz, double kd,
                               const double* __restrict__ dirs, C* __restrict__ tabs) {
    const int64_t total = nq * 3 * Lm;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(e % Lm);
        const int64_t qa = e / Lm;
        const int a = (int)(qa % 3);
        const double c = a == 0 ? cx : (a == 1 ? cy : cz);
        double sn, cs;
        sincos(-kd * dirs[qa] * (i - c), &sn, &cs);
        tabs[e] = ccast<C>(make_double2(cs, sn));
    }
}

}  // namespace

template <typename C>
cudaError_t launch_phase_tables(int64_t nq, int Lm, const double c[3], double kd, const double* dirs, C* tabs,
                                cudaStream_t st) {
    const int64_t total = nq * 3 * Lm;
    const int blocks = (int)std::min<int64_t>((total + 255) / 256, 152 * 16);
    PROF_BEGIN(st);
    k_phase_tables<C><<<blocks, 256, 0, st>>>(nq, Lm, c[0], c[1], c[2], kd, dirs, tabs);
    PROF_END(KK_FARFIELD, 1, st);
    return cudaGetLastError();
}
template cudaError_t launch_phase_tables<float2>(int64_t, int, const double*, double, const double*, float2*,
                                                 cudaStream_t);
template cudaError_t launch_phase_tables<double2>(int64_t, int, const double*, double, const double*, double2*,
                                                  cudaStream_t);

template <typename C>
cudaError_t launch_farfield(int R, int64_t N, const unsigned* site_xyz, const C* P, int ndir, int tab_len,
                            const C* tabs, const double* dirs, double kd, double2* F, cudaStream_t st) {
    if (tab_len % 3) return cudaErrorInvalidValue;
    cudaError_t e = cudaMemsetAsync(F, 0, (size_t)R * ndir * 3 * sizeof(double2), st);
    if (e != cudaSuccess) return e;
    const size_t sm = (size_t)kTD * tab_len * sizeof(C);
    if (sm > 48 * 1024) {
        e = cudaFuncSetAttribute(k_farfield<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
    }
    // site chunks per (direction tile, RHS): enough blocks to fill the GPU
    const int tiles = (ndir + kTD - 1) / kTD;
    const int64_t want = 4 * 152;
    int chunks = (int)std::max<int64_t>(1, std::min<int64_t>((N + kFFThreads - 1) / kFFThreads,
                                                             (want + (int64_t)tiles * R - 1) / ((int64_t)tiles * R)));
    chunks = std::min(chunks, 65535);
    PROF_BEGIN(st);
    k_farfield<C><<<dim3(tiles, R, chunks), kFFThreads, sm, st>>>(N, site_xyz, P, ndir, tab_len, tabs, dirs, kd, F);
    PROF_END(KK_FARFIELD, R, st);
    return cudaGetLastError();
}

template cudaError_t launch_farfield<float2>(int, int64_t, const unsigned*, const float2*, int, int, const float2*,
                                             const double*, double, double2*, cudaStream_t);
template cudaError_t launch_farfield<double2>(int, int64_t, const unsigned*, const double2*, int, int, const double2*,
                                              const double*, double, double2*, cudaStream_t);

}  // namespace dda
