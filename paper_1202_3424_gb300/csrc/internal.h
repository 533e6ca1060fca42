// Internal (non-ABI) declarations shared by the CUDA translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <complex>
#include <string>
#include <vector>

#include "common.cuh"

namespace dda {

// Lattice and padded-grid geometry.  The caller's lattice ox*oy*oz is
// extended with vacuum to nx*ny*nz = (Lx/2)*(Ly/2)*(Lz/2), where Lx,Ly,Lz are
// the supported FFT lengths >= 2*ox, ...; the kernels only ever see the
// extended lattice.  Lattice index of site (ix,iy,iz) is (iz*ny + iy)*nx + ix
// on the extended lattice; positions use the original box centre.  The stored
// octant of the transformed Green tensor has (Lz/2+1)(Ly/2+1)(Lx/2+1) points
// per component.
struct Geom {
    int ox = 0, oy = 0, oz = 0;  // caller's lattice
    int nx = 0, ny = 0, nz = 0;  // extended lattice (L/2 per axis)
    int Lx = 0, Ly = 0, Lz = 0;
    int64_t N = 0;  // occupied sites
    int hx() const { return Lx / 2 + 1; }
    int hy() const { return Ly / 2 + 1; }
    int hz() const { return Lz / 2 + 1; }
    int64_t M() const { return (int64_t)nx * ny * nz; }
    int64_t u1_per_comp() const { return (int64_t)nz * ny * Lx; }
    int64_t u2_per_comp() const { return (int64_t)nz * Ly * Lx; }
    int64_t oct_per_comp() const { return (int64_t)hz() * hy() * hx(); }
};

// Device-side target description.
struct DevTarget {
    int* site_of = nullptr;        // [M] lattice -> site index, -1 for vacuum
    int* lat_of = nullptr;         // [N] site -> lattice index
    uint8_t* comp_of = nullptr;    // [N] composition code 1..ncomp
    // the x rows (iz * ny + iy of the extended lattice) holding at least one
    // site, ascending: the x-inverse pass reads and transforms only these
    // (a row without sites has no output); null: every row
    const int* rows = nullptr;
    int nrows = 0;
};

// Twiddle tables, one per padded axis: exp(-2 pi i m/L), m < L.
template <typename T> struct Twiddles {
    const cx<T>* x = nullptr;
    const cx<T>* y = nullptr;
    const cx<T>* z = nullptr;
};

// The x passes write and read the rows (iz, iy < ny) of one buffer
// U [R][3][nz][Ly][Lx], row (iz, iy) at ky = iy of z-plane iz.  So the y
// passes run in place (a block reads all positions of its pencils before it
// writes any), the z pass works in place on the same buffer, and no
// separate [nz][ny][Lx] buffer occupies L2 or HBM.
struct RowMap {
    int ny;               // lattice rows per z-plane
    int pitch;            // rows per z-plane in the buffer (Ly)
    int64_t comp_stride;  // elements per (RHS, component) slab: nz Ly Lx
    __device__ __forceinline__ int64_t at(int r, int c, int row, int lx) const {
        return ((int64_t)r * 3 + c) * comp_stride + ((int64_t)(row / ny) * pitch + row % ny) * lx;
    }
};

// Workspace for the padded passes of one matvec of R right-hand sides.
template <typename T> struct PadWork {
    cx<T>* u1 = nullptr;  // unused (the x passes use the rows of u2, RowMap)
    cx<T>* u2 = nullptr;  // [R][3][nz][Ly][Lx]
    int zvar = 0;         // z-pass schedule, see zconv_schedules
    int xfwd = 0;         // x-forward schedule, see xpass_schedules
    int xinv = 0;         // x-inverse schedule, likewise
    int yvar = 0;         // y-pass radix plan variant, see ypass_schedules
    int slices = 1;       // fused x+y slice passes where built (see slice_passes)
    // The 1/alpha table holds 3x3 tensors (anisotropic materials): per RHS
    // [3 rows c][comp][3 columns], so row c of composition comp's tensor is at
    // beta[r*beta_stride + c*(beta_stride/3) + comp*3].  The slice passes
    // handle only the isotropic table and are skipped.
    bool beta_tensor = false;
};

int pick_fft_length(int n);  // smallest supported length >= 2n, or 0

struct KState;

// BiCGstab updates fused into the x passes of a matvec (mode 0: none).
//   mode 1: gather p <- r + beta (p - omega v) (written back to x);
//           scatter v = A p and sigma = <rhat, v> -> alpha
//   mode 2: gather s <- r - alpha v (written back to x);
//           scatter t = A s and <t, s>, <t, t>, <s, s>, <rhat, s>,
//           <rhat, t> -> omega, |r'|, rho', beta and the stopping tests
//   mode 3: gather of the BiCGstab iteration's first matvec: the previous
//           iteration's r' = s - omega t and x += alpha p + omega s, then
//           p <- r' + beta (p - omega v) (written back to x); scatter as mode 1
// (BiCGstab runs modes 3 and 2; BiCGstab(2) uses mode 1.)
// part/cnt: per-RHS partial sums (part_stride double2 per RHS) and tickets.
template <typename T> struct FusedKrylov {
    int mode = 0;
    cx<T>* r = nullptr;  // read by modes 1 and 2, written by mode 3
    const cx<T>* v = nullptr;
    const cx<T>* rhat = nullptr;
    const cx<T>* s = nullptr;  // mode 3: the previous iteration's s and t = A s
    const cx<T>* t = nullptr;
    cx<T>* x = nullptr;  // mode 3: the solution, updated in the gather
    KState* st = nullptr;
    double2* part = nullptr;
    unsigned* cnt = nullptr;
    int part_stride = 0;
};

int xinv_blocks_per_rhs(const Geom& g);

// Number of z-pass schedules for this grid and arithmetic type: schedule 0
// (three component groups per column, spectra exchanged through shared
// memory) always; for complex64 when the z plan keeps at most 8 points per
// thread, schedule 1 (register-resident, one thread holds all three
// components of its points) and schedule 2 (the same with the octant column
// mapping: one staged Green tile serves the four columns +-kx, +-ky).  All
// compute the same product; the context times them per RHS count and keeps
// the fastest (dda_set_schedule can force one).
template <typename T> int zconv_schedules(const Geom& g);

// Number of x-pass schedules for this grid and arithmetic type: 0, the rows
// staged through shared memory (k_xfwd, k_xinv), always; for complex64 also
// 1 + V for the warp-local passes with radix plan variant V (xwarp.cuh).
// Timed by the context like the z schedules.
template <typename T> int xpass_schedules(const Geom& g);

// Number of y-pass schedules (radix plan variants of the strided y passes,
// complex64 only), timed like the others.
template <typename T> int ypass_schedules(const Geom& g);

// Fused x+y passes over whole z-slices (slice_impl.cuh): built for this
// grid and element type?  Then the matvec runs xy-fwd, z, yx-inv instead of
// the five separate passes, and needs no U1 workspace.
template <typename T> bool slice_passes(const Geom& g);
template <typename T>
cudaError_t launch_slice_fwd(const Geom& g, int R, cx<T>* x, cx<T>* u2, const int* site_of, const Twiddles<T>& tw,
                             const int* active, const FusedKrylov<T>& fk, cudaStream_t st);
template <typename T>
cudaError_t launch_slice_inv(const Geom& g, int R, const cx<T>* u2, cx<T>* y, const cx<T>* x, const DevTarget& tg,
                             const cx<T>* beta, int beta_stride, const Twiddles<T>& tw, int* active,
                             const FusedKrylov<T>& fk, cudaStream_t st);

// The z pass alone, in place on u2 (used to time the schedules).
template <typename T>
cudaError_t launch_zconv(const Geom& g, int R, cx<T>* u2, const cx<T>* ghat, const cx<T>* twz, const int* active,
                         int zvar, cudaStream_t st);

template <typename T>
cudaError_t launch_matvec_fused(const Geom& g, int R, cx<T>* x, cx<T>* y, const PadWork<T>& w,
                                const DevTarget& tg, const cx<T>* beta, int beta_stride, const cx<T>* ghat,
                                const Twiddles<T>& tw, int* active, const FusedKrylov<T>& fk, cudaStream_t st);

// y = A x for R right-hand sides, vectors [R][3][N].  beta[r*beta_stride + comp]
// is 1/alpha of composition comp for RHS r (or, with w.beta_tensor, the rows
// of its 1/alpha tensor, see PadWork).  active (nullable): RHS r is skipped
// when active[r] == 0.
template <typename T>
cudaError_t launch_matvec(const Geom& g, int R, const cx<T>* x, cx<T>* y, const PadWork<T>& w,
                          const DevTarget& tg, const cx<T>* beta, int beta_stride, const cx<T>* ghat,
                          const Twiddles<T>& tw, const int* active, cudaStream_t st);

// Build the octant of FFT(g)/(Lx Ly Lz) of the six Green-tensor components
// (xx, xy, xz, yy, yz, zz) in FP64.  scratch: 6*Lx*Ly*Lz double2.
cudaError_t launch_green_fft(const Geom& g, double kd, double2* scratch, double2* ghat64,
                             const Twiddles<double>& tw, cudaStream_t st);

cudaError_t launch_convert_c128_to_c64(const double2* src, float2* dst, int64_t n, cudaStream_t st);
cudaError_t launch_convert_c128_to_df(const double2* src, cdfl* dst, int64_t n, cudaStream_t st);
cudaError_t launch_convert_df_to_c128(const cdfl* src, double2* dst, int64_t n, cudaStream_t st);

}  // namespace dda
