// Far-field amplitude kernel (farfield.cu).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace dda {

// F[r][d][a] (complex128, zeroed here) = kd^2 ((I - n n) sum_j P[r][.][j] phase_{r,d}(j))_a for
// R RHS x ndir directions.  site_xyz[j] = ix | iy << 10 | iz << 20 (lattice indices < 1024);
// tabs[(r*ndir + d)*tab_len + a*(tab_len/3) + i] = exp(-i kd n_a (i - c_a)) for axis a;
// dirs[(r*ndir + d)*3 + a] the unit vectors n.  C = float2 or double2.
template <typename C>
cudaError_t launch_farfield(int R, int64_t N, const unsigned* site_xyz, const C* P, int ndir, int tab_len,
                            const C* tabs, const double* dirs, double kd, double2* F, cudaStream_t st);

// The per-axis phase tables above for nq = R*ndir unit vectors dirs[q*3 + a]:
// tabs[(q*3 + a)*Lm + i] = exp(-i kd dirs[q*3 + a] (i - c[a])), i < Lm (tab_len = 3 Lm).
template <typename C>
cudaError_t launch_phase_tables(int64_t nq, int Lm, const double c[3], double kd, const double* dirs, C* tabs,
                                cudaStream_t st);

}  // namespace dda
