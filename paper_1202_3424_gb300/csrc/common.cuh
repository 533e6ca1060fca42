// Shared device/host helpers for the DDA CUDA path: complex types and
// arithmetic, error plumbing.  Nothing here is specific to one kernel.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdio>
#include <string>

namespace dda {

template <typename T> struct cplx_of;
template <> struct cplx_of<float> { using type = float2; };
template <> struct cplx_of<double> { using type = double2; };
template <typename T> using cx = typename cplx_of<T>::type;

template <typename C> struct real_of;
template <> struct real_of<float2> { using type = float; };
template <> struct real_of<double2> { using type = double; };

__host__ __device__ __forceinline__ float2 mk(float re, float im) { return make_float2(re, im); }
__host__ __device__ __forceinline__ double2 mk(double re, double im) { return make_double2(re, im); }

template <typename C> __host__ __device__ __forceinline__ C cadd(C a, C b) { C r; r.x = a.x + b.x; r.y = a.y + b.y; return r; }
template <typename C> __host__ __device__ __forceinline__ C csub(C a, C b) { C r; r.x = a.x - b.x; r.y = a.y - b.y; return r; }
template <typename C> __host__ __device__ __forceinline__ C cmul(C a, C b) {
    C r;
    r.x = a.x * b.x - a.y * b.y;
    r.y = a.x * b.y + a.y * b.x;
    return r;
}
// a * conj(b)
template <typename C> __host__ __device__ __forceinline__ C cmulc(C a, C b) {
    C r;
    r.x = a.x * b.x + a.y * b.y;
    r.y = a.y * b.x - a.x * b.y;
    return r;
}
template <typename C, typename S> __host__ __device__ __forceinline__ C cscale(C a, S s) { C r; r.x = a.x * s; r.y = a.y * s; return r; }
template <typename C> __host__ __device__ __forceinline__ C czero() { C r; r.x = 0; r.y = 0; return r; }
// multiply by +i (sgn > 0) or -i (sgn < 0)
template <int SGN, typename C> __host__ __device__ __forceinline__ C cmul_i(C a) {
    C r;
    if (SGN > 0) { r.x = -a.y; r.y = a.x; }
    else         { r.x = a.y;  r.y = -a.x; }
    return r;
}
template <typename D, typename S> __host__ __device__ __forceinline__ D ccast(S a) {
    D r;
    r.x = (typename real_of<D>::type)a.x;
    r.y = (typename real_of<D>::type)a.y;
    return r;
}

}  // namespace dda
