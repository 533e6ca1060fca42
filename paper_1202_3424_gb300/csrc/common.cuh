// Shared device/host helpers for the DDA CUDA path: complex types and
// arithmetic, error plumbing.  Nothing here is specific to one kernel.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <cstdio>
#include <type_traits>
#include <string>

namespace dda {

// ---- double-float reals -------------------------------------------------------
// A value hi + lo held in two floats (|lo| <= ulp(hi)/2), with arithmetic by
// error-free transformations: Knuth's two-sum for addition and the FMA
// two-product (exact product of two floats as p + fma(a, b, -p)) for
// multiplication (Dekker 1971; Shewchuk 1997).  About 44 significant bits:
// an FFT matvec in this arithmetic is accurate to ~1e-12 relative, far below
// the residual tolerances it checks, and runs on the FP32 pipes, which on
// GB300 have ~58x the FP64 throughput.  Addition uses the cheaper variant
// whose error is bounded relative to |a| + |b| (enough for FFT sums).
struct dfl {
    float hi, lo;
    dfl() = default;
    __host__ __device__ constexpr dfl(float h, float l) : hi(h), lo(l) {}
    __host__ __device__ dfl(double d) : hi((float)d), lo((float)(d - (double)(float)d)) {}
    __host__ __device__ dfl(int i) : hi((float)i), lo(0.f) {}
    __host__ __device__ explicit operator double() const { return (double)hi + (double)lo; }
};

__host__ __device__ __forceinline__ dfl operator-(dfl a) { return dfl(-a.hi, -a.lo); }
__host__ __device__ __forceinline__ dfl operator+(dfl a, dfl b) {
    const float s = a.hi + b.hi;
    const float bb = s - a.hi;
    float e = (a.hi - (s - bb)) + (b.hi - bb);  // two-sum error of the leading parts
    e += a.lo + b.lo;
    const float h = s + e;
    return dfl(h, e - (h - s));
}
__host__ __device__ __forceinline__ dfl operator-(dfl a, dfl b) { return a + (-b); }
__host__ __device__ __forceinline__ dfl operator*(dfl a, dfl b) {
    const float p = a.hi * b.hi;
    float e = fmaf(a.hi, b.hi, -p);  // exact error of the float product
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    const float h = p + e;
    return dfl(h, e - (h - p));
}

struct cdfl {
    dfl x, y;
};

template <typename T> struct cplx_of;
template <> struct cplx_of<float> { using type = float2; };
template <> struct cplx_of<double> { using type = double2; };
template <> struct cplx_of<dfl> { using type = cdfl; };
template <typename T> using cx = typename cplx_of<T>::type;

template <typename C> struct real_of;
template <> struct real_of<float2> { using type = float; };
template <> struct real_of<double2> { using type = double; };
template <> struct real_of<cdfl> { using type = dfl; };

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
// g0 p0 + g1 p1 + g2 p2 (a row of the 3x3 product in Fourier space) as one
// FMA chain per part: 12 instructions for complex64 instead of the 16 of
// three products and two sums (IEEE rules forbid the compiler this
// reassociation)
template <typename C> __host__ __device__ __forceinline__ C cdot3(C g0, C p0, C g1, C p1, C g2, C p2) {
    C r;
    if constexpr (std::is_same<C, float2>::value) {
        r.x = fmaf(g0.x, p0.x, fmaf(-g0.y, p0.y, fmaf(g1.x, p1.x, fmaf(-g1.y, p1.y, fmaf(g2.x, p2.x, -g2.y * p2.y)))));
        r.y = fmaf(g0.x, p0.y, fmaf(g0.y, p0.x, fmaf(g1.x, p1.y, fmaf(g1.y, p1.x, fmaf(g2.x, p2.y, g2.y * p2.x)))));
    } else if constexpr (std::is_same<C, double2>::value) {
        r.x = fma(g0.x, p0.x, fma(-g0.y, p0.y, fma(g1.x, p1.x, fma(-g1.y, p1.y, fma(g2.x, p2.x, -g2.y * p2.y)))));
        r.y = fma(g0.x, p0.y, fma(g0.y, p0.x, fma(g1.x, p1.y, fma(g1.y, p1.x, fma(g2.x, p2.y, g2.y * p2.x)))));
    } else {
        r.x = g0.x * p0.x - g0.y * p0.y + (g1.x * p1.x - g1.y * p1.y) + (g2.x * p2.x - g2.y * p2.y);
        r.y = g0.x * p0.y + g0.y * p0.x + (g1.x * p1.y + g1.y * p1.x) + (g2.x * p2.y + g2.y * p2.x);
    }
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
    r.x = static_cast<typename real_of<D>::type>(a.x);
    r.y = static_cast<typename real_of<D>::type>(a.y);
    return r;
}

// Index of site s in the per-RHS 1/alpha and weight tables: its composition
// code, or, with per-site materials (no composition array), s + 1.
__device__ __forceinline__ int table_index(const uint8_t* __restrict__ comp_of, int64_t s) {
    return comp_of != nullptr ? (int)comp_of[s] : (int)(s + 1);
}

// How the x-inverse pass finds a site's 1/alpha (a template parameter of its
// kernels): the scalar of the site's composition, row c of its composition's
// tensor, or the scalar of the site itself (per-site materials).
enum { kDiagComp = 0, kDiagTensor = 1, kDiagSite = 2 };
template <int DIAG, typename C>
__device__ __forceinline__ C diag_entry(const C* __restrict__ br, const uint8_t* __restrict__ comp_of, int64_t s,
                                        int c) {
    if constexpr (DIAG == kDiagTensor) return br[comp_of[s] * 3 + c];
    else if constexpr (DIAG == kDiagSite) return br[s + 1];
    else return br[comp_of[s]];
}

}  // namespace dda
