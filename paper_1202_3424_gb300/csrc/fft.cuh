// Mixed-radix Stockham FFT on pencils held by a group of threads.
//
// The DDA matvec (Goodman, Draine & Flatau 1990, the FFT method the user
// guide cites under "Choice of FFT Algorithm") needs 1-D transforms of
// length L = 2^a 3^b along each lattice axis of the zero-padded grid.
// One pencil of length L is owned by NT threads; every thread holds
// E = L/NT points in registers.  A stage of radix R (p = product of the
// radices already applied) takes butterfly i in [0, L/R) with inputs at
// positions i + j*L/R, multiplies input j by w^(j*k) (k = i mod p,
// w = exp(sgn 2 pi i/(p R))), applies a length-R DFT and writes output m to
// position (i-k)*R + k + m*p (Stockham autosort, natural order in and out).
//
// Data enters the first stage straight from the caller (global memory or a
// staging buffer) and leaves the last stage straight to the caller: the last
// stage's outputs sit at positions i + m*L/R, which are exactly the inputs of
// a first stage of the same radix -- the z-pass exploits this to apply the
// Fourier-space product in registers between its forward and inverse
// transforms.  Intermediate stages exchange through shared memory with two
// block barriers each, so every thread of the block must call these
// routines the same number of times.
#pragma once

#include "common.cuh"

namespace dda {

// Radix schedules.  NT divides L/R for every radix R of the schedule, so that
// every thread runs exactly E/R butterflies per stage.
template <int L_, int NT_, int... Rs> struct PlanDef {
    static constexpr int L = L_;
    static constexpr int NT = NT_;
    static constexpr int E = L_ / NT_;
    static constexpr int NS = sizeof...(Rs);
    static constexpr int rad[NS] = {Rs...};
};

template <int L> struct Plan;
template <> struct Plan<16> : PlanDef<16, 4, 4, 4> {};
template <> struct Plan<32> : PlanDef<32, 4, 4, 8> {};
template <> struct Plan<48> : PlanDef<48, 4, 3, 4, 4> {};
template <> struct Plan<64> : PlanDef<64, 8, 8, 8> {};
template <> struct Plan<96> : PlanDef<96, 8, 3, 4, 4, 2> {};
template <> struct Plan<128> : PlanDef<128, 16, 4, 4, 8> {};
template <> struct Plan<192> : PlanDef<192, 16, 3, 4, 4, 4> {};
template <> struct Plan<256> : PlanDef<256, 32, 4, 8, 8> {};
template <> struct Plan<384> : PlanDef<384, 32, 3, 4, 4, 4, 2> {};
template <> struct Plan<512> : PlanDef<512, 64, 8, 8, 8> {};

// Supported padded lengths, ascending (host side picks the smallest >= 2n).
static constexpr int kSupportedLengths[] = {16, 32, 48, 64, 96, 128, 192, 256, 384, 512};

// radix of stage S for direction DIR (forward uses the schedule as listed,
// inverse in reverse order so that its first radix equals the forward's last)
template <class PL, int DIR, int S> struct StageRadix {
    static constexpr int value = (DIR < 0) ? PL::rad[S] : PL::rad[PL::NS - 1 - S];
};

// ---- small DFTs, sign convention exp(SGN * 2 pi i j k / R) ----------------
template <int R, int SGN, typename C> struct Dft;

template <int SGN, typename C> struct Dft<2, SGN, C> {
    __device__ __forceinline__ static void run(C* v) {
        C a = v[0], b = v[1];
        v[0] = cadd(a, b);
        v[1] = csub(a, b);
    }
};

template <int SGN, typename C> struct Dft<3, SGN, C> {
    __device__ __forceinline__ static void run(C* v) {
        using T = typename real_of<C>::type;
        const T h = T(0.5), s3 = T(0.86602540378443864676);  // cos(pi/3), sin(pi/3)
        C s = cadd(v[1], v[2]);
        C d = csub(v[1], v[2]);
        C a0 = v[0];
        C m = csub(a0, cscale(s, h));
        C r = cmul_i<SGN>(cscale(d, s3));
        v[0] = cadd(a0, s);
        v[1] = cadd(m, r);
        v[2] = csub(m, r);
    }
};

template <int SGN, typename C> struct Dft<4, SGN, C> {
    __device__ __forceinline__ static void run(C* v) {
        C t0 = cadd(v[0], v[2]);
        C t1 = csub(v[0], v[2]);
        C t2 = cadd(v[1], v[3]);
        C t3 = cmul_i<SGN>(csub(v[1], v[3]));
        v[0] = cadd(t0, t2);
        v[2] = csub(t0, t2);
        v[1] = cadd(t1, t3);
        v[3] = csub(t1, t3);
    }
};

template <int SGN, typename C> struct Dft<8, SGN, C> {
    __device__ __forceinline__ static void run(C* v) {
        using T = typename real_of<C>::type;
        const T r2 = T(0.70710678118654752440);  // 1/sqrt(2)
        C e[4] = {v[0], v[2], v[4], v[6]};
        C o[4] = {v[1], v[3], v[5], v[7]};
        Dft<4, SGN, C>::run(e);
        Dft<4, SGN, C>::run(o);
        // w8^1 = (1 + SGN i)/sqrt2, w8^2 = SGN i, w8^3 = (-1 + SGN i)/sqrt2
        C o1 = cscale(cadd(o[1], cmul_i<SGN>(o[1])), r2);
        C o2 = cmul_i<SGN>(o[2]);
        C o3 = cscale(csub(cmul_i<SGN>(o[3]), o[3]), r2);
        v[0] = cadd(e[0], o[0]);
        v[4] = csub(e[0], o[0]);
        v[1] = cadd(e[1], o1);
        v[5] = csub(e[1], o1);
        v[2] = cadd(e[2], o2);
        v[6] = csub(e[2], o2);
        v[3] = cadd(e[3], o3);
        v[7] = csub(e[3], o3);
    }
};

// ---- stage recursion -----------------------------------------------------
// v: E registers; u: thread index within the pencil (0..NT-1);
// tw: forward twiddle table of L entries exp(-2 pi i m/L) (shared or global);
// ld(pos) / st(pos, val): shared-memory exchange for this thread's pencil;
// last(q, m, pos, val): consumer of the final outputs (pos = i + m L/R).
template <typename C, class PL, int DIR, int S, int P, class Ld, class St, class Last>
__device__ __forceinline__ void fft_stages(C (&v)[PL::E], int u, const C* __restrict__ tw,
                                           Ld& ld, St& st, Last& last) {
    constexpr int L = PL::L, NT = PL::NT, E = PL::E, NS = PL::NS;
    constexpr int R = StageRadix<PL, DIR, S>::value;
    constexpr int NB = E / R;
#pragma unroll
    for (int q = 0; q < NB; ++q) {
        const int i = u + q * NT;
        if constexpr (P > 1) {
            const int k = i % P;
#pragma unroll
            for (int j = 1; j < R; ++j) {
                C w = tw[j * k * (L / (P * R))];
                if constexpr (DIR > 0) w.y = -w.y;
                v[q * R + j] = cmul(v[q * R + j], w);
            }
        }
        Dft<R, DIR, C>::run(&v[q * R]);
    }
    if constexpr (S == NS - 1) {
        static_assert(P * R == L, "radix schedule must multiply to L");
#pragma unroll
        for (int q = 0; q < NB; ++q)
#pragma unroll
            for (int m = 0; m < R; ++m) last(q, m, u + q * NT + m * (L / R), v[q * R + m]);
    } else {
        __syncthreads();
#pragma unroll
        for (int q = 0; q < NB; ++q) {
            const int i = u + q * NT;
            const int k = i % P;
#pragma unroll
            for (int m = 0; m < R; ++m) st((i - k) * R + k + m * P, v[q * R + m]);
        }
        __syncthreads();
        constexpr int R2 = StageRadix<PL, DIR, S + 1>::value;
        constexpr int NB2 = E / R2;
#pragma unroll
        for (int q = 0; q < NB2; ++q)
#pragma unroll
            for (int j = 0; j < R2; ++j) v[q * R2 + j] = ld(u + q * NT + j * (L / R2));
        fft_stages<C, PL, DIR, S + 1, P * R>(v, u, tw, ld, st, last);
    }
}

// Load the first stage's inputs through first(pos), then run all stages.
template <typename C, class PL, int DIR, class First, class Ld, class St, class Last>
__device__ __forceinline__ void pencil_fft(C (&v)[PL::E], int u, const C* __restrict__ tw, First& first,
                                           Ld& ld, St& st, Last& last) {
    constexpr int R0 = StageRadix<PL, DIR, 0>::value;
    constexpr int NB0 = PL::E / R0;
#pragma unroll
    for (int q = 0; q < NB0; ++q)
#pragma unroll
        for (int j = 0; j < R0; ++j) v[q * R0 + j] = first(u + q * PL::NT + j * (PL::L / R0));
    fft_stages<C, PL, DIR, 0, 1>(v, u, tw, ld, st, last);
}

// Run all stages on data already in registers, laid out as the first stage
// expects (inputs of butterfly q at v[q*R0 + j], positions i + j*L/R0).
template <typename C, class PL, int DIR, class Ld, class St, class Last>
__device__ __forceinline__ void pencil_fft_regs(C (&v)[PL::E], int u, const C* __restrict__ tw, Ld& ld, St& st,
                                                Last& last) {
    fft_stages<C, PL, DIR, 0, 1>(v, u, tw, ld, st, last);
}

}  // namespace dda
