// Mixed-radix Stockham FFT on pencils held by a group of threads.
//
// The DDA matvec (Goodman, Draine & Flatau 1990, the FFT method the user
// guide cites under "Choice of FFT Algorithm") needs 1-D transforms of
// length L = 2^a 3^b along each axis of the zero-padded grid.  The lattice
// is padded with vacuum to exactly L/2 sites per axis, so every forward
// transform sees zeros in its upper half and every inverse transform is
// needed only on its lower half; both facts are compile-time here.
//
// One pencil of length L is owned by NT threads; every thread holds
// E = L/NT points in registers.  A stage of radix R (p = product of the
// radices already applied) takes butterfly i in [0, L/R) with inputs at
// positions i + j*L/R, multiplies input j by w^(j*k) (k = i mod p,
// w = exp(sgn 2 pi i/(p R))), applies a length-R DFT and writes output m to
// position (i-k)*R + k + m*p (Stockham autosort, natural order in and out).
// Thread u runs butterflies i = u + q*NT.  Whenever p divides NT or NT
// divides p, k and the output positions are a per-thread base plus
// compile-time offsets, and (p | NT) the twiddles are shared by all of the
// thread's butterflies, so they are loaded once per stage.
//
// The last stage's outputs sit at positions i + m*L/R, exactly the inputs of
// a first stage of the same radix: the inverse uses the forward radices in
// reverse order, so a forward transform can be followed by a pointwise
// product and the inverse without leaving registers.  Intermediate stages
// exchange through shared memory with two barriers each -- block barriers,
// or warp barriers when every pencil lies within one warp (WARP) -- so every
// thread of the block must run these routines the same number of times.
// Two-stage plans whose pencil lies in consecutive lanes can exchange by
// warp shuffles instead (ShflExchange), with no shared memory and no barrier.
#pragma once

#include "common.cuh"

namespace dda {

template <int L_, int NT_, int... Rs> struct PlanDef {
    static constexpr int L = L_;
    static constexpr int NT = NT_;
    static constexpr int E = L_ / NT_;
    static constexpr int NS = sizeof...(Rs);
    static constexpr int rad[NS] = {Rs...};
};

// Radix schedules: the first forward radix (= last inverse radix) is even,
// and NT divides L/R for every radix R.
template <int L> struct Plan;
template <> struct Plan<16> : PlanDef<16, 4, 4, 4> {};
template <> struct Plan<32> : PlanDef<32, 4, 4, 8> {};
template <> struct Plan<48> : PlanDef<48, 4, 4, 4, 3> {};
template <> struct Plan<64> : PlanDef<64, 8, 8, 8> {};
template <> struct Plan<96> : PlanDef<96, 8, 4, 4, 3, 2> {};
template <> struct Plan<128> : PlanDef<128, 16, 4, 4, 8> {};
template <> struct Plan<192> : PlanDef<192, 16, 4, 4, 4, 3> {};
template <> struct Plan<256> : PlanDef<256, 32, 4, 8, 8> {};
template <> struct Plan<384> : PlanDef<384, 32, 4, 4, 4, 3, 2> {};
template <> struct Plan<512> : PlanDef<512, 64, 8, 8, 8> {};

// Schedules of the z pass (three component groups per block): as Plan<L>,
// except that L = 512 uses 32 threads per pencil (16 points each) so that
// eight adjacent columns fit in one block.
template <int L> struct ZPlan : Plan<L> {};
template <> struct ZPlan<512> : PlanDef<512, 32, 8, 8, 8> {};

// Supported padded lengths, ascending (the host picks the smallest >= 2n).
static constexpr int kSupportedLengths[] = {16, 32, 48, 64, 96, 128, 192, 256, 384, 512};

template <class PL, int DIR> __host__ __device__ constexpr int stage_radix(int s) {
    return DIR < 0 ? PL::rad[s] : PL::rad[PL::NS - 1 - s];
}
template <class PL, int DIR> __host__ __device__ constexpr int stage_p(int s) {
    int p = 1;
    for (int i = 0; i < s; ++i) p *= stage_radix<PL, DIR>(i);
    return p;
}

// ---- exchange-plane row padding --------------------------------------------
// Kernels that stage TP pencils side by side in shared memory ([row][TP]
// complex64 elements) insert one padding row after every 2^S rows: position
// pos lives in row pos + (pos >> S).  With narrow tiles (TP * 8 bytes < 128)
// several rows share one bank window, and the stride patterns of the stage
// exchanges put whole half-warps on the same banks; the padding moves those
// rows apart.  Every exchange position is a per-thread base plus a multiple
// of the stage's radix stride, so the shift folds into constant offsets.
// S per (plan, tile width) is the choice of
// paper_1202_3424_gb300/bank_model.py, which counts the shared-memory
// wavefronts of every exchange instruction of every warp; S = 0: no padding.
__host__ __device__ constexpr int exchange_pad_shift(int L, int NT, int TP) {
    if (L == 256 && NT == 32 && TP == 4) return 3;
    if (L == 512 && NT == 64 && TP == 4) return 3;
    return 0;
}
// Rows of one padded plane of 8-byte elements.
__host__ __device__ constexpr int exchange_rows8(int L, int NT, int TP) {
    return exchange_pad_shift(L, NT, TP) ? L + ((L - 1) >> exchange_pad_shift(L, NT, TP)) : L;
}
// (tabulated for 8-byte elements; planes of wider elements are not padded)
template <int L, int NT, int TP, int ES> __host__ __device__ constexpr int exchange_shift() {
    return ES == 8 ? exchange_pad_shift(L, NT, TP) : 0;
}
// Rows of one padded plane.
template <int L, int NT, int TP, int ES> __host__ __device__ constexpr int exchange_rows() {
    constexpr int s = exchange_shift<L, NT, TP, ES>();
    return s ? L + ((L - 1) >> s) : L;
}
template <int L, int NT, int TP, int ES> __device__ __forceinline__ int exchange_row(int pos) {
    constexpr int s = exchange_shift<L, NT, TP, ES>();
    if constexpr (s == 0) return pos;
    else return pos + (pos >> s);
}

// ---- small DFTs, sign convention exp(SGN * 2 pi i j k / R) ----------------
template <int R, int SGN, typename C> struct Dft;

template <int SGN, typename C> struct Dft<2, SGN, C> {
    __device__ __forceinline__ static void run(C* v) {
        C a = v[0], b = v[1];
        v[0] = cadd(a, b);
        v[1] = csub(a, b);
    }
    __device__ __forceinline__ static void run_half(C* v) { v[1] = v[0]; }
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
    // inputs 2 and 3 are zero
    __device__ __forceinline__ static void run_half(C* v) {
        C a = v[0], b = v[1];
        C t3 = cmul_i<SGN>(b);
        v[0] = cadd(a, b);
        v[2] = csub(a, b);
        v[1] = cadd(a, t3);
        v[3] = csub(a, t3);
    }
};

template <int SGN, typename C> struct Dft<8, SGN, C> {
    __device__ __forceinline__ static void combine(C* v, C (&e)[4], C (&o)[4]) {
        using T = typename real_of<C>::type;
        const T r2 = T(0.70710678118654752440);  // 1/sqrt(2)
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
    __device__ __forceinline__ static void run(C* v) {
        C e[4] = {v[0], v[2], v[4], v[6]};
        C o[4] = {v[1], v[3], v[5], v[7]};
        Dft<4, SGN, C>::run(e);
        Dft<4, SGN, C>::run(o);
        combine(v, e, o);
    }
    // inputs 4..7 are zero
    __device__ __forceinline__ static void run_half(C* v) {
        C e[4] = {v[0], v[2], v[0], v[0]};
        C o[4] = {v[1], v[3], v[1], v[1]};
        Dft<4, SGN, C>::run_half(e);
        Dft<4, SGN, C>::run_half(o);
        combine(v, e, o);
    }
};

// Radix 16 as 4 x 4: n = 4 n1 + n2, k = k1 + 4 k2; four length-4 DFTs over
// n1, the twiddles W16^(n2 k1), four length-4 DFTs over n2.
template <int SGN, typename C> struct Dft<16, SGN, C> {
    template <int J> __device__ __forceinline__ static C w16(C a) {
        using T = typename real_of<C>::type;
        const T c1 = T(0.92387953251128675613), s1 = T(0.38268343236508977173);  // cos, sin(pi/8)
        const T r2 = T(0.70710678118654752440);
        auto w = [](T re, T im) { C r; r.x = re; r.y = im; return r; };
        if constexpr (J == 1) return cmul(a, w(c1, SGN > 0 ? s1 : -s1));
        else if constexpr (J == 2) return cscale(cadd(a, cmul_i<SGN>(a)), r2);
        else if constexpr (J == 3) return cmul(a, w(s1, SGN > 0 ? c1 : -c1));
        else if constexpr (J == 4) return cmul_i<SGN>(a);
        else if constexpr (J == 6) return cscale(csub(cmul_i<SGN>(a), a), r2);
        else return cmul(a, w(-c1, SGN > 0 ? -s1 : s1));  // J == 9
    }
    __device__ __forceinline__ static void finish(C* v, C (&y)[4][4]) {
        y[1][1] = w16<1>(y[1][1]);
        y[1][2] = w16<2>(y[1][2]);
        y[1][3] = w16<3>(y[1][3]);
        y[2][1] = w16<2>(y[2][1]);
        y[2][2] = w16<4>(y[2][2]);
        y[2][3] = w16<6>(y[2][3]);
        y[3][1] = w16<3>(y[3][1]);
        y[3][2] = w16<6>(y[3][2]);
        y[3][3] = w16<9>(y[3][3]);
#pragma unroll
        for (int k1 = 0; k1 < 4; ++k1) {
            C z[4] = {y[0][k1], y[1][k1], y[2][k1], y[3][k1]};
            Dft<4, SGN, C>::run(z);
#pragma unroll
            for (int k2 = 0; k2 < 4; ++k2) v[k1 + 4 * k2] = z[k2];
        }
    }
    __device__ __forceinline__ static void run(C* v) {
        C y[4][4];
#pragma unroll
        for (int n2 = 0; n2 < 4; ++n2) {
#pragma unroll
            for (int n1 = 0; n1 < 4; ++n1) y[n2][n1] = v[4 * n1 + n2];
            Dft<4, SGN, C>::run(y[n2]);
        }
        finish(v, y);
    }
    // inputs 8..15 are zero
    __device__ __forceinline__ static void run_half(C* v) {
        C y[4][4];
#pragma unroll
        for (int n2 = 0; n2 < 4; ++n2) {
            y[n2][0] = v[n2];
            y[n2][1] = v[4 + n2];
            Dft<4, SGN, C>::run_half(y[n2]);
        }
        finish(v, y);
    }
};

// Radix 32 as 4 x 8: n = 8 n1 + n2, k = k1 + 4 k2; eight length-4 DFTs over
// n1, the twiddles W32^(n2 k1) (n2 k1 <= 21), four length-8 DFTs over n2.
struct W32Table {
    // cos and sin of pi j / 16, j = 0..21
    static constexpr double c[22] = {1, 0.98078528040323043, 0.92387953251128674, 0.83146961230254524, 0.70710678118654757, 0.55557023301960229, 0.38268343236508984, 0.19509032201612833, 6.123233995736766e-17, -0.19509032201612819, -0.38268343236508973, -0.55557023301960196, -0.70710678118654746, -0.83146961230254535, -0.92387953251128674, -0.98078528040323043, -1, -0.98078528040323043, -0.92387953251128685, -0.83146961230254546, -0.70710678118654768, -0.55557023301960218};
    static constexpr double s[22] = {0, 0.19509032201612825, 0.38268343236508978, 0.55557023301960218, 0.70710678118654746, 0.83146961230254524, 0.92387953251128674, 0.98078528040323043, 1, 0.98078528040323043, 0.92387953251128674, 0.83146961230254546, 0.70710678118654757, 0.55557023301960218, 0.38268343236508989, 0.19509032201612861, 1.2246467991473532e-16, -0.19509032201612836, -0.38268343236508967, -0.55557023301960196, -0.70710678118654746, -0.83146961230254524};
};
template <int SGN, typename C> struct Dft<32, SGN, C> {
    template <int J> __device__ __forceinline__ static C w32(C a) {
        using T = typename real_of<C>::type;
        if constexpr (J == 0) return a;
        else if constexpr (J == 8) return cmul_i<SGN>(a);
        else if constexpr (J == 16) return cscale(a, T(-1));
        else {
            constexpr double cj = W32Table::c[J], sj = SGN > 0 ? W32Table::s[J] : -W32Table::s[J];
            C w;
            w.x = T(cj);
            w.y = T(sj);
            return cmul(a, w);
        }
    }
    template <int N2> __device__ __forceinline__ static void twiddle_row(C (&y)[8][4]) {
        y[N2][1] = w32<N2>(y[N2][1]);
        y[N2][2] = w32<2 * N2>(y[N2][2]);
        y[N2][3] = w32<3 * N2>(y[N2][3]);
    }
    __device__ __forceinline__ static void finish(C* v, C (&y)[8][4]) {
        twiddle_row<1>(y);
        twiddle_row<2>(y);
        twiddle_row<3>(y);
        twiddle_row<4>(y);
        twiddle_row<5>(y);
        twiddle_row<6>(y);
        twiddle_row<7>(y);
#pragma unroll
        for (int k1 = 0; k1 < 4; ++k1) {
            C z[8] = {y[0][k1], y[1][k1], y[2][k1], y[3][k1], y[4][k1], y[5][k1], y[6][k1], y[7][k1]};
            Dft<8, SGN, C>::run(z);
#pragma unroll
            for (int k2 = 0; k2 < 8; ++k2) v[k1 + 4 * k2] = z[k2];
        }
    }
    __device__ __forceinline__ static void run(C* v) {
        C y[8][4];
#pragma unroll
        for (int n2 = 0; n2 < 8; ++n2) {
#pragma unroll
            for (int n1 = 0; n1 < 4; ++n1) y[n2][n1] = v[8 * n1 + n2];
            Dft<4, SGN, C>::run(y[n2]);
        }
        finish(v, y);
    }
    // inputs 16..31 are zero
    __device__ __forceinline__ static void run_half(C* v) {
        C y[8][4];
#pragma unroll
        for (int n2 = 0; n2 < 8; ++n2) {
            y[n2][0] = v[n2];
            y[n2][1] = v[8 + n2];
            Dft<4, SGN, C>::run_half(y[n2]);
        }
        finish(v, y);
    }
};

// ---- exchange-plane address maps -------------------------------------------
// Kernels whose pencils lie within one warp give each pencil its own plane
// and map position pos of the exchange after stage S to a swizzled slot;
// the default keeps the position.
struct NoSwizzle {
    static constexpr bool kShuffle = false;
    template <int DIR, int S> __device__ __forceinline__ static int map(int pos) { return pos; }
};

// ---- exchange by warp shuffles ---------------------------------------------
// For a two-stage plan whose first radix R is a multiple of NT and whose
// pencil lies in NT consecutive lanes, the exchange is a set of NT x NT
// transposes: the first stage leaves output position (u + q NT) R + m in
// register q R + m of lane u (P = 1), and the second stage wants position
// u' + NT c (c = q2 + j E/R2) in register q2 R2 + j of lane u'.  Writing the
// register as h NT + l, lane u's register h NT + l goes to lane l, register
// h NT + u.  shfl_exchange_ok checks that for every lane and register.
template <class PL, int DIR> __host__ __device__ constexpr bool shfl_exchange_ok() {
    constexpr int L = PL::L, NT = PL::NT, E = PL::E;
    if (PL::NS != 2 || E % NT != 0 || NT > 32 || (NT & (NT - 1)) != 0) return false;
    constexpr int R = stage_radix<PL, DIR>(0), R2 = stage_radix<PL, DIR>(1);
    constexpr int NB = E / R, NB2 = E / R2;
    if (L / R2 != NT * NB2) return false;
    for (int u = 0; u < NT; ++u)
        for (int q = 0; q < NB; ++q)
            for (int m = 0; m < R; ++m) {
                const int pos = (u + q * NT) * R + m, reg = q * R + m;
                const int h = reg / NT, l = reg % NT;
                const int c = pos / NT, want = (c % NB2) * R2 + c / NB2;
                if (pos % NT != l || want != h * NT + u) return false;
            }
    return true;
}

// In-register transpose of the NT x NT blocks v[h NT + i] across NT
// consecutive lanes (u = lane within the group), in log2(NT) rounds: round b
// swaps the entries whose lane bit b and register bit b differ with lane
// u ^ b, so after all rounds lane u holds register u of every lane.
template <int NT, int E, typename C> __device__ __forceinline__ void shfl_transpose(C (&v)[E], int u) {
#pragma unroll
    for (int b = 1; b < NT; b <<= 1) {
        const bool hi = (u & b) != 0;
#pragma unroll
        for (int h = 0; h < E / NT; ++h)
#pragma unroll
            for (int i = 0; i < NT; ++i) {
                if (i & b) continue;
                C& lo_reg = v[h * NT + i];
                C& hi_reg = v[h * NT + (i | b)];
                const C send = hi ? lo_reg : hi_reg;
                C recv;
                recv.x = __shfl_xor_sync(0xffffffffu, send.x, b);
                recv.y = __shfl_xor_sync(0xffffffffu, send.y, b);
                if (hi) lo_reg = recv;
                else hi_reg = recv;
            }
    }
}
struct ShflExchange {
    static constexpr bool kShuffle = true;
    template <int DIR, int S> __device__ __forceinline__ static int map(int pos) { return pos; }
};

// ---- stage recursion -----------------------------------------------------
// v: E registers; u: thread index within the pencil (0..NT-1);
// tw: forward twiddle table of L entries exp(-2 pi i m/L);
// ld(pos) / st(pos, val): shared-memory exchange for this thread's pencil.
// On return v[q*R + m] holds output position u + q*NT + m*L/R (R = last radix).
template <bool WARP> __device__ __forceinline__ void stage_sync() {
    if constexpr (WARP) __syncwarp();
    else __syncthreads();
}

template <typename C, class PL, int DIR, int S, class Ld, class St, bool WARP = false, class SWZ = NoSwizzle>
__device__ __forceinline__ void fft_stages(C (&v)[PL::E], int u, const C* __restrict__ tw, Ld& ld, St& st,
                                           bool half_first) {
    constexpr int L = PL::L, NT = PL::NT, E = PL::E, NS = PL::NS;
    constexpr int R = stage_radix<PL, DIR>(S);
    constexpr int P = stage_p<PL, DIR>(S);
    constexpr int NB = E / R;
    constexpr int STEP = L / (P * R);
    static_assert(E % R == 0, "radix must divide the points per thread");
    if constexpr (P > 1) {
        if constexpr (NT % P == 0) {
            const int k = u % P;  // shared by all butterflies of this thread
            C w[R];
#pragma unroll
            for (int j = 1; j < R; ++j) {
                w[j] = tw[j * k * STEP];
                if constexpr (DIR > 0) w[j].y = -w[j].y;
            }
#pragma unroll
            for (int q = 0; q < NB; ++q)
#pragma unroll
                for (int j = 1; j < R; ++j) v[q * R + j] = cmul(v[q * R + j], w[j]);
        } else {
#pragma unroll
            for (int q = 0; q < NB; ++q) {
                int k;
                if constexpr (P % NT == 0) k = u + (q % (P / NT)) * NT;
                else k = (u + q * NT) % P;
#pragma unroll
                for (int j = 1; j < R; ++j) {
                    C w = tw[j * k * STEP];
                    if constexpr (DIR > 0) w.y = -w.y;
                    v[q * R + j] = cmul(v[q * R + j], w);
                }
            }
        }
    }
#pragma unroll
    for (int q = 0; q < NB; ++q) {
        if constexpr (S == 0 && (R % 2 == 0)) {
            if (half_first) Dft<R, DIR, C>::run_half(&v[q * R]);
            else Dft<R, DIR, C>::run(&v[q * R]);
        } else {
            Dft<R, DIR, C>::run(&v[q * R]);
        }
    }
    if constexpr (S < NS - 1 && SWZ::kShuffle) {
        static_assert(S == 0 && shfl_exchange_ok<PL, DIR>(), "the shuffle exchange needs a two-stage transpose plan");
        shfl_transpose<NT>(v, u);
        fft_stages<C, PL, DIR, S + 1, Ld, St, WARP, SWZ>(v, u, tw, ld, st, false);
    } else if constexpr (S < NS - 1) {
        stage_sync<WARP>();
        if constexpr (NT % P == 0) {
            const int base = (u / P) * (P * R) + (u % P);
#pragma unroll
            for (int q = 0; q < NB; ++q)
#pragma unroll
                for (int m = 0; m < R; ++m) st(SWZ::template map<DIR, S>(base + q * NT * R + m * P), v[q * R + m]);
        } else if constexpr (P % NT == 0) {
#pragma unroll
            for (int q = 0; q < NB; ++q)
#pragma unroll
                for (int m = 0; m < R; ++m)
                    st(SWZ::template map<DIR, S>(u + (q - q % (P / NT)) * NT * R + (q % (P / NT)) * NT + m * P),
                       v[q * R + m]);
        } else {
#pragma unroll
            for (int q = 0; q < NB; ++q) {
                const int i = u + q * NT, k = i % P;
#pragma unroll
                for (int m = 0; m < R; ++m) st(SWZ::template map<DIR, S>((i - k) * R + k + m * P), v[q * R + m]);
            }
        }
        stage_sync<WARP>();
        constexpr int R2 = stage_radix<PL, DIR>(S + 1);
        constexpr int NB2 = E / R2;
#pragma unroll
        for (int q = 0; q < NB2; ++q)
#pragma unroll
            for (int j = 0; j < R2; ++j) v[q * R2 + j] = ld(SWZ::template map<DIR, S>(u + q * NT + j * (L / R2)));
        fft_stages<C, PL, DIR, S + 1, Ld, St, WARP, SWZ>(v, u, tw, ld, st, false);
    }
}

// NP pencils of one thread in lockstep: every stage runs on all NP before
// the exchange, so a stage's twiddles are loaded once for all of them and
// the NP exchanges share one pair of barriers.  ld(p, pos) / st(p, pos, val)
// address pencil p's own exchange plane.
template <typename C, class PL, int DIR, int S, int NP, class Ld, class St>
__device__ __forceinline__ void fft_stages_np(C (&v)[NP][PL::E], int u, const C* __restrict__ tw, Ld& ld, St& st,
                                              bool half_first) {
    constexpr int L = PL::L, NT = PL::NT, E = PL::E, NS = PL::NS;
    constexpr int R = stage_radix<PL, DIR>(S);
    constexpr int P = stage_p<PL, DIR>(S);
    constexpr int NB = E / R;
    constexpr int STEP = L / (P * R);
    static_assert(E % R == 0, "radix must divide the points per thread");
    if constexpr (P > 1) {
        if constexpr (NT % P == 0) {
            const int k = u % P;
            C w[R];
#pragma unroll
            for (int j = 1; j < R; ++j) {
                w[j] = tw[j * k * STEP];
                if constexpr (DIR > 0) w[j].y = -w[j].y;
            }
#pragma unroll
            for (int p = 0; p < NP; ++p)
#pragma unroll
                for (int q = 0; q < NB; ++q)
#pragma unroll
                    for (int j = 1; j < R; ++j) v[p][q * R + j] = cmul(v[p][q * R + j], w[j]);
        } else {
#pragma unroll
            for (int q = 0; q < NB; ++q) {
                int k;
                if constexpr (P % NT == 0) k = u + (q % (P / NT)) * NT;
                else k = (u + q * NT) % P;
#pragma unroll
                for (int j = 1; j < R; ++j) {
                    C w = tw[j * k * STEP];
                    if constexpr (DIR > 0) w.y = -w.y;
#pragma unroll
                    for (int p = 0; p < NP; ++p) v[p][q * R + j] = cmul(v[p][q * R + j], w);
                }
            }
        }
    }
#pragma unroll
    for (int p = 0; p < NP; ++p)
#pragma unroll
        for (int q = 0; q < NB; ++q) {
            if constexpr (S == 0 && (R % 2 == 0)) {
                if (half_first) Dft<R, DIR, C>::run_half(&v[p][q * R]);
                else Dft<R, DIR, C>::run(&v[p][q * R]);
            } else {
                Dft<R, DIR, C>::run(&v[p][q * R]);
            }
        }
    if constexpr (S < NS - 1) {
        __syncthreads();
#pragma unroll
        for (int p = 0; p < NP; ++p) {
            if constexpr (NT % P == 0) {
                const int base = (u / P) * (P * R) + (u % P);
#pragma unroll
                for (int q = 0; q < NB; ++q)
#pragma unroll
                    for (int m = 0; m < R; ++m) st(p, base + q * NT * R + m * P, v[p][q * R + m]);
            } else if constexpr (P % NT == 0) {
#pragma unroll
                for (int q = 0; q < NB; ++q)
#pragma unroll
                    for (int m = 0; m < R; ++m)
                        st(p, u + (q - q % (P / NT)) * NT * R + (q % (P / NT)) * NT + m * P, v[p][q * R + m]);
            } else {
#pragma unroll
                for (int q = 0; q < NB; ++q) {
                    const int i = u + q * NT, k = i % P;
#pragma unroll
                    for (int m = 0; m < R; ++m) st(p, (i - k) * R + k + m * P, v[p][q * R + m]);
                }
            }
        }
        __syncthreads();
        constexpr int R2 = stage_radix<PL, DIR>(S + 1);
        constexpr int NB2 = E / R2;
#pragma unroll
        for (int p = 0; p < NP; ++p)
#pragma unroll
            for (int q = 0; q < NB2; ++q)
#pragma unroll
                for (int j = 0; j < R2; ++j) v[p][q * R2 + j] = ld(p, u + q * NT + j * (L / R2));
        fft_stages_np<C, PL, DIR, S + 1, NP, Ld, St>(v, u, tw, ld, st, false);
    }
}

// Load the first stage's inputs through first(pos), then run all stages.
// HALF_IN: positions >= L/2 are zero and are neither loaded nor transformed.
template <typename C, class PL, int DIR, bool HALF_IN, class First, class Ld, class St, bool WARP = false>
__device__ __forceinline__ void pencil_fft(C (&v)[PL::E], int u, const C* __restrict__ tw, First& first, Ld& ld,
                                           St& st) {
    constexpr int R0 = stage_radix<PL, DIR>(0);
    constexpr int NB0 = PL::E / R0;
    static_assert(!HALF_IN || R0 % 2 == 0, "a half-zero input needs an even first radix");
    constexpr int JN = HALF_IN ? R0 / 2 : R0;
#pragma unroll
    for (int q = 0; q < NB0; ++q)
#pragma unroll
        for (int j = 0; j < JN; ++j) v[q * R0 + j] = first(u + q * PL::NT + j * (PL::L / R0));
    fft_stages<C, PL, DIR, 0, Ld, St, WARP>(v, u, tw, ld, st, HALF_IN);
}

// Run all stages on data already in registers, laid out as the first stage
// expects (inputs of butterfly q at v[q*R0 + j], positions i + j*L/R0).
template <typename C, class PL, int DIR, class Ld, class St, bool WARP = false>
__device__ __forceinline__ void pencil_fft_regs(C (&v)[PL::E], int u, const C* __restrict__ tw, Ld& ld, St& st) {
    fft_stages<C, PL, DIR, 0, Ld, St, WARP>(v, u, tw, ld, st, false);
}

// Final outputs of a pencil transform: v[idx] holds position pos.
// HALF_OUT: only positions < L/2 (the lattice half of an inverse transform).
template <class PL, int DIR, bool HALF_OUT, class F>
__device__ __forceinline__ void for_each_out(int u, F&& f) {
    constexpr int R = stage_radix<PL, DIR>(PL::NS - 1);
    constexpr int NB = PL::E / R;
    static_assert(!HALF_OUT || R % 2 == 0, "half outputs need an even last radix");
    constexpr int MN = HALF_OUT ? R / 2 : R;
#pragma unroll
    for (int q = 0; q < NB; ++q)
#pragma unroll
        for (int m = 0; m < MN; ++m) f(q * R + m, u + q * PL::NT + m * (PL::L / R));
}

}  // namespace dda
