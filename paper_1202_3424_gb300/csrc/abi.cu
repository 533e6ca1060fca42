// C ABI of the DDA hot path: context, target/material/wavelength set-up,
// matvec, the BiCGstab solve with FP64 iterative refinement, Q reductions and
// the adjoint gradient.  Declarations and conventions: include/dda.h.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <cmath>
#include <complex>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "dda.h"
#include "farfield.h"
#include "internal.h"
#include "krylov.h"
#include "profiler.h"

using cd = std::complex<double>;
using namespace dda;

namespace {

constexpr double kPi = 3.14159265358979323846;
// LATTDR coefficients (Draine & Goodman 1993), the guide's "LATTDR" option.
constexpr double kB1 = -1.8915316, kB2 = 0.1648469, kB3 = -1.7700004;

struct DevMem {
    void* p = nullptr;
    size_t bytes = 0;
};

// Inner-solve vectors.  BiCGstab: b, x, r, rhat, p, v, s, t.  BiCGstab(2)
// keeps r0, r1, r2 in r, s, t and u0, u1, u2 in p, v, u2 (shadow residual rhat).
template <typename T> struct Inner {
    cx<T>*b = nullptr, *x = nullptr, *r = nullptr, *rhat = nullptr, *p = nullptr, *v = nullptr, *s = nullptr,
    *t = nullptr, *u2 = nullptr;
};

struct GraphEntry {
    cudaGraphExec_t exec = nullptr;
    bool traced = false;  // captured with launch tracing on
    int R = 0;
    int prec = -1;
    int K = 0;
    int solver = 0;
    cudaStream_t stream = nullptr;
};

}  // namespace

struct dda_ctx {
    int device = 0;
    cudaStream_t own_stream = nullptr;
    cudaStream_t stream = nullptr;
    std::string err;

    // target
    Geom g;
    bool has_target = false;
    int max_code = 0;
    DevTarget tg;
    DevMem m_site_of, m_lat_of, m_comp_of, m_rows;

    // materials
    std::vector<cd> m;
    double m_amb = 1.0;
    bool has_materials = false;
    // anisotropic compositions (dda_set_anisotropic_materials): refractive
    // indices along the principal axes e_1..e_3 and the dielectric-frame
    // angles (theta_DF, phi_DF, beta_DF) of each
    bool aniso = false;
    std::vector<std::array<cd, 3>> m3;
    std::vector<std::array<double, 3>> df_angles;
    // per-site materials (dda_set_site_materials): m holds one index per
    // occupied site, and site j takes table entry j + 1 (tg.comp_of is null)
    bool site_mode = false;

    // prepared wavelength
    bool prepared = false, has32 = false;
    double kd = 0.0, aeff_lat = 0.0;
    DevMem m_gh64, m_gh32, m_tw64[3], m_tw32[3];
    DevMem m_ghdf, m_twdf[3];  // double-float copies for the refinement residual

    // workspace
    std::vector<DevMem> pool;  // generic named slots, see slot()
    int ws_R = 0;
    GraphEntry graph;
    // z-pass schedule per (element bytes, RHS count), timed on first use;
    // force_z >= 0 overrides (dda_set_schedule)
    std::map<std::pair<int, int>, std::array<int, 5>> zsched;  // -> (z, slice passes, x-fwd, x-inv, y)
    int force_z = -1;
    int force_xf = -1, force_xi = -1;  // x-pass schedules: -1 timed, else forced (dda_set_xpass)
    int force_y = -1;                   // y-pass radix plan: -1 timed, else forced (dda_set_ypass)
    // -1 timed, 0 separate passes (default), 1 slice passes where built.
    // Measured on GB300 the slice passes win only on small grids outside a
    // solve (64^3 sphere, 2 RHS: 0.163 vs 0.175 ms per matvec) and lose inside
    // the BiCGstab solve and on the 128-RHS ellipsoid (1 block of 512 threads
    // per SM), so they are opt-in.
    int force_slices = 0;
    int* h_count = nullptr;  // pinned
    Profiler prof;

    dda_status fail(dda_status code, const char* fmt, ...) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        err = buf;
        return code;
    }
    dda_status cuda_fail(cudaError_t e, const char* what) {
        cudaGetLastError();
        return fail(e == cudaErrorMemoryAllocation ? DDA_ERR_OOM : DDA_ERR_CUDA, "%s: %s", what,
                    cudaGetErrorString(e));
    }
};

#define CU(call)                                                   \
    do {                                                           \
        cudaError_t _e = (call);                                   \
        if (_e != cudaSuccess) return ctx->cuda_fail(_e, #call);   \
    } while (0)

namespace {

// Synchronize the context stream and, with tracing on, read the launch events.
cudaError_t sync_collect(dda_ctx* ctx) {
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (e == cudaSuccess && ctx->prof.on) e = ctx->prof.collect();
    return e;
}

struct ProfScope {
    explicit ProfScope(dda_ctx* c) { set_current_profiler(c ? &c->prof : nullptr); }
    ~ProfScope() { set_current_profiler(nullptr); }
};

// Workspace slots (each a device buffer grown on demand).
enum Slot {
    S_E64, S_X64, S_R64, S_Y64,
    S_IN_B, S_IN_X, S_IN_R, S_IN_RHAT, S_IN_P, S_IN_V, S_IN_S, S_IN_T,
    S_PAD2_32, S_PAD2_64,
    S_STATE, S_ACTIVE, S_WANT, S_OUTER, S_TOLREL, S_SCALE, S_COEF, S_NORM_B, S_NORM_R,
    S_PART, S_CNT, S_QSUM, S_COUNT,
    S_BETA64, S_BETA32, S_W, S_KHAT, S_EPOL,
    S_MV_X32, S_MV_Y32, S_GRAD, S_DBETA,
    S_BETADF, S_XDF, S_YDF, S_TUNE, S_IN_U2,
    S_NSLOTS
};

dda_status ensure(dda_ctx* ctx, DevMem& m, size_t bytes, bool zero = false) {
    if (m.bytes >= bytes && m.p != nullptr) {
        if (zero) CU(cudaMemsetAsync(m.p, 0, bytes, ctx->stream));
        return DDA_OK;
    }
    if (m.p) {
        cudaFree(m.p);
        m.p = nullptr;
        m.bytes = 0;
    }
    // any cached graph may reference the old buffer
    if (ctx->graph.exec) {
        cudaGraphExecDestroy(ctx->graph.exec);
        ctx->graph.exec = nullptr;
    }
    CU(cudaMalloc(&m.p, bytes < 256 ? 256 : bytes));
    m.bytes = bytes < 256 ? 256 : bytes;
    if (zero) CU(cudaMemsetAsync(m.p, 0, m.bytes, ctx->stream));
    return DDA_OK;
}

template <typename P> P* slot(dda_ctx* ctx, int s) { return reinterpret_cast<P*>(ctx->pool[s].p); }

size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

void free_mem(DevMem& m) {
    if (m.p) cudaFree(m.p);
    m.p = nullptr;
    m.bytes = 0;
}

// S = sum_a khat_a^2 |e_a|^2 for a unit e: for a real e this is Draine &
// Goodman's sum_a (khat_a e_a)^2; for a complex e it is the form that keeps
// the lattice dispersion relation exact on the cube's 3-fold axes, where every
// transverse polarization (circular ones too) is a lattice mode.
double ldr_s(const double* khat, const cd* e) {
    double S = 0.0;
    for (int a = 0; a < 3; ++a) S += khat[a] * khat[a] * std::norm(e[a]);
    return S;
}

cd ldr_inverse_alpha(cd eps, double kd, const double* khat, const cd* e) {
    const double S = ldr_s(khat, e);
    const cd inv_acm = (4.0 * kPi / 3.0) * (eps + 2.0) / (eps - 1.0);
    return inv_acm + (kB1 + kB2 * eps + kB3 * eps * S) * (kd * kd) - cd(0.0, 2.0 / 3.0) * (kd * kd * kd);
}

cd ldr_inverse_alpha_deps(cd eps, double kd, const double* khat, const cd* e) {
    const double S = ldr_s(khat, e);
    return -4.0 * kPi / ((eps - 1.0) * (eps - 1.0)) + (kB2 + kB3 * S) * (kd * kd);
}

// Validate and normalize the RHS description; fills host copies.
dda_status check_rhs(dda_ctx* ctx, int R, const double* khat, const double* e, std::vector<double>& k_out,
                     std::vector<cd>& e_out) {
    if (R <= 0 || khat == nullptr || e == nullptr) return ctx->fail(DDA_ERR_ARG, "R must be > 0 with khat and e given");
    k_out.assign(3 * (size_t)R, 0.0);
    e_out.assign(3 * (size_t)R, 0.0);
    for (int r = 0; r < R; ++r) {
        double kn = 0.0, en = 0.0;
        for (int a = 0; a < 3; ++a) {
            const double kv = khat[3 * r + a], er = e[6 * r + 2 * a], ei = e[6 * r + 2 * a + 1];
            if (!std::isfinite(kv) || !std::isfinite(er) || !std::isfinite(ei))
                return ctx->fail(DDA_ERR_NONFINITE, "non-finite direction or polarization for RHS %d", r);
            kn += kv * kv;
            en += er * er + ei * ei;
        }
        if (std::fabs(std::sqrt(kn) - 1.0) > 1e-6) return ctx->fail(DDA_ERR_ARG, "khat of RHS %d is not a unit vector", r);
        if (en == 0.0) return ctx->fail(DDA_ERR_ARG, "polarization of RHS %d is zero", r);
        cd dot = 0.0;
        for (int a = 0; a < 3; ++a) {
            k_out[3 * r + a] = khat[3 * r + a] / std::sqrt(kn);
            e_out[3 * r + a] = cd(e[6 * r + 2 * a], e[6 * r + 2 * a + 1]) / std::sqrt(en);
            dot += k_out[3 * r + a] * e_out[3 * r + a];
        }
        if (std::abs(dot) > 1e-6) return ctx->fail(DDA_ERR_ARG, "polarization of RHS %d is not transverse to khat", r);
    }
    return DDA_OK;
}

// Compositions + 1 (code 0, vacuum, unused).
int beta_stride(const dda_ctx* ctx) { return (int)ctx->m.size() + 1; }
// Entries per RHS of the 1/alpha table: one per composition, or the three
// rows of each composition's tensor (layout in PadWork::beta_tensor).
int beta_rhs_stride(const dda_ctx* ctx) { return beta_stride(ctx) * (ctx->aniso ? 9 : 1); }
// Entries per RHS of the absorption weights (k_qsums): one or six per composition.
int qweight_stride(const dda_ctx* ctx) { return beta_stride(ctx) * (ctx->aniso ? 6 : 1); }

// Principal axes e_1, e_2, e_3 (rows of ax) of a dielectric frame rotated by
// (theta_DF, phi_DF, beta_DF) from the Target Frame ("Composite Targets with
// Anisotropic Constituents").
void dielectric_axes(const std::array<double, 3>& a, double ax[3][3]) {
    const double ct = std::cos(a[0]), st = std::sin(a[0]), cp = std::cos(a[1]), sp = std::sin(a[1]),
                 cb = std::cos(a[2]), sb = std::sin(a[2]);
    const double e[3][3] = {{ct, st * cp, st * sp},
                            {-st * cb, ct * cb * cp - sb * sp, ct * cb * sp + sb * cp},
                            {st * sb, -(ct * sb * cp + cb * sp), -(ct * sb * sp - cb * cp)}};
    std::memcpy(ax, e, sizeof e);
}

// 1/alpha table of R RHS (beta_rhs_stride entries each) and, if w is given,
// the absorption weights (qweight_stride each).  Isotropic: 1/alpha and
// w = -Im(1/alpha) - (2/3)k^3.  Anisotropic: B = sum_j (1/alpha_j) e_j e_j^T,
// 1/alpha_j the LATTDR value of the j-th principal index (the same S for all
// three), and the six weights of Im(P . B^* P^*) - (2/3)k^3 |P|^2.
dda_status diag_tables(dda_ctx* ctx, int R, const std::vector<double>& k, const std::vector<cd>& e, std::vector<cd>& b,
                       std::vector<double>* w) {
    const int BS = beta_stride(ctx), RS = beta_rhs_stride(ctx), WS = qweight_stride(ctx);
    const double kd = ctx->kd, rad = (2.0 / 3.0) * kd * kd * kd;
    b.assign((size_t)R * RS, cd(0.0));
    if (w) w->assign((size_t)R * WS, 0.0);
    auto inv_alpha = [&](cd m, int r, cd* out) -> bool {
        const cd mrel = m / ctx->m_amb;
        *out = ldr_inverse_alpha(mrel * mrel, kd, &k[3 * r], &e[3 * r]);
        return std::isfinite(out->real()) && std::isfinite(out->imag());
    };
    for (int r = 0; r < R; ++r) {
        for (int c = 1; c < BS; ++c) {
            if (!ctx->aniso) {
                cd be;
                if (!inv_alpha(ctx->m[c - 1], r, &be))
                    return ctx->fail(DDA_ERR_NONFINITE, "polarizability of composition %d is not finite", c);
                b[(size_t)r * RS + c] = be;
                if (w) (*w)[(size_t)r * WS + c] = -be.imag() - rad;
                continue;
            }
            double ax[3][3];
            dielectric_axes(ctx->df_angles[c - 1], ax);
            cd bj[3];
            for (int j = 0; j < 3; ++j)
                if (!inv_alpha(ctx->m3[c - 1][j], r, &bj[j]))
                    return ctx->fail(DDA_ERR_NONFINITE, "polarizability of composition %d is not finite", c);
            cd B[3][3];
            for (int a = 0; a < 3; ++a)
                for (int d = 0; d < 3; ++d) {
                    B[a][d] = 0.0;
                    for (int j = 0; j < 3; ++j) B[a][d] += bj[j] * (ax[j][a] * ax[j][d]);
                }
            for (int a = 0; a < 3; ++a)
                for (int d = 0; d < 3; ++d) b[(size_t)r * RS + (size_t)a * 3 * BS + c * 3 + d] = B[a][d];
            if (w) {
                double* wt = w->data() + (size_t)r * WS + c * 6;
                for (int a = 0; a < 3; ++a) wt[a] = -B[a][a].imag() - rad;
                wt[3] = -2.0 * B[0][1].imag();
                wt[4] = -2.0 * B[0][2].imag();
                wt[5] = -2.0 * B[1][2].imag();
            }
        }
    }
    return DDA_OK;
}

// Per-(RHS, composition) device tables: 1/alpha in FP64, FP32 and double-float
// (diag_tables), the absorption weights, and the RHS directions and polarizations.
dda_status upload_tables(dda_ctx* ctx, int R, const std::vector<double>& k, const std::vector<cd>& e) {
    std::vector<cd> b;
    std::vector<double> w;
    dda_status s;
    if ((s = diag_tables(ctx, R, k, e, b, &w)) != DDA_OK) return s;
    std::vector<double2> b64(b.size());
    std::vector<float2> b32(b.size());
    std::vector<cdfl> bdf(b.size());
    for (size_t i = 0; i < b.size(); ++i) {
        b64[i] = make_double2(b[i].real(), b[i].imag());
        b32[i] = make_float2((float)b[i].real(), (float)b[i].imag());
        bdf[i] = cdfl{dfl(b[i].real()), dfl(b[i].imag())};
    }
    if ((s = ensure(ctx, ctx->pool[S_BETA64], b64.size() * sizeof(double2))) != DDA_OK) return s;
    if ((s = ensure(ctx, ctx->pool[S_BETA32], b32.size() * sizeof(float2))) != DDA_OK) return s;
    if ((s = ensure(ctx, ctx->pool[S_W], w.size() * sizeof(double))) != DDA_OK) return s;
    CU(cudaMemcpyAsync(ctx->pool[S_BETA64].p, b64.data(), b64.size() * sizeof(double2), cudaMemcpyHostToDevice, ctx->stream));
    CU(cudaMemcpyAsync(ctx->pool[S_BETA32].p, b32.data(), b32.size() * sizeof(float2), cudaMemcpyHostToDevice, ctx->stream));
    if ((s = ensure(ctx, ctx->pool[S_BETADF], bdf.size() * sizeof(cdfl))) != DDA_OK) return s;
    CU(cudaMemcpyAsync(ctx->pool[S_BETADF].p, bdf.data(), bdf.size() * sizeof(cdfl), cudaMemcpyHostToDevice, ctx->stream));
    CU(cudaMemcpyAsync(ctx->pool[S_W].p, w.data(), w.size() * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
    std::vector<double2> e2(3 * (size_t)R);
    for (size_t i = 0; i < e2.size(); ++i) e2[i] = make_double2(e[i].real(), e[i].imag());
    if ((s = ensure(ctx, ctx->pool[S_KHAT], k.size() * sizeof(double))) != DDA_OK) return s;
    if ((s = ensure(ctx, ctx->pool[S_EPOL], e2.size() * sizeof(double2))) != DDA_OK) return s;
    CU(cudaMemcpyAsync(ctx->pool[S_KHAT].p, k.data(), k.size() * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
    CU(cudaMemcpyAsync(ctx->pool[S_EPOL].p, e2.data(), e2.size() * sizeof(double2), cudaMemcpyHostToDevice, ctx->stream));
    // the host vectors go out of scope: finish the copies first
    CU(sync_collect(ctx));
    return DDA_OK;
}

// Chunk of RHS whose padded work (one [3][nz][Ly][Lx] buffer per RHS: the x
// passes use its rows, see RowMap) fits the budget.
template <typename T> int matvec_chunk(const dda_ctx* ctx, int R) {
    const size_t per = (size_t)3 * ctx->g.u2_per_comp() * sizeof(cx<T>);
    const size_t budget = (size_t)48 << 30;
    int c = (int)std::max<size_t>(1, budget / per);
    return std::min(c, R);
}

template <typename T> struct PadSlots;
template <> struct PadSlots<float> { static constexpr int b = S_PAD2_32; };
template <> struct PadSlots<double> { static constexpr int b = S_PAD2_64; };
// double-float elements are 16 bytes like complex128: share its work buffers
template <> struct PadSlots<dfl> { static constexpr int b = S_PAD2_64; };

template <typename T> const cx<T>* ghat_of(const dda_ctx* ctx);
template <> const float2* ghat_of<float>(const dda_ctx* ctx) { return (const float2*)ctx->m_gh32.p; }
template <> const double2* ghat_of<double>(const dda_ctx* ctx) { return (const double2*)ctx->m_gh64.p; }
template <> const cdfl* ghat_of<dfl>(const dda_ctx* ctx) { return (const cdfl*)ctx->m_ghdf.p; }
template <typename T> Twiddles<T> tw_of(const dda_ctx* ctx);
template <> Twiddles<float> tw_of<float>(const dda_ctx* ctx) {
    return {(const float2*)ctx->m_tw32[0].p, (const float2*)ctx->m_tw32[1].p, (const float2*)ctx->m_tw32[2].p};
}
template <> Twiddles<double> tw_of<double>(const dda_ctx* ctx) {
    return {(const double2*)ctx->m_tw64[0].p, (const double2*)ctx->m_tw64[1].p, (const double2*)ctx->m_tw64[2].p};
}
template <> Twiddles<dfl> tw_of<dfl>(const dda_ctx* ctx) {
    return {(const cdfl*)ctx->m_twdf[0].p, (const cdfl*)ctx->m_twdf[1].p, (const cdfl*)ctx->m_twdf[2].p};
}
template <typename T> const cx<T>* beta_of(dda_ctx* ctx);
template <> const float2* beta_of<float>(dda_ctx* ctx) { return slot<float2>(ctx, S_BETA32); }
template <> const double2* beta_of<double>(dda_ctx* ctx) { return slot<double2>(ctx, S_BETA64); }
template <> const cdfl* beta_of<dfl>(dda_ctx* ctx) { return slot<cdfl>(ctx, S_BETADF); }

template <typename T> dda_status ensure_pad(dda_ctx* ctx, int R) {
    const int rc = matvec_chunk<T>(ctx, R);
    return ensure(ctx, ctx->pool[PadSlots<T>::b], (size_t)rc * 3 * ctx->g.u2_per_comp() * sizeof(cx<T>));
}

// Schedule of the matvec passes for R right-hand sides: the z-pass variant
// (zconv_schedules), whether the fused x+y slice passes run (slice_passes),
// and the x-forward and x-inverse schedules (xpass_schedules).  Where more
// than one choice exists they are timed inside whole plain matvecs of R RHS
// (the passes decide what their neighbours find in L2) on the context's
// workspace plus a transient pair of vectors, one coordinate at a time (z
// and slices, then x-forward, then x-inverse), and the fastest is kept.  The
// workspace must hold R RHS (ensure_pad<T>).  Inside a stream capture, or
// with may_time false, an untimed choice is returned: the cached one, else
// the register-resident z schedule (octant mapping below 8 RHS), the slice
// passes where built and forced, and the warp-local x passes with plan 0.
int partial_stride(const dda_ctx* ctx);

template <typename T>
dda_status pick_schedule(dda_ctx* ctx, int R, bool may_time, PadWork<T>* out, bool fused = false) {
    const int nv = zconv_schedules<T>(ctx->g);
    const int nx = xpass_schedules<T>(ctx->g);
    const bool sl = slice_passes<T>(ctx->g) && !ctx->aniso && !ctx->site_mode;
    std::vector<int> zs, ss;
    if (nv <= 1) zs = {0};
    else if (ctx->force_z >= 0) {
        // a plan-variant schedule (3, 4) falls back to its plan-0 schedule
        // (1, 2) where the length has one plan, and anything to 0 where the
        // register schedules do not exist
        int fz = ctx->force_z;
        if (fz >= nv) fz = (nv >= 3 && fz >= 3) ? fz - 2 : nv - 1;
        zs = {fz};
    }
    else for (int z = 0; z < nv; ++z) zs.push_back(z);
    if (!sl) ss = {0};
    else if (ctx->force_slices >= 0) ss = {ctx->force_slices};
    else ss = {1, 0};
    auto xlist = [&](int force) {
        std::vector<int> xs;
        if (nx <= 1) {
            xs = {0};
        } else if (force >= 0) {
            xs = {std::min(force, nx - 1)};
        } else {
            for (int x = 1; x < nx; ++x) xs.push_back(x);
            xs.push_back(0);
        }
        return xs;
    };
    const std::vector<int> xfs = xlist(ctx->force_xf), xis = xlist(ctx->force_xi);
    const int ny = ypass_schedules<T>(ctx->g);
    std::vector<int> ys;
    if (ny <= 1) ys = {0};
    else if (ctx->force_y >= 0) ys = {std::min(ctx->force_y, ny - 1)};
    else ys = {0, 1};
    // untimed choice: the first of each list (warp-local x passes, plan 0;
    // y passes plan 0)
    auto apply = [&](const std::array<int, 5>& c) {
        out->zvar = c[0];
        out->slices = c[1];
        out->xfwd = c[2];
        out->xinv = c[3];
        out->yvar = c[4];
    };
    std::array<int, 5> cur = {zs[0], ss[0], xfs[0], xis[0], ys[0]};
    apply(cur);
    if (zs.size() * ss.size() == 1 && xfs.size() == 1 && xis.size() == 1 && ys.size() == 1) return DDA_OK;
    // plain matvecs and the BiCGstab matvecs with fused updates (the solves)
    // are tuned apart: the fused gather and scatter change what is fastest
    const std::pair<int, int> key((int)sizeof(cx<T>) * (fused ? -1 : 1), R);
    auto it = ctx->zsched.find(key);
    if (it != ctx->zsched.end()) {
        apply(it->second);
        return DDA_OK;
    }
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    CU(cudaStreamIsCapturing(ctx->stream, &cs));
    if (!may_time || cs != cudaStreamCaptureStatusNone) {
        if (zs.size() > 1) out->zvar = R >= 8 ? 1 : 2;
        return DDA_OK;
    }
    // x, y and 1/alpha table filled with one byte pattern (finite, nonzero
    // values; they do not change the timing), and for the fused matvecs a
    // scratch Krylov state, partial sums, tickets and active flags
    const int BS = beta_rhs_stride(ctx);
    const size_t vec = align256((size_t)R * 3 * ctx->g.N * sizeof(cx<T>));
    const size_t tab = align256((size_t)R * BS * sizeof(cx<T>));
    const int ps = partial_stride(ctx);
    const size_t stb = align256((size_t)R * sizeof(KState)), pb = align256((size_t)R * ps * sizeof(double2));
    const size_t cb = align256((size_t)R * sizeof(unsigned)), ab = align256((size_t)R * sizeof(int));
    dda_status s;
    if ((s = ensure(ctx, ctx->pool[S_TUNE], 2 * vec + tab + (fused ? stb + pb + cb + ab : 0), true)) != DDA_OK)
        return s;
    char* base = static_cast<char*>(ctx->pool[S_TUNE].p);
    cx<T>* x = reinterpret_cast<cx<T>*>(base);
    cx<T>* y = reinterpret_cast<cx<T>*>(base + vec);
    const cx<T>* beta = reinterpret_cast<const cx<T>*>(base + 2 * vec);
    KState* kst = reinterpret_cast<KState*>(base + 2 * vec + tab);
    double2* part = reinterpret_cast<double2*>(base + 2 * vec + tab + stb);
    unsigned* cnt = reinterpret_cast<unsigned*>(base + 2 * vec + tab + stb + pb);
    int* act = reinterpret_cast<int*>(base + 2 * vec + tab + stb + pb + cb);
    CU(cudaMemsetAsync(base, 0x3c, 2 * vec + tab, ctx->stream));
    PadWork<T> w{nullptr, slot<cx<T>>(ctx, PadSlots<T>::b)};
    w.beta_tensor = ctx->aniso;
    auto run = [&](const std::array<int, 5>& c) -> cudaError_t {
        w.zvar = c[0];
        w.slices = c[1];
        w.xfwd = c[2];
        w.xinv = c[3];
        w.yvar = c[4];
        if (!fused)
            return launch_matvec<T>(ctx->g, R, x, y, w, ctx->tg, beta, BS, ghat_of<T>(ctx), tw_of<T>(ctx), nullptr,
                                    ctx->stream);
        // the two matvecs of a BiCGstab iteration, on a fresh scratch state
        // (the fused scatters write alpha and omega, and clear the flag of a
        // RHS that breaks down)
        cudaError_t e = cudaMemsetAsync(kst, 0x3c, R * sizeof(KState), ctx->stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(act, 0x01, R * sizeof(int), ctx->stream);
        // (BiCGstab's modes 3 and 2; the scratch vectors stand in for all of
        // the Krylov vectors, whose values do not matter here)
        for (int mode : {3, 2}) {
            if (e != cudaSuccess) break;
            FusedKrylov<T> fk;
            fk.mode = mode;
            fk.r = x;
            fk.v = y;
            fk.rhat = x;
            fk.s = x;
            fk.t = y;
            fk.x = y;
            fk.st = kst;
            fk.part = part;
            fk.cnt = cnt;
            fk.part_stride = ps;
            e = launch_matvec_fused<T>(ctx->g, R, x, y, w, ctx->tg, beta, BS, ghat_of<T>(ctx), tw_of<T>(ctx), act,
                                       fk, ctx->stream);
        }
        return e;
    };
    const bool was_on = ctx->prof.on;
    ctx->prof.on = false;  // tuning launches are not part of the traced work
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t ce = cudaEventCreate(&e0);
    if (ce == cudaSuccess) ce = cudaEventCreate(&e1);
    // The fastest of a set of candidates: one warm-up matvec each, then
    // rounds that alternate the candidates (so a clock ramp or a neighbour's
    // burst does not favour one); each keeps its best round.
    auto fastest = [&](const std::vector<std::array<int, 5>>& combos) -> size_t {
        constexpr int kRounds = 3, kReps = 2;
        std::vector<float> best(combos.size(), 0.f);
        for (size_t i = 0; i < combos.size() && ce == cudaSuccess; ++i) ce = run(combos[i]);
        for (int round = 0; round < kRounds && ce == cudaSuccess; ++round) {
            for (size_t i = 0; i < combos.size() && ce == cudaSuccess; ++i) {
                ce = cudaEventRecord(e0, ctx->stream);
                for (int k = 0; k < kReps && ce == cudaSuccess; ++k) ce = run(combos[i]);
                if (ce == cudaSuccess) ce = cudaEventRecord(e1, ctx->stream);
                if (ce == cudaSuccess) ce = cudaEventSynchronize(e1);
                float ms = 0.f;
                if (ce == cudaSuccess) ce = cudaEventElapsedTime(&ms, e0, e1);
                if (ce == cudaSuccess && (round == 0 || ms < best[i])) best[i] = ms;
            }
        }
        size_t pick = 0;
        for (size_t i = 1; i < combos.size(); ++i)
            if (best[i] < best[pick]) pick = i;
        return pick;
    };
    // One coordinate at a time (the passes are separate kernels): the z
    // schedule and slice passes with the default x and y passes, then the
    // x-forward schedule, the x-inverse schedule and the y-pass plan.
    std::vector<std::array<int, 5>> combos;
    for (int zv : zs)
        for (int sv : ss) combos.push_back({zv, sv, cur[2], cur[3], cur[4]});
    if (combos.size() > 1) cur = combos[fastest(combos)];
    if (!cur[1] && xfs.size() > 1 && ce == cudaSuccess) {
        combos.clear();
        for (int xv : xfs) combos.push_back({cur[0], 0, xv, cur[3], cur[4]});
        cur = combos[fastest(combos)];
    }
    if (!cur[1] && xis.size() > 1 && ce == cudaSuccess) {
        combos.clear();
        for (int xv : xis) combos.push_back({cur[0], 0, cur[2], xv, cur[4]});
        cur = combos[fastest(combos)];
    }
    if (!cur[1] && ys.size() > 1 && ce == cudaSuccess) {
        combos.clear();
        for (int yv : ys) combos.push_back({cur[0], 0, cur[2], cur[3], yv});
        cur = combos[fastest(combos)];
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    ctx->prof.on = was_on;
    free_mem(ctx->pool[S_TUNE]);
    if (ce != cudaSuccess) return ctx->cuda_fail(ce, "matvec schedule timing");
    ctx->zsched[key] = cur;
    apply(cur);
    return DDA_OK;
}

// y = A x over R RHS in chunks (workspace from ensure_pad<T>).
template <typename T>
dda_status run_matvec(dda_ctx* ctx, int R, const cx<T>* x, cx<T>* y, const int* active) {
    const int rc = matvec_chunk<T>(ctx, R);
    const int64_t n = 3 * ctx->g.N;
    PadWork<T> w{nullptr, slot<cx<T>>(ctx, PadSlots<T>::b)};
    w.beta_tensor = ctx->aniso;
    const int BS = beta_rhs_stride(ctx);
    dda_status zs;
    for (int r0 = 0; r0 < R; r0 += rc) {
        const int rn = std::min(rc, R - r0);
        if ((zs = pick_schedule<T>(ctx, rn, true, &w)) != DDA_OK) return zs;
        CU(launch_matvec<T>(ctx->g, rn, x + (int64_t)r0 * n, y + (int64_t)r0 * n, w, ctx->tg,
                            beta_of<T>(ctx) + (int64_t)r0 * BS, BS, ghat_of<T>(ctx), tw_of<T>(ctx),
                            active ? active + r0 : nullptr, ctx->stream));
    }
    return DDA_OK;
}

// Y = A X for FP64 vectors: native complex128 arithmetic, or (df) the
// double-float matvec on converted copies.
dda_status matvec64(dda_ctx* ctx, int R, const double2* X, double2* Y, const int* active, bool df) {
    if (!df) return run_matvec<double>(ctx, R, X, Y, active);
    const int64_t n = (int64_t)R * 3 * ctx->g.N;
    dda_status rs;
    if ((rs = ensure(ctx, ctx->pool[S_XDF], n * sizeof(cdfl))) != DDA_OK) return rs;
    if ((rs = ensure(ctx, ctx->pool[S_YDF], n * sizeof(cdfl))) != DDA_OK) return rs;
    if ((rs = ensure_pad<dfl>(ctx, R)) != DDA_OK) return rs;
    CU(launch_convert_c128_to_df(X, slot<cdfl>(ctx, S_XDF), n, ctx->stream));
    if ((rs = run_matvec<dfl>(ctx, R, slot<cdfl>(ctx, S_XDF), slot<cdfl>(ctx, S_YDF), active)) != DDA_OK) return rs;
    CU(launch_convert_df_to_c128(slot<cdfl>(ctx, S_YDF), Y, n, ctx->stream));
    return DDA_OK;
}

template <typename T> struct InnerSlots {
    static Inner<T> get(dda_ctx* ctx) {
        Inner<T> in;
        in.b = slot<cx<T>>(ctx, S_IN_B);
        in.x = slot<cx<T>>(ctx, S_IN_X);
        in.r = slot<cx<T>>(ctx, S_IN_R);
        in.rhat = slot<cx<T>>(ctx, S_IN_RHAT);
        in.p = slot<cx<T>>(ctx, S_IN_P);
        in.v = slot<cx<T>>(ctx, S_IN_V);
        in.s = slot<cx<T>>(ctx, S_IN_S);
        in.t = slot<cx<T>>(ctx, S_IN_T);
        in.u2 = slot<cx<T>>(ctx, S_IN_U2);
        return in;
    }
};

// Per-RHS stride (in double2) of the partial-sum buffer: enough for the
// reduction kernels (<= kMaxReduceBlocks blocks, 2 sums) and for the fused
// x-inverse scatter (one partial per block of that pass, 2 sums).
int partial_stride(const dda_ctx* ctx) {
    // 5 sums: the BiCGstab(2) Gram step; 4 per block: the BiCGstab t = A s scatter
    return std::max(5 * kMaxReduceBlocks, 4 * xinv_blocks_per_rhs(ctx->g));
}

// Matvec over R RHS in chunks with the BiCGstab updates of `mode` fused into
// its x passes (see FusedKrylov).
template <typename T>
dda_status run_matvec_fused(dda_ctx* ctx, int R, int mode, cx<T>* x, cx<T>* y, cx<T>* r, const cx<T>* v,
                            const cx<T>* rhat, const cx<T>* s_ = nullptr, const cx<T>* t = nullptr,
                            cx<T>* xsol = nullptr) {
    const int rc = matvec_chunk<T>(ctx, R);
    const int64_t n = 3 * ctx->g.N;
    PadWork<T> w{nullptr, slot<cx<T>>(ctx, PadSlots<T>::b)};
    w.beta_tensor = ctx->aniso;
    const int BS = beta_rhs_stride(ctx);
    const int ps = partial_stride(ctx);
    int* act = slot<int>(ctx, S_ACTIVE);
    dda_status zs;
    for (int r0 = 0; r0 < R; r0 += rc) {
        const int rn = std::min(rc, R - r0);
        const int64_t o = (int64_t)r0 * n;
        if ((zs = pick_schedule<T>(ctx, rn, true, &w, true)) != DDA_OK) return zs;
        FusedKrylov<T> fk;
        fk.mode = mode;
        fk.r = r + o;
        fk.v = v + o;
        fk.rhat = rhat + o;
        if (mode == 3) {
            fk.s = s_ + o;
            fk.t = t + o;
            fk.x = xsol + o;
        }
        fk.st = slot<KState>(ctx, S_STATE) + r0;
        fk.part = slot<double2>(ctx, S_PART) + (int64_t)r0 * ps;
        fk.cnt = slot<unsigned>(ctx, S_CNT) + r0;
        fk.part_stride = ps;
        CU(launch_matvec_fused<T>(ctx->g, rn, x + o, y + o, w, ctx->tg, beta_of<T>(ctx) + (int64_t)r0 * BS, BS,
                                  ghat_of<T>(ctx), tw_of<T>(ctx), act + r0, fk, ctx->stream));
    }
    return DDA_OK;
}

// One BiCGstab iteration for every active RHS, two matvecs and no other
// kernel: the first one's gather applies the previous iteration's end
// (r <- s - omega t, x += alpha p + omega s) and forms p <- r + beta (p -
// omega v), its scatter alpha; the second one's gather forms s <- r -
// alpha v, its scatter omega, |r|, rho', beta and the stopping tests
// (FusedKrylov modes 3 and 2).
template <typename T> dda_status inner_iteration(dda_ctx* ctx, int R) {
    Inner<T> in = InnerSlots<T>::get(ctx);
    dda_status rs;
    if ((rs = run_matvec_fused<T>(ctx, R, 3, in.p, in.v, in.r, in.v, in.rhat, in.s, in.t, in.x)) != DDA_OK) return rs;
    return run_matvec_fused<T>(ctx, R, 2, in.s, in.t, in.r, in.v, in.rhat);
}

// One BiCGstab(2) iteration for every active RHS (bicgstab2.cu): two BiCG
// steps and the degree-2 minimal-residual step, 4 matvecs.  The matvecs of
// u1 = A u0 and u2 = A u1 take the update u <- r - beta u in their gather
// and alpha = rho / <rt, A u> in their scatter (the BiCGstab mode-1 fusion,
// fed beta -> -beta and omega = 0 by the BiCGstab(2) kernels).
template <typename T> dda_status inner_iteration_b2(dda_ctx* ctx, int R) {
    using B2 = BiCGstab2Ops<cx<T>>;
    const int64_t n = 3 * ctx->g.N;
    Inner<T> in = InnerSlots<T>::get(ctx);
    cx<T>*r0 = in.r, *r1 = in.s, *r2 = in.t, *u0 = in.p, *u1 = in.v, *u2 = in.u2;
    KState* st = slot<KState>(ctx, S_STATE);
    int* act = slot<int>(ctx, S_ACTIVE);
    double2* part = slot<double2>(ctx, S_PART);
    unsigned* cnt = slot<unsigned>(ctx, S_CNT);
    cudaStream_t s = ctx->stream;
    dda_status rs;
    if ((rs = run_matvec_fused<T>(ctx, R, 1, u0, u1, r0, r0, in.rhat)) != DDA_OK) return rs;
    CU(B2::r0(R, n, r0, u1, in.x, u0, st, act, s));
    if ((rs = run_matvec<T>(ctx, R, r0, r1, act)) != DDA_OK) return rs;
    CU(B2::rho(R, n, in.rhat, r1, st, act, part, cnt, s));
    if ((rs = run_matvec_fused<T>(ctx, R, 1, u1, u2, r1, r1, in.rhat)) != DDA_OK) return rs;
    CU(B2::r1(R, n, r0, r1, u0, u1, u2, in.x, st, act, s));
    if ((rs = run_matvec<T>(ctx, R, r1, r2, act)) != DDA_OK) return rs;
    CU(B2::gram(R, n, r0, r1, r2, st, act, part, cnt, s));
    CU(B2::mr(R, n, in.x, r0, r1, r2, u0, u1, u2, in.rhat, st, act, part, cnt, s));
    return DDA_OK;
}

// One QMR iteration for every active RHS (qmr.cu): w = A v, alpha, the
// Lanczos vector with the rotations, the updates.  v, p and A p each rotate
// through two slots; `odd` selects the assignment of this iteration.
//   slots: x, r, w = t; v / v_prev = s / rhat; p1 / p2 = p / v; Ap1 / Ap2 = u2 / b
template <typename T> dda_status inner_iteration_qmr(dda_ctx* ctx, int R, bool odd) {
    using Q = QmrOps<cx<T>>;
    const int64_t n = 3 * ctx->g.N;
    Inner<T> in = InnerSlots<T>::get(ctx);
    cx<T>*v = in.s, *vp = in.rhat, *p1 = in.p, *p2 = in.v, *ap1 = in.u2, *ap2 = in.b;
    if (odd) {
        std::swap(v, vp);
        std::swap(p1, p2);
        std::swap(ap1, ap2);
    }
    KState* st = slot<KState>(ctx, S_STATE);
    int* act = slot<int>(ctx, S_ACTIVE);
    double2* part = slot<double2>(ctx, S_PART);
    unsigned* cnt = slot<unsigned>(ctx, S_CNT);
    cudaStream_t s = ctx->stream;
    dda_status rs;
    if ((rs = run_matvec<T>(ctx, R, v, in.t, act)) != DDA_OK) return rs;
    CU(Q::alpha(R, n, v, in.t, st, act, part, cnt, s));
    CU(Q::lanczos(R, n, in.t, v, vp, st, act, part, cnt, s));
    CU(Q::update(R, n, v, vp, in.t, p1, p2, ap1, ap2, in.x, in.r, st, act, part, cnt, s));
    return DDA_OK;
}

// Iterations per captured block: 8 matvecs per RHS for every solver (an even
// count, so the QMR slot rotation is the same at every block start).
int block_iterations(int solver) {
    return solver == DDA_SOLVER_BICGSTAB2 ? 2 : (solver == DDA_SOLVER_QMR ? 8 : 4);
}
int matvecs_per_iteration(int solver) {
    return solver == DDA_SOLVER_BICGSTAB2 ? 4 : (solver == DDA_SOLVER_QMR ? 1 : 2);
}

template <typename T> dda_status inner_block(dda_ctx* ctx, int R, int K, int solver) {
    dda_status rs;
    for (int k = 0; k < K; ++k) {
        if (solver == DDA_SOLVER_BICGSTAB2) rs = inner_iteration_b2<T>(ctx, R);
        else if (solver == DDA_SOLVER_QMR) rs = inner_iteration_qmr<T>(ctx, R, (k & 1) != 0);
        else rs = inner_iteration<T>(ctx, R);
        if (rs != DDA_OK) return rs;
    }
    CU(launch_count_active(slot<int>(ctx, S_ACTIVE), R, slot<int>(ctx, S_COUNT), ctx->stream));
    CU(cudaMemcpyAsync(ctx->h_count, ctx->pool[S_COUNT].p, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    return DDA_OK;
}

// Iterate until no RHS is active (the device decides convergence and maxit).
// The first block of K iterations runs eagerly; with use_graph the block is
// then captured once and replayed.
template <typename T> dda_status inner_solve(dda_ctx* ctx, int R, int maxit, bool use_graph, int solver) {
    const int K = block_iterations(solver);
    const int prec = sizeof(T) == 4 ? 1 : 0;
    const int max_blocks = maxit / K + 2;
    dda_status rs;
    bool have_graph = ctx->graph.exec && ctx->graph.R == R && ctx->graph.prec == prec && ctx->graph.K == K &&
                      ctx->graph.solver == solver && ctx->graph.stream == ctx->stream &&
                      ctx->graph.traced == ctx->prof.on;
    for (int b = 0; b < max_blocks; ++b) {
        if (use_graph && have_graph) {
            CU(cudaGraphLaunch(ctx->graph.exec, ctx->stream));
            if (ctx->prof.on) ctx->prof.graph_launched();
        } else if ((rs = inner_block<T>(ctx, R, K, solver)) != DDA_OK) {
            return rs;
        }
        CU(sync_collect(ctx));
        if (*ctx->h_count == 0) break;
        if (use_graph && !have_graph) {
            if (ctx->graph.exec) {
                cudaGraphExecDestroy(ctx->graph.exec);
                ctx->graph.exec = nullptr;
            }
            cudaGraph_t graph = nullptr;
            ctx->prof.capture_begin();
            CU(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
            rs = inner_block<T>(ctx, R, K, solver);
            cudaError_t ce = cudaStreamEndCapture(ctx->stream, &graph);
            ctx->prof.capture_end();
            if (rs != DDA_OK) {
                if (graph) cudaGraphDestroy(graph);
                return rs;
            }
            if (ce != cudaSuccess) return ctx->cuda_fail(ce, "cudaStreamEndCapture");
            ce = cudaGraphInstantiate(&ctx->graph.exec, graph, 0);
            cudaGraphDestroy(graph);
            if (ce != cudaSuccess) return ctx->cuda_fail(ce, "cudaGraphInstantiate");
            ctx->graph.R = R;
            ctx->graph.prec = prec;
            ctx->graph.K = K;
            ctx->graph.solver = solver;
            ctx->graph.stream = ctx->stream;
            ctx->graph.traced = ctx->prof.on;
            have_graph = true;
        }
    }
    // BiCGstab: the last x update of a RHS that stopped in the second matvec's
    // scatter is still to be applied
    if (solver == DDA_SOLVER_BICGSTAB) {
        Inner<T> in = InnerSlots<T>::get(ctx);
        CU(KrylovOps<cx<T>>::finish_x(R, 3 * ctx->g.N, in.x, in.p, in.s, slot<KState>(ctx, S_STATE), ctx->stream));
    }
    return DDA_OK;
}

struct RhsTrack {
    double bn = 0.0, rn = 0.0;
    int iters = 0, outer = 0, mv = 0;
    int status = KS_RUNNING;
    bool done = false;
};

dda_status ensure_common(dda_ctx* ctx, int R) {
    dda_status s;
    const size_t nb = (size_t)R * partial_stride(ctx) * sizeof(double2);
    if ((s = ensure(ctx, ctx->pool[S_PART], nb)) != DDA_OK) return s;
    if (ctx->pool[S_CNT].bytes < R * sizeof(unsigned)) {
        if ((s = ensure(ctx, ctx->pool[S_CNT], R * sizeof(unsigned), true)) != DDA_OK) return s;
    }
    for (int sl : {S_ACTIVE, S_WANT, S_OUTER})
        if ((s = ensure(ctx, ctx->pool[sl], R * sizeof(int))) != DDA_OK) return s;
    for (int sl : {S_TOLREL, S_SCALE, S_COEF, S_NORM_B, S_NORM_R})
        if ((s = ensure(ctx, ctx->pool[sl], R * sizeof(double))) != DDA_OK) return s;
    if ((s = ensure(ctx, ctx->pool[S_STATE], R * sizeof(KState))) != DDA_OK) return s;
    if ((s = ensure(ctx, ctx->pool[S_QSUM], R * sizeof(double2))) != DDA_OK) return s;
    if ((s = ensure(ctx, ctx->pool[S_COUNT], sizeof(int))) != DDA_OK) return s;
    return DDA_OK;
}

template <typename T> dda_status ensure_inner(dda_ctx* ctx, int R, int solver) {
    const size_t vb = (size_t)R * 3 * ctx->g.N * sizeof(cx<T>);
    dda_status s;
    for (int sl = S_IN_B; sl <= S_IN_T; ++sl)
        if ((s = ensure(ctx, ctx->pool[sl], vb)) != DDA_OK) return s;
    if (solver != DDA_SOLVER_BICGSTAB && (s = ensure(ctx, ctx->pool[S_IN_U2], vb)) != DDA_OK) return s;
    return ensure_pad<T>(ctx, R);
}

// Solve A x = b (b = S_E64, x -> S_X64) for R RHS with inner precision T.
// refine: FP64 outer residual loop; otherwise a single inner solve.
template <typename T>
dda_status solve_core(dda_ctx* ctx, int R, const dda_opts& o, bool refine, bool have_x0,
                      std::vector<RhsTrack>& tr) {
    const int64_t n = 3 * ctx->g.N;
    cudaStream_t s = ctx->stream;
    dda_status rs;
    // refinement residuals of the complex64 modes in double-float unless FP64 is asked for
    const bool df_resid = (sizeof(T) == 4) && !o.residual_fp64 && ctx->m_ghdf.p != nullptr;
    if ((rs = ensure_common(ctx, R)) != DDA_OK) return rs;
    if ((rs = ensure_inner<T>(ctx, R, o.solver)) != DDA_OK) return rs;
    if ((rs = ensure_pad<double>(ctx, R)) != DDA_OK) return rs;
    const size_t vb64 = (size_t)R * n * sizeof(double2);
    for (int sl : {S_X64, S_R64, S_Y64})
        if ((rs = ensure(ctx, ctx->pool[sl], vb64)) != DDA_OK) return rs;
    double2* E = slot<double2>(ctx, S_E64);
    double2* X = slot<double2>(ctx, S_X64);
    double2* Rr = slot<double2>(ctx, S_R64);
    double2* Y = slot<double2>(ctx, S_Y64);
    double2* part = slot<double2>(ctx, S_PART);
    unsigned* cnt = slot<unsigned>(ctx, S_CNT);
    int* outer = slot<int>(ctx, S_OUTER);
    std::vector<double> hb(R), hr(R), tmp(R);
    std::vector<int> hact(R, 1);

    CU(launch_residual(R, n, E, nullptr, nullptr, slot<double>(ctx, S_NORM_B), nullptr, part, cnt, s));
    if (have_x0) {
        CU(cudaMemcpyAsync(outer, hact.data(), R * sizeof(int), cudaMemcpyHostToDevice, s));
        if ((rs = matvec64(ctx, R, X, Y, nullptr, df_resid)) != DDA_OK) return rs;
        CU(launch_residual(R, n, E, Y, Rr, slot<double>(ctx, S_NORM_R), nullptr, part, cnt, s));
        for (auto& t : tr) t.mv += 1;
    } else {
        CU(cudaMemsetAsync(X, 0, vb64, s));
        CU(launch_residual(R, n, E, nullptr, Rr, slot<double>(ctx, S_NORM_R), nullptr, part, cnt, s));
    }
    CU(cudaMemcpyAsync(hb.data(), ctx->pool[S_NORM_B].p, R * sizeof(double), cudaMemcpyDeviceToHost, s));
    CU(cudaMemcpyAsync(hr.data(), ctx->pool[S_NORM_R].p, R * sizeof(double), cudaMemcpyDeviceToHost, s));
    CU(sync_collect(ctx));
    for (int r = 0; r < R; ++r) {
        tr[r].bn = std::sqrt(hb[r]);
        tr[r].rn = std::sqrt(hr[r]);
        if (!std::isfinite(tr[r].bn)) return ctx->fail(DDA_ERR_NONFINITE, "non-finite right-hand side");
    }
    const int max_outer = refine ? (o.max_outer > 0 ? o.max_outer : 8) : 1;
    const double floor_tol = (sizeof(T) == 4) ? (o.inner_tol > 0 ? o.inner_tol : 2e-6) : 1e-15;
    Inner<T> in = InnerSlots<T>::get(ctx);
    std::vector<KState> hst(R);
    for (int it = 0; it < max_outer; ++it) {
        int nact = 0;
        std::vector<double> tolrel(R, 0.0), scale(R, 0.0), coef(R, 0.0);
        for (int r = 0; r < R; ++r) {
            RhsTrack& t = tr[r];
            hact[r] = 0;
            if (t.done) continue;
            if (t.rn <= o.tol * t.bn) {
                t.done = true;
                t.status = KS_CONVERGED;
                continue;
            }
            if (t.iters >= o.maxit) {
                t.done = true;
                if (t.status == KS_RUNNING || t.status == KS_CONVERGED) t.status = KS_MAXIT;
                continue;
            }
            hact[r] = 1;
            ++nact;
            scale[r] = 1.0 / t.rn;
            coef[r] = t.rn;
            const double want = refine ? 0.5 * o.tol * t.bn / t.rn : o.tol * t.bn / t.rn;
            tolrel[r] = std::max(want, floor_tol);
        }
        if (nact == 0) break;
        CU(cudaMemcpyAsync(outer, hact.data(), R * sizeof(int), cudaMemcpyHostToDevice, s));
        CU(cudaMemcpyAsync(ctx->pool[S_TOLREL].p, tolrel.data(), R * sizeof(double), cudaMemcpyHostToDevice, s));
        CU(cudaMemcpyAsync(ctx->pool[S_SCALE].p, scale.data(), R * sizeof(double), cudaMemcpyHostToDevice, s));
        CU(cudaMemcpyAsync(ctx->pool[S_COEF].p, coef.data(), R * sizeof(double), cudaMemcpyHostToDevice, s));
        for (int r = 0; r < R; ++r) {
            std::memset(&hst[r], 0, sizeof(KState));
            hst[r].maxit = std::max(1, o.maxit - tr[r].iters);
        }
        CU(cudaMemcpyAsync(ctx->pool[S_STATE].p, hst.data(), R * sizeof(KState), cudaMemcpyHostToDevice, s));
        CU(KrylovOps<cx<T>>::to_inner(R, n, Rr, in.b, slot<double>(ctx, S_SCALE), outer, s));
        CU(KrylovOps<cx<T>>::init(R, n, in.b, in.x, in.r, in.rhat, in.p, in.v,
                                  o.solver == DDA_SOLVER_BICGSTAB ? in.s : nullptr, slot<KState>(ctx, S_STATE),
                                  slot<double>(ctx, S_TOLREL), outer, slot<int>(ctx, S_ACTIVE), part, cnt, s));
        if (o.solver == DDA_SOLVER_QMR)
            CU(QmrOps<cx<T>>::init(R, n, in.r, in.s, in.rhat, in.u2, in.b, slot<KState>(ctx, S_STATE),
                                   slot<int>(ctx, S_ACTIVE), part, cnt, s));
        if ((rs = inner_solve<T>(ctx, R, o.maxit, o.use_graph != 0, o.solver)) != DDA_OK) return rs;
        CU(cudaMemcpyAsync(hst.data(), ctx->pool[S_STATE].p, R * sizeof(KState), cudaMemcpyDeviceToHost, s));
        CU(KrylovOps<cx<T>>::accumulate(R, n, X, in.x, slot<double>(ctx, S_COEF), outer, s));
        if ((rs = matvec64(ctx, R, X, Y, outer, df_resid)) != DDA_OK) return rs;
        CU(launch_residual(R, n, E, Y, Rr, slot<double>(ctx, S_NORM_R), outer, part, cnt, s));
        CU(cudaMemcpyAsync(hr.data(), ctx->pool[S_NORM_R].p, R * sizeof(double), cudaMemcpyDeviceToHost, s));
        CU(sync_collect(ctx));
        for (int r = 0; r < R; ++r) {
            if (!hact[r]) continue;
            RhsTrack& t = tr[r];
            t.iters += hst[r].iter;
            t.mv += matvecs_per_iteration(o.solver) * hst[r].iter + 1;
            t.outer += 1;
            const double prev = t.rn;
            t.rn = std::sqrt(hr[r]);
            if (hst[r].status == KS_NONFINITE || !std::isfinite(t.rn)) {
                t.status = KS_NONFINITE;
                t.done = true;
            } else if (t.rn <= o.tol * t.bn) {
                t.status = KS_CONVERGED;
                t.done = true;
            } else if (!refine) {
                t.status = hst[r].status == KS_CONVERGED ? KS_MAXIT : hst[r].status;
                t.done = true;
            } else if (hst[r].status == KS_BREAKDOWN && hst[r].iter == 0) {
                t.status = KS_BREAKDOWN;
                t.done = true;
            } else if (t.rn > 0.9 * prev && hst[r].status != KS_CONVERGED) {
                t.status = hst[r].status == KS_BREAKDOWN ? KS_BREAKDOWN : KS_MAXIT;
                t.done = true;
            }
        }
    }
    for (auto& t : tr)
        if (!t.done) {
            t.done = true;
            t.status = (t.rn <= o.tol * t.bn) ? KS_CONVERGED : KS_MAXIT;
        }
    return DDA_OK;
}

dda_status map_status(int ks) {
    switch (ks) {
        case KS_CONVERGED: return DDA_OK;
        case KS_BREAKDOWN: return DDA_ERR_BREAKDOWN;
        case KS_NONFINITE: return DDA_ERR_NONFINITE;
        default: return DDA_ERR_NOT_CONVERGED;
    }
}

dda_status check_ready(dda_ctx* ctx, dda_precision prec) {
    if (!ctx) return DDA_ERR_ARG;
    if (!ctx->prepared) return ctx->fail(DDA_ERR_ARG, "dda_prepare has not been called for the current target");
    if (prec != DDA_FP64 && prec != DDA_FP32 && prec != DDA_FP32_REFINED)
        return ctx->fail(DDA_ERR_ARG, "unknown precision %d", (int)prec);
    if (prec != DDA_FP64 && !ctx->has32)
        return ctx->fail(DDA_ERR_ARG, "precision needs the complex64 Green tensor: prepare with an FP32 mode");
    return DDA_OK;
}

dda_opts default_opts() {
    dda_opts o;
    o.tol = 1e-5;
    o.maxit = 1000;
    o.use_graph = 1;
    o.inner_tol = 0.0;
    o.max_outer = 0;
    o.normal_eq = 0;
    o.x0 = nullptr;
    o.residual_fp64 = 0;
    o.solver = DDA_SOLVER_BICGSTAB;
    return o;
}

// Forward solve of A P = E_inc; P left in S_X64, E in S_E64.
dda_status forward_solve(dda_ctx* ctx, dda_precision prec, int R, const double* khat, const double* e,
                         const dda_opts* opts_in, dda_result* res) {
    dda_status rs;
    if ((rs = check_ready(ctx, prec)) != DDA_OK) return rs;
    if (res == nullptr) return ctx->fail(DDA_ERR_ARG, "res must not be NULL");
    dda_opts o = opts_in ? *opts_in : default_opts();
    if (!(o.tol > 0.0) || o.maxit <= 0) return ctx->fail(DDA_ERR_ARG, "tol must be > 0 and maxit > 0");
    if (o.solver != DDA_SOLVER_BICGSTAB && o.solver != DDA_SOLVER_BICGSTAB2 && o.solver != DDA_SOLVER_QMR)
        return ctx->fail(DDA_ERR_ARG, "unknown solver %d", o.solver);
    std::vector<double> k;
    std::vector<cd> ev;
    if ((rs = check_rhs(ctx, R, khat, e, k, ev)) != DDA_OK) return rs;
    if ((rs = upload_tables(ctx, R, k, ev)) != DDA_OK) return rs;
    const int64_t n = 3 * ctx->g.N;
    const size_t vb64 = (size_t)R * n * sizeof(double2);
    for (int sl : {S_E64, S_X64})
        if ((rs = ensure(ctx, ctx->pool[sl], vb64)) != DDA_OK) return rs;
    CU(launch_einc(R, ctx->g.N, ctx->tg.lat_of, ctx->g, ctx->kd, slot<double>(ctx, S_KHAT),
                   slot<double2>(ctx, S_EPOL), slot<double2>(ctx, S_E64), ctx->stream));
    const bool have_x0 = o.x0 != nullptr;
    if (have_x0) {
        for (size_t i = 0; i < (size_t)R * n * 2; ++i)
            if (!std::isfinite(o.x0[i])) return ctx->fail(DDA_ERR_NONFINITE, "non-finite initial guess");
        CU(cudaMemcpyAsync(ctx->pool[S_X64].p, o.x0, vb64, cudaMemcpyHostToDevice, ctx->stream));
    }
    std::vector<RhsTrack> tr(R);
    if (prec == DDA_FP64)
        rs = solve_core<double>(ctx, R, o, true, have_x0, tr);
    else
        rs = solve_core<float>(ctx, R, o, prec == DDA_FP32_REFINED, have_x0, tr);
    if (rs != DDA_OK) return rs;
    // Q reductions (FP64)
    CU(launch_qsums(R, ctx->g.N, slot<double2>(ctx, S_E64), slot<double2>(ctx, S_X64), ctx->tg.comp_of,
                    slot<double>(ctx, S_W), qweight_stride(ctx), ctx->aniso, slot<double2>(ctx, S_QSUM),
                    slot<double2>(ctx, S_PART),
                    slot<unsigned>(ctx, S_CNT), ctx->stream));
    std::vector<double2> q(R);
    CU(cudaMemcpyAsync(q.data(), ctx->pool[S_QSUM].p, R * sizeof(double2), cudaMemcpyDeviceToHost, ctx->stream));
    std::vector<double> ne(R, -1.0);
    if (o.normal_eq) {
        // |A^H (A P - E)| / |A^H E| with A^H y = conj(A conj(y)); S_Y64 holds A P
        double2* Y = slot<double2>(ctx, S_Y64);
        double2* Rr = slot<double2>(ctx, S_R64);
        double2* E = slot<double2>(ctx, S_E64);
        dda_status s2;
        if ((s2 = run_matvec<double>(ctx, R, slot<double2>(ctx, S_X64), Y, nullptr)) != DDA_OK) return s2;
        CU(launch_conj_diff(R, n, Y, E, Rr, ctx->stream));
        if ((s2 = run_matvec<double>(ctx, R, Rr, Y, nullptr)) != DDA_OK) return s2;
        CU(launch_residual(R, n, Y, nullptr, nullptr, slot<double>(ctx, S_NORM_R), nullptr, slot<double2>(ctx, S_PART),
                           slot<unsigned>(ctx, S_CNT), ctx->stream));
        CU(launch_conj_diff(R, n, E, nullptr, Rr, ctx->stream));
        if ((s2 = run_matvec<double>(ctx, R, Rr, Y, nullptr)) != DDA_OK) return s2;
        CU(launch_residual(R, n, Y, nullptr, nullptr, slot<double>(ctx, S_NORM_B), nullptr, slot<double2>(ctx, S_PART),
                           slot<unsigned>(ctx, S_CNT), ctx->stream));
        std::vector<double> a(R), b(R);
        CU(cudaMemcpyAsync(a.data(), ctx->pool[S_NORM_R].p, R * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
        CU(cudaMemcpyAsync(b.data(), ctx->pool[S_NORM_B].p, R * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
        CU(sync_collect(ctx));
        for (int r = 0; r < R; ++r) ne[r] = std::sqrt(a[r] / b[r]);
    }
    CU(sync_collect(ctx));
    const double kd = ctx->kd, a2 = ctx->aeff_lat * ctx->aeff_lat;
    dda_status worst = DDA_OK;
    for (int r = 0; r < R; ++r) {
        dda_result& out = res[r];
        const double cext = 4.0 * kPi * kd * q[r].x, cabs = 4.0 * kPi * kd * q[r].y;
        out.qext = cext / (kPi * a2);
        out.qabs = cabs / (kPi * a2);
        out.qsca = out.qext - out.qabs;
        out.resid_rel = tr[r].bn > 0 ? tr[r].rn / tr[r].bn : 0.0;
        out.resid_normal_eq = ne[r];
        out.iters = tr[r].iters;
        out.outer_iters = tr[r].outer;
        out.matvecs = tr[r].mv;
        out.status = map_status(tr[r].status);
        if (out.status != DDA_OK && worst == DDA_OK) worst = out.status;
    }
    if (worst != DDA_OK) ctx->fail(worst, "some right-hand sides did not converge (see per-RHS status)");
    return worst;
}

void host_twiddles(int L, std::vector<double2>& t64, std::vector<float2>& t32) {
    t64.resize(L);
    t32.resize(L);
    for (int m = 0; m < L; ++m) {
        const double a = -2.0 * kPi * (double)m / (double)L;
        t64[m] = make_double2(std::cos(a), std::sin(a));
        t32[m] = make_float2((float)t64[m].x, (float)t64[m].y);
    }
}

}  // namespace

// ---- no-allocation matvec scratch ------------------------------------------------
// The padded work buffers and the 1/alpha table of dda_matvec_device_noalloc
// live in this file-scope device array.  Every GPU that loads the library
// holds it until the process exits.  In host code `g_noalloc_scratch` names
// a host-side stand-in, not device memory: kernels only ever receive the
// address returned by cudaGetSymbolAddress below.
static constexpr size_t kNoAllocScratchBytes = size_t(64) << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_ptr[kMaxDevices] = {};
unsigned long long g_noalloc_ctx[kMaxDevices] = {};

// Unique id of the calling thread's current CUDA context, through the driver
// entry points that the runtime hands out (the library does not link the
// driver library itself).  0 if the driver does not offer them.
unsigned long long current_context_id() {
    static PFN_cuCtxGetCurrent_v4000 get_current = nullptr;
    static PFN_cuCtxGetId_v12000 get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        cudaDriverEntryPointQueryResult q;
        void* f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 4000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = reinterpret_cast<PFN_cuCtxGetCurrent_v4000>(f);
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<PFN_cuCtxGetId_v12000>(f);
    });
    CUcontext c = nullptr;
    unsigned long long id = 0;
    if (get_current && get_id && get_current(&c) == CUDA_SUCCESS && c && get_id(c, &id) == CUDA_SUCCESS) return id;
    return 0;
}

// Device address of the scratch array on `device` (which must be current).
// It is looked up on the first call for that device, and again when the
// device's context has been destroyed and re-created since (cudaDeviceReset
// reloads the library's module, and the array may then sit elsewhere).
cudaError_t noalloc_scratch(int device, unsigned char** out) {
    if (device < 0 || device >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    const unsigned long long ctx_id = current_context_id();
    if (g_noalloc_ptr[device] == nullptr || (ctx_id != 0 && ctx_id != g_noalloc_ctx[device])) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_noalloc_ptr[device] = p;
        g_noalloc_ctx[device] = ctx_id;
    }
    *out = static_cast<unsigned char*>(g_noalloc_ptr[device]);
    return cudaSuccess;
}

template <typename T>
dda_status matvec_noalloc(dda_ctx* ctx, int R, const std::vector<double>& k, const std::vector<cd>& ev,
                          const void* x_dev, void* y_dev) {
    using C = cx<T>;
    const int BS = beta_rhs_stride(ctx);
    const size_t beta_bytes = align256((size_t)R * BS * sizeof(C));
    const size_t u2_bytes = (size_t)R * 3 * ctx->g.u2_per_comp() * sizeof(C);
    const size_t need = beta_bytes + u2_bytes;
    if (need > kNoAllocScratchBytes)
        return ctx->fail(DDA_ERR_SIZE,
                         "dda_matvec_device_noalloc needs %zu bytes of scratch for R=%d on this lattice; "
                         "its fixed scratch holds %zu bytes (use dda_matvec_device or fewer RHS)",
                         need, R, kNoAllocScratchBytes);
    unsigned char* base = nullptr;
    CU(noalloc_scratch(ctx->device, &base));
    std::vector<cd> bt;
    dda_status ts;
    if ((ts = diag_tables(ctx, R, k, ev, bt, nullptr)) != DDA_OK) return ts;
    std::vector<C> beta(bt.size());
    for (size_t i = 0; i < bt.size(); ++i) beta[i] = ccast<C>(make_double2(bt[i].real(), bt[i].imag()));
    C* d_beta = reinterpret_cast<C*>(base);
    PadWork<T> w{nullptr, reinterpret_cast<C*>(base + beta_bytes)};
    w.beta_tensor = ctx->aniso;
    CU(cudaMemcpyAsync(d_beta, beta.data(), beta.size() * sizeof(C), cudaMemcpyHostToDevice, ctx->stream));
    dda_status zs;
    if ((zs = pick_schedule<T>(ctx, R, false, &w)) != DDA_OK) return zs;  // no timing here
    CU(launch_matvec<T>(ctx->g, R, static_cast<const C*>(x_dev), static_cast<C*>(y_dev), w, ctx->tg, d_beta, BS,
                        ghat_of<T>(ctx), tw_of<T>(ctx), nullptr, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    return DDA_OK;
}
}  // namespace

namespace {
// Back to composition codes after per-site materials: the device composition
// array of the target serves the tables again.
void leave_site_mode(dda_ctx* ctx) {
    if (!ctx->site_mode) return;
    ctx->site_mode = false;
    ctx->tg.comp_of = (uint8_t*)ctx->m_comp_of.p;
    ctx->zsched.clear();
    if (ctx->graph.exec) {
        cudaGraphExecDestroy(ctx->graph.exec);
        ctx->graph.exec = nullptr;
    }
}

// Switch between the scalar and the tensor 1/alpha tables: the cached
// schedules (slice passes) and the captured solve graph depend on it.
void set_isotropy(dda_ctx* ctx, bool aniso) {
    if (ctx->aniso == aniso) return;
    ctx->aniso = aniso;
    if (!aniso) {
        ctx->m3.clear();
        ctx->df_angles.clear();
    }
    ctx->zsched.clear();
    if (ctx->graph.exec) {
        cudaGraphExecDestroy(ctx->graph.exec);
        ctx->graph.exec = nullptr;
    }
}
}  // namespace

// ================================================================== ABI ===
extern "C" {

dda_status dda_create(int device, dda_ctx** out) {
    if (out == nullptr) return DDA_ERR_ARG;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return DDA_ERR_CUDA;
    }
    dda_ctx* ctx = new dda_ctx();
    ctx->device = device;
    ctx->pool.resize(S_NSLOTS);
    if (cudaSetDevice(device) != cudaSuccess || cudaStreamCreateWithFlags(&ctx->own_stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaMallocHost(&ctx->h_count, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        delete ctx;
        return DDA_ERR_CUDA;
    }
    ctx->stream = ctx->own_stream;
    *out = ctx;
    return DDA_OK;
}

dda_status dda_destroy(dda_ctx* ctx) {
    if (!ctx) return DDA_OK;
    cudaSetDevice(ctx->device);
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    if (ctx->graph.exec) cudaGraphExecDestroy(ctx->graph.exec);
    for (auto& m : ctx->pool) free_mem(m);
    free_mem(ctx->m_site_of);
    free_mem(ctx->m_rows);
    free_mem(ctx->m_lat_of);
    free_mem(ctx->m_comp_of);
    free_mem(ctx->m_gh64);
    free_mem(ctx->m_gh32);
    free_mem(ctx->m_ghdf);
    for (int a = 0; a < 3; ++a) {
        free_mem(ctx->m_tw64[a]);
        free_mem(ctx->m_tw32[a]);
        free_mem(ctx->m_twdf[a]);
    }
    ctx->prof.release();
    if (ctx->h_count) cudaFreeHost(ctx->h_count);
    if (ctx->own_stream) cudaStreamDestroy(ctx->own_stream);
    delete ctx;
    return DDA_OK;
}

const char* dda_last_error(const dda_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

dda_status dda_set_stream(dda_ctx* ctx, void* stream) {
    if (!ctx) return DDA_ERR_ARG;
    cudaSetDevice(ctx->device);
    ctx->stream = stream ? (cudaStream_t)stream : ctx->own_stream;
    return DDA_OK;
}

dda_status dda_set_target(dda_ctx* ctx, int nx, int ny, int nz, const uint8_t* comp) {
    if (!ctx) return DDA_ERR_ARG;
    if (nx <= 0 || ny <= 0 || nz <= 0 || comp == nullptr) return ctx->fail(DDA_ERR_ARG, "bad lattice dimensions");
    Geom g;
    g.ox = nx;
    g.oy = ny;
    g.oz = nz;
    g.Lx = pick_fft_length(nx);
    g.Ly = pick_fft_length(ny);
    g.Lz = pick_fft_length(nz);
    if (!g.Lx || !g.Ly || !g.Lz)
        return ctx->fail(DDA_ERR_SIZE, "lattice %dx%dx%d exceeds the largest supported padded length", nx, ny, nz);
    // the kernels work on the lattice extended with vacuum to L/2 per axis
    g.nx = g.Lx / 2;
    g.ny = g.Ly / 2;
    g.nz = g.Lz / 2;
    const int64_t M = g.M();
    if (M > (int64_t)INT32_MAX) return ctx->fail(DDA_ERR_SIZE, "lattice too large");
    std::vector<int> site_of(M, -1), lat_of;
    std::vector<uint8_t> comp_of;
    int maxc = 0;
    for (int iz = 0; iz < nz; ++iz)
        for (int iy = 0; iy < ny; ++iy)
            for (int ix = 0; ix < nx; ++ix) {
                const uint8_t cv = comp[((int64_t)iz * ny + iy) * nx + ix];
                if (!cv) continue;
                const int64_t li = ((int64_t)iz * g.ny + iy) * g.nx + ix;
                site_of[li] = (int)lat_of.size();
                lat_of.push_back((int)li);
                comp_of.push_back(cv);
                maxc = std::max<int>(maxc, cv);
            }
    if (lat_of.empty()) return ctx->fail(DDA_ERR_ARG, "target has no occupied site");
    g.N = (int64_t)lat_of.size();
    // the x rows with at least one site (the x-inverse pass transforms only these)
    std::vector<int> rows;
    for (int iz = 0; iz < g.nz; ++iz)
        for (int iy = 0; iy < g.ny; ++iy) {
            const int64_t r0 = ((int64_t)iz * g.ny + iy) * g.nx;
            for (int ix = 0; ix < g.nx; ++ix)
                if (site_of[r0 + ix] >= 0) {
                    rows.push_back(iz * g.ny + iy);
                    break;
                }
        }
    cudaSetDevice(ctx->device);
    ctx->prepared = false;
    ctx->has32 = false;
    dda_status s;
    if ((s = ensure(ctx, ctx->m_site_of, M * sizeof(int))) != DDA_OK) return s;
    if ((s = ensure(ctx, ctx->m_lat_of, g.N * sizeof(int))) != DDA_OK) return s;
    if ((s = ensure(ctx, ctx->m_comp_of, g.N)) != DDA_OK) return s;
    CU(cudaMemcpy(ctx->m_site_of.p, site_of.data(), M * sizeof(int), cudaMemcpyHostToDevice));
    CU(cudaMemcpy(ctx->m_lat_of.p, lat_of.data(), g.N * sizeof(int), cudaMemcpyHostToDevice));
    CU(cudaMemcpy(ctx->m_comp_of.p, comp_of.data(), g.N, cudaMemcpyHostToDevice));
    if ((s = ensure(ctx, ctx->m_rows, rows.size() * sizeof(int))) != DDA_OK) return s;
    CU(cudaMemcpy(ctx->m_rows.p, rows.data(), rows.size() * sizeof(int), cudaMemcpyHostToDevice));
    ctx->tg.site_of = (int*)ctx->m_site_of.p;
    ctx->tg.lat_of = (int*)ctx->m_lat_of.p;
    ctx->tg.comp_of = (uint8_t*)ctx->m_comp_of.p;
    ctx->tg.rows = (const int*)ctx->m_rows.p;
    ctx->tg.nrows = (int)rows.size();
    ctx->g = g;
    ctx->zsched.clear();
    ctx->max_code = maxc;
    ctx->has_target = true;
    if (ctx->site_mode) {  // per-site materials belong to the previous target
        ctx->site_mode = false;
        ctx->has_materials = false;
        ctx->m.clear();
    }
    if (ctx->graph.exec) {
        cudaGraphExecDestroy(ctx->graph.exec);
        ctx->graph.exec = nullptr;
    }
    return DDA_OK;
}

dda_status dda_set_materials(dda_ctx* ctx, int ncomp, const double* m_complex, double m_ambient) {
    if (!ctx) return DDA_ERR_ARG;
    if (ncomp <= 0 || ncomp > 255 || m_complex == nullptr) return ctx->fail(DDA_ERR_ARG, "bad ncomp or NULL indices");
    if (!(m_ambient > 0.0) || !std::isfinite(m_ambient)) return ctx->fail(DDA_ERR_ARG, "ambient index must be > 0");
    std::vector<cd> m(ncomp);
    for (int c = 0; c < ncomp; ++c) {
        m[c] = cd(m_complex[2 * c], m_complex[2 * c + 1]);
        if (!std::isfinite(m[c].real()) || !std::isfinite(m[c].imag()))
            return ctx->fail(DDA_ERR_NONFINITE, "refractive index of composition %d is not finite", c + 1);
        const cd mr = m[c] / m_ambient;
        if (std::abs(mr * mr - 1.0) == 0.0)
            return ctx->fail(DDA_ERR_ARG, "composition %d matches the ambient medium (zero polarizability)", c + 1);
    }
    leave_site_mode(ctx);
    ctx->m = m;
    ctx->m_amb = m_ambient;
    set_isotropy(ctx, false);
    ctx->has_materials = true;
    ctx->prepared = false;
    ctx->has32 = false;
    return DDA_OK;
}

dda_status dda_set_site_materials(dda_ctx* ctx, const double* m_site, double m_ambient) {
    if (!ctx) return DDA_ERR_ARG;
    if (!ctx->has_target) return ctx->fail(DDA_ERR_ARG, "dda_set_target first (one index per occupied site)");
    if (m_site == nullptr) return ctx->fail(DDA_ERR_ARG, "NULL indices");
    if (!(m_ambient > 0.0) || !std::isfinite(m_ambient)) return ctx->fail(DDA_ERR_ARG, "ambient index must be > 0");
    const int64_t N = ctx->g.N;
    std::vector<cd> m((size_t)N);
    for (int64_t j = 0; j < N; ++j) {
        m[j] = cd(m_site[2 * j], m_site[2 * j + 1]);
        if (!std::isfinite(m[j].real()) || !std::isfinite(m[j].imag()))
            return ctx->fail(DDA_ERR_NONFINITE, "refractive index of site %lld is not finite", (long long)j);
        const cd mr = m[j] / m_ambient;
        if (std::abs(mr * mr - 1.0) == 0.0)
            return ctx->fail(DDA_ERR_ARG, "site %lld matches the ambient medium (zero polarizability)", (long long)j);
    }
    set_isotropy(ctx, false);
    ctx->m = std::move(m);
    ctx->m_amb = m_ambient;
    ctx->site_mode = true;
    ctx->tg.comp_of = nullptr;
    ctx->zsched.clear();
    if (ctx->graph.exec) {
        cudaGraphExecDestroy(ctx->graph.exec);
        ctx->graph.exec = nullptr;
    }
    ctx->has_materials = true;
    ctx->prepared = false;
    ctx->has32 = false;
    return DDA_OK;
}

dda_status dda_set_anisotropic_materials(dda_ctx* ctx, int ncomp, const double* m_principal,
                                         const double* df_angles, double m_ambient) {
    if (!ctx) return DDA_ERR_ARG;
    if (ncomp <= 0 || ncomp > 255 || m_principal == nullptr || df_angles == nullptr)
        return ctx->fail(DDA_ERR_ARG, "bad ncomp or NULL indices/angles");
    if (!(m_ambient > 0.0) || !std::isfinite(m_ambient)) return ctx->fail(DDA_ERR_ARG, "ambient index must be > 0");
    std::vector<std::array<cd, 3>> m3(ncomp);
    std::vector<std::array<double, 3>> ang(ncomp);
    for (int c = 0; c < ncomp; ++c) {
        for (int j = 0; j < 3; ++j) {
            const cd mj(m_principal[6 * c + 2 * j], m_principal[6 * c + 2 * j + 1]);
            if (!std::isfinite(mj.real()) || !std::isfinite(mj.imag()))
                return ctx->fail(DDA_ERR_NONFINITE, "refractive index %d of composition %d is not finite", j + 1, c + 1);
            const cd mr = mj / m_ambient;
            if (std::abs(mr * mr - 1.0) == 0.0)
                return ctx->fail(DDA_ERR_ARG, "principal index %d of composition %d matches the ambient medium", j + 1,
                                 c + 1);
            m3[c][j] = mj;
            ang[c][j] = df_angles[3 * c + j];
            if (!std::isfinite(ang[c][j]))
                return ctx->fail(DDA_ERR_NONFINITE, "dielectric-frame angle of composition %d is not finite", c + 1);
        }
    }
    leave_site_mode(ctx);
    ctx->m.resize(ncomp);
    for (int c = 0; c < ncomp; ++c) ctx->m[c] = m3[c][0];
    ctx->m3 = m3;
    ctx->df_angles = ang;
    ctx->m_amb = m_ambient;
    set_isotropy(ctx, true);
    ctx->has_materials = true;
    ctx->prepared = false;
    ctx->has32 = false;
    return DDA_OK;
}

dda_status dda_prepare(dda_ctx* ctx, double lambda_vac, double aeff, dda_precision precision) {
    if (!ctx) return DDA_ERR_ARG;
    ProfScope prof_scope(ctx);
    if (!ctx->has_target || !ctx->has_materials) return ctx->fail(DDA_ERR_ARG, "set target and materials first");
    if (!ctx->site_mode && (int)ctx->m.size() < ctx->max_code)
        return ctx->fail(DDA_ERR_ARG, "grid uses composition %d but only %d indices given", ctx->max_code, (int)ctx->m.size());
    if (!(lambda_vac > 0.0) || !(aeff > 0.0) || !std::isfinite(lambda_vac) || !std::isfinite(aeff))
        return ctx->fail(DDA_ERR_ARG, "wavelength and aeff must be positive and finite");
    cudaSetDevice(ctx->device);
    const Geom& g = ctx->g;
    ctx->aeff_lat = std::cbrt(3.0 * (double)g.N / (4.0 * kPi));
    const double d = aeff / ctx->aeff_lat;
    ctx->kd = 2.0 * kPi * ctx->m_amb / lambda_vac * d;
    dda_status s;
    const int Ls[3] = {g.Lx, g.Ly, g.Lz};
    for (int a = 0; a < 3; ++a) {
        std::vector<double2> t64;
        std::vector<float2> t32;
        host_twiddles(Ls[a], t64, t32);
        if ((s = ensure(ctx, ctx->m_tw64[a], t64.size() * sizeof(double2))) != DDA_OK) return s;
        if ((s = ensure(ctx, ctx->m_tw32[a], t32.size() * sizeof(float2))) != DDA_OK) return s;
        CU(cudaMemcpy(ctx->m_tw64[a].p, t64.data(), t64.size() * sizeof(double2), cudaMemcpyHostToDevice));
        CU(cudaMemcpy(ctx->m_tw32[a].p, t32.data(), t32.size() * sizeof(float2), cudaMemcpyHostToDevice));
        std::vector<cdfl> tdf(t64.size());
        for (size_t i = 0; i < t64.size(); ++i) tdf[i] = cdfl{dfl(t64[i].x), dfl(t64[i].y)};
        if ((s = ensure(ctx, ctx->m_twdf[a], tdf.size() * sizeof(cdfl))) != DDA_OK) return s;
        CU(cudaMemcpy(ctx->m_twdf[a].p, tdf.data(), tdf.size() * sizeof(cdfl), cudaMemcpyHostToDevice));
    }
    const int64_t oct = 6 * g.oct_per_comp();
    if ((s = ensure(ctx, ctx->m_gh64, oct * sizeof(double2))) != DDA_OK) return s;
    DevMem scratch;
    const size_t sb = (size_t)6 * g.Lx * g.Ly * g.Lz * sizeof(double2);
    cudaError_t e = cudaMalloc(&scratch.p, sb);
    if (e != cudaSuccess) return ctx->cuda_fail(e, "cudaMalloc(Green tensor scratch)");
    e = launch_green_fft(g, ctx->kd, (double2*)scratch.p, (double2*)ctx->m_gh64.p, tw_of<double>(ctx), ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    cudaFree(scratch.p);
    if (e != cudaSuccess) return ctx->cuda_fail(e, "Green tensor FFT");
    ctx->has32 = false;
    if (precision != DDA_FP64) {
        if ((s = ensure(ctx, ctx->m_gh32, oct * sizeof(float2))) != DDA_OK) return s;
        CU(launch_convert_c128_to_c64((const double2*)ctx->m_gh64.p, (float2*)ctx->m_gh32.p, oct, ctx->stream));
        if ((s = ensure(ctx, ctx->m_ghdf, oct * sizeof(cdfl))) != DDA_OK) return s;
        CU(launch_convert_c128_to_df((const double2*)ctx->m_gh64.p, (cdfl*)ctx->m_ghdf.p, oct, ctx->stream));
        CU(sync_collect(ctx));
        ctx->has32 = true;
    }
    ctx->prepared = true;
    if (ctx->graph.exec) {
        cudaGraphExecDestroy(ctx->graph.exec);
        ctx->graph.exec = nullptr;
    }
    return DDA_OK;
}

dda_status dda_get_info(const dda_ctx* ctx, dda_info* info) {
    if (!ctx || !info) return DDA_ERR_ARG;
    std::memset(info, 0, sizeof *info);
    info->nx = ctx->g.ox;
    info->ny = ctx->g.oy;
    info->nz = ctx->g.oz;
    info->Lx = ctx->g.Lx;
    info->Ly = ctx->g.Ly;
    info->Lz = ctx->g.Lz;
    info->ndipoles = ctx->g.N;
    info->ncomp = (int)ctx->m.size();
    info->aeff_lattice = ctx->has_target ? std::cbrt(3.0 * (double)ctx->g.N / (4.0 * kPi)) : 0.0;
    info->kd = ctx->prepared ? ctx->kd : 0.0;
    info->x = ctx->prepared ? ctx->kd * ctx->aeff_lat : 0.0;
    return DDA_OK;
}

dda_status dda_solve(dda_ctx* ctx, dda_precision precision, int R, const double* khat, const double* e,
                     const dda_opts* opts, double* P_out, dda_result* res) {
    if (!ctx) return DDA_ERR_ARG;
    ProfScope prof_scope(ctx);
    cudaSetDevice(ctx->device);
    dda_status st = forward_solve(ctx, precision, R, khat, e, opts, res);
    if (st != DDA_OK && st != DDA_ERR_NOT_CONVERGED && st != DDA_ERR_BREAKDOWN) return st;
    if (P_out) {
        const size_t bytes = (size_t)R * 3 * ctx->g.N * sizeof(double2);
        CU(cudaMemcpyAsync(P_out, ctx->pool[S_X64].p, bytes, cudaMemcpyDeviceToHost, ctx->stream));
        CU(sync_collect(ctx));
    }
    return st;
}

dda_status dda_solve_device(dda_ctx* ctx, dda_precision precision, int R, const double* khat, const double* e,
                            const dda_opts* opts, void* P_dev, dda_result* res) {
    if (!ctx) return DDA_ERR_ARG;
    ProfScope prof_scope(ctx);
    cudaSetDevice(ctx->device);
    dda_status st = forward_solve(ctx, precision, R, khat, e, opts, res);
    if (st != DDA_OK && st != DDA_ERR_NOT_CONVERGED && st != DDA_ERR_BREAKDOWN) return st;
    if (P_dev) {
        const size_t bytes = (size_t)R * 3 * ctx->g.N * sizeof(double2);
        CU(cudaMemcpyAsync(P_dev, ctx->pool[S_X64].p, bytes, cudaMemcpyDeviceToDevice, ctx->stream));
        CU(sync_collect(ctx));
    }
    return st;
}

static dda_status matvec_common(dda_ctx* ctx, dda_precision precision, int R, const double* khat, const double* e,
                                const void* x_dev, void* y_dev) {
    dda_status rs;
    if (precision == DDA_FP32_REFINED)
        return ctx->fail(DDA_ERR_ARG, "matvec precision must be DDA_FP64, DDA_FP32 or DDA_DF64");
    if (precision == DDA_DF64) {
        if ((rs = check_ready(ctx, DDA_FP32_REFINED)) != DDA_OK) return rs;
        std::vector<double> k;
        std::vector<cd> ev;
        if ((rs = check_rhs(ctx, R, khat, e, k, ev)) != DDA_OK) return rs;
        if ((rs = upload_tables(ctx, R, k, ev)) != DDA_OK) return rs;
        return matvec64(ctx, R, (const double2*)x_dev, (double2*)y_dev, nullptr, true);
    }
    if ((rs = check_ready(ctx, precision)) != DDA_OK) return rs;
    std::vector<double> k;
    std::vector<cd> ev;
    if ((rs = check_rhs(ctx, R, khat, e, k, ev)) != DDA_OK) return rs;
    if ((rs = upload_tables(ctx, R, k, ev)) != DDA_OK) return rs;
    if (precision == DDA_FP64) {
        if ((rs = ensure_pad<double>(ctx, R)) != DDA_OK) return rs;
        return run_matvec<double>(ctx, R, (const double2*)x_dev, (double2*)y_dev, nullptr);
    }
    if ((rs = ensure_pad<float>(ctx, R)) != DDA_OK) return rs;
    return run_matvec<float>(ctx, R, (const float2*)x_dev, (float2*)y_dev, nullptr);
}

dda_status dda_matvec_device(dda_ctx* ctx, dda_precision precision, int R, const double* khat, const double* e,
                             const void* x_dev, void* y_dev) {
    if (!ctx) return DDA_ERR_ARG;
    ProfScope prof_scope(ctx);
    if (!x_dev || !y_dev) return ctx->fail(DDA_ERR_ARG, "NULL vector");
    cudaSetDevice(ctx->device);
    dda_status rs = matvec_common(ctx, precision, R, khat, e, x_dev, y_dev);
    if (rs != DDA_OK) return rs;
    CU(sync_collect(ctx));
    return DDA_OK;
}

dda_status dda_matvec_device_noalloc(dda_ctx* ctx, dda_precision precision, int R, const double* khat,
                                     const double* e, const void* x_dev, void* y_dev) {
    if (!ctx) return DDA_ERR_ARG;
    if (!x_dev || !y_dev) return ctx->fail(DDA_ERR_ARG, "NULL vector");
    if (precision != DDA_FP64 && precision != DDA_FP32)
        return ctx->fail(DDA_ERR_ARG,
                         "dda_matvec_device_noalloc takes DDA_FP64 or DDA_FP32 (got %d); the double-float "
                         "DDA_DF64 matvec is available through dda_matvec_device only", (int)precision);
    // (it copies its 1/alpha table from host memory and synchronizes the
    // stream: neither may happen inside a stream capture)
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    CU(cudaStreamIsCapturing(ctx->stream, &cs));
    if (cs != cudaStreamCaptureStatusNone)
        return ctx->fail(DDA_ERR_ARG, "dda_matvec_device_noalloc cannot run inside a stream capture (it synchronizes "
                                      "the context stream)");
    dda_status rs;
    if ((rs = check_ready(ctx, precision)) != DDA_OK) return rs;
    CU(cudaSetDevice(ctx->device));
    std::vector<double> k;
    std::vector<cd> ev;
    if ((rs = check_rhs(ctx, R, khat, e, k, ev)) != DDA_OK) return rs;
    if (precision == DDA_FP64) return matvec_noalloc<double>(ctx, R, k, ev, x_dev, y_dev);
    return matvec_noalloc<float>(ctx, R, k, ev, x_dev, y_dev);
}

dda_status dda_matvec(dda_ctx* ctx, dda_precision precision, int R, const double* khat, const double* e,
                      const double* x, double* y) {
    if (!ctx) return DDA_ERR_ARG;
    ProfScope prof_scope(ctx);
    if (!x || !y) return ctx->fail(DDA_ERR_ARG, "NULL vector");
    if (!ctx->prepared) return ctx->fail(DDA_ERR_ARG, "dda_prepare has not been called");
    if (R <= 0) return ctx->fail(DDA_ERR_ARG, "R must be > 0");
    cudaSetDevice(ctx->device);
    const int64_t n = (int64_t)R * 3 * ctx->g.N;
    dda_status rs;
    for (int64_t i = 0; i < 2 * n; ++i)
        if (!std::isfinite(x[i])) return ctx->fail(DDA_ERR_NONFINITE, "non-finite input vector");
    if ((rs = ensure(ctx, ctx->pool[S_X64], n * sizeof(double2))) != DDA_OK) return rs;
    if ((rs = ensure(ctx, ctx->pool[S_Y64], n * sizeof(double2))) != DDA_OK) return rs;
    CU(cudaMemcpyAsync(ctx->pool[S_X64].p, x, n * sizeof(double2), cudaMemcpyHostToDevice, ctx->stream));
    if (precision == DDA_FP32) {
        if ((rs = ensure(ctx, ctx->pool[S_MV_X32], n * sizeof(float2))) != DDA_OK) return rs;
        if ((rs = ensure(ctx, ctx->pool[S_MV_Y32], n * sizeof(float2))) != DDA_OK) return rs;
        CU(launch_c128_to_c64v(n, slot<double2>(ctx, S_X64), slot<float2>(ctx, S_MV_X32), ctx->stream));
        if ((rs = matvec_common(ctx, precision, R, khat, e, ctx->pool[S_MV_X32].p, ctx->pool[S_MV_Y32].p)) != DDA_OK)
            return rs;
        CU(launch_c64_to_c128(n, slot<float2>(ctx, S_MV_Y32), slot<double2>(ctx, S_Y64), ctx->stream));
    } else {
        if ((rs = matvec_common(ctx, precision, R, khat, e, ctx->pool[S_X64].p, ctx->pool[S_Y64].p)) != DDA_OK)
            return rs;
    }
    CU(cudaMemcpyAsync(y, ctx->pool[S_Y64].p, n * sizeof(double2), cudaMemcpyDeviceToHost, ctx->stream));
    CU(sync_collect(ctx));
    return DDA_OK;
}

dda_status dda_incident_field(dda_ctx* ctx, int R, const double* khat, const double* e, double* E_out) {
    if (!ctx) return DDA_ERR_ARG;
    ProfScope prof_scope(ctx);
    if (!E_out) return ctx->fail(DDA_ERR_ARG, "NULL output");
    dda_status rs;
    if ((rs = check_ready(ctx, DDA_FP64)) != DDA_OK) return rs;
    cudaSetDevice(ctx->device);
    std::vector<double> k;
    std::vector<cd> ev;
    if ((rs = check_rhs(ctx, R, khat, e, k, ev)) != DDA_OK) return rs;
    if ((rs = upload_tables(ctx, R, k, ev)) != DDA_OK) return rs;
    const size_t bytes = (size_t)R * 3 * ctx->g.N * sizeof(double2);
    if ((rs = ensure(ctx, ctx->pool[S_E64], bytes)) != DDA_OK) return rs;
    CU(launch_einc(R, ctx->g.N, ctx->tg.lat_of, ctx->g, ctx->kd, slot<double>(ctx, S_KHAT),
                   slot<double2>(ctx, S_EPOL), slot<double2>(ctx, S_E64), ctx->stream));
    CU(cudaMemcpyAsync(E_out, ctx->pool[S_E64].p, bytes, cudaMemcpyDeviceToHost, ctx->stream));
    CU(sync_collect(ctx));
    return DDA_OK;
}

}  // extern "C"

// ---- near field ------------------------------------------------------------
namespace {

// Extended volume of the near-field calculation: nint(r n) lattice points
// added on each side of an axis of n points (the guide's NRFLD extension
// fractions r1..r6 of the computational volume).
dda_status nf_box(dda_ctx* ctx, const double* ext, int dims[3], int off[3]) {
    if (!ext) return ctx->fail(DDA_ERR_ARG, "NULL extension fractions");
    const int n[3] = {ctx->g.ox, ctx->g.oy, ctx->g.oz};
    for (int a = 0; a < 3; ++a) {
        const double lo = ext[2 * a], hi = ext[2 * a + 1];
        if (!std::isfinite(lo) || !std::isfinite(hi) || lo < 0.0 || hi < 0.0 || lo > 64.0 || hi > 64.0)
            return ctx->fail(DDA_ERR_ARG, "extension fractions must be finite, in [0, 64]");
        const int add_lo = (int)std::floor(lo * n[a] + 0.5), add_hi = (int)std::floor(hi * n[a] + 0.5);
        off[a] = add_lo;
        dims[a] = n[a] + add_lo + add_hi;
        if (!pick_fft_length(dims[a]))
            return ctx->fail(DDA_ERR_SIZE, "extended volume has %d points along axis %d: above the largest padded length",
                             dims[a], a);
    }
    return DDA_OK;
}

struct NearWork {
    std::vector<DevMem> mem;
    ~NearWork() {
        for (auto& m : mem) free_mem(m);
    }
    void* get(size_t bytes, cudaError_t& e) {
        mem.emplace_back();
        e = cudaMalloc(&mem.back().p, bytes < 256 ? 256 : bytes);
        return mem.back().p;
    }
};

template <typename T>
dda_status nearfield_run(dda_ctx* ctx, int R, const double* P_host, const int dims[3], const int off[3],
                         const std::vector<double>& khat, const std::vector<cd>& e, double* Einc_out, double* Esca_out) {
    using C = cx<T>;
    cudaStream_t st = ctx->stream;
    // geometry of the extended box: every box point is an output site
    Geom g;
    g.ox = dims[0];
    g.oy = dims[1];
    g.oz = dims[2];
    g.Lx = pick_fft_length(dims[0]);
    g.Ly = pick_fft_length(dims[1]);
    g.Lz = pick_fft_length(dims[2]);
    g.nx = g.Lx / 2;
    g.ny = g.Ly / 2;
    g.nz = g.Lz / 2;
    const int64_t Ne = (int64_t)dims[0] * dims[1] * dims[2], M = g.M(), N = ctx->g.N;
    if (M > (int64_t)INT32_MAX) return ctx->fail(DDA_ERR_SIZE, "extended volume too large");
    g.N = Ne;
    std::vector<int> site_of(M, -1), lat_of(Ne);
    for (int iz = 0; iz < dims[2]; ++iz)
        for (int iy = 0; iy < dims[1]; ++iy)
            for (int ix = 0; ix < dims[0]; ++ix) {
                const int64_t b = ((int64_t)iz * dims[1] + iy) * dims[0] + ix;
                const int64_t li = ((int64_t)iz * g.ny + iy) * g.nx + ix;
                site_of[li] = (int)b;
                lat_of[b] = (int)li;
            }
    // target site -> box point (target lattice indices from the context's map)
    std::vector<int> tlat(N), box_of(N);
    CU(cudaMemcpy(tlat.data(), ctx->tg.lat_of, N * sizeof(int), cudaMemcpyDeviceToHost));
    for (int64_t j = 0; j < N; ++j) {
        const int l = tlat[j];
        const int ix = l % ctx->g.nx, iy = (l / ctx->g.nx) % ctx->g.ny, iz = l / (ctx->g.nx * ctx->g.ny);
        box_of[j] = (int)(((int64_t)(iz + off[2]) * dims[1] + (iy + off[1])) * dims[0] + (ix + off[0]));
    }
    NearWork w;
    cudaError_t ce = cudaSuccess;
    auto alloc = [&](size_t bytes) { return ce == cudaSuccess ? w.get(bytes, ce) : nullptr; };
    int* d_site = (int*)alloc(M * sizeof(int));
    int* d_lat = (int*)alloc(Ne * sizeof(int));
    int* d_box = (int*)alloc(N * sizeof(int));
    uint8_t* d_comp = (uint8_t*)alloc(Ne);
    const int64_t oct = 6 * g.oct_per_comp();
    double2* gh64 = (double2*)alloc(oct * sizeof(double2));
    double2* tw64[3];
    void* twT[3];
    for (int a = 0; a < 3; ++a) {
        const int L = a == 0 ? g.Lx : (a == 1 ? g.Ly : g.Lz);
        tw64[a] = (double2*)alloc(L * sizeof(double2));
        twT[a] = sizeof(T) == 8 ? (void*)tw64[a] : alloc(L * sizeof(C));
    }
    C* ghT = sizeof(T) == 8 ? (C*)gh64 : (C*)alloc(oct * sizeof(C));
    const int rc = std::max(1, std::min(R, 8));  // RHS per pass over the box
    C* Pbox = (C*)alloc((size_t)rc * 3 * Ne * sizeof(C));
    C* Ybox = (C*)alloc((size_t)rc * 3 * Ne * sizeof(C));
    C* u2 = (C*)alloc((size_t)rc * 3 * g.u2_per_comp() * sizeof(C));
    C* beta0 = (C*)alloc((size_t)rc * 2 * sizeof(C));
    double2* d_P = (double2*)alloc((size_t)rc * 3 * N * sizeof(double2));
    double2* d_E = (double2*)alloc((size_t)rc * 3 * Ne * sizeof(double2));
    double* d_k = (double*)alloc((size_t)R * 3 * sizeof(double));
    double2* d_e = (double2*)alloc((size_t)R * 3 * sizeof(double2));
    if (ce != cudaSuccess) return ctx->cuda_fail(ce, "near-field workspace");
    CU(cudaMemcpy(d_site, site_of.data(), M * sizeof(int), cudaMemcpyHostToDevice));
    CU(cudaMemcpy(d_lat, lat_of.data(), Ne * sizeof(int), cudaMemcpyHostToDevice));
    CU(cudaMemcpy(d_box, box_of.data(), N * sizeof(int), cudaMemcpyHostToDevice));
    CU(cudaMemset(d_comp, 1, Ne));
    CU(cudaMemset(beta0, 0, (size_t)rc * 2 * sizeof(C)));
    std::vector<double2> e2(3 * (size_t)R);
    for (size_t i = 0; i < e2.size(); ++i) e2[i] = make_double2(e[i].real(), e[i].imag());
    CU(cudaMemcpy(d_k, khat.data(), khat.size() * sizeof(double), cudaMemcpyHostToDevice));
    CU(cudaMemcpy(d_e, e2.data(), e2.size() * sizeof(double2), cudaMemcpyHostToDevice));
    for (int a = 0; a < 3; ++a) {
        const int L = a == 0 ? g.Lx : (a == 1 ? g.Ly : g.Lz);
        std::vector<double2> t64;
        std::vector<float2> t32;
        host_twiddles(L, t64, t32);
        CU(cudaMemcpy(tw64[a], t64.data(), L * sizeof(double2), cudaMemcpyHostToDevice));
        if (sizeof(T) != 8) CU(cudaMemcpy(twT[a], t32.data(), L * sizeof(float2), cudaMemcpyHostToDevice));
    }
    {
        DevMem scratch;
        CU(cudaMalloc(&scratch.p, (size_t)6 * g.Lx * g.Ly * g.Lz * sizeof(double2)));
        Twiddles<double> t{tw64[0], tw64[1], tw64[2]};
        cudaError_t e1 = launch_green_fft(g, ctx->kd, (double2*)scratch.p, gh64, t, st);
        if (e1 == cudaSuccess) e1 = cudaStreamSynchronize(st);
        cudaFree(scratch.p);
        if (e1 != cudaSuccess) return ctx->cuda_fail(e1, "near-field Green tensor FFT");
    }
    if (sizeof(T) != 8) CU(launch_convert_c128_to_c64(gh64, (float2*)ghT, oct, st));
    DevTarget tg;
    tg.site_of = d_site;
    tg.lat_of = d_lat;
    tg.comp_of = d_comp;
    Twiddles<T> tw{(const C*)twT[0], (const C*)twT[1], (const C*)twT[2]};
    PadWork<T> pw{nullptr, u2};
    pw.slices = ctx->force_slices != 0;
    // phase origin: the target's own centre, in box index space
    const double cx = off[0] + 0.5 * (ctx->g.ox - 1), cy = off[1] + 0.5 * (ctx->g.oy - 1),
                 cz = off[2] + 0.5 * (ctx->g.oz - 1);
    for (int r0 = 0; r0 < R; r0 += rc) {
        const int rn = std::min(rc, R - r0);
        const size_t nb = (size_t)rn * 3 * Ne;
        CU(cudaMemcpyAsync(d_P, P_host + (size_t)r0 * 6 * N, (size_t)rn * 3 * N * sizeof(double2),
                           cudaMemcpyHostToDevice, st));
        CU(cudaMemsetAsync(Pbox, 0, nb * sizeof(C), st));
        CU(launch_scatter_sites<C>(rn, N, Ne, d_box, d_P, Pbox, st));
        // y = sum_{l != j} A_jl P_l: the matvec on the box with 1/alpha = 0
        CU(launch_matvec<T>(g, rn, Pbox, Ybox, pw, tg, beta0, 2, ghT, tw, nullptr, st));
        CU(launch_negate_c128<C>((int64_t)nb, Ybox, d_E, st));
        CU(cudaMemcpyAsync(Esca_out + (size_t)r0 * 6 * Ne, d_E, nb * sizeof(double2), cudaMemcpyDeviceToHost, st));
        if (Einc_out) {
            CU(launch_einc_at(rn, Ne, d_lat, g.nx, g.ny, cx, cy, cz, ctx->kd, d_k + 3 * r0, d_e + 3 * r0, d_E, st));
            CU(cudaMemcpyAsync(Einc_out + (size_t)r0 * 6 * Ne, d_E, nb * sizeof(double2), cudaMemcpyDeviceToHost, st));
        }
        CU(sync_collect(ctx));
    }
    return DDA_OK;
}

}  // namespace

extern "C" {

dda_status dda_nearfield_dims(dda_ctx* ctx, const double* ext, int* dims, int* offset) {
    if (!ctx) return DDA_ERR_ARG;
    if (!dims || !offset) return ctx->fail(DDA_ERR_ARG, "NULL output");
    if (!ctx->has_target) return ctx->fail(DDA_ERR_ARG, "set a target first");
    int d[3], o[3];
    dda_status s = nf_box(ctx, ext, d, o);
    if (s != DDA_OK) return s;
    for (int a = 0; a < 3; ++a) {
        dims[a] = d[a];
        offset[a] = o[a];
    }
    return DDA_OK;
}

dda_status dda_nearfield(dda_ctx* ctx, dda_precision precision, int R, const double* khat, const double* e,
                         const double* P, const double* ext, double* E_inc_out, double* E_sca_out) {
    if (!ctx) return DDA_ERR_ARG;
    ProfScope prof_scope(ctx);
    if (!P || !E_sca_out) return ctx->fail(DDA_ERR_ARG, "NULL P or E_sca");
    dda_status rs;
    if (!ctx->prepared) return ctx->fail(DDA_ERR_ARG, "dda_prepare has not been called for the current target");
    if (precision != DDA_FP64 && precision != DDA_FP32 && precision != DDA_FP32_REFINED)
        return ctx->fail(DDA_ERR_ARG, "near field: precision must be DDA_FP64 or a complex64 mode");
    cudaSetDevice(ctx->device);
    std::vector<double> k;
    std::vector<cd> ev;
    if ((rs = check_rhs(ctx, R, khat, e, k, ev)) != DDA_OK) return rs;
    int dims[3], off[3];
    if ((rs = nf_box(ctx, ext, dims, off)) != DDA_OK) return rs;
    if (precision == DDA_FP64) return nearfield_run<double>(ctx, R, P, dims, off, k, ev, E_inc_out, E_sca_out);
    return nearfield_run<float>(ctx, R, P, dims, off, k, ev, E_inc_out, E_sca_out);
}

}  // extern "C"

// ---- far field ---------------------------------------------------------------
namespace {

// The guide's scattering directions for angular averages ("Selection of
// Scattering Angles"): theta equally spaced in s(theta) = theta + theta /
// (theta + theta0), theta0 = 2 pi / (1 + x), N_theta the nearest integer to
// its expression in x and eta; nint(4 pi sin(theta_j) / (theta_{j+1} -
// theta_{j-1})) (at least 3) azimuths at each interior theta, one at 0 and
// pi; solid-angle weights from its quadrature ("Angular Averaging").
void scat_dirs(double x, double eta, std::vector<double>& th_out, std::vector<double>& ph_out,
               std::vector<double>& om_out) {
    const double th0 = 2.0 * kPi / (1.0 + x);
    const double ntr = 1.0 + (2.0 * (3.0 + x) / eta) * (1.0 + 1.0 / (kPi + th0)) / (1.0 + th0 / ((kPi + th0) * (kPi + th0)));
    const int nth = std::max(2, (int)std::floor(ntr + 0.5));
    std::vector<double> th(nth);
    for (int j = 0; j < nth; ++j) {
        const double sj = j * kPi / (nth - 1) * (1.0 + 1.0 / (kPi + th0));
        th[j] = ((sj - 1.0 - th0) + std::sqrt((1.0 + th0 - sj) * (1.0 + th0 - sj) + 4.0 * th0 * sj)) / 2.0;
    }
    th[0] = 0.0;
    th[nth - 1] = kPi;
    th_out.clear();
    ph_out.clear();
    om_out.clear();
    for (int j = 0; j < nth; ++j) {
        int nph = 1;
        double om;
        if (j == 0) {
            om = 2.0 * kPi * (1.0 - (std::cos(th[0]) + std::cos(th[1])) / 2.0);
        } else if (j == nth - 1) {
            om = 2.0 * kPi * ((std::cos(th[j - 1]) + std::cos(th[j])) / 2.0 + 1.0);
        } else {
            nph = std::max(3, (int)std::floor(4.0 * kPi * std::sin(th[j]) / (th[j + 1] - th[j - 1]) + 0.5));
            om = kPi * (std::cos(th[j - 1]) - std::cos(th[j + 1]));
        }
        for (int k = 0; k < nph; ++k) {
            th_out.push_back(th[j]);
            ph_out.push_back(2.0 * kPi * k / nph);
            om_out.push_back(om / nph);
        }
    }
}

// Lab Frame of a RHS: x_L = khat, y_L = normalize(z x khat) (x if khat is
// along z), z_L = x_L x y_L.
void lab_frame(const double* k, double xl[3], double yl[3], double zl[3]) {
    for (int a = 0; a < 3; ++a) xl[a] = k[a];
    double y[3] = {-k[1], k[0], 0.0};  // z x k
    double n = std::sqrt(y[0] * y[0] + y[1] * y[1]);
    if (n < 1e-8) {
        y[0] = 1.0;
        y[1] = 0.0;
        n = 1.0;
    }
    for (int a = 0; a < 3; ++a) yl[a] = y[a] / n;
    zl[0] = xl[1] * yl[2] - xl[2] * yl[1];
    zl[1] = xl[2] * yl[0] - xl[0] * yl[2];
    zl[2] = xl[0] * yl[1] - xl[1] * yl[0];
}

template <typename T>
dda_status farfield_run(dda_ctx* ctx, int R, const std::vector<double>& khat, const double* P_host, int ndir,
                        const double* theta, const double* phi, std::vector<double2>& F) {
    using C = cx<T>;
    const Geom& g = ctx->g;
    const int64_t N = g.N;
    if (g.ox > 1024 || g.oy > 1024 || g.oz > 1024) return ctx->fail(DDA_ERR_SIZE, "far field: lattice above 1024");
    const int Lm = std::max(g.ox, std::max(g.oy, g.oz)), tab_len = 3 * Lm;
    const double kd = ctx->kd, c[3] = {0.5 * (g.ox - 1), 0.5 * (g.oy - 1), 0.5 * (g.oz - 1)};
    std::vector<double> dirs((size_t)R * ndir * 3);
    for (int r = 0; r < R; ++r) {
        double xl[3], yl[3], zl[3];
        lab_frame(&khat[3 * r], xl, yl, zl);
        for (int d = 0; d < ndir; ++d) {
            const double ct = std::cos(theta[d]), st = std::sin(theta[d]), cp = std::cos(phi[d]), sp = std::sin(phi[d]);
            double* n = &dirs[((size_t)r * ndir + d) * 3];
            for (int a = 0; a < 3; ++a) n[a] = ct * xl[a] + st * cp * yl[a] + st * sp * zl[a];
        }
    }
    const size_t ntab = (size_t)R * ndir * tab_len;
    std::vector<int> lat(N);
    std::vector<unsigned> xyz(N);
    CU(cudaMemcpy(lat.data(), ctx->tg.lat_of, N * sizeof(int), cudaMemcpyDeviceToHost));
    for (int64_t j = 0; j < N; ++j) {
        const int l = lat[j];
        const unsigned ix = l % g.nx, iy = (l / g.nx) % g.ny, iz = l / (g.nx * g.ny);
        xyz[j] = ix | (iy << 10) | (iz << 20);
    }
    NearWork w;
    cudaError_t ce = cudaSuccess;
    auto alloc = [&](size_t bytes) { return ce == cudaSuccess ? w.get(bytes, ce) : nullptr; };
    unsigned* d_xyz = (unsigned*)alloc(N * sizeof(unsigned));
    double2* d_P64 = (double2*)alloc((size_t)R * 3 * N * sizeof(double2));
    C* d_P = sizeof(T) == 8 ? (C*)d_P64 : (C*)alloc((size_t)R * 3 * N * sizeof(C));
    C* d_tabs = (C*)alloc(ntab * sizeof(C));
    double* d_dirs = (double*)alloc(dirs.size() * sizeof(double));
    double2* d_F = (double2*)alloc((size_t)R * ndir * 3 * sizeof(double2));
    if (ce != cudaSuccess) return ctx->cuda_fail(ce, "far-field workspace");
    cudaStream_t st = ctx->stream;
    CU(cudaMemcpyAsync(d_xyz, xyz.data(), N * sizeof(unsigned), cudaMemcpyHostToDevice, st));
    CU(cudaMemcpyAsync(d_P64, P_host, (size_t)R * 3 * N * sizeof(double2), cudaMemcpyHostToDevice, st));
    if (sizeof(T) != 8) CU(launch_c128_to_c64v((int64_t)R * 3 * N, d_P64, (float2*)d_P, st));
    CU(cudaMemcpyAsync(d_dirs, dirs.data(), dirs.size() * sizeof(double), cudaMemcpyHostToDevice, st));
    CU(launch_phase_tables<C>((int64_t)R * ndir, Lm, c, kd, d_dirs, d_tabs, st));
    CU(launch_farfield<C>(R, N, d_xyz, d_P, ndir, tab_len, d_tabs, d_dirs, kd, d_F, st));
    F.resize((size_t)R * ndir * 3);
    CU(cudaMemcpyAsync(F.data(), d_F, F.size() * sizeof(double2), cudaMemcpyDeviceToHost, st));
    CU(sync_collect(ctx));
    return DDA_OK;
}

dda_status farfield_common(dda_ctx* ctx, dda_precision prec, int R, const double* khat, const double* P,
                           std::vector<double>& k) {
    if (!ctx->prepared) return ctx->fail(DDA_ERR_ARG, "dda_prepare has not been called for the current target");
    if (prec != DDA_FP64 && prec != DDA_FP32 && prec != DDA_FP32_REFINED)
        return ctx->fail(DDA_ERR_ARG, "far field: precision must be DDA_FP64 or a complex64 mode");
    if (R <= 0 || !khat || !P) return ctx->fail(DDA_ERR_ARG, "R > 0 with khat and P required");
    k.assign(3 * (size_t)R, 0.0);
    for (int r = 0; r < R; ++r) {
        double n = 0.0;
        for (int a = 0; a < 3; ++a) n += khat[3 * r + a] * khat[3 * r + a];
        if (!std::isfinite(n) || std::fabs(std::sqrt(n) - 1.0) > 1e-6)
            return ctx->fail(DDA_ERR_ARG, "khat of RHS %d is not a unit vector", r);
        for (int a = 0; a < 3; ++a) k[3 * r + a] = khat[3 * r + a] / std::sqrt(n);
    }
    cudaSetDevice(ctx->device);
    return DDA_OK;
}

}  // namespace

extern "C" {

dda_status dda_scattering_directions(double x, double eta, int capacity, double* theta, double* phi, double* omega,
                                     int* count) {
    if (!count || !(x > 0.0) || !(eta > 0.0) || !std::isfinite(x) || !std::isfinite(eta) || capacity < 0)
        return DDA_ERR_ARG;
    if (x / eta > 1e5) return DDA_ERR_SIZE;
    std::vector<double> th, ph, om;
    scat_dirs(x, eta, th, ph, om);
    *count = (int)th.size();
    if (capacity >= (int)th.size()) {
        if (!theta || !phi || !omega) return DDA_ERR_ARG;
        std::copy(th.begin(), th.end(), theta);
        std::copy(ph.begin(), ph.end(), phi);
        std::copy(om.begin(), om.end(), omega);
    }
    return DDA_OK;
}

dda_status dda_farfield(dda_ctx* ctx, dda_precision precision, int R, const double* khat, const double* P, int ndir,
                        const double* theta, const double* phi, double* F_out) {
    if (!ctx) return DDA_ERR_ARG;
    ProfScope prof_scope(ctx);
    if (ndir <= 0 || !theta || !phi || !F_out) return ctx->fail(DDA_ERR_ARG, "ndir > 0 with theta, phi, F_out");
    std::vector<double> k;
    dda_status rs = farfield_common(ctx, precision, R, khat, P, k);
    if (rs != DDA_OK) return rs;
    std::vector<double2> F;
    rs = precision == DDA_FP64 ? farfield_run<double>(ctx, R, k, P, ndir, theta, phi, F)
                               : farfield_run<float>(ctx, R, k, P, ndir, theta, phi, F);
    if (rs != DDA_OK) return rs;
    std::memcpy(F_out, F.data(), F.size() * sizeof(double2));
    return DDA_OK;
}

dda_status dda_mueller(dda_ctx* ctx, dda_precision precision, const double* khat, const double* e01, const double* e02,
                       const double* P, int ndir, const double* theta, const double* phi, double* S_out,
                       double* amp_out) {
    if (!ctx) return DDA_ERR_ARG;
    ProfScope prof_scope(ctx);
    if (ndir <= 0 || !theta || !phi || !S_out || !e01 || !e02)
        return ctx->fail(DDA_ERR_ARG, "ndir > 0 with e01, e02, theta, phi and S_out required");
    std::vector<double> k;
    const double kk[6] = {khat ? khat[0] : 0.0, khat ? khat[1] : 0.0, khat ? khat[2] : 0.0,
                          khat ? khat[0] : 0.0, khat ? khat[1] : 0.0, khat ? khat[2] : 0.0};
    dda_status rs = farfield_common(ctx, precision, 2, khat ? kk : nullptr, P, k);
    if (rs != DDA_OK) return rs;
    std::vector<double2> F;  // [2][ndir][3]: far fields of the two incident states
    rs = precision == DDA_FP64 ? farfield_run<double>(ctx, 2, k, P, ndir, theta, phi, F)
                               : farfield_run<float>(ctx, 2, k, P, ndir, theta, phi, F);
    if (rs != DDA_OK) return rs;
    double xl[3], yl[3], zl[3];
    lab_frame(k.data(), xl, yl, zl);
    // conj(e0l) . y_L and . z_L
    cd a = 0.0, b = 0.0, c = 0.0, d = 0.0;
    for (int q = 0; q < 3; ++q) {
        const cd u = std::conj(cd(e01[2 * q], e01[2 * q + 1])), v = std::conj(cd(e02[2 * q], e02[2 * q + 1]));
        a += u * yl[q];
        b += u * zl[q];
        c += v * yl[q];
        d += v * zl[q];
    }
    const cd I(0.0, 1.0);
    for (int dd = 0; dd < ndir; ++dd) {
        const double ct = std::cos(theta[dd]), st = std::sin(theta[dd]), cp = std::cos(phi[dd]), sp = std::sin(phi[dd]);
        double th_hat[3], ph_hat[3];
        for (int q = 0; q < 3; ++q) {
            th_hat[q] = -st * xl[q] + ct * cp * yl[q] + ct * sp * zl[q];
            ph_hat[q] = -sp * yl[q] + cp * zl[q];
        }
        // f_ml = k F_l . e_m, e_1 = theta_hat, e_2 = phi_hat
        cd f[2][2];
        for (int l = 0; l < 2; ++l) {
            const double2* Fl = &F[((size_t)l * ndir + dd) * 3];
            cd ft = 0.0, fp = 0.0;
            for (int q = 0; q < 3; ++q) {
                const cd v(Fl[q].x, Fl[q].y);
                ft += v * th_hat[q];
                fp += v * ph_hat[q];
            }
            f[0][l] = ctx->kd * ft;
            f[1][l] = ctx->kd * fp;
        }
        const cd S1 = -I * (f[1][0] * (b * cp - a * sp) + f[1][1] * (d * cp - c * sp));
        const cd S2 = -I * (f[0][0] * (a * cp + b * sp) + f[0][1] * (c * cp + d * sp));
        const cd S3 = I * (f[0][0] * (b * cp - a * sp) + f[0][1] * (d * cp - c * sp));
        const cd S4 = I * (f[1][0] * (a * cp + b * sp) + f[1][1] * (c * cp + d * sp));
        if (amp_out) {
            const cd Sv[4] = {S1, S2, S3, S4};
            for (int q = 0; q < 4; ++q) {
                amp_out[(size_t)dd * 8 + 2 * q] = Sv[q].real();
                amp_out[(size_t)dd * 8 + 2 * q + 1] = Sv[q].imag();
            }
        }
        // Mueller matrix: Stokes-vector transformation of (S1, S2, S3, S4)
        const double n1 = std::norm(S1), n2 = std::norm(S2), n3 = std::norm(S3), n4 = std::norm(S4);
        const cd s23 = S2 * std::conj(S3), s14 = S1 * std::conj(S4), s24 = S2 * std::conj(S4),
                 s13 = S1 * std::conj(S3), s12 = S1 * std::conj(S2), s34 = S3 * std::conj(S4);
        double* M = S_out + (size_t)dd * 16;
        M[0] = 0.5 * (n1 + n2 + n3 + n4);
        M[1] = 0.5 * (n2 - n1 + n4 - n3);
        M[2] = (s23 + s14).real();
        M[3] = (s23 - s14).imag();
        M[4] = 0.5 * (n2 - n1 + n3 - n4);
        M[5] = 0.5 * (n1 + n2 - n3 - n4);
        M[6] = (s23 - s14).real();
        M[7] = (s23 + s14).imag();
        M[8] = (s24 + s13).real();
        M[9] = (s24 - s13).real();
        M[10] = (s12 + s34).real();
        M[11] = -(s12 + s34).imag();     // Im(S2 S1^* + S4 S3^*)
        M[12] = (std::conj(s24) + s13).imag();  // Im(S4 S2^* + S1 S3^*)
        M[13] = (std::conj(s24) - s13).imag();  // Im(S4 S2^* - S1 S3^*)
        M[14] = (s12 - s34).imag();
        M[15] = (s12 - s34).real();
    }
    return DDA_OK;
}

dda_status dda_angular_averages(dda_ctx* ctx, dda_precision precision, int R, const double* khat, const double* P,
                                double eta, double* out, int* ndir_out) {
    if (!ctx) return DDA_ERR_ARG;
    ProfScope prof_scope(ctx);
    if (!out || !(eta > 0.0) || !std::isfinite(eta)) return ctx->fail(DDA_ERR_ARG, "eta > 0 and out required");
    std::vector<double> k;
    dda_status rs = farfield_common(ctx, precision, R, khat, P, k);
    if (rs != DDA_OK) return rs;
    const double x = ctx->kd * ctx->aeff_lat;
    if (x / eta > 1e5) return ctx->fail(DDA_ERR_SIZE, "eta too small for x = %g", x);
    std::vector<double> th, ph, om;
    scat_dirs(x, eta, th, ph, om);
    const int nd = (int)th.size();
    std::vector<double2> F;
    rs = precision == DDA_FP64 ? farfield_run<double>(ctx, R, k, P, nd, th.data(), ph.data(), F)
                               : farfield_run<float>(ctx, R, k, P, nd, th.data(), ph.data(), F);
    if (rs != DDA_OK) return rs;
    for (int r = 0; r < R; ++r) {
        double c = 0.0, s1 = 0.0, s2 = 0.0, gy = 0.0, gz = 0.0;
        for (int d = 0; d < nd; ++d) {
            const double2* f = &F[((size_t)r * nd + d) * 3];
            const double w = om[d] * (f[0].x * f[0].x + f[0].y * f[0].y + f[1].x * f[1].x + f[1].y * f[1].y +
                                      f[2].x * f[2].x + f[2].y * f[2].y);
            const double ct = std::cos(th[d]), st = std::sin(th[d]);
            c += w;
            s1 += w * ct;
            s2 += w * ct * ct;
            gy += w * st * std::cos(ph[d]);
            gz += w * st * std::sin(ph[d]);
        }
        double* o = out + 6 * (size_t)r;
        o[0] = c / (kPi * ctx->aeff_lat * ctx->aeff_lat);
        o[1] = s1 / c;
        o[2] = s2 / c;
        o[3] = s1 / c;
        o[4] = gy / c;
        o[5] = gz / c;
    }
    if (ndir_out) *ndir_out = nd;
    return DDA_OK;
}

dda_status dda_grad_qabs(dda_ctx* ctx, dda_precision precision, const double* khat, const double* e,
                         const dda_opts* opts, double* dq_dre_eps, double* dq_dim_eps, double* P_out,
                         dda_result* res) {
    if (!ctx) return DDA_ERR_ARG;
    ProfScope prof_scope(ctx);
    if (!dq_dre_eps || !dq_dim_eps || !res) return ctx->fail(DDA_ERR_ARG, "NULL output");
    if (ctx->aniso)
        return ctx->fail(DDA_ERR_ARG, "the gradient is defined for isotropic materials (one eps per site)");
    cudaSetDevice(ctx->device);
    dda_status st = forward_solve(ctx, precision, 1, khat, e, opts, &res[0]);
    if (st != DDA_OK) return st;
    const int64_t N = ctx->g.N, n = 3 * N;
    dda_status rs;
    // keep P, build the adjoint RHS W P^* in S_E64, solve A nu = W P^*
    if ((rs = ensure(ctx, ctx->pool[S_GRAD], (size_t)n * sizeof(double2))) != DDA_OK) return rs;
    double2* Pkeep = slot<double2>(ctx, S_GRAD);
    CU(cudaMemcpyAsync(Pkeep, ctx->pool[S_X64].p, n * sizeof(double2), cudaMemcpyDeviceToDevice, ctx->stream));
    CU(launch_adjoint_rhs(N, Pkeep, ctx->tg.comp_of, slot<double>(ctx, S_W), slot<double2>(ctx, S_E64), ctx->stream));
    dda_opts o = opts ? *opts : default_opts();
    o.x0 = nullptr;
    std::vector<RhsTrack> tr(1);
    if (precision == DDA_FP64)
        rs = solve_core<double>(ctx, 1, o, true, false, tr);
    else
        rs = solve_core<float>(ctx, 1, o, precision == DDA_FP32_REFINED, false, tr);
    if (rs != DDA_OK) return rs;
    res[1].qext = res[1].qabs = res[1].qsca = 0.0;
    res[1].resid_rel = tr[0].bn > 0 ? tr[0].rn / tr[0].bn : 0.0;
    res[1].resid_normal_eq = -1.0;
    res[1].iters = tr[0].iters;
    res[1].outer_iters = tr[0].outer;
    res[1].matvecs = tr[0].mv;
    res[1].status = map_status(tr[0].status);
    if (res[1].status != DDA_OK) return ctx->fail(res[1].status, "adjoint solve did not converge");
    // d(1/alpha)/d(eps) per composition for this RHS
    std::vector<double> k;
    std::vector<cd> ev;
    if ((rs = check_rhs(ctx, 1, khat, e, k, ev)) != DDA_OK) return rs;
    const int BS = beta_stride(ctx);
    std::vector<double2> db(BS, make_double2(0.0, 0.0));
    for (int c = 1; c < BS; ++c) {
        const cd mr = ctx->m[c - 1] / ctx->m_amb;
        const cd v = ldr_inverse_alpha_deps(mr * mr, ctx->kd, k.data(), ev.data());
        db[c] = make_double2(v.real(), v.imag());
    }
    if ((rs = ensure(ctx, ctx->pool[S_DBETA], BS * sizeof(double2))) != DDA_OK) return rs;
    CU(cudaMemcpyAsync(ctx->pool[S_DBETA].p, db.data(), BS * sizeof(double2), cudaMemcpyHostToDevice, ctx->stream));
    if ((rs = ensure(ctx, ctx->pool[S_MV_X32], (size_t)2 * N * sizeof(double))) != DDA_OK) return rs;
    double* g = slot<double>(ctx, S_MV_X32);
    const double K = 4.0 * ctx->kd / (ctx->aeff_lat * ctx->aeff_lat);
    CU(launch_grad(N, Pkeep, slot<double2>(ctx, S_X64), ctx->tg.comp_of, slot<double2>(ctx, S_DBETA), K, g, g + N,
                   ctx->stream));
    CU(cudaMemcpyAsync(dq_dre_eps, g, N * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaMemcpyAsync(dq_dim_eps, g + N, N * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    if (P_out) CU(cudaMemcpyAsync(P_out, Pkeep, n * sizeof(double2), cudaMemcpyDeviceToHost, ctx->stream));
    CU(sync_collect(ctx));
    return DDA_OK;
}

dda_status dda_set_schedule(dda_ctx* ctx, int zpass) {
    if (!ctx) return DDA_ERR_ARG;
    if (zpass < -1 || zpass > 4)
        return ctx->fail(DDA_ERR_ARG, "z-pass schedule must be -1 or 0..4 (got %d)", zpass);
    ctx->force_z = zpass;
    ctx->zsched.clear();
    if (ctx->graph.exec) {
        cudaGraphExecDestroy(ctx->graph.exec);
        ctx->graph.exec = nullptr;
    }
    return DDA_OK;
}

dda_status dda_set_slice_passes(dda_ctx* ctx, int on) {
    if (!ctx) return DDA_ERR_ARG;
    if (on < -1 || on > 1) return ctx->fail(DDA_ERR_ARG, "slice passes: -1, 0 or 1 (got %d)", on);
    ctx->force_slices = on;
    ctx->zsched.clear();
    if (ctx->graph.exec) {
        cudaGraphExecDestroy(ctx->graph.exec);
        ctx->graph.exec = nullptr;
    }
    return DDA_OK;
}

dda_status dda_get_schedule(dda_ctx* ctx, int R, int* zpass, int* slices) {
    if (!ctx || !zpass) return DDA_ERR_ARG;
    if (R <= 0) return ctx->fail(DDA_ERR_ARG, "R must be > 0");
    if (!ctx->prepared || !ctx->has32)
        return ctx->fail(DDA_ERR_ARG, "dda_prepare with a complex64-capable precision has not been called");
    ProfScope prof_scope(ctx);
    cudaSetDevice(ctx->device);
    dda_status s;
    if ((s = ensure_pad<float>(ctx, R)) != DDA_OK) return s;
    PadWork<float> w;
    s = pick_schedule<float>(ctx, matvec_chunk<float>(ctx, R), true, &w);
    *zpass = w.zvar;
    if (slices) *slices = w.slices;
    return s;
}

dda_status dda_get_solve_schedule(dda_ctx* ctx, int R, int* zpass, int* xfwd, int* xinv, int* ypass) {
    if (!ctx || !zpass || !xfwd || !xinv || !ypass) return DDA_ERR_ARG;
    if (R <= 0) return ctx->fail(DDA_ERR_ARG, "R must be > 0");
    if (!ctx->prepared || !ctx->has32)
        return ctx->fail(DDA_ERR_ARG, "dda_prepare with a complex64-capable precision has not been called");
    ProfScope prof_scope(ctx);
    cudaSetDevice(ctx->device);
    dda_status s;
    if ((s = ensure_pad<float>(ctx, R)) != DDA_OK) return s;
    PadWork<float> w;
    s = pick_schedule<float>(ctx, matvec_chunk<float>(ctx, R), true, &w, true);
    *zpass = w.zvar;
    *xfwd = w.xfwd;
    *xinv = w.xinv;
    *ypass = w.yvar;
    return s;
}

dda_status dda_set_ypass(dda_ctx* ctx, int ypass) {
    if (!ctx) return DDA_ERR_ARG;
    if (ypass < -1 || ypass > 1) return ctx->fail(DDA_ERR_ARG, "y-pass schedule must be -1, 0 or 1 (got %d)", ypass);
    ctx->force_y = ypass;
    ctx->zsched.clear();
    if (ctx->graph.exec) {
        cudaGraphExecDestroy(ctx->graph.exec);
        ctx->graph.exec = nullptr;
    }
    return DDA_OK;
}

dda_status dda_get_ypass(dda_ctx* ctx, int R, int* ypass) {
    if (!ctx || !ypass) return DDA_ERR_ARG;
    if (R <= 0) return ctx->fail(DDA_ERR_ARG, "R must be > 0");
    if (!ctx->prepared || !ctx->has32)
        return ctx->fail(DDA_ERR_ARG, "dda_prepare with a complex64-capable precision has not been called");
    ProfScope prof_scope(ctx);
    cudaSetDevice(ctx->device);
    dda_status s;
    if ((s = ensure_pad<float>(ctx, R)) != DDA_OK) return s;
    PadWork<float> w;
    s = pick_schedule<float>(ctx, matvec_chunk<float>(ctx, R), true, &w);
    *ypass = w.yvar;
    return s;
}

dda_status dda_set_xpass(dda_ctx* ctx, int xfwd, int xinv) {
    if (!ctx) return DDA_ERR_ARG;
    if (xfwd < -1 || xfwd > 3 || xinv < -1 || xinv > 3)
        return ctx->fail(DDA_ERR_ARG, "x-pass schedules must be -1, 0, 1, 2 or 3 (got %d, %d)", xfwd, xinv);
    ctx->force_xf = xfwd;
    ctx->force_xi = xinv;
    ctx->zsched.clear();
    if (ctx->graph.exec) {
        cudaGraphExecDestroy(ctx->graph.exec);
        ctx->graph.exec = nullptr;
    }
    return DDA_OK;
}

dda_status dda_get_xpass(dda_ctx* ctx, int R, int* xfwd, int* xinv) {
    if (!ctx || !xfwd || !xinv) return DDA_ERR_ARG;
    if (R <= 0) return ctx->fail(DDA_ERR_ARG, "R must be > 0");
    if (!ctx->prepared || !ctx->has32)
        return ctx->fail(DDA_ERR_ARG, "dda_prepare with a complex64-capable precision has not been called");
    ProfScope prof_scope(ctx);
    cudaSetDevice(ctx->device);
    dda_status s;
    if ((s = ensure_pad<float>(ctx, R)) != DDA_OK) return s;
    PadWork<float> w;
    s = pick_schedule<float>(ctx, matvec_chunk<float>(ctx, R), true, &w);
    *xfwd = w.xfwd;
    *xinv = w.xinv;
    return s;
}

dda_status dda_profile_enable(dda_ctx* ctx, int on) {
    if (!ctx) return DDA_ERR_ARG;
    cudaSetDevice(ctx->device);
    if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) return ctx->cuda_fail(cudaGetLastError(), "sync");
    ctx->prof.reset();
    ctx->prof.on = on != 0;
    return DDA_OK;
}

dda_status dda_profile_read(const dda_ctx* ctx, dda_kernel_stat* out, int max_entries, int* n_entries) {
    if (!ctx || !n_entries || (max_entries > 0 && !out)) return DDA_ERR_ARG;
    int n = 0;
    for (int k = 0; k < KK_COUNT; ++k) {
        if (ctx->prof.launches[k] == 0) continue;
        if (n < max_entries) {
            dda_kernel_stat& st = out[n];
            std::memset(&st, 0, sizeof st);
            std::snprintf(st.name, sizeof st.name, "%s", kernel_kind_name(k));
            st.launches = ctx->prof.launches[k];
            st.total_ms = ctx->prof.ms[k];
            st.units = ctx->prof.unit_sum[k];
        }
        ++n;
    }
    *n_entries = n;
    return DDA_OK;
}

}  // extern "C"
