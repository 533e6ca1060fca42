// Launch tracing (see profiler.h).
#include "profiler.h"

namespace dda {

static thread_local Profiler* t_current = nullptr;

// Inside stream capture a plain event record only orders graph nodes; the
// external flag makes it a record node that runs on every graph launch.
static cudaError_t record(cudaEvent_t e, cudaStream_t st) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaError_t err = cudaStreamIsCapturing(st, &cs);
    if (err != cudaSuccess) return err;
    return cs == cudaStreamCaptureStatusActive ? cudaEventRecordWithFlags(e, st, cudaEventRecordExternal)
                                               : cudaEventRecord(e, st);
}
Profiler* current_profiler() { return t_current; }
void set_current_profiler(Profiler* p) { t_current = p; }

const char* kernel_kind_name(int kind) {
    static const char* names[KK_COUNT] = {
        "x_fwd_c64", "y_fwd_c64", "z_conv_c64", "y_inv_c64", "x_inv_c64",
        "x_fwd_c128", "y_fwd_c128", "z_conv_c128", "y_inv_c128", "x_inv_c128",
        "x_fwd_df", "y_fwd_df", "z_conv_df", "y_inv_df", "x_inv_df",
        "bicgstab_c64", "bicgstab_c128", "refine_c128", "incident_field", "q_sums", "green_fft", "other",
        "xy_fwd_c64", "yx_inv_c64", "xy_fwd_c128", "yx_inv_c128", "xy_fwd_df", "yx_inv_df", "far_field"};
    return (kind >= 0 && kind < KK_COUNT) ? names[kind] : "?";
}

void Profiler::reset() {
    cursor = 0;
    gkinds.clear();
    gunits.clear();
    for (int k = 0; k < KK_COUNT; ++k) {
        ms[k] = 0.0;
        unit_sum[k] = 0.0;
        launches[k] = 0;
    }
}

void Profiler::release() {
    for (cudaEvent_t e : ev) cudaEventDestroy(e);
    ev.clear();
    kinds.clear();
    units.clear();
    reset();
}

cudaError_t Profiler::begin(cudaStream_t st) {
    if (2 * cursor + 2 > ev.size()) {
        for (int i = 0; i < 2; ++i) {
            cudaEvent_t e;
            cudaError_t err = cudaEventCreate(&e);
            if (err != cudaSuccess) return err;
            ev.push_back(e);
        }
        kinds.push_back(KK_OTHER);
        units.push_back(0.0);
    }
    return record(ev[2 * cursor], st);
}

cudaError_t Profiler::end(int kind, double u, cudaStream_t st) {
    kinds[cursor] = kind;
    units[cursor] = u;
    cudaError_t err = record(ev[2 * cursor + 1], st);
    ++cursor;
    return err;
}

cudaError_t Profiler::collect() {
    for (size_t i = 0; i < cursor; ++i) {
        float t = 0.f;
        cudaError_t err = cudaEventElapsedTime(&t, ev[2 * i], ev[2 * i + 1]);
        if (err != cudaSuccess) {
            cursor = 0;
            return err;
        }
        ms[kinds[i]] += t;
        unit_sum[kinds[i]] += units[i];
        launches[kinds[i]] += 1;
    }
    cursor = 0;
    return cudaSuccess;
}

void Profiler::capture_end() {
    gkinds.assign(kinds.begin(), kinds.begin() + cursor);
    gunits.assign(units.begin(), units.begin() + cursor);
    cursor = 0;
}

void Profiler::graph_launched() {
    for (size_t i = 0; i < gkinds.size(); ++i) {
        kinds[i] = gkinds[i];
        units[i] = gunits[i];
    }
    cursor = gkinds.size();
}

}  // namespace dda
