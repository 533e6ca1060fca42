// Launch tracing: CUDA events around each hot-path kernel launch, on the
// stream the kernel is launched on, accumulated per kernel kind.  Off by
// default; when on, events recorded while a stream is captured become event
// nodes of the graph and are read back after each replay.
#pragma once

#include <cuda_runtime.h>

#include <vector>

namespace dda {

enum KernelKind : int {
    KK_XFWD_C64, KK_YFWD_C64, KK_ZCONV_C64, KK_YINV_C64, KK_XINV_C64,
    KK_XFWD_C128, KK_YFWD_C128, KK_ZCONV_C128, KK_YINV_C128, KK_XINV_C128,
    KK_XFWD_DF, KK_YFWD_DF, KK_ZCONV_DF, KK_YINV_DF, KK_XINV_DF,
    KK_KRYLOV_C64, KK_KRYLOV_C128, KK_REFINE, KK_EINC, KK_QSUMS, KK_GREEN, KK_OTHER,
    KK_XYFWD_C64, KK_YXINV_C64, KK_XYFWD_C128, KK_YXINV_C128, KK_XYFWD_DF, KK_YXINV_DF,
    KK_FARFIELD,
    KK_COUNT
};

const char* kernel_kind_name(int kind);

struct Profiler {
    bool on = false;
    std::vector<cudaEvent_t> ev;  // 2 per slot
    std::vector<int> kinds;
    std::vector<double> units;
    size_t cursor = 0;
    std::vector<int> gkinds;      // slots captured in the current graph
    std::vector<double> gunits;
    double ms[KK_COUNT] = {};
    double unit_sum[KK_COUNT] = {};
    long long launches[KK_COUNT] = {};

    void reset();
    void release();
    cudaError_t begin(cudaStream_t st);
    cudaError_t end(int kind, double u, cudaStream_t st);
    cudaError_t collect();        // call after the recorded work has completed
    void capture_begin() { cursor = 0; }
    void capture_end();
    void graph_launched();
};

// The profiler of the context whose ABI call is running on this thread (or null).
Profiler* current_profiler();
void set_current_profiler(Profiler* p);

// Bracket a launch: PROF_BEGIN(st); kernel<<<...>>>; PROF_END(kind, units, st);
#define PROF_BEGIN(st)                                                 \
    do {                                                               \
        ::dda::Profiler* _p = ::dda::current_profiler();               \
        if (_p && _p->on) { cudaError_t _pe = _p->begin(st); if (_pe != cudaSuccess) return _pe; } \
    } while (0)
#define PROF_END(kind, u, st)                                          \
    do {                                                               \
        ::dda::Profiler* _p = ::dda::current_profiler();               \
        if (_p && _p->on) { cudaError_t _pe = _p->end(kind, u, st); if (_pe != cudaSuccess) return _pe; } \
    } while (0)

}  // namespace dda
