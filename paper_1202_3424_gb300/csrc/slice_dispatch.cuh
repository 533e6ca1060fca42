// Runtime dispatch over (Lx, Ly) for the slice passes; included by the
// translation units that instantiate them.
#pragma once

#include "slice_impl.cuh"

namespace dda {

#define DDA_SLICE_LY(LXV, LYV, FN, ...)                                  \
    switch (LYV) {                                                       \
        case 64: return FN<LXV, 64>(__VA_ARGS__);                        \
        case 96: return FN<LXV, 96>(__VA_ARGS__);                        \
        case 128: return FN<LXV, 128>(__VA_ARGS__);                      \
        case 192: return FN<LXV, 192>(__VA_ARGS__);                      \
        default: return cudaErrorInvalidValue;                           \
    }
#define DDA_SLICE_DISPATCH(LXV, LYV, FN, ...)                            \
    switch (LXV) {                                                       \
        case 64: DDA_SLICE_LY(64, LYV, FN, __VA_ARGS__)                  \
        case 96: DDA_SLICE_LY(96, LYV, FN, __VA_ARGS__)                  \
        case 128: DDA_SLICE_LY(128, LYV, FN, __VA_ARGS__)                \
        case 192: DDA_SLICE_LY(192, LYV, FN, __VA_ARGS__)                \
        default: return cudaErrorInvalidValue;                           \
    }

template <int ES> bool slice_built_rt(int Lx, int Ly) {
#define DDA_SB(a, b) \
    if (Lx == a && Ly == b) return slice_built<a, b, ES>();
    DDA_SB(64, 64) DDA_SB(64, 96) DDA_SB(64, 128) DDA_SB(64, 192)
    DDA_SB(96, 64) DDA_SB(96, 96) DDA_SB(96, 128) DDA_SB(96, 192)
    DDA_SB(128, 64) DDA_SB(128, 96) DDA_SB(128, 128) DDA_SB(128, 192)
    DDA_SB(192, 64) DDA_SB(192, 96) DDA_SB(192, 128) DDA_SB(192, 192)
#undef DDA_SB
    return false;
}

template <typename T> struct SliceKinds;
template <> struct SliceKinds<float> { static constexpr int fwd = KK_XYFWD_C64, inv = KK_YXINV_C64; };
template <> struct SliceKinds<double> { static constexpr int fwd = KK_XYFWD_C128, inv = KK_YXINV_C128; };
template <> struct SliceKinds<dfl> { static constexpr int fwd = KK_XYFWD_DF, inv = KK_YXINV_DF; };

template <typename T> bool slice_passes(const Geom& g) { return slice_built_rt<sizeof(cx<T>)>(g.Lx, g.Ly); }

template <typename T>
cudaError_t launch_slice_fwd(const Geom& g, int R, cx<T>* x, cx<T>* u2, const int* site_of, const Twiddles<T>& tw,
                             const int* active, const FusedKrylov<T>& fk, cudaStream_t st) {
    DDA_SLICE_DISPATCH(g.Lx, g.Ly, LaunchSlice<T>::template fwd, g, R, x, u2, site_of, tw.x, tw.y, active, fk, st,
                       SliceKinds<T>::fwd)
}

template <typename T>
cudaError_t launch_slice_inv(const Geom& g, int R, const cx<T>* u2, cx<T>* y, const cx<T>* x, const DevTarget& tg,
                             const cx<T>* beta, int beta_stride, const Twiddles<T>& tw, int* active,
                             const FusedKrylov<T>& fk, cudaStream_t st) {
    DDA_SLICE_DISPATCH(g.Lx, g.Ly, LaunchSlice<T>::template inv, g, R, u2, y, x, tg, beta, beta_stride, tw.x, tw.y,
                       active, fk, st, SliceKinds<T>::inv)
}

#define DDA_SLICE_INSTANTIATE(T)                                                                                  \
    template bool slice_passes<T>(const Geom&);                                                                   \
    template cudaError_t launch_slice_fwd<T>(const Geom&, int, cx<T>*, cx<T>*, const int*, const Twiddles<T>&,   \
                                             const int*, const FusedKrylov<T>&, cudaStream_t);                    \
    template cudaError_t launch_slice_inv<T>(const Geom&, int, const cx<T>*, cx<T>*, const cx<T>*,               \
                                             const DevTarget&, const cx<T>*, int, const Twiddles<T>&, int*,       \
                                             const FusedKrylov<T>&, cudaStream_t);

}  // namespace dda
