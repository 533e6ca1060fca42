// complex64 instantiation of the matvec passes (see matvec_impl.cuh).
#include "matvec_impl.cuh"

namespace dda {

template int zconv_schedules<float>(const Geom&);
template int xpass_schedules<float>(const Geom&);
template int ypass_schedules<float>(const Geom&);
template cudaError_t launch_zconv<float>(const Geom&, int, float2*, const float2*, const float2*, const int*, int, cudaStream_t);
template cudaError_t launch_matvec<float>(const Geom&, int, const float2*, float2*, const PadWork<float>&,
                                          const DevTarget&, const float2*, int, const float2*, const Twiddles<float>&,
                                          const int*, cudaStream_t);
template cudaError_t launch_matvec_fused<float>(const Geom&, int, float2*, float2*, const PadWork<float>&,
                                                const DevTarget&, const float2*, int, const float2*,
                                                const Twiddles<float>&, int*, const FusedKrylov<float>&,
                                                cudaStream_t);

}  // namespace dda
