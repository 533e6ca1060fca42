// double-float instantiation of the matvec passes (see matvec_impl.cuh).
#include "matvec_impl.cuh"

namespace dda {

template int zconv_schedules<dfl>(const Geom&);
template int xpass_schedules<dfl>(const Geom&);
template int ypass_schedules<dfl>(const Geom&);
template cudaError_t launch_zconv<dfl>(const Geom&, int, cdfl*, const cdfl*, const cdfl*, const int*, int, cudaStream_t);
template cudaError_t launch_matvec<dfl>(const Geom&, int, const cdfl*, cdfl*, const PadWork<dfl>&, const DevTarget&,
                                        const cdfl*, int, const cdfl*, const Twiddles<dfl>&, const int*, cudaStream_t);
// (the double-float passes run no fused Krylov modes; this keeps the generic
// schedule code linkable)
template cudaError_t launch_matvec_fused<dfl>(const Geom&, int, cdfl*, cdfl*, const PadWork<dfl>&, const DevTarget&,
                                              const cdfl*, int, const cdfl*, const Twiddles<dfl>&, int*,
                                              const FusedKrylov<dfl>&, cudaStream_t);

}  // namespace dda
