// double-float instantiation of the matvec passes (see matvec_impl.cuh).
#include "matvec_impl.cuh"

namespace dda {

template int zconv_schedules<dfl>(const Geom&);
template cudaError_t launch_zconv<dfl>(const Geom&, int, cdfl*, const cdfl*, const cdfl*, const int*, int, cudaStream_t);
template cudaError_t launch_matvec<dfl>(const Geom&, int, const cdfl*, cdfl*, const PadWork<dfl>&, const DevTarget&,
                                        const cdfl*, int, const cdfl*, const Twiddles<dfl>&, const int*, cudaStream_t);

}  // namespace dda
