// double-float instantiation of the matvec passes (see matvec_impl.cuh).
#include "matvec_impl.cuh"

namespace dda {

template cudaError_t launch_matvec<dfl>(const Geom&, int, const cdfl*, cdfl*, const PadWork<dfl>&, const DevTarget&,
                                        const cdfl*, int, const cdfl*, const Twiddles<dfl>&, const int*, cudaStream_t);

}  // namespace dda
