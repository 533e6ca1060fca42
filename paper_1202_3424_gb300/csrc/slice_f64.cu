// complex128 and double-float instantiations of the fused x+y slice passes
// (see slice_impl.cuh).
#include "slice_impl.cuh"
#include "slice_dispatch.cuh"

namespace dda {

DDA_SLICE_INSTANTIATE(double)
DDA_SLICE_INSTANTIATE(dfl)

}  // namespace dda
