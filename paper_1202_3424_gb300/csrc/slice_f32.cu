// complex64 instantiation of the fused x+y slice passes (see slice_impl.cuh).
#include "slice_impl.cuh"
#include "slice_dispatch.cuh"

namespace dda {

DDA_SLICE_INSTANTIATE(float)

}  // namespace dda
