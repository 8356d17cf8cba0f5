// Reflection bound kernel in float32 with 320-thread blocks (one of the block-size schedules the
// autotuner chooses from; the default, 384, is compiled in bnb_bound.cu); a translation unit of
// its own so the build parallelizes.
#include "bnb_bound_impl.cuh"

namespace bnb {
template cudaError_t launch_bound_base_T<float, 0, 320>(const BoundParams&, cudaStream_t);
}  // namespace bnb
