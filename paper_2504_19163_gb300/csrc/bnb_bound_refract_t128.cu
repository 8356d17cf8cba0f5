// Refraction bound kernel in float32 with 128-thread blocks (a block-size schedule the autotuner
// chooses from; the default, 256, is compiled in bnb_bound_refract.cu); a translation unit of its own
// so the build parallelizes.
#include "bnb_bound_impl.cuh"

namespace bnb {
template cudaError_t launch_bound_base_T<float, 1, 128>(const BoundParams&, cudaStream_t);
}  // namespace bnb
