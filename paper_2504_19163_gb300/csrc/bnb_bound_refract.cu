// Refraction instantiation of the bound kernel in float32 (with the float64 sign fallback);
// compiled separately so the build parallelizes.
#include "bnb_bound_impl.cuh"

namespace bnb {
template cudaError_t launch_bound_base_T<float, 1>(const BoundParams&, cudaStream_t);
template cudaError_t launch_bound_split_T<float, 1>(const BoundParams&, const SplitItem*, const int64_t*,
                                                    cudaStream_t);
}  // namespace bnb
