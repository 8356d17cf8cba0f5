// Refraction instantiation of the bound kernel with the whole pass in float64 (position bound; the
// irradiance of refraction is bounded in the float32 pass only); compiled separately.
#include "bnb_bound_impl.cuh"

namespace bnb {
template cudaError_t launch_bound_base_T<double, 1>(const BoundParams&, cudaStream_t);
template cudaError_t launch_bound_split_T<double, 1>(const BoundParams&, const SplitItem*, const int64_t*,
                                                     cudaStream_t);
}  // namespace bnb
