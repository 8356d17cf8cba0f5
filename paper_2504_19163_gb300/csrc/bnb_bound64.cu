// Float64 instantiation of the bound kernel (bound pass run entirely in double,
// same arithmetic with u = 2^-53); compiled separately so the build parallelizes.
#include "bnb_bound_impl.cuh"

namespace bnb {
template cudaError_t launch_bound_base_T<double, 0>(const BoundParams&, cudaStream_t);
template cudaError_t launch_bound_split_T<double, 0>(const BoundParams&, const SplitItem*, const int64_t*,
                                                     cudaStream_t);
}  // namespace bnb
