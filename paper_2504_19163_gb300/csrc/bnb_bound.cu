// Bound kernel launchers and the float32 instantiation (the kernel itself is in
// bnb_bound_impl.cuh; the float64 instantiation is compiled in bnb_bound64.cu).
#include "bnb_bound_impl.cuh"

namespace bnb {

template cudaError_t launch_bound_base_T<float, 0>(const BoundParams&, cudaStream_t);
template cudaError_t launch_bound_split_T<float, 0>(const BoundParams&, const SplitItem*, const int64_t*,
                                                    cudaStream_t);
// instantiated in bnb_bound64.cu (float64 reflection) and bnb_bound_refract.cu (refraction)
extern template cudaError_t launch_bound_base_T<double, 0>(const BoundParams&, cudaStream_t);
extern template cudaError_t launch_bound_split_T<double, 0>(const BoundParams&, const SplitItem*, const int64_t*,
                                                            cudaStream_t);
extern template cudaError_t launch_bound_base_T<float, 1>(const BoundParams&, cudaStream_t);
extern template cudaError_t launch_bound_split_T<float, 1>(const BoundParams&, const SplitItem*, const int64_t*,
                                                           cudaStream_t);
extern template cudaError_t launch_bound_base_T<double, 1>(const BoundParams&, cudaStream_t);
extern template cudaError_t launch_bound_split_T<double, 1>(const BoundParams&, const SplitItem*, const int64_t*,
                                                            cudaStream_t);
// block-size schedules of the float32 reflection pass (bnb_bound_t256.cu, bnb_bound_t320.cu)
extern template cudaError_t launch_bound_base_T<float, 0, 256>(const BoundParams&, cudaStream_t);
extern template cudaError_t launch_bound_base_T<float, 0, 320>(const BoundParams&, cudaStream_t);
extern template cudaError_t launch_bound_base_T<float, 1, 128>(const BoundParams&, cudaStream_t);  // bnb_bound_refract_t128.cu

__global__ void pack_tris_k(const float* __restrict__ px, const float* __restrict__ py, const float* __restrict__ pz,
                            const float* __restrict__ nx, const float* __restrict__ ny, const float* __restrict__ nz,
                            const int32_t* __restrict__ i0, const int32_t* __restrict__ i1,
                            const int32_t* __restrict__ i2, int n_tris, int n_verts, float4* __restrict__ out) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n_tris) return;
  int v[3] = {i0[t], i1[t], i2[t]};
  // an out-of-range vertex index degenerates the triangle to vertex 0 instead of reading outside
  for (int k = 0; k < 3; ++k) v[k] = (v[k] >= 0 && v[k] < n_verts) ? v[k] : 0;
  float f[20];
  for (int k = 0; k < 3; ++k) {
    f[3 * k + 0] = px[v[k]];
    f[3 * k + 1] = py[v[k]];
    f[3 * k + 2] = pz[v[k]];
    f[9 + 3 * k + 0] = nx[v[k]];
    f[9 + 3 * k + 1] = ny[v[k]];
    f[9 + 3 * k + 2] = nz[v[k]];
  }
  f[18] = 0.f;
  f[19] = 0.f;
  float4* o = out + (int64_t)t * kTriF4;
  for (int q = 0; q < kTriF4; ++q) o[q] = make_float4(f[4 * q], f[4 * q + 1], f[4 * q + 2], f[4 * q + 3]);
}

cudaError_t launch_pack_tris(const bnb_surface* s, float4* out, cudaStream_t st) {
  if (s->n_tris <= 0 || s->n_verts <= 0) return cudaSuccess;
  pack_tris_k<<<(s->n_tris + 255) / 256, 256, 0, st>>>(s->px, s->py, s->pz, s->nx, s->ny, s->nz, s->i0, s->i1, s->i2,
                                                        s->n_tris, s->n_verts, out);
  return cudaGetLastError();
}

cudaError_t launch_bound_base(const BoundParams& p, bool fp64, cudaStream_t st) {
  if (p.kind == BNB_REFRACT) {
    if (fp64) return launch_bound_base_T<double, 1>(p, st);
    if (p.block_threads == 128) return launch_bound_base_T<float, 1, 128>(p, st);
    return launch_bound_base_T<float, 1>(p, st);
  }
  if (fp64) return launch_bound_base_T<double, 0>(p, st);
  if (p.block_threads == 256) return launch_bound_base_T<float, 0, 256>(p, st);
  if (p.block_threads == 320) return launch_bound_base_T<float, 0, 320>(p, st);
  return launch_bound_base_T<float, 0>(p, st);
}

cudaError_t launch_bound_split(const BoundParams& p, const SplitItem* q_in, const int64_t* q_in_count, bool fp64,
                               cudaStream_t st) {
  if (p.kind == BNB_REFRACT)
    return fp64 ? launch_bound_split_T<double, 1>(p, q_in, q_in_count, st)
                : launch_bound_split_T<float, 1>(p, q_in, q_in_count, st);
  return fp64 ? launch_bound_split_T<double, 0>(p, q_in, q_in_count, st)
              : launch_bound_split_T<float, 0>(p, q_in, q_in_count, st);
}

}  // namespace bnb
