// Exhaustive check of the reciprocal approximation the bound kernel uses in its ratio bounds
// (rcp.approx.ftz.f32): the largest relative error |r x - 1| over every normal float x in
// [lo_bits, hi_bits] (bit patterns), computed exactly in float64.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

__global__ void rcp_err_k(uint32_t lo_bits, uint32_t hi_bits, unsigned long long* max_err_bits) {
  double mx = 0.0;
  const uint64_t n = (uint64_t)hi_bits - lo_bits + 1;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
    const float x = __uint_as_float(lo_bits + (uint32_t)i);
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    // r * x has at most 48 significant bits: exact in float64, and so is the difference to 1.
    const double e = fabs((double)r * (double)x - 1.0);
    mx = e > mx ? e : mx;
  }
  for (int o = 16; o > 0; o >>= 1) {
    const double y = __shfl_xor_sync(0xffffffffu, mx, o);
    mx = y > mx ? y : mx;
  }
  if ((threadIdx.x & 31) == 0) atomicMax(max_err_bits, (unsigned long long)__double_as_longlong(mx));
}

extern "C" int rcp_max_rel_err(uint32_t lo_bits, uint32_t hi_bits, double* out) {
  unsigned long long* d = nullptr;
  if (cudaMalloc(&d, sizeof(*d)) != cudaSuccess) return 1;
  cudaMemset(d, 0, sizeof(*d));
  rcp_err_k<<<152 * 16, 256>>>(lo_bits, hi_bits, d);
  unsigned long long h = 0;
  const cudaError_t e = cudaMemcpy(&h, d, sizeof(h), cudaMemcpyDeviceToHost);
  cudaFree(d);
  if (e != cudaSuccess) return 2;
  memcpy(out, &h, sizeof(h));
  return 0;
}
