// bnb_ffma_probe: FP32 fused multiply-add throughput of this GPU, the denominator of the roofline
// of the ALU-bound bound kernels (no counterpart in the paper).
//
// Every thread runs `iters` rounds of kChains independent FMA chains x <- x * a + b (a, b kernel
// arguments, so nothing folds at compile time), either as scalar FFMA or as paired FFMA2
// (__ffma2_rn: two lanes' worth of FMAs per instruction, the form the bound kernels use for
// independent same-shape products), then writes the sum of its chains to sink[thread] so no chain
// is dead code.  With kChains = 16 per thread and >= 8 warps per scheduler, the FMA latency is
// hidden and the pipe, not issue or dependences, sets the rate.  FLOPs per launch =
// grid_blocks * block_threads * iters * kChains * 2 (x2 again with paired = 1).
#include "bnb_internal.cuh"

namespace bnb {

namespace {

constexpr int kChains = 16;

__global__ void __launch_bounds__(1024) ffma_probe_k(int iters, float a, float b, float* __restrict__ sink) {
  float x[kChains];
#pragma unroll
  for (int j = 0; j < kChains; ++j) x[j] = (float)(threadIdx.x + j) * 1e-3f;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int j = 0; j < kChains; ++j) x[j] = __fmaf_rn(x[j], a, b);
  }
  float s = 0.0f;
#pragma unroll
  for (int j = 0; j < kChains; ++j) s += x[j];
  sink[(int64_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(1024) ffma2_probe_k(int iters, float a, float b, float* __restrict__ sink) {
  float2 x[kChains];
#pragma unroll
  for (int j = 0; j < kChains; ++j) x[j] = make_float2((float)(threadIdx.x + j) * 1e-3f, (float)j * 1e-3f);
  const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int j = 0; j < kChains; ++j) x[j] = __ffma2_rn(x[j], a2, b2);
  }
  float s = 0.0f;
#pragma unroll
  for (int j = 0; j < kChains; ++j) s += x[j].x + x[j].y;
  sink[(int64_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

}  // namespace bnb

extern "C" int32_t bnb_ffma_probe(int32_t grid_blocks, int32_t block_threads, int32_t iters, int32_t paired,
                                  float* sink, void* stream) {
  if (grid_blocks < 1 || grid_blocks > (1 << 20) || block_threads < 32 || block_threads > 1024 ||
      block_threads % 32 != 0 || iters < 1 || (paired != 0 && paired != 1) || !sink)
    return BNB_ERR_INVALID;
  cudaStream_t st = (cudaStream_t)stream;
  // a = 1 - 2^-20 and b = 2^-10 keep every chain finite and away from denormals for any iters
  const float a = 0.99999905f, b = 0.0009765625f;
  if (paired)
    bnb::ffma2_probe_k<<<grid_blocks, block_threads, 0, st>>>(iters, a, b, sink);
  else
    bnb::ffma_probe_k<<<grid_blocks, block_threads, 0, st>>>(iters, a, b, sink);
  return cudaGetLastError() == cudaSuccess ? BNB_OK : BNB_ERR_CUDA;
}
