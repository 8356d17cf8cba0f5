// gamma for a target expected |S| (Sec. 5.4): the smallest float32 gamma whose expected number of
// selected tuples per shading point reaches the target, found on the device.
//
// Sec. 5.4 notes that gamma and the expected sample count E|S| are in one-to-one correspondence,
// so a render can be configured by E|S|.  With the selection rule of bnb_sample_and_solve (tuple
// T of a point's list selected when a 24-bit uniform r = k 2^-24 is below P_T = min(gamma (x) E~_T,
// 1), the product rounded up), the exact probability of selecting T is ceil(P_T 2^24) / 2^24, so
//     E|S|(gamma) = sum_g w_g sum_{T listed in g} ceil(P_T 2^24) / (2^24 W),
// w_g the number of shading points in grid cell g and W their total.  The sum is formed in
// integers (exact, the same on every run), and it is non-decreasing in gamma, so a bisection over
// the bit patterns of the positive finite floats (31 steps) finds the smallest gamma with
// E|S|(gamma) >= target.  Every step is two launches on the stream (evaluate, then update the
// bracket in a one-thread kernel), so nothing returns to the host in between.
#include <stdint.h>

#include <algorithm>

#include "bnb_internal.cuh"

namespace bnb {

struct GammaState {
  unsigned long long sum;  // integer E|S| numerator at `mid`
  uint32_t lo, hi, mid;    // bracket over float bit patterns: f(lo) < target <= f(hi) (hi may be unreachable)
  uint32_t pad;
  double thresh;           // target * W * 2^24
};

namespace {

constexpr uint32_t kMaxFiniteBits = 0x7f7fffffu;

__global__ void gamma_points_k(const float* __restrict__ su, const float* __restrict__ sv, int64_t n, int G,
                               int32_t* __restrict__ w) {
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
    const int gi = min(G - 1, max(0, (int)floorf(__fmul_rn(fminf(fmaxf(su[p], 0.0f), 1.0f), (float)G))));
    const int gj = min(G - 1, max(0, (int)floorf(__fmul_rn(fminf(fmaxf(sv[p], 0.0f), 1.0f), (float)G))));
    atomicAdd(w + (int64_t)gj * G + gi, 1);
  }
}

__global__ void gamma_init_k(GammaState* s, double target, double W) {
  s->sum = 0ull;
  s->lo = 0u;
  s->hi = kMaxFiniteBits;
  s->mid = s->lo + (s->hi - s->lo) / 2u;
  s->thresh = target * W * 16777216.0;
}

// Integer E|S| numerator at gamma = bits(mid): one warp per grid cell (grid-stride), lanes over the
// cell's list; one atomic per block.
__global__ void __launch_bounds__(256) gamma_eval_k(const int64_t* __restrict__ offsets, const float* __restrict__ et,
                                                    int64_t capacity, int64_t n_cells,
                                                    const int32_t* __restrict__ w, GammaState* s) {
  const float gamma = __uint_as_float(s->mid);
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t n_warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  unsigned long long acc = 0ull;
  for (int64_t g = warp; g < n_cells; g += n_warps) {
    const unsigned long long wg = w ? (unsigned long long)w[g] : 1ull;
    if (wg == 0ull) continue;
    const int64_t a = offsets[g], b = min(offsets[g + 1], capacity);
    unsigned long long c = 0ull;
    for (int64_t j = a + lane; j < b; j += 32) {
      const float P = fminf(__fmul_ru(gamma, et[j]), 1.0f);
      c += (unsigned long long)ceilf(P * 16777216.0f);  // exact: a power-of-two scaling of P <= 1
    }
    acc += wg * c;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  __shared__ unsigned long long part[8];
  if (lane == 0) part[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long t = 0ull;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += part[i];
    if (t) atomicAdd(&s->sum, t);
  }
}

__global__ void gamma_step_k(GammaState* s) {
  if ((double)s->sum >= s->thresh)
    s->hi = s->mid;
  else
    s->lo = s->mid;
  s->mid = s->lo + (s->hi - s->lo) / 2u;
  s->sum = 0ull;
}

__global__ void gamma_out_k(const GammaState* s, float* out) { *out = __uint_as_float(s->hi); }

}  // namespace

size_t gamma_ws_bytes(int32_t G) {
  return (size_t)round_up((int64_t)sizeof(GammaState), 256) + (size_t)round_up((int64_t)G * G * 4, 256);
}

cudaError_t launch_gamma_for_target(const bnb_index* idx, const float* su, const float* sv, int64_t n_points,
                                    double target, float* gamma_out, void* ws, cudaStream_t st) {
  const int G = idx->grid_res;
  const int64_t n_cells = (int64_t)G * G;
  GammaState* s = (GammaState*)ws;
  int32_t* w = (int32_t*)((char*)ws + round_up((int64_t)sizeof(GammaState), 256));
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaError_t e;
  const bool weighted = su != nullptr;
  if (weighted) {
    if ((e = cudaMemsetAsync(w, 0, (size_t)n_cells * 4, st)) != cudaSuccess) return e;
    if (n_points > 0) {
      const int64_t pb = std::min<int64_t>((n_points + 255) / 256, (int64_t)sms * 16);
      gamma_points_k<<<(unsigned)pb, 256, 0, st>>>(su, sv, n_points, G, w);
    }
  }
  const double W = weighted ? (double)n_points : (double)n_cells;
  gamma_init_k<<<1, 1, 0, st>>>(s, target, W);
  const int blocks = sms * 8;
  for (int it = 0; it < 31; ++it) {  // hi - lo < 2^31 halves to 1
    gamma_eval_k<<<blocks, 256, 0, st>>>(idx->offsets, idx->etilde, idx->capacity, n_cells, weighted ? w : nullptr,
                                         s);
    gamma_step_k<<<1, 1, 0, st>>>(s);
  }
  gamma_out_k<<<1, 1, 0, st>>>(s, gamma_out);
  return cudaGetLastError();
}

}  // namespace bnb
