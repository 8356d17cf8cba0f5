// Batched bound pass: the base cells of many scenes in one persistent launch.  Every cell finds its
// job by binary search over the jobs' cell offsets, builds the job's parameters and runs the same
// cell program as the single-scene pass (reflection inline, refraction through its compiled-once
// function).  Jobs take no extra split levels (max_depth = depth).
#include "bnb_bound_impl.cuh"

namespace bnb {

constexpr int kJobThreads = 1024;

// Cell offsets of the jobs (one block), and each job's base-cell count added to its *count.
__global__ void __launch_bounds__(kJobThreads) bound_jobs_k(const bnb_bound_job* __restrict__ jobs,
                                                            const int32_t* __restrict__ n_jobs_p, int32_t max_jobs,
                                                            int64_t* __restrict__ job_off) {
  __shared__ int64_t warp_sum[kJobThreads / 32];
  const int32_t n = max(0, min(*n_jobs_p, max_jobs));
  const int chunk = (max_jobs + kJobThreads - 1) / kJobThreads;
  const int j0 = threadIdx.x * chunk;
  auto cells_of = [&](int j) -> int64_t {
    const bnb_bound_job& J = jobs[j];
    if (J.depth < 0 || J.depth > 10 || J.n_tris < 0 || J.n_emitters < 0) return 0;
    return (int64_t)J.n_emitters * J.n_tris * ((int64_t)1 << (2 * J.depth));
  };
  int64_t mine = 0;
  for (int j = j0; j < min(j0 + chunk, n); ++j) mine += cells_of(j);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int64_t x = mine;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int64_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_sum[wid] = x;
  __syncthreads();
  if (wid == 0) {
    int64_t w = warp_sum[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int64_t y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    warp_sum[lane] = w;
  }
  __syncthreads();
  int64_t acc = x - mine + (wid > 0 ? warp_sum[wid - 1] : 0);
  if (threadIdx.x == 0) job_off[0] = 0;
  for (int j = j0; j < min(j0 + chunk, max_jobs); ++j) {
    if (j < n) {
      const int64_t c = cells_of(j);
      acc += c;
      if (c > jobs[j].capacity) {
        raise_status(jobs[j].status, BNB_ERR_CAPACITY);
      } else if (c > 0) {
        atomicAdd((unsigned long long*)jobs[j].count, (unsigned long long)c);
      }
    }
    job_off[j + 1] = acc;
  }
}

__device__ __forceinline__ int bound_job_of(const int64_t* __restrict__ job_off, int n, int64_t w) {
  int lo = 0, hi = n - 1;  // largest j with job_off[j] <= w
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (job_off[mid] <= w) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ BoundParams params_of(const bnb_bound_job& J) {
  BoundParams P{};
  P.tri = (const float4*)J.packed_tris;
  P.n_tris = J.n_tris;
  P.n_emitters = J.n_emitters;
  P.ex = J.ex;
  P.ey = J.ey;
  P.ez = J.ez;
  P.ei = J.ei;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    P.rp0[c] = J.rp0[c];
    P.re1[c] = J.re1[c];
    P.re2[c] = J.re2[c];
  }
  P.depth = J.depth;
  P.max_depth = J.depth;
  P.irradiance = J.irradiance;
  P.kind = J.kind;
  P.eta = J.eta;
  P.n_base = (int64_t)J.n_emitters * J.n_tris * ((int64_t)1 << (2 * J.depth));
  P.capacity = J.capacity;
  P.count = J.count;
  P.status = J.status;
  P.u_lo = J.u_lo;
  P.u_hi = J.u_hi;
  P.v_lo = J.v_lo;
  P.v_hi = J.v_hi;
  P.e_lo = J.e_lo;
  P.e_hi = J.e_hi;
  P.emitter = J.emitter;
  P.tri0 = J.tri0;
  P.tri1 = J.tri1;
  P.cell = J.cell;
  P.flags = J.flags;
  P.e_hi_min = nullptr;
  P.q_out = nullptr;
  P.q_out_count = nullptr;
  P.q_cap = 0;
  return P;
}

// Persistent: one block per SM, a block barrier per round (uniform round count: the total is read
// from device memory by every thread).
__global__ void __launch_bounds__(kBoundThreads, 1) bound_batched_k(const bnb_bound_job* __restrict__ jobs,
                                                                   const int32_t* __restrict__ n_jobs_p,
                                                                   int32_t max_jobs,
                                                                   const int64_t* __restrict__ job_off) {
  const int n = max(0, min(*n_jobs_p, max_jobs));
  const int64_t total = job_off[n];
  const int64_t stride = (int64_t)gridDim.x * kBoundThreads;
  const int64_t rounds = (total + stride - 1) / stride;
  for (int64_t r = 0; r < rounds; ++r) {
    __syncthreads();
    const int64_t w = r * stride + (int64_t)blockIdx.x * kBoundThreads + threadIdx.x;
    if (w < total) {
      const int j = bound_job_of(job_off, n, w);
      const bnb_bound_job& J = jobs[j];
      if (J.capacity >= job_off[j + 1] - job_off[j]) {  // else reported by bound_jobs_k
        const BoundParams P = params_of(J);
        const int64_t lw = w - job_off[j];
        const int64_t per_tuple = (int64_t)1 << (2 * J.depth);
        const int64_t per_em = per_tuple * J.n_tris;
        const int e = (int)(lw / per_em);
        const int64_t rr = lw - (int64_t)e * per_em;
        const int t = (int)(rr / per_tuple);
        const uint32_t c = (uint32_t)(rr - (int64_t)t * per_tuple);
        if (J.kind == BNB_REFRACT)
          process_cell_refract_f32(P, e, t, c, J.depth, lw);
        else
          process_cell<float>(P, e, t, c, J.depth, lw);
      }
    }
  }
}

size_t bound_batch_ws_bytes(int32_t max_jobs) { return (size_t)round_up((int64_t)(max_jobs + 1) * 8, 256); }

cudaError_t launch_bound_batched(const bnb_bound_job* jobs, const int32_t* n_jobs, int32_t max_jobs, void* ws,
                                 cudaStream_t st) {
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int64_t* job_off = (int64_t*)ws;
  bound_jobs_k<<<1, kJobThreads, 0, st>>>(jobs, n_jobs, max_jobs, job_off);
  bound_batched_k<<<sms, kBoundThreads, 0, st>>>(jobs, n_jobs, max_jobs, job_off);
  return cudaGetLastError();
}

}  // namespace bnb
