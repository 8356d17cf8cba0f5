// Batched rendering pass: many jobs (one request's shading points against one resident
// (scene, emitter) index) in one launch sequence.
//
// The job table and the job count live in device memory and every launch is sized from the
// batch capacities only (max points, worklist capacity), so the same launch sequence can be
// captured once in a CUDA graph and replayed for any batch that fits: the host only rewrites
// the job table between replays.  Per point and per selected tuple the arithmetic is the one
// of bnb_sample_and_solve (Algorithm 1 with P = min(gamma E~, 1), Newton with float64 polish),
// with the point's index *within its job* as the Philox counter, so a job's result does not
// depend on the other jobs in the batch.
#include <stdint.h>

#include <algorithm>

#include "bnb_internal.cuh"
#include "bnb_path.cuh"

namespace bnb {

struct BatchWs {
  int64_t* job_off;  // max_jobs + 1
  int64_t* n_sel;    // max_points
  int64_t* woff;     // max_points + 1
  int64_t* wl_point; // worklist: global point
  uint64_t* wl_key;
  float* wl_p;
  float* contrib;
  int64_t* pl_count;  // float32 survivors handed to the float64 polish
  int64_t* pl_idx;
  float *pl_u, *pl_v;
  void* scan;
  size_t bytes;
};

static BatchWs carve_batch_ws(void* base, const bnb_batch_cfg* c) {
  BatchWs w{};
  size_t o = 0;
  auto take = [&](size_t b) -> char* {
    char* p = (char*)base + o;
    o += (size_t)round_up((int64_t)b, 256);
    return p;
  };
  w.job_off = (int64_t*)take((size_t)(c->max_jobs + 1) * 8);
  w.n_sel = (int64_t*)take((size_t)c->max_points * 8);
  w.woff = (int64_t*)take((size_t)(c->max_points + 1) * 8);
  w.wl_point = (int64_t*)take((size_t)c->worklist_capacity * 8);
  w.wl_key = (uint64_t*)take((size_t)c->worklist_capacity * 8);
  w.wl_p = (float*)take((size_t)c->worklist_capacity * 4);
  w.contrib = (float*)take((size_t)c->worklist_capacity * 4);
  w.pl_count = (int64_t*)take(8);
  w.pl_idx = (int64_t*)take((size_t)c->worklist_capacity * 8);
  w.pl_u = (float*)take((size_t)c->worklist_capacity * 4);
  w.pl_v = (float*)take((size_t)c->worklist_capacity * 4);
  w.scan = take(scan_ws_bytes(c->max_points));
  w.bytes = o;
  return w;
}

size_t batch_ws_bytes(const bnb_batch_cfg* c) { return carve_batch_ws(nullptr, c).bytes; }

// Prefix sums of the jobs' point counts: one block of kJobScanThreads threads, each summing a
// contiguous chunk of jobs, then a block-wide exclusive scan of the chunk sums.
constexpr int kJobScanThreads = 1024;

__global__ void __launch_bounds__(kJobScanThreads) job_offsets_k(const bnb_job* __restrict__ jobs,
                                                               const int32_t* __restrict__ n_jobs_p,
                                                               int32_t max_jobs, int64_t max_points,
                                                               int64_t* __restrict__ job_off,
                                                               int32_t* __restrict__ status) {
  __shared__ int64_t warp_sum[kJobScanThreads / 32];
  const int32_t n_req = *n_jobs_p;
  const int32_t n = max(0, min(n_req, max_jobs));
  const int chunk = (max_jobs + kJobScanThreads - 1) / kJobScanThreads;
  const int j0 = threadIdx.x * chunk;
  const int j1 = min(j0 + chunk, n);
  int64_t mine = 0;
  for (int j = j0; j < j1; ++j) mine += (jobs[j].n_points > 0 ? jobs[j].n_points : (int64_t)0);
  // inclusive scan across the block
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
  int64_t acc = x - mine + (wid > 0 ? warp_sum[wid - 1] : 0);  // exclusive prefix of this chunk
  if (threadIdx.x == 0) job_off[0] = 0;
  for (int j = j0; j < min(j0 + chunk, max_jobs); ++j) {
    if (j < n) acc += (jobs[j].n_points > 0 ? jobs[j].n_points : (int64_t)0);
    job_off[j + 1] = acc;
  }
  if (threadIdx.x == kJobScanThreads - 1 && (warp_sum[31] > max_points || n_req > max_jobs || n_req < 0))
    raise_status(status, BNB_ERR_CAPACITY);
}

__device__ __forceinline__ int job_of(const int64_t* __restrict__ job_off, int n_jobs, int64_t p) {
  int lo = 0, hi = n_jobs - 1;  // largest j with job_off[j] <= p
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (job_off[mid] <= p) lo = mid; else hi = mid - 1;
  }
  return lo;
}

struct BatchParams {
  const bnb_job* jobs;
  const int32_t* n_jobs;
  int32_t max_jobs;
  int64_t max_points;
  const int64_t* job_off;
  int64_t* n_sel;
  const int64_t* woff;
  int64_t wl_cap;
  int64_t* wl_point;
  uint64_t* wl_key;
  float* wl_p;
  float* contrib;
  int64_t* pl_count;
  int64_t* pl_idx;
  float *pl_u, *pl_v;
  int64_t* counters;
  int32_t* status;
  int32_t newton_iters, polish_iters;
  float tol;
};

template <bool FILL>
__global__ void __launch_bounds__(512) sample_b_k(BatchParams B) {
  const int nj = max(0, min(*B.n_jobs, B.max_jobs));
  const int64_t total = min(B.job_off[nj], B.max_points);
  long long nu = 0, ns = 0;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < B.max_points;
       p += (int64_t)gridDim.x * blockDim.x) {
    if (p >= total) {
      if (!FILL) B.n_sel[p] = 0;
      continue;
    }
    const int j = job_of(B.job_off, nj, p);
    const bnb_job& J = B.jobs[j];
    const int64_t lp = p - B.job_off[j];
    const int G = J.grid_res;
    const int g = grid_col_s(J.sv[lp], G) * G + grid_col_s(J.su[lp], G);
    const int64_t s = J.offsets[g];
    const int64_t e = min(J.offsets[g + 1], J.index_capacity);
    int64_t cnt = 0;
    int64_t out = FILL ? B.woff[p] : 0;
    const uint8_t* on = J.emitter_on;
    int64_t listed = 0;
    for (int64_t k = s; k < e; ++k) {
      const uint64_t key = J.key[k];
      if (on != nullptr) {
        const int em = (int)(key >> 48);
        if (em >= J.n_emitters || on[em] == 0) continue;
      }
      ++listed;
      const float Pt = fminf(__fmul_ru(J.gamma, J.etilde[k]), 1.0f);
      if (uniform24(J.seed, lp, key) < Pt) {
        if (FILL) {
          if (out < B.wl_cap) {
            B.wl_point[out] = p;
            B.wl_key[out] = key;
            B.wl_p[out] = Pt;
          } else {
            raise_status(B.status, BNB_ERR_CAPACITY);
          }
          ++out;
        }
        ++cnt;
      }
    }
    if (!FILL) B.n_sel[p] = cnt;
    nu += listed;
    ns += cnt;
  }
  if (!FILL) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      nu += __shfl_xor_sync(0xffffffffu, nu, o);
      ns += __shfl_xor_sync(0xffffffffu, ns, o);
    }
    if ((threadIdx.x & 31) == 0) {
      if (nu) atomicAdd((unsigned long long*)&B.counters[0], (unsigned long long)nu);
      if (ns) atomicAdd((unsigned long long*)&B.counters[1], (unsigned long long)ns);
    }
  }
}

// float32 Newton phase over every selection of the batch (see newton32); survivors are listed.
__global__ void __launch_bounds__(512) solve32_b_k(BatchParams B) {
  const int nj = max(0, min(*B.n_jobs, B.max_jobs));
  const int64_t n = min(B.woff[B.max_points], B.wl_cap);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p = B.wl_point[i];
    const int j = job_of(B.job_off, nj, p);
    const bnb_job& J = B.jobs[j];
    const int64_t lp = p - B.job_off[j];
    const uint64_t k = B.wl_key[i];
    const int e = (int)(k >> 48), t = (int)(k & 0xFFFFFFull);
    bool need = false;
    float u = 0.0f, v = 0.0f;
    if (t < J.n_tris && e < J.n_emitters) {
      float pf[3][3], nf[3][3];
      load_tri_s((const float4*)J.packed_tris, t, pf, nf);
      const float x0[3] = {__ldg(J.ex + e), __ldg(J.ey + e), __ldg(J.ez + e)};
      if (J.kind == BNB_REFRACT)
        need = newton32<true>(pf, nf, x0, __ldg(J.ei + e), J.rp0, J.re1, J.re2, J.su[lp], J.sv[lp], B.newton_iters,
                              J.eta, u, v);
      else
        need = newton32<false>(pf, nf, x0, __ldg(J.ei + e), J.rp0, J.re1, J.re2, J.su[lp], J.sv[lp], B.newton_iters,
                               J.eta, u, v);
    }
    if (!need) B.contrib[i] = 0.0f;
    const int64_t q = warp_append(need, B.pl_count);
    if (need) {
      B.pl_idx[q] = i;
      B.pl_u[q] = u;
      B.pl_v[q] = v;
    }
  }
}

// float64 polish of the listed selections, acceptance tests, contribution E(root) / P.
__global__ void __launch_bounds__(512) polish_b_k(BatchParams B) {
  const int nj = max(0, min(*B.n_jobs, B.max_jobs));
  const int64_t n = *B.pl_count;
  long long roots = 0;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = B.pl_idx[q];
    const int64_t p = B.wl_point[i];
    const int j = job_of(B.job_off, nj, p);
    const bnb_job& J = B.jobs[j];
    const int64_t lp = p - B.job_off[j];
    const uint64_t k = B.wl_key[i];
    const int e = (int)(k >> 48), t = (int)(k & 0xFFFFFFull);
    float pf[3][3], nf[3][3];
    load_tri_s((const float4*)J.packed_tris, t, pf, nf);
    const float x0[3] = {__ldg(J.ex + e), __ldg(J.ey + e), __ldg(J.ez + e)};
    const double E =
        J.kind == BNB_REFRACT
            ? polish64<true>(pf, nf, x0, __ldg(J.ei + e), J.rp0, J.re1, J.re2, J.su[lp], J.sv[lp], B.polish_iters,
                             B.tol, J.eta, B.pl_u[q], B.pl_v[q])
            : polish64<false>(pf, nf, x0, __ldg(J.ei + e), J.rp0, J.re1, J.re2, J.su[lp], J.sv[lp], B.polish_iters,
                              B.tol, J.eta, B.pl_u[q], B.pl_v[q]);
    float c = 0.0f;
    if (E >= 0.0) {
      c = (float)(E / (double)B.wl_p[i]);
      ++roots;
    }
    B.contrib[i] = c;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) roots += __shfl_xor_sync(0xffffffffu, roots, o);
  if ((threadIdx.x & 31) == 0 && roots) atomicAdd((unsigned long long*)&B.counters[2], (unsigned long long)roots);
}

__global__ void __launch_bounds__(512) reduce_b_k(BatchParams B) {
  const int nj = max(0, min(*B.n_jobs, B.max_jobs));
  const int64_t total = min(B.job_off[nj], B.max_points);
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < total; p += (int64_t)gridDim.x * blockDim.x) {
    const int j = job_of(B.job_off, nj, p);
    const int64_t a = B.woff[p], b = min(B.woff[p + 1], B.wl_cap);
    float s = 0.0f;
    for (int64_t i = a; i < b; ++i) s += B.contrib[i];
    B.jobs[j].E_out[p - B.job_off[j]] = s;
  }
}

cudaError_t launch_sample_and_solve_batched(const bnb_job* jobs, const int32_t* n_jobs, const bnb_batch_cfg* c,
                                            bnb_sample_stats* stats, void* ws, cudaStream_t st) {
  BatchWs w = carve_batch_ws(ws, c);
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int threads = c->block_threads > 0 ? c->block_threads : 256;
  const int per_sm = c->blocks_per_sm > 0 ? c->blocks_per_sm : 8;
  BatchParams B{};
  B.jobs = jobs;
  B.n_jobs = n_jobs;
  B.max_jobs = c->max_jobs;
  B.max_points = c->max_points;
  B.job_off = w.job_off;
  B.n_sel = w.n_sel;
  B.woff = w.woff;
  B.wl_cap = c->worklist_capacity;
  B.wl_point = w.wl_point;
  B.wl_key = w.wl_key;
  B.wl_p = w.wl_p;
  B.contrib = w.contrib;
  B.pl_count = w.pl_count;
  B.pl_idx = w.pl_idx;
  B.pl_u = w.pl_u;
  B.pl_v = w.pl_v;
  B.counters = stats->counters;
  B.status = stats->status;
  B.newton_iters = c->newton_iters;
  B.polish_iters = c->polish_iters;
  B.tol = c->tol;
  job_offsets_k<<<1, kJobScanThreads, 0, st>>>(jobs, n_jobs, c->max_jobs, c->max_points, w.job_off, stats->status);
  if (c->max_points == 0) return cudaGetLastError();
  const int64_t pblocks = std::min<int64_t>((c->max_points + threads - 1) / threads, (int64_t)sms * per_sm);
  sample_b_k<false><<<(unsigned)pblocks, threads, 0, st>>>(B);
  cudaError_t e = launch_exclusive_scan(w.n_sel, w.woff, c->max_points, w.scan, st);
  if (e != cudaSuccess) return e;
  sample_b_k<true><<<(unsigned)pblocks, threads, 0, st>>>(B);
  if ((e = cudaMemsetAsync(w.pl_count, 0, sizeof(int64_t), st)) != cudaSuccess) return e;
  solve32_b_k<<<sms * per_sm, threads, 0, st>>>(B);
  polish_b_k<<<sms * per_sm, threads, 0, st>>>(B);
  reduce_b_k<<<(unsigned)pblocks, threads, 0, st>>>(B);
  return cudaGetLastError();
}

}  // namespace bnb
