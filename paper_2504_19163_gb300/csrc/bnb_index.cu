// Index kernel: bound storage on a uniform texture-space grid (Sec. 6.1 "Bound
// storage") with the per-tuple bound of Eq. eq_pertuple_b.
//
// Pass structure (all on the caller's stream, no host synchronization):
//   1. tuple_merge_k  one warp per tuple: the 4^D base records of a tuple are
//                     contiguous; their boxes are rasterized into a warp-private
//                     shared-memory tile over the tuple's footprint, keeping the
//                     max E_hi per grid cell, so each (grid cell, tuple) pair is
//                     emitted once.  Footprints larger than the tile fall back to
//                     per-record emission (merged in step 4).
//      overflow_k    children of split cells, one thread per record.
//   2. exclusive scan of the per-grid-cell counts.
//   3. scatter_k     counting sort of the entries by grid cell.
//   4. segsort_k     per grid cell: bitonic sort by tuple key in shared memory,
//                    duplicates merged with max (oversized cells: segsort_big_k).
//   5. scan of the merged counts -> CSR offsets; compact_k writes key/etilde.
// A record covers grid columns floor(u_lo G) .. min(G-1, floor(u_hi G)) (float32
// product), rows likewise.
#include <stdint.h>

#include <algorithm>

#include "bnb_internal.cuh"

namespace bnb {

// ------------------------------------------------------------------ scan
constexpr int kScanThreads = 256;
constexpr int kScanPer = 8;
constexpr int64_t kScanTile = kScanThreads * kScanPer;

__global__ void __launch_bounds__(kScanThreads) scan_tile_k(const int64_t* __restrict__ in, int64_t* __restrict__ out,
                                                             int64_t n, int64_t* __restrict__ tile_sums) {
  __shared__ int64_t wsum[kScanThreads / 32];
  const int64_t base = (int64_t)blockIdx.x * kScanTile;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  int64_t v[kScanPer];
  int64_t s = 0;
#pragma unroll
  for (int k = 0; k < kScanPer; ++k) {
    const int64_t i = base + (int64_t)tid * kScanPer + k;
    v[k] = i < n ? in[i] : 0;
    s += v[k];
  }
  int64_t x = s;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int64_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) wsum[wid] = x;
  __syncthreads();
  if (wid == 0) {
    int64_t w = lane < kScanThreads / 32 ? wsum[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int64_t y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    if (lane < kScanThreads / 32) wsum[lane] = w;
  }
  __syncthreads();
  int64_t ex = x - s + (wid > 0 ? wsum[wid - 1] : 0);
#pragma unroll
  for (int k = 0; k < kScanPer; ++k) {
    const int64_t i = base + (int64_t)tid * kScanPer + k;
    if (i < n) out[i] = ex;
    ex += v[k];
  }
  if (tid == kScanThreads - 1) tile_sums[blockIdx.x] = ex;
}

__global__ void scan_add_k(int64_t* __restrict__ out, int64_t n, const int64_t* __restrict__ offs) {
  const int64_t base = (int64_t)blockIdx.x * kScanTile;
  const int64_t add = offs[blockIdx.x];
  for (int64_t i = base + threadIdx.x; i < min(n, base + kScanTile); i += blockDim.x) out[i] += add;
}

__global__ void copy_one_k(const int64_t* __restrict__ src, int64_t* __restrict__ dst) { *dst = *src; }

size_t scan_ws_bytes(int64_t n) {
  size_t b = 0;
  while (n > 1) {
    const int64_t tiles = (n + kScanTile - 1) / kScanTile;
    b += (size_t)round_up((2 * tiles + 1) * (int64_t)sizeof(int64_t), 256);
    if (tiles == 1) break;
    n = tiles;
  }
  return b + 256;
}

cudaError_t launch_exclusive_scan(const int64_t* in, int64_t* out, int64_t n, void* ws, cudaStream_t st) {
  if (n <= 0) return cudaMemsetAsync(out, 0, sizeof(int64_t), st);
  const int64_t tiles = (n + kScanTile - 1) / kScanTile;
  int64_t* sums = (int64_t*)ws;
  int64_t* sums_scan = sums + tiles;
  void* next = (char*)ws + round_up((2 * tiles + 1) * (int64_t)sizeof(int64_t), 256);
  scan_tile_k<<<(unsigned)tiles, kScanThreads, 0, st>>>(in, out, n, sums);
  if (tiles == 1) {
    copy_one_k<<<1, 1, 0, st>>>(sums, out + n);
    return cudaGetLastError();
  }
  cudaError_t e = launch_exclusive_scan(sums, sums_scan, tiles, next, st);
  if (e != cudaSuccess) return e;
  scan_add_k<<<(unsigned)tiles, 256, 0, st>>>(out, n, sums_scan);
  copy_one_k<<<1, 1, 0, st>>>(sums_scan + tiles, out + n);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ index kernels
struct IndexParams {
  const float *u_lo, *u_hi, *v_lo, *v_hi, *e_hi;
  const int32_t *emitter, *tri0, *tri1;
  const uint32_t* flags;
  const int64_t* rec_count;  // device: records produced
  int64_t rec_capacity, n_base;
  int32_t cells_per_tuple;
  int64_t n_tuples;
  int32_t G;
  float m;
  // pre-merge entries
  uint32_t* pre_g;
  uint64_t* pre_key;
  float* pre_e;
  int64_t pre_cap;
  int64_t* pre_count;    // device
  int64_t* gcount;       // device, G*G (zeroed)
  int32_t* status;
};

__device__ __forceinline__ int grid_col(float x, int G) {
  const float p = __fmul_rn(fminf(fmaxf(x, 0.0f), 1.0f), (float)G);
  return min(G - 1, max(0, (int)floorf(p)));
}

__device__ __forceinline__ uint64_t tuple_key(int e, int t0, int t1) {
  return ((uint64_t)(uint32_t)e << 48) | ((uint64_t)(uint32_t)(t1 + 1) << 24) | (uint64_t)(uint32_t)t0;
}

__device__ __forceinline__ void emit(const IndexParams& P, int64_t slot, int g, uint64_t key, float e) {
  if (slot < P.pre_cap) {
    P.pre_g[slot] = (uint32_t)g;
    P.pre_key[slot] = key;
    P.pre_e[slot] = e;
    atomicAdd((unsigned long long*)(P.gcount + g), 1ull);
  } else {
    raise_status(P.status, BNB_ERR_CAPACITY);
  }
}

// Per-record emission (no merge): every grid cell of the record's box.
__device__ __forceinline__ void emit_record(const IndexParams& P, int64_t r) {
  const int i0 = grid_col(P.u_lo[r], P.G), i1 = grid_col(P.u_hi[r], P.G);
  const int j0 = grid_col(P.v_lo[r], P.G), j1 = grid_col(P.v_hi[r], P.G);
  const int64_t n = (int64_t)(i1 - i0 + 1) * (j1 - j0 + 1);
  const int64_t base = (int64_t)atomicAdd((unsigned long long*)P.pre_count, (unsigned long long)n);
  const uint64_t key = tuple_key(P.emitter[r], P.tri0[r], P.tri1[r]);
  const float e = P.e_hi[r];
  int64_t k = 0;
  for (int j = j0; j <= j1; ++j)
    for (int i = i0; i <= i1; ++i) emit(P, base + (k++), j * P.G + i, key, e);
}

constexpr int kMergeWarps = 4;
constexpr int kMergeTile = 512;  // grid cells per warp-private tile

__global__ void __launch_bounds__(32 * kMergeWarps) tuple_merge_k(IndexParams P) {
  __shared__ uint32_t tile[kMergeWarps][kMergeTile];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  uint32_t* loc = tile[wid];
  for (int64_t T = (int64_t)blockIdx.x * kMergeWarps + wid; T < P.n_tuples; T += (int64_t)gridDim.x * kMergeWarps) {
    const int64_t r0 = T * P.cells_per_tuple;
    int bi0 = 1 << 30, bi1 = -1, bj0 = 1 << 30, bj1 = -1;
    int64_t any_rec = -1;
    for (int k = lane; k < P.cells_per_tuple; k += 32) {
      const int64_t r = r0 + k;
      if (!(P.flags[r] & BNB_CELL_LIVE)) continue;
      any_rec = r;
      bi0 = min(bi0, grid_col(P.u_lo[r], P.G));
      bi1 = max(bi1, grid_col(P.u_hi[r], P.G));
      bj0 = min(bj0, grid_col(P.v_lo[r], P.G));
      bj1 = max(bj1, grid_col(P.v_hi[r], P.G));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      bi0 = min(bi0, __shfl_xor_sync(0xffffffffu, bi0, o));
      bi1 = max(bi1, __shfl_xor_sync(0xffffffffu, bi1, o));
      bj0 = min(bj0, __shfl_xor_sync(0xffffffffu, bj0, o));
      bj1 = max(bj1, __shfl_xor_sync(0xffffffffu, bj1, o));
      any_rec = max(any_rec, (int64_t)__shfl_xor_sync(0xffffffffu, (long long)any_rec, o));
    }
    if (any_rec < 0) continue;  // no live cell in this tuple
    const int W = bi1 - bi0 + 1, H = bj1 - bj0 + 1;
    if ((int64_t)W * H > kMergeTile) {
      for (int k = lane; k < P.cells_per_tuple; k += 32) {
        const int64_t r = r0 + k;
        if (P.flags[r] & BNB_CELL_LIVE) emit_record(P, r);
      }
      continue;
    }
    for (int k = lane; k < W * H; k += 32) loc[k] = 0u;
    __syncwarp();
    for (int k = lane; k < P.cells_per_tuple; k += 32) {
      const int64_t r = r0 + k;
      if (!(P.flags[r] & BNB_CELL_LIVE)) continue;
      const int i0 = grid_col(P.u_lo[r], P.G) - bi0, i1 = grid_col(P.u_hi[r], P.G) - bi0;
      const int j0 = grid_col(P.v_lo[r], P.G) - bj0, j1 = grid_col(P.v_hi[r], P.G) - bj0;
      // E_hi >= 0: the float bit pattern orders like the value; +1 marks "covered".
      const uint32_t bits = __float_as_uint(fmaxf(P.e_hi[r], 0.0f)) + 1u;
      for (int j = j0; j <= j1; ++j)
        for (int i = i0; i <= i1; ++i) atomicMax(&loc[j * W + i], bits);
    }
    __syncwarp();
    const uint64_t key = tuple_key(P.emitter[any_rec], P.tri0[any_rec], P.tri1[any_rec]);
    int cnt = 0;
    for (int k = lane; k < W * H; k += 32) cnt += loc[k] != 0u;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    long long base = 0;
    if (lane == 0) base = (long long)atomicAdd((unsigned long long*)P.pre_count, (unsigned long long)cnt);
    base = __shfl_sync(0xffffffffu, base, 0);
    int done = 0;
    for (int k0 = 0; k0 < W * H; k0 += 32) {
      const int k = k0 + lane;
      const uint32_t b = k < W * H ? loc[k] : 0u;
      const unsigned m = __ballot_sync(0xffffffffu, b != 0u);
      if (b != 0u) {
        const int pos = done + __popc(m & ((1u << lane) - 1u));
        const int g = (bj0 + k / W) * P.G + (bi0 + k % W);
        emit(P, base + pos, g, key, __uint_as_float(b - 1u));
      }
      done += __popc(m);
    }
    __syncwarp();
  }
}

__global__ void overflow_k(IndexParams P) {
  const int64_t n = min(*P.rec_count, P.rec_capacity);
  for (int64_t r = P.n_base + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n;
       r += (int64_t)gridDim.x * blockDim.x) {
    if (P.flags[r] & BNB_CELL_LIVE) emit_record(P, r);
  }
}

__global__ void scatter_k(const uint32_t* __restrict__ pre_g, const uint64_t* __restrict__ pre_key,
                          const float* __restrict__ pre_e, const int64_t* __restrict__ pre_count, int64_t pre_cap,
                          const int64_t* __restrict__ goff, int64_t* __restrict__ gcur, uint64_t* __restrict__ s_key,
                          float* __restrict__ s_e) {
  const int64_t n = min(*pre_count, pre_cap);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t g = pre_g[i];
    const int64_t pos = goff[g] + (int64_t)atomicAdd((unsigned long long*)(gcur + g), 1ull);
    s_key[pos] = pre_key[i];
    s_e[pos] = pre_e[i];
  }
}

// All-ascending bitonic network over n elements (virtual +inf padding to a power of two):
// every comparator puts the smaller key at the lower index, so padding never moves.
template <typename KeyAt, typename Swap>
__device__ __forceinline__ void bitonic_all_asc(int n, int n2, KeyAt key, Swap swp, bool block_sync) {
  for (int k = 2; k <= n2; k <<= 1) {
    for (int i = threadIdx.x; i < n2 / 2; i += blockDim.x) {
      const int h = k >> 1, blk = i / h, off = i % h;
      const int a = blk * k + off, b = blk * k + k - 1 - off;
      if (b < n && key(b) < key(a)) swp(a, b);
    }
    if (block_sync) __syncthreads();
    for (int j = k >> 2; j >= 1; j >>= 1) {
      for (int i = threadIdx.x; i < n2 / 2; i += blockDim.x) {
        const int a = (i / j) * 2 * j + i % j, b = a + j;
        if (b < n && key(b) < key(a)) swp(a, b);
      }
      if (block_sync) __syncthreads();
    }
  }
}

constexpr int kSegCap = 1024;
constexpr int kSegThreads = 128;

__global__ void __launch_bounds__(kSegThreads) segsort_k(const int64_t* __restrict__ goff, uint64_t* __restrict__ s_key,
                                                         float* __restrict__ s_e, int64_t* __restrict__ rcount,
                                                         int32_t* __restrict__ big, int32_t* __restrict__ n_big,
                                                         int n_cells) {
  __shared__ uint64_t K[kSegCap];
  __shared__ float V[kSegCap];
  const int g = blockIdx.x;
  if (g >= n_cells) return;
  const int64_t s = goff[g];
  const int64_t nn = goff[g + 1] - s;
  const int n = (int)(nn < ((int64_t)1 << 30) ? nn : ((int64_t)1 << 30));
  if (n == 0) {
    if (threadIdx.x == 0) rcount[g] = 0;
    return;
  }
  if (n > kSegCap) {
    if (threadIdx.x == 0) {
      rcount[g] = 0;
      big[atomicAdd(n_big, 1)] = g;
    }
    return;
  }
  int n2 = 1;
  while (n2 < n) n2 <<= 1;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    K[i] = s_key[s + i];
    V[i] = s_e[s + i];
  }
  __syncthreads();
  bitonic_all_asc(
      n, n2, [&](int i) { return K[i]; },
      [&](int a, int b) {
        const uint64_t tk = K[a];
        K[a] = K[b];
        K[b] = tk;
        const float tv = V[a];
        V[a] = V[b];
        V[b] = tv;
      },
      true);
  // Merge runs of equal keys (max of E~) in parallel: each thread takes a contiguous chunk, counts
  // the run heads in it, a block scan turns the counts into output positions, and each head writes
  // its key with the max over its run (runs are short: a tuple is usually listed once per cell).
  const int per = (n + kSegThreads - 1) / kSegThreads;
  const int i0 = min(n, (int)threadIdx.x * per), i1 = min(n, i0 + per);
  int heads = 0;
  for (int i = i0; i < i1; ++i) heads += (i == 0 || K[i] != K[i - 1]);
  __shared__ int wsum[kSegThreads / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int incl = heads;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) wsum[wid] = incl;
  __syncthreads();
  int before = 0;
  for (int w = 0; w < wid; ++w) before += wsum[w];
  int pos = before + incl - heads;
  for (int i = i0; i < i1; ++i) {
    if (i == 0 || K[i] != K[i - 1]) {
      float m = V[i];
      for (int j = i + 1; j < n && K[j] == K[i]; ++j) m = fmaxf(m, V[j]);
      s_key[s + pos] = K[i];
      s_e[s + pos] = m;
      ++pos;
    }
  }
  if (threadIdx.x == kSegThreads - 1) {
    int total = 0;
    for (int w = 0; w < kSegThreads / 32; ++w) total += wsum[w];
    rcount[g] = total;
  }
}

__global__ void __launch_bounds__(512) segsort_big_k(const int64_t* __restrict__ goff, uint64_t* __restrict__ s_key,
                                                     float* __restrict__ s_e, int64_t* __restrict__ rcount,
                                                     const int32_t* __restrict__ big,
                                                     const int32_t* __restrict__ n_big) {
  for (int b = blockIdx.x; b < *n_big; b += gridDim.x) {
    const int g = big[b];
    const int64_t s = goff[g];
    const int n = (int)(goff[g + 1] - s);
    int n2 = 1;
    while (n2 < n) n2 <<= 1;
    uint64_t* K = s_key + s;
    float* V = s_e + s;
    bitonic_all_asc(
        n, n2, [&](int i) { return K[i]; },
        [&](int a, int c) {
          const uint64_t tk = K[a];
          K[a] = K[c];
          K[c] = tk;
          const float tv = V[a];
          V[a] = V[c];
          V[c] = tv;
        },
        true);
    __syncthreads();
    if (threadIdx.x == 0) {
      int o = 0;
      for (int i = 0; i < n; ++i) {
        if (o > 0 && K[o - 1] == K[i]) {
          V[o - 1] = fmaxf(V[o - 1], V[i]);
        } else {
          K[o] = K[i];
          V[o] = V[i];
          ++o;
        }
      }
      rcount[g] = o;
    }
    __syncthreads();
  }
}

__global__ void compact_k(const int64_t* __restrict__ goff, const uint64_t* __restrict__ s_key,
                          const float* __restrict__ s_e, const int64_t* __restrict__ offsets, int n_cells, float m,
                          int64_t capacity, uint64_t* __restrict__ key, float* __restrict__ et,
                          int64_t* __restrict__ count, int32_t* __restrict__ status) {
  const int lane = threadIdx.x & 31;
  const int g = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (g == 0 && lane == 0) {
    count[0] = offsets[n_cells];
    if (offsets[n_cells] > capacity) raise_status(status, BNB_ERR_CAPACITY);
  }
  if (g >= n_cells) return;
  const int64_t src = goff[g], dst = offsets[g], n = offsets[g + 1] - dst;
  for (int64_t i = lane; i < n; i += 32) {
    if (dst + i < capacity) {
      key[dst + i] = s_key[src + i];
      et[dst + i] = __fmul_ru(m, s_e[src + i]);
    }
  }
}

__global__ void store_pre_count_k(const int64_t* __restrict__ pre_count, int64_t* __restrict__ count) {
  count[1] = *pre_count;
}

// ------------------------------------------------------------------ host side
struct IndexWs {
  int64_t* gcount;   // G*G
  int64_t* goff;     // G*G + 1
  int64_t* gcur;     // G*G
  int64_t* rcount;   // G*G
  int64_t* pre_count;
  int32_t* n_big;
  int32_t* big;      // G*G
  uint32_t* pre_g;
  uint64_t* pre_key;
  float* pre_e;
  uint64_t* s_key;
  float* s_e;
  void* scan;
  size_t bytes;
};

static IndexWs carve_index_ws(void* base, int32_t G, int64_t pre_cap) {
  IndexWs w{};
  const int64_t cells = (int64_t)G * G;
  size_t o = 0;
  auto take = [&](size_t b) -> char* {
    char* p = (char*)base + o;
    o += (size_t)round_up((int64_t)b, 256);
    return p;
  };
  w.gcount = (int64_t*)take(cells * 8);
  w.gcur = (int64_t*)take(cells * 8);
  w.pre_count = (int64_t*)take(8);
  w.n_big = (int32_t*)take(8);
  const size_t zero_end = o;  // everything above is zeroed per call
  w.goff = (int64_t*)take((cells + 1) * 8);
  w.rcount = (int64_t*)take(cells * 8);
  w.big = (int32_t*)take(cells * 4);
  w.pre_g = (uint32_t*)take(pre_cap * 4);
  w.pre_key = (uint64_t*)take(pre_cap * 8);
  w.pre_e = (float*)take(pre_cap * 4);
  w.s_key = (uint64_t*)take(pre_cap * 8);
  w.s_e = (float*)take(pre_cap * 4);
  w.scan = take(scan_ws_bytes(cells + 1));
  w.bytes = o;
  (void)zero_end;
  return w;
}

size_t index_ws_bytes(int32_t G, int64_t pre_cap) { return carve_index_ws(nullptr, G, pre_cap).bytes; }

static int sm_count() {
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms;
}

cudaError_t launch_build_index(const bnb_cell_bounds* c, float m, int64_t pre_cap, bnb_index* out, void* ws,
                               cudaStream_t st) {
  const int32_t G = out->grid_res;
  const int64_t cells = (int64_t)G * G;
  IndexWs w = carve_index_ws(ws, G, pre_cap);
  cudaError_t e;
  // zero the counters (gcount, gcur, pre_count, n_big are laid out first and contiguous)
  const size_t zero_bytes = (size_t)((char*)w.goff - (char*)w.gcount);
  if ((e = cudaMemsetAsync(w.gcount, 0, zero_bytes, st)) != cudaSuccess) return e;
  IndexParams P{};
  P.u_lo = c->u_lo;
  P.u_hi = c->u_hi;
  P.v_lo = c->v_lo;
  P.v_hi = c->v_hi;
  P.e_hi = c->e_hi;
  P.emitter = c->emitter;
  P.tri0 = c->tri0;
  P.tri1 = c->tri1;
  P.flags = c->flags;
  P.rec_count = c->count;
  P.rec_capacity = c->capacity;
  P.n_base = c->n_base;
  P.cells_per_tuple = 1 << (2 * c->depth);
  P.n_tuples = c->n_base / P.cells_per_tuple;
  P.G = G;
  P.m = m;
  P.pre_g = w.pre_g;
  P.pre_key = w.pre_key;
  P.pre_e = w.pre_e;
  P.pre_cap = pre_cap;
  P.pre_count = w.pre_count;
  P.gcount = w.gcount;
  P.status = out->status;
  const int sms = sm_count();
  if (P.n_tuples > 0) {
    const int64_t blocks = std::min<int64_t>((P.n_tuples + kMergeWarps - 1) / kMergeWarps, (int64_t)sms * 64);
    tuple_merge_k<<<(unsigned)blocks, 32 * kMergeWarps, 0, st>>>(P);
  }
  overflow_k<<<sms * 2, 256, 0, st>>>(P);
  if ((e = launch_exclusive_scan(w.gcount, w.goff, cells, w.scan, st)) != cudaSuccess) return e;
  scatter_k<<<sms * 8, 256, 0, st>>>(w.pre_g, w.pre_key, w.pre_e, w.pre_count, pre_cap, w.goff, w.gcur, w.s_key,
                                      w.s_e);
  segsort_k<<<(unsigned)cells, kSegThreads, 0, st>>>(w.goff, w.s_key, w.s_e, w.rcount, w.big, w.n_big, (int)cells);
  segsort_big_k<<<sms, 512, 0, st>>>(w.goff, w.s_key, w.s_e, w.rcount, w.big, w.n_big);
  if ((e = launch_exclusive_scan(w.rcount, out->offsets, cells, w.scan, st)) != cudaSuccess) return e;
  compact_k<<<(unsigned)((cells + 7) / 8), 256, 0, st>>>(w.goff, w.s_key, w.s_e, out->offsets, (int)cells, m,
                                                          out->capacity, out->key, out->etilde, out->count,
                                                          out->status);
  store_pre_count_k<<<1, 1, 0, st>>>(w.pre_count, out->count);
  return cudaGetLastError();
}

}  // namespace bnb
