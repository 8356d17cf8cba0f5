// Index kernel: bound storage on a uniform texture-space grid (Sec. 6.1 "Bound
// storage") with the per-tuple bound of Eq. eq_pertuple_b.
//
// Pass structure (all on the caller's stream, no host synchronization):
//   1. tuple_merge64_k / tuple_merge_k  one warp per tuple: the 4^D base records
//                     of a tuple are contiguous; their boxes are rasterized into a
//                     warp-private shared-memory tile over the tuple's footprint,
//                     keeping the max E_hi per grid cell, so each (grid cell, tuple)
//                     pair is emitted once (tuples of <= 64 cells hold their records
//                     in registers, one round of loads).  Footprints larger than the
//                     tile fall back to per-record emission (merged in step 4).
//      overflow_k    children of split cells, one thread per record.
//   2. exclusive scan of the per-grid-cell counts.
//   3. scatter_k     counting sort of the entries by grid cell.
//   4. segrank_k     a warp per grid cell: lists of <= 128 entries by rank (each
//                    entry's place in key order is the number of keys below it,
//                    counted against the list in shared memory), duplicates merged
//                    with max.  Per-record emission is the only source of duplicate
//                    keys; when none happened, segrank_k writes the final CSR directly
//                    (the merged counts equal the counts of step 2), and also orders
//                    lists of <= 512 entries whose keys have an order-preserving
//                    32-bit form, by a warp bitonic sort.  Other lists: segsort_k
//                    (block bitonic sort, <= 1024) and segsort_big_k.
//   5. scan of the merged counts -> CSR offsets; compact_k writes key/etilde of
//      the cells not written in step 4.
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
// A pre-merge or grid-cell-sorted entry: one 16-byte store or load per entry.
struct __align__(16) Ent {
  uint64_t key;
  float e;
  uint32_t g;  // grid cell
};

// The pre-merge entries are split into kPreParts partitions of part_cap entries, each with its own
// counter (128 bytes apart): a tuple T (or a record r emitted on its own) appends to the partition
// given by the top 6 bits of T * 2654435761 mod 2^32 (Knuth's multiplicative hash, which spreads
// the regular triangle numbering of a mesh evenly), so no single counter takes every tuple's
// reservation.  The capacity needed is kPreParts x the largest partition's count, which depends
// only on the records.
constexpr int kPreParts = 64;
constexpr int kPartStride = 16;  // int64 units between partition counters

__device__ __forceinline__ int part_of(int64_t t) { return (int)(((uint32_t)t * 2654435761u) >> 26); }

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
  Ent* pre;
  int64_t part_cap;
  int64_t* pre_count;    // device, kPreParts counters kPartStride apart (zeroed)
  int64_t* gcount;       // device, G*G (zeroed)
  int32_t* dup;          // device (zeroed): set when an entry was emitted per record
  int32_t* status;
};

__device__ __forceinline__ int grid_col(float x, int G) {
  const float p = __fmul_rn(fminf(fmaxf(x, 0.0f), 1.0f), (float)G);
  return min(G - 1, max(0, (int)floorf(p)));
}

__device__ __forceinline__ uint64_t tuple_key(int e, int t0, int t1) {
  return ((uint64_t)(uint32_t)e << 48) | ((uint64_t)(uint32_t)(t1 + 1) << 24) | (uint64_t)(uint32_t)t0;
}

__device__ __forceinline__ int64_t reserve(const IndexParams& P, int part, int64_t n) {
  return (int64_t)atomicAdd((unsigned long long*)(P.pre_count + part * kPartStride), (unsigned long long)n);
}

__device__ __forceinline__ void emit(const IndexParams& P, int part, int64_t slot, int g, uint64_t key, float e) {
  if (slot < P.part_cap) {
    Ent x;
    x.key = key;
    x.e = e;
    x.g = (uint32_t)g;
    P.pre[part * P.part_cap + slot] = x;
    atomicAdd((unsigned long long*)(P.gcount + g), 1ull);
  } else {
    raise_status(P.status, BNB_ERR_CAPACITY);
  }
}

// Per-record emission (no merge): every grid cell of the record's box.
__device__ __forceinline__ void emit_record(const IndexParams& P, int64_t r) {
  *P.dup = 1;
  const int i0 = grid_col(P.u_lo[r], P.G), i1 = grid_col(P.u_hi[r], P.G);
  const int j0 = grid_col(P.v_lo[r], P.G), j1 = grid_col(P.v_hi[r], P.G);
  const int64_t n = (int64_t)(i1 - i0 + 1) * (j1 - j0 + 1);
  const int part = part_of(r);
  const int64_t base = reserve(P, part, n);
  const uint64_t key = tuple_key(P.emitter[r], P.tri0[r], P.tri1[r]);
  const float e = P.e_hi[r];
  int64_t k = 0;
  for (int j = j0; j <= j1; ++j)
    for (int i = i0; i <= i1; ++i) emit(P, part, base + (k++), j * P.G + i, key, e);
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
    const int part = part_of(T);
    long long base = 0;
    if (lane == 0) base = (long long)reserve(P, part, cnt);
    base = __shfl_sync(0xffffffffu, base, 0);
    int done = 0;
    for (int k0 = 0; k0 < W * H; k0 += 32) {
      const int k = k0 + lane;
      const uint32_t b = k < W * H ? loc[k] : 0u;
      const unsigned m = __ballot_sync(0xffffffffu, b != 0u);
      if (b != 0u) {
        const int pos = done + __popc(m & ((1u << lane) - 1u));
        const int g = (bj0 + k / W) * P.G + (bi0 + k % W);
        emit(P, part, base + pos, g, key, __uint_as_float(b - 1u));
      }
      done += __popc(m);
    }
    __syncwarp();
  }
}

// One tuple of at most 64 records held two per lane (record lane + 32 c in slot c): footprint,
// rasterization into the warp's tile with the max E_hi per grid cell, and emission of one entry
// per covered grid cell.  The key comes from the tuple's first record (all 4^D records of a tuple
// share it) unless that record is dead.
__device__ __forceinline__ void merge_tuple64(const IndexParams& P, int64_t T, int64_t r0, uint32_t* loc,
                                              const float (&ulo)[2], const float (&uhi)[2], const float (&vlo)[2],
                                              const float (&vhi)[2], const float (&eh)[2], const uint32_t (&fl)[2],
                                              int e0, int t0, int t1) {
  const int lane = threadIdx.x & 31;
  int ci0[2], ci1[2], cj0[2], cj1[2];
  int bi0 = 1 << 30, bi1 = -1, bj0 = 1 << 30, bj1 = -1;
#pragma unroll
  for (int c = 0; c < 2; ++c) {
    ci0[c] = grid_col(ulo[c], P.G);
    ci1[c] = grid_col(uhi[c], P.G);
    cj0[c] = grid_col(vlo[c], P.G);
    cj1[c] = grid_col(vhi[c], P.G);
    if (fl[c] & BNB_CELL_LIVE) {
      bi0 = min(bi0, ci0[c]);
      bi1 = max(bi1, ci1[c]);
      bj0 = min(bj0, cj0[c]);
      bj1 = max(bj1, cj1[c]);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    bi0 = min(bi0, __shfl_xor_sync(0xffffffffu, bi0, o));
    bi1 = max(bi1, __shfl_xor_sync(0xffffffffu, bi1, o));
    bj0 = min(bj0, __shfl_xor_sync(0xffffffffu, bj0, o));
    bj1 = max(bj1, __shfl_xor_sync(0xffffffffu, bj1, o));
  }
  if (bi1 < 0) return;  // no live record in this tuple
  const int W = bi1 - bi0 + 1, H = bj1 - bj0 + 1;
  if ((int64_t)W * H > kMergeTile) {
#pragma unroll
    for (int c = 0; c < 2; ++c)
      if (fl[c] & BNB_CELL_LIVE) emit_record(P, r0 + lane + 32 * c);
    return;
  }
  for (int k = lane; k < W * H; k += 32) loc[k] = 0u;
  __syncwarp();
#pragma unroll
  for (int c = 0; c < 2; ++c) {
    if (!(fl[c] & BNB_CELL_LIVE)) continue;
    // E_hi >= 0: the float bit pattern orders like the value; +1 marks "covered".
    const uint32_t bits = __float_as_uint(fmaxf(eh[c], 0.0f)) + 1u;
    for (int j = cj0[c] - bj0; j <= cj1[c] - bj0; ++j)
      for (int i = ci0[c] - bi0; i <= ci1[c] - bi0; ++i) atomicMax(&loc[j * W + i], bits);
  }
  __syncwarp();
  // the key of the tuple's first live record (the first record's, loaded above, unless it is dead)
  uint64_t key = tuple_key(e0, t0, t1);
  const unsigned l0 = __ballot_sync(0xffffffffu, (fl[0] & BNB_CELL_LIVE) != 0u);
  const unsigned l1 = __ballot_sync(0xffffffffu, (fl[1] & BNB_CELL_LIVE) != 0u);
  const int first = l0 ? __ffs(l0) - 1 : 32 + __ffs(l1) - 1;
  if (first != 0) key = tuple_key(P.emitter[r0 + first], P.tri0[r0 + first], P.tri1[r0 + first]);
  int cnt = 0;
  for (int k = lane; k < W * H; k += 32) cnt += loc[k] != 0u;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
  const int part = part_of(T);
  long long base = 0;
  if (lane == 0) base = (long long)reserve(P, part, cnt);
  base = __shfl_sync(0xffffffffu, base, 0);
  int done = 0;
  for (int k0 = 0; k0 < W * H; k0 += 32) {
    const int k = k0 + lane;
    const uint32_t b = k < W * H ? loc[k] : 0u;
    const unsigned m = __ballot_sync(0xffffffffu, b != 0u);
    if (b != 0u) {
      const int pos = done + __popc(m & ((1u << lane) - 1u));
      const int g = (bj0 + k / W) * P.G + (bi0 + k % W);
      emit(P, part, base + pos, g, key, __uint_as_float(b - 1u));
    }
    done += __popc(m);
  }
  __syncwarp();
}

// Tuples of at most 64 records: each lane holds two records in registers, loaded in one round
// (box, E_hi and flags of both at once), so the footprint and the rasterization need no second
// read; the tuple's key is loaded beside them from its first record.
__global__ void __launch_bounds__(32 * kMergeWarps) tuple_merge64_k(IndexParams P) {
  __shared__ uint32_t tile[kMergeWarps][kMergeTile];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int cpt = P.cells_per_tuple;
  for (int64_t T = (int64_t)blockIdx.x * kMergeWarps + wid; T < P.n_tuples; T += (int64_t)gridDim.x * kMergeWarps) {
    const int64_t r0 = T * cpt;
    float ulo[2], uhi[2], vlo[2], vhi[2], eh[2];
    uint32_t fl[2];
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      const int k = lane + 32 * c;
      const int64_t r = r0 + (k < cpt ? k : 0);
      fl[c] = k < cpt ? P.flags[r] : 0u;
      ulo[c] = P.u_lo[r];
      uhi[c] = P.u_hi[r];
      vlo[c] = P.v_lo[r];
      vhi[c] = P.v_hi[r];
      eh[c] = P.e_hi[r];
    }
    merge_tuple64(P, T, r0, tile[wid], ulo, uhi, vlo, vhi, eh, fl, P.emitter[r0], P.tri0[r0], P.tri1[r0]);
  }
}

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const uint32_t sa = (uint32_t)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Tuples of exactly 64 records with 16-byte aligned record arrays: each warp double-buffers its
// tuples' records (box, E_hi, flags: 6 x 256 B) in shared memory with cp.async, so the next
// tuple's records are in flight while this one is rasterized.
__global__ void __launch_bounds__(32 * kMergeWarps) tuple_merge64_async_k(IndexParams P) {
  __shared__ uint32_t tile[kMergeWarps][kMergeTile];
  __shared__ __align__(16) float rec[kMergeWarps][2][6][64];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int64_t step = (int64_t)gridDim.x * kMergeWarps;
  auto fetch = [&](int64_t T, int b) {
#pragma unroll
    for (int q = 0; q < 3; ++q) {  // 6 arrays x 16 chunks of 16 B, 3 chunks per lane
      const int c = lane + 32 * q, a = c >> 4, o = (c & 15) * 4;
      const float* g = a == 0 ? P.u_lo
                              : a == 1 ? P.u_hi
                                       : a == 2 ? P.v_lo : a == 3 ? P.v_hi : a == 4 ? P.e_hi : (const float*)P.flags;
      cp_async16(&rec[wid][b][a][o], g + T * 64 + o);
    }
  };
  int64_t T = (int64_t)blockIdx.x * kMergeWarps + wid;
  if (T < P.n_tuples) fetch(T, 0);
  cp_async_commit();
  for (int b = 0; T < P.n_tuples; T += step, b ^= 1) {
    if (T + step < P.n_tuples) fetch(T + step, b ^ 1);
    cp_async_commit();
    cp_async_wait<1>();  // this tuple's group has landed (the next one may be in flight)
    __syncwarp();
    const int64_t r0 = T * 64;
    float ulo[2], uhi[2], vlo[2], vhi[2], eh[2];
    uint32_t fl[2];
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      const int k = lane + 32 * c;
      ulo[c] = rec[wid][b][0][k];
      uhi[c] = rec[wid][b][1][k];
      vlo[c] = rec[wid][b][2][k];
      vhi[c] = rec[wid][b][3][k];
      eh[c] = rec[wid][b][4][k];
      fl[c] = __float_as_uint(rec[wid][b][5][k]);
    }
    merge_tuple64(P, T, r0, tile[wid], ulo, uhi, vlo, vhi, eh, fl, P.emitter[r0], P.tri0[r0], P.tri1[r0]);
    __syncwarp();  // every lane has read buffer b before it is refilled
  }
  cp_async_wait<0>();
}

__global__ void overflow_k(IndexParams P) {
  const int64_t n = min(*P.rec_count, P.rec_capacity);
  for (int64_t r = P.n_base + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n;
       r += (int64_t)gridDim.x * blockDim.x) {
    if (P.flags[r] & BNB_CELL_LIVE) emit_record(P, r);
  }
}

// Counting sort by grid cell, one partition per grid row (blockIdx.y): four entries per thread per
// round, their cursor atomics issued together so their latencies overlap.
__global__ void scatter_k(const Ent* __restrict__ pre, int64_t part_cap, const int64_t* __restrict__ pre_count,
                          const int64_t* __restrict__ goff, int64_t* __restrict__ gcur, Ent* __restrict__ sent) {
  const int part = blockIdx.y;
  const int64_t n = min(pre_count[part * kPartStride], part_cap);
  const Ent* src = pre + part * part_cap;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i0 < n; i0 += 4 * stride) {
    Ent x[4];
    int64_t pos[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int64_t i = i0 + q * stride;
      if (i < n) x[q] = src[i];
    }
#pragma unroll
    for (int q = 0; q < 4; ++q)
      if (i0 + q * stride < n)
        pos[q] = goff[x[q].g] + (int64_t)atomicAdd((unsigned long long*)(gcur + x[q].g), 1ull);
#pragma unroll
    for (int q = 0; q < 4; ++q)
      if (i0 + q * stride < n) sent[pos[q]] = x[q];
  }
}

// ------------------------------------------------------------------ per-cell ordering
constexpr int kRankWarps = 8;   // grid cells in flight per 256-thread block, one per warp
constexpr int kRankCap = 128;   // longest list a warp orders by rank (4 entries per lane)
constexpr int kSegCap = 1024;   // longest list a block orders in shared memory (segsort_k)

// Ranks of the lane's EPL keys k[q] against the n keys SK[0..n): lt[q] = #{j : SK[j] < k[q]}.
template <typename KT, int EPL>
__device__ __forceinline__ void rank_below(const KT* SK, int n, const KT (&k)[EPL], int (&lt)[EPL]) {
#pragma unroll
  for (int q = 0; q < EPL; ++q) lt[q] = 0;
#pragma unroll 4
  for (int j = 0; j < n; ++j) {
    const KT kj = SK[j];
#pragma unroll
    for (int q = 0; q < EPL; ++q) lt[q] += kj < k[q] ? 1 : 0;
  }
}

// One grid cell's list of n <= 32 * EPL entries, in the warp's shared arrays K (keys), V (E),
// S (ranking keys), I (ints): sorted by key, equal keys merged with the max of E (with `merge`);
// writes the list through `put` and returns its length.
// Entry i is lane i % 32's element i / 32.  Where the cell's keys span less than 2^32, or share
// the tuple's second-triangle field and span fewer than 256 emitters, the ranks are computed on
// an order-preserving 32-bit form of the key.
// Writers of an ordered list: straight to the index arrays (E~ = m E rounded up), or back into
// the grid-cell-sorted entries.
struct PutIndex {
  uint64_t* key;
  float* et;
  float m;
  __device__ __forceinline__ void operator()(int p, uint64_t k, float e) const {
    key[p] = k;
    et[p] = __fmul_ru(m, e);
  }
};
struct PutEnt {
  Ent* ent;
  __device__ __forceinline__ void operator()(int p, uint64_t k, float e) const {
    Ent x;
    x.key = k;
    x.e = e;
    x.g = 0u;
    ent[p] = x;
  }
};

template <int EPL, typename Put>
__device__ int order_cell(uint64_t* K, float* V, uint32_t* S, int* I, int n, const Put& put, bool merge) {
  const int lane = threadIdx.x & 31;
  uint64_t k[EPL];
  uint64_t kmin = ~0ull, kmax = 0ull, mid_or = 0ull, mid_and = ~0ull;
#pragma unroll
  for (int q = 0; q < EPL; ++q) {
    const int i = lane + 32 * q;
    k[q] = i < n ? K[i] : ~0ull;
    if (i < n) {
      kmin = min(kmin, k[q]);
      kmax = max(kmax, k[q]);
      mid_or |= k[q] >> 24;
      mid_and &= k[q] >> 24;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    kmin = min(kmin, (uint64_t)__shfl_xor_sync(0xffffffffu, (unsigned long long)kmin, o));
    kmax = max(kmax, (uint64_t)__shfl_xor_sync(0xffffffffu, (unsigned long long)kmax, o));
    mid_or |= (uint64_t)__shfl_xor_sync(0xffffffffu, (unsigned long long)mid_or, o);
    mid_and &= (uint64_t)__shfl_xor_sync(0xffffffffu, (unsigned long long)mid_and, o);
  }
  int lt[EPL];
  const uint64_t emin = kmin >> 48, emax = kmax >> 48;
  // key = emitter << 48 | (t1 + 1) << 24 | t0: with (t1 + 1) the same for every entry, the order
  // is (emitter, t0), which (emitter - emin) << 24 | t0 keeps in 32 bits
  const bool span32 = kmax - kmin <= 0xffffffffull;
  const bool same_t1 = ((mid_or ^ mid_and) & 0xffffffull) == 0ull && emax - emin < 256ull;
  if (span32 || same_t1) {
    uint32_t k32[EPL];
#pragma unroll
    for (int q = 0; q < EPL; ++q) {
      const int i = lane + 32 * q;
      k32[q] = span32 ? (uint32_t)(k[q] - kmin)
                      : (uint32_t)((((k[q] >> 48) - emin) << 24) | (k[q] & 0xffffffull));
      if (i < n) S[i] = k32[q];
    }
    __syncwarp();
    rank_below<uint32_t, EPL>(S, n, k32, lt);
  } else {
    rank_below<uint64_t, EPL>(K, n, k, lt);
  }
  // equal keys share a rank: each entry claims its rank's slot, a lost claim means a duplicate
#pragma unroll
  for (int q = 0; q < EPL; ++q) {
    const int i = lane + 32 * q;
    if (i < n) I[lt[q]] = i;
  }
  __syncwarp();
  bool dup = false;
#pragma unroll
  for (int q = 0; q < EPL; ++q) {
    const int i = lane + 32 * q;
    if (i < n && I[lt[q]] != i) dup = true;
  }
  if (!__any_sync(0xffffffffu, dup)) {
#pragma unroll
    for (int q = 0; q < EPL; ++q) {
      const int i = lane + 32 * q;
      if (i < n) put(lt[q], k[q], V[i]);
    }
    return n;
  }
  // duplicates: the first entry of each key (lowest index) is its head and carries the max of E
  // over the key; the head's place is the number of heads with a smaller key.  Without `merge`,
  // every entry is kept in (key, index) order instead.
  __syncwarp();
  bool head[EPL];
  float vmax[EPL];
  int eqb[EPL];
#pragma unroll
  for (int q = 0; q < EPL; ++q) {
    const int i = lane + 32 * q;
    head[q] = i < n;
    vmax[q] = i < n ? V[i] : 0.0f;
    eqb[q] = 0;
  }
  for (int j = 0; j < n; ++j) {
    const uint64_t kj = K[j];
    const float vj = V[j];
#pragma unroll
    for (int q = 0; q < EPL; ++q) {
      if (kj == k[q]) {
        if (j < lane + 32 * q) {
          head[q] = false;
          ++eqb[q];
        }
        vmax[q] = fmaxf(vmax[q], vj);
      }
    }
  }
  if (!merge) {
#pragma unroll
    for (int q = 0; q < EPL; ++q) {
      const int i = lane + 32 * q;
      if (i < n) put(lt[q] + eqb[q], k[q], V[i]);
    }
    return n;
  }
#pragma unroll
  for (int q = 0; q < EPL; ++q) {
    const int i = lane + 32 * q;
    if (i < n) I[i] = head[q] ? 1 : 0;
  }
  __syncwarp();
  int heads = 0;
#pragma unroll
  for (int q = 0; q < EPL; ++q) heads += head[q] ? 1 : 0;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) heads += __shfl_xor_sync(0xffffffffu, heads, o);
  int pos[EPL];
#pragma unroll
  for (int q = 0; q < EPL; ++q) pos[q] = 0;
  for (int j = 0; j < n; ++j) {
    const uint64_t kj = K[j];
    const int hj = I[j];
#pragma unroll
    for (int q = 0; q < EPL; ++q) pos[q] += (hj && kj < k[q]) ? 1 : 0;
  }
#pragma unroll
  for (int q = 0; q < EPL; ++q) {
    if (head[q]) put(pos[q], k[q], vmax[q]);
  }
  return heads;
}

// Warp-wide all-ascending bitonic network over W[0..n) (virtual +inf padding to 2^ln2): every
// comparator puts the smaller word at the lower index, so padding never moves.
__device__ __forceinline__ void warp_bitonic(uint64_t* W, int n, int ln2) {
  const int lane = threadIdx.x & 31;
  const int half = 1 << (ln2 - 1);
  for (int lk = 1; lk <= ln2; ++lk) {
    const int k = 1 << lk, lh = lk - 1;
    for (int i = lane; i < half; i += 32) {
      const int blk = i >> lh, off = i & ((1 << lh) - 1);
      const int a = blk * k + off, b = blk * k + k - 1 - off;
      if (b < n) {
        const uint64_t wa = W[a], wb = W[b];
        if (wb < wa) {
          W[a] = wb;
          W[b] = wa;
        }
      }
    }
    __syncwarp();
    for (int lj = lk - 2; lj >= 0; --lj) {
      const int j = 1 << lj;
      for (int i = lane; i < half; i += 32) {
        const int a = ((i >> lj) << (lj + 1)) | (i & (j - 1)), b = a + j;
        if (b < n) {
          const uint64_t wa = W[a], wb = W[b];
          if (wb < wa) {
            W[a] = wb;
            W[b] = wa;
          }
        }
      }
      __syncwarp();
    }
  }
}

constexpr int kWarpSortCap = 512;                    // longest list the warp bitonic path orders
constexpr int kRankWarpBytes = kWarpSortCap * 8;     // shared memory per warp
static_assert(kRankCap * (8 + 4 + 4 + 4) <= kRankWarpBytes, "rank arrays fit the warp's buffer");

__device__ __forceinline__ uint64_t shfl_xor64(uint64_t v, int m) {
  return (uint64_t)__shfl_xor_sync(0xffffffffu, (unsigned long long)v, m);
}

// The order-preserving 32-bit form of a grid cell's keys, if it has one: key = emitter << 48 |
// (t1 + 1) << 24 | t0; keys spanning < 2^32 map to key - kmin, keys sharing the (t1 + 1) field
// over < 256 emitters to (emitter - emin) << 24 | t0.  Reductions over the warp.
struct Form32 {
  uint64_t kmin, emin;
  bool span32, ok;
  __device__ __forceinline__ uint32_t operator()(uint64_t k) const {
    return span32 ? (uint32_t)(k - kmin) : (uint32_t)((((k >> 48) - emin) << 24) | (k & 0xffffffull));
  }
};

__device__ __forceinline__ Form32 form32(uint64_t kmin, uint64_t kmax, uint64_t mid_or, uint64_t mid_and) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    kmin = min(kmin, shfl_xor64(kmin, o));
    kmax = max(kmax, shfl_xor64(kmax, o));
    mid_or |= shfl_xor64(mid_or, o);
    mid_and &= shfl_xor64(mid_and, o);
  }
  Form32 f;
  f.kmin = kmin;
  f.emin = kmin >> 48;
  f.span32 = kmax - kmin <= 0xffffffffull;
  f.ok = f.span32 || (((mid_or ^ mid_and) & 0xffffffull) == 0ull && (kmax >> 48) - f.emin < 256ull);
  return f;
}

// A warp per grid cell.  Lists of <= kRankCap entries are ordered by rank (order_cell).  With no
// per-record emission (*dup == 0) no cell holds a duplicate key (the base tuples' keys are
// distinct and each tuple lists a grid cell once), so the merged counts are the pre-merge counts,
// the CSR offsets are goff, and the ordered list goes straight to the index arrays (E~ = m E_hi
// rounded up); then lists of <= kWarpSortCap entries whose keys have an order-preserving 32-bit
// form are ordered here too, by a warp bitonic sort of (32-bit key << 32 | entry) words in shared
// memory.  Other lists are listed for segsort_k (<= kSegCap) or segsort_big_k, and with per-record
// emission the ordered lists go back to the sorted entries, merged, for compact_k.  (Base records
// that repeat a tuple's key would stay unmerged in direct mode, in (key, index) order: a valid CSR
// either way.)
__global__ void __launch_bounds__(32 * kRankWarps) segrank_k(const int64_t* __restrict__ goff,
                                                            Ent* __restrict__ sent, int64_t* __restrict__ rcount,
                                                            int32_t* __restrict__ mid, int32_t* __restrict__ n_mid,
                                                            int32_t* __restrict__ big, int32_t* __restrict__ n_big,
                                                            int n_cells, const int32_t* __restrict__ dup, float m,
                                                            int64_t capacity, uint64_t* __restrict__ key,
                                                            float* __restrict__ et) {
  extern __shared__ __align__(16) unsigned char rank_smem[];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  unsigned char* buf = rank_smem + (size_t)wid * kRankWarpBytes;
  uint64_t* K = (uint64_t*)buf;
  float* V = (float*)(buf + kRankCap * 8);
  uint32_t* S = (uint32_t*)(buf + kRankCap * 12);
  int* I = (int*)(buf + kRankCap * 16);
  uint64_t* W = (uint64_t*)buf;
  const bool direct = *dup == 0;
  for (int g = blockIdx.x * kRankWarps + wid; g < n_cells; g += gridDim.x * kRankWarps) {
    const int64_t s = goff[g];
    const int64_t nn = goff[g + 1] - s;
    if (nn == 0) {
      if (lane == 0) rcount[g] = 0;
      continue;
    }
    if (direct && s + nn > capacity) {  // the index arrays are too small: compact_k raises the status
      if (lane == 0) rcount[g] = nn;
      continue;
    }
    const int n = (int)min(nn, (int64_t)(1 << 30));
    if (n <= kRankCap) {
      for (int i = lane; i < n; i += 32) {
        const Ent x = sent[s + i];
        K[i] = x.key;
        V[i] = x.e;
      }
      __syncwarp();
      const int epl = (n + 31) >> 5;
      int u;
      if (direct) {
        const PutIndex put{key + s, et + s, m};
        switch (epl) {
          case 1: u = order_cell<1>(K, V, S, I, n, put, false); break;
          case 2: u = order_cell<2>(K, V, S, I, n, put, false); break;
          case 3: u = order_cell<3>(K, V, S, I, n, put, false); break;
          default: u = order_cell<4>(K, V, S, I, n, put, false); break;
        }
      } else {
        const PutEnt put{sent + s};
        switch (epl) {
          case 1: u = order_cell<1>(K, V, S, I, n, put, true); break;
          case 2: u = order_cell<2>(K, V, S, I, n, put, true); break;
          case 3: u = order_cell<3>(K, V, S, I, n, put, true); break;
          default: u = order_cell<4>(K, V, S, I, n, put, true); break;
        }
      }
      if (lane == 0) rcount[g] = u;
      __syncwarp();
      continue;
    }
    Form32 f;
    f.ok = false;
    if (direct && n <= kWarpSortCap) {
      uint64_t kmin = ~0ull, kmax = 0ull, mid_or = 0ull, mid_and = ~0ull;
      for (int i = lane; i < n; i += 32) {
        const uint64_t k = sent[s + i].key;
        kmin = min(kmin, k);
        kmax = max(kmax, k);
        mid_or |= k >> 24;
        mid_and &= k >> 24;
      }
      f = form32(kmin, kmax, mid_or, mid_and);
    }
    if (!f.ok) {
      if (lane == 0) {
        rcount[g] = 0;
        if (n > kSegCap)
          big[atomicAdd(n_big, 1)] = g;
        else
          mid[atomicAdd(n_mid, 1)] = g;
      }
      continue;
    }
    // direct mode, 32-bit keys, a long list: sort (key32 << 32 | entry) words in shared memory
    int ln2 = 6;
    while ((1 << ln2) < n) ++ln2;
    for (int i = lane; i < n; i += 32) W[i] = ((uint64_t)f(sent[s + i].key) << 32) | (uint32_t)i;
    __syncwarp();
    warp_bitonic(W, n, ln2);
    for (int p = lane; p < n; p += 32) {
      const Ent x = sent[s + (int)(uint32_t)W[p]];
      key[s + p] = x.key;
      et[s + p] = __fmul_ru(m, x.e);
    }
    if (lane == 0) rcount[g] = n;
    __syncwarp();
  }
}

// All-ascending bitonic network over n elements (virtual +inf padding to 2^ln2): every comparator
// puts the smaller key at the lower index, so padding never moves.  Block-wide.
template <typename KeyAt, typename Swap>
__device__ __forceinline__ void bitonic_all_asc(int n, int ln2, KeyAt key, Swap swp) {
  const int half = 1 << (ln2 - 1);
  for (int lk = 1; lk <= ln2; ++lk) {
    const int k = 1 << lk, lh = lk - 1;
    for (int i = threadIdx.x; i < half; i += blockDim.x) {
      const int blk = i >> lh, off = i & ((1 << lh) - 1);
      const int a = blk * k + off, b = blk * k + k - 1 - off;
      if (b < n && key(b) < key(a)) swp(a, b);
    }
    __syncthreads();
    for (int lj = lk - 2; lj >= 0; --lj) {
      const int j = 1 << lj;
      for (int i = threadIdx.x; i < half; i += blockDim.x) {
        const int a = ((i >> lj) << (lj + 1)) | (i & (j - 1)), b = a + j;
        if (b < n && key(b) < key(a)) swp(a, b);
      }
      __syncthreads();
    }
  }
}

constexpr int kSegThreads = 128;

// Grid cells of kRankCap < n <= kSegCap entries (listed by segrank_k), a block each: bitonic sort
// by key in shared memory, then runs of equal keys merged with the max of E (`merge`, i.e. when
// per-record emission happened; otherwise every entry is kept).
__global__ void __launch_bounds__(kSegThreads) segsort_k(const int64_t* __restrict__ goff, Ent* __restrict__ sent,
                                                         int64_t* __restrict__ rcount,
                                                         const int32_t* __restrict__ mid,
                                                         const int32_t* __restrict__ n_mid,
                                                         const int32_t* __restrict__ dup) {
  __shared__ uint64_t K[kSegCap];
  __shared__ float V[kSegCap];
  __shared__ int wsum[kSegThreads / 32];
  const bool merge = *dup != 0;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int b = blockIdx.x; b < *n_mid; b += gridDim.x) {
    const int g = mid[b];
    const int64_t s = goff[g];
    const int n = (int)(goff[g + 1] - s);
    int ln2 = 1;
    while ((1 << ln2) < n) ++ln2;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      const Ent x = sent[s + i];
      K[i] = x.key;
      V[i] = x.e;
    }
    __syncthreads();
    bitonic_all_asc(
        n, ln2, [&](int i) { return K[i]; },
        [&](int a, int c) {
          const uint64_t tk = K[a];
          K[a] = K[c];
          K[c] = tk;
          const float tv = V[a];
          V[a] = V[c];
          V[c] = tv;
        });
    // Merge runs of equal keys (max of E~) in parallel: each thread takes a contiguous chunk,
    // counts the run heads in it, a block scan turns the counts into output positions, and each
    // head writes its key with the max over its run.
    const int per = (n + kSegThreads - 1) / kSegThreads;
    const int i0 = min(n, (int)threadIdx.x * per), i1 = min(n, i0 + per);
    int heads = 0;
    for (int i = i0; i < i1; ++i) heads += (!merge || i == 0 || K[i] != K[i - 1]);
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
      if (!merge || i == 0 || K[i] != K[i - 1]) {
        float m = V[i];
        if (merge)
          for (int j = i + 1; j < n && K[j] == K[i]; ++j) m = fmaxf(m, V[j]);
        Ent x;
        x.key = K[i];
        x.e = m;
        x.g = 0u;
        sent[s + pos] = x;
        ++pos;
      }
    }
    if (threadIdx.x == kSegThreads - 1) {
      int total = 0;
      for (int w = 0; w < kSegThreads / 32; ++w) total += wsum[w];
      rcount[g] = total;
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(512) segsort_big_k(const int64_t* __restrict__ goff, Ent* __restrict__ sent,
                                                     int64_t* __restrict__ rcount, const int32_t* __restrict__ big,
                                                     const int32_t* __restrict__ n_big,
                                                     const int32_t* __restrict__ dup) {
  const bool merge = *dup != 0;
  for (int b = blockIdx.x; b < *n_big; b += gridDim.x) {
    const int g = big[b];
    const int64_t s = goff[g];
    const int n = (int)(goff[g + 1] - s);
    int ln2 = 1;
    while ((1 << ln2) < n) ++ln2;
    Ent* X = sent + s;
    bitonic_all_asc(
        n, ln2, [&](int i) { return X[i].key; },
        [&](int a, int c) {
          const Ent t = X[a];
          X[a] = X[c];
          X[c] = t;
        });
    if (threadIdx.x == 0) {
      int o = 0;
      for (int i = 0; i < n; ++i) {
        if (merge && o > 0 && X[o - 1].key == X[i].key) {
          X[o - 1].e = fmaxf(X[o - 1].e, X[i].e);
        } else {
          X[o] = X[i];
          ++o;
        }
      }
      rcount[g] = o;
    }
    __syncthreads();
  }
}

// Copies each grid cell's merged list from the sorted entries to its CSR place, E~ = m E_hi
// rounded up;
// in direct mode (*dup == 0) only the cells segrank_k did not write (those listed for segsort_k
// and segsort_big_k) are copied.
__global__ void compact_k(const int64_t* __restrict__ goff, const Ent* __restrict__ sent,
                          const int64_t* __restrict__ offsets, int n_cells, float m,
                          int64_t capacity, uint64_t* __restrict__ key, float* __restrict__ et,
                          int64_t* __restrict__ count, const int32_t* __restrict__ dup,
                          const int32_t* __restrict__ mid, const int32_t* __restrict__ n_mid,
                          const int32_t* __restrict__ big, const int32_t* __restrict__ n_big,
                          int32_t* __restrict__ status) {
  const int lane = threadIdx.x & 31;
  int g = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (g == 0 && lane == 0) {
    count[0] = offsets[n_cells];
    if (offsets[n_cells] > capacity) raise_status(status, BNB_ERR_CAPACITY);
  }
  if (*dup == 0) {
    const int a = *n_mid, b = *n_big;
    if (g < a)
      g = mid[g];
    else if (g < a + b)
      g = big[g - a];
    else
      return;
  }
  if (g >= n_cells) return;
  const int64_t src = goff[g];
  const int64_t dst = offsets[g], n = offsets[g + 1] - dst;
  for (int64_t i = lane; i < n; i += 32) {
    if (dst + i < capacity) {
      const Ent x = sent[src + i];
      key[dst + i] = x.key;
      et[dst + i] = __fmul_ru(m, x.e);
    }
  }
}

// The pre-merge capacity the records need: kPreParts x the largest partition's count.
__global__ void store_pre_count_k(const int64_t* __restrict__ pre_count, int64_t* __restrict__ count) {
  int64_t mx = 0;
  for (int p = 0; p < kPreParts; ++p) mx = max(mx, pre_count[p * kPartStride]);
  count[1] = mx * kPreParts;
}

// ------------------------------------------------------------------ host side
struct IndexWs {
  int64_t* gcount;   // G*G
  int64_t* goff;     // G*G + 1
  int64_t* gcur;     // G*G
  int64_t* rcount;   // G*G
  int64_t* pre_count;
  int32_t* n_big;
  int32_t* n_mid;
  int32_t* dup;
  int32_t* big;      // G*G
  int32_t* mid;      // G*G
  Ent* pre;          // pre_cap: kPreParts partitions of pre_cap / kPreParts
  Ent* sent;         // pre_cap: sorted by grid cell
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
  w.pre_count = (int64_t*)take(kPreParts * kPartStride * 8);
  w.n_big = (int32_t*)take(8);
  w.n_mid = (int32_t*)take(8);
  w.dup = (int32_t*)take(8);
  const size_t zero_end = o;  // everything above is zeroed per call
  w.goff = (int64_t*)take((cells + 1) * 8);
  w.rcount = (int64_t*)take(cells * 8);
  w.big = (int32_t*)take(cells * 4);
  w.mid = (int32_t*)take(cells * 4);
  w.pre = (Ent*)take(pre_cap * sizeof(Ent));
  w.sent = (Ent*)take(pre_cap * sizeof(Ent));
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
  // zero the counters (gcount, gcur, the partition counters, n_big, n_mid, dup: laid out first, contiguous)
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
  P.pre = w.pre;
  P.part_cap = pre_cap / kPreParts;
  P.pre_count = w.pre_count;
  P.gcount = w.gcount;
  P.dup = w.dup;
  P.status = out->status;
  const int sms = sm_count();
  if (P.n_tuples > 0) {
    const int64_t blocks = std::min<int64_t>((P.n_tuples + kMergeWarps - 1) / kMergeWarps, (int64_t)sms * 64);
    auto al16 = [](const void* q) { return ((uintptr_t)q & 15u) == 0; };
    if (P.cells_per_tuple == 64 && al16(P.u_lo) && al16(P.u_hi) && al16(P.v_lo) && al16(P.v_hi) && al16(P.e_hi) &&
        al16(P.flags))
      tuple_merge64_async_k<<<(unsigned)blocks, 32 * kMergeWarps, 0, st>>>(P);
    else if (P.cells_per_tuple <= 64)
      tuple_merge64_k<<<(unsigned)blocks, 32 * kMergeWarps, 0, st>>>(P);
    else
      tuple_merge_k<<<(unsigned)blocks, 32 * kMergeWarps, 0, st>>>(P);
  }
  overflow_k<<<sms * 2, 256, 0, st>>>(P);
  if ((e = launch_exclusive_scan(w.gcount, w.goff, cells, w.scan, st)) != cudaSuccess) return e;
  scatter_k<<<dim3((unsigned)std::max(1, sms * 8 / kPreParts), kPreParts), 256, 0, st>>>(
      w.pre, P.part_cap, w.pre_count, w.goff, w.gcur, w.sent);
  const int64_t rank_blocks = std::min<int64_t>((cells + kRankWarps - 1) / kRankWarps, (int64_t)sms * 24);
  const int rank_smem = kRankWarps * kRankWarpBytes;
  if ((e = cudaFuncSetAttribute(segrank_k, cudaFuncAttributeMaxDynamicSharedMemorySize, rank_smem)) != cudaSuccess)
    return e;
  segrank_k<<<(unsigned)rank_blocks, 32 * kRankWarps, rank_smem, st>>>(w.goff, w.sent, w.rcount, w.mid, w.n_mid,
                                                                        w.big, w.n_big, (int)cells, w.dup, m,
                                                                        out->capacity, out->key, out->etilde);
  segsort_k<<<sms * 16, kSegThreads, 0, st>>>(w.goff, w.sent, w.rcount, w.mid, w.n_mid, w.dup);
  segsort_big_k<<<sms, 512, 0, st>>>(w.goff, w.sent, w.rcount, w.big, w.n_big, w.dup);
  if ((e = launch_exclusive_scan(w.rcount, out->offsets, cells, w.scan, st)) != cudaSuccess) return e;
  compact_k<<<(unsigned)((cells + 7) / 8), 256, 0, st>>>(w.goff, w.sent, out->offsets, (int)cells, m, out->capacity,
                                                          out->key, out->etilde, out->count, w.dup, w.mid, w.n_mid,
                                                          w.big, w.n_big, out->status);
  store_pre_count_k<<<1, 1, 0, st>>>(w.pre_count, out->count);
  return cudaGetLastError();
}

}  // namespace bnb
