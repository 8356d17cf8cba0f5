// Internal declarations shared by the libbnb translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/bnb.h"

namespace bnb {

constexpr int kMaxDepth = 15;  // depth + extra splits: 2 bits per level in a uint32 cell id

// Packed triangle: p0, p1, p2, n0, n1, n2 as 18 floats in 5 float4 (80 bytes, 16-byte aligned).
constexpr int kTriF4 = 5;

struct SplitItem {
  int32_t emitter, tri;
  uint32_t cell;
  int32_t depth;
};

struct BoundParams {
  const float4* tri;  // packed triangles
  int32_t n_tris, n_emitters;
  const float *ex, *ey, *ez, *ei;
  float rp0[3], re1[3], re2[3];
  int32_t depth, max_depth, irradiance;
  int32_t kind;  // BNB_REFLECT or BNB_REFRACT
  float eta;     // refraction: eta' = incident / transmitted index
  int32_t adapt_depth;  // adaptive subdivision above this depth (0: off)
  int32_t block_threads;  // block size of the float32 reflection base pass (0: the default, 384)
  float sigma, alpha;   // its stopping thresholds (box area, E_hi / E_lo)
  int64_t n_base;
  // outputs
  int64_t capacity;
  int64_t* count;
  int32_t* status;
  float *u_lo, *u_hi, *v_lo, *v_hi, *e_lo, *e_hi;
  int32_t *emitter, *tri0, *tri1;
  uint32_t *cell, *flags;
  float* e_hi_min;  // optional
  // split queues
  SplitItem* q_out;
  int64_t* q_out_count;
  int64_t q_cap;
};

// Launchers (bnb_bound.cu)
cudaError_t launch_pack_tris(const bnb_surface* s, float4* out, cudaStream_t st);
cudaError_t launch_bound_base(const BoundParams& p, bool fp64, cudaStream_t st);
cudaError_t launch_bound_split(const BoundParams& p, const SplitItem* q_in, const int64_t* q_in_count, bool fp64,
                               cudaStream_t st);

// Scan (bnb_index.cu): exclusive prefix sum of n int64 values into out[0..n], out[n] = total.
size_t scan_ws_bytes(int64_t n);
cudaError_t launch_exclusive_scan(const int64_t* in, int64_t* out, int64_t n, void* ws, cudaStream_t st);

__host__ __device__ inline int64_t round_up(int64_t x, int64_t a) { return (x + a - 1) / a * a; }

// ---- device error word (read and cleared by bnb_stream_status)
// Each translation unit holds its own word (the library is built without relocatable device code,
// so a __device__ variable cannot be shared between units).  A kernel that meets a condition only
// the device can see records it in the status word of the call's output struct and in its unit's
// word; the first code since the last read is kept.  Every unit registers, at load time, a host
// function that takes its word on a stream (an atomic exchange with 0 in a one-thread kernel, then
// a copy of the old value to the host), so a read never loses a code raised concurrently.
static __device__ int32_t g_device_error;
static __device__ int32_t g_device_error_taken;

__device__ __forceinline__ void raise_status(int32_t* status, int32_t code) {
  if (status) atomicCAS(status, 0, code);
  atomicCAS(&g_device_error, 0, code);
}

static __global__ void take_device_error_k() { g_device_error_taken = atomicExch(&g_device_error, 0); }

// Enqueues the exchange on `st` and copies the taken code to *host_out (a pageable copy: it returns
// once the value is on the host).
static cudaError_t take_device_error(cudaStream_t st, int32_t* host_out) {
  take_device_error_k<<<1, 1, 0, st>>>();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return cudaMemcpyFromSymbolAsync(host_out, g_device_error_taken, sizeof(int32_t), 0, cudaMemcpyDeviceToHost, st);
}

typedef cudaError_t (*TakeErrorFn)(cudaStream_t, int32_t*);
int register_error_word(TakeErrorFn f);  // bnb_status.cu
static const int g_error_word_registered = register_error_word(&take_device_error);

}  // namespace bnb
