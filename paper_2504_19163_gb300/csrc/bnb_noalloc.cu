// bnb_bound_tuples_noalloc: the bound pass for callers that cannot allocate device memory.
//
// Some callers have no way to obtain a device workspace: a plug-in or callback running inside a
// host application whose device memory is owned by another runtime (no allocator is exposed to
// it), or a program that forbids any allocation after start-up.  For them this entry point runs
// bnb_bound_tuples with its scratch (packed triangles and the split queues) in a fixed-size array
// that lives in this library's device memory.  The caller still passes inputs and outputs.
//
// The array is a file-scope static __device__ variable: every GPU that loads the library holds
// kNoallocScratchBytes of it until the process exits.  In host code its name only stands in for
// the device object, so its device address is taken with cudaGetSymbolAddress, once per device,
// on the first call made with that device current; calls made afterwards reuse the address.
#include <mutex>

#include "bnb_internal.cuh"

namespace {

constexpr size_t kNoallocScratchBytes = size_t(8) << 20;  // 8 MiB
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_bound_scratch[kNoallocScratchBytes];

std::mutex g_scratch_mu;
void* g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device (set up on first use).
int32_t scratch_for_current_device(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return BNB_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (g_scratch_addr[dev] == nullptr) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_bound_scratch) != cudaSuccess || p == nullptr) return BNB_ERR_CUDA;
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return BNB_OK;
}

}  // namespace

extern "C" int32_t bnb_bound_tuples_noalloc(const bnb_surface* s1, const bnb_surface* s2, const bnb_receiver* rec,
                                            const bnb_emitters* em, const bnb_bound_cfg* cfg, bnb_cell_bounds* out,
                                            void* stream) {
  const size_t need = bnb_bound_tuples_ws(s1, s2, em, cfg);
  if (need == 0) return BNB_ERR_INVALID;
  if (need > kNoallocScratchBytes) return BNB_ERR_CAPACITY;  // nothing launched
  void* scratch = nullptr;
  const int32_t st = scratch_for_current_device(&scratch);
  if (st != BNB_OK) return st;
  // bnb_bound_tuples clears the queue counters it reads on the stream before its first kernel,
  // and writes the packed triangles before reading them, so the previous call's contents of the
  // shared array do not leak into this one.
  return bnb_bound_tuples(s1, s2, rec, em, cfg, out, scratch, kNoallocScratchBytes, stream);
}
