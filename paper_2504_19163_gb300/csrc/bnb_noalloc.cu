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
// the device object, so its device address is taken with cudaGetSymbolAddress.  That address is
// valid in the CUDA context that was current when it was looked up (each context loads its own
// copy of the module), so it is cached per context: the key is the unique id the driver gives the
// current context (cuCtxGetId), and a call made under a context not seen before (another device, a
// context created by the driver API, a primary context re-created after cudaDeviceReset) looks
// the address up again.  The driver functions are resolved at run time through the runtime, so the
// library does not link the driver library.
#include <cuda.h>  // CUcontext and CUresult only; the driver functions are resolved at run time

#include <mutex>

#include "bnb_internal.cuh"

namespace {

constexpr size_t kNoallocScratchBytes = size_t(8) << 20;  // 8 MiB
constexpr int kMaxContexts = 64;

static __device__ __align__(256) unsigned char g_bound_scratch[kNoallocScratchBytes];

typedef CUresult (*CtxGetCurrentFn)(CUcontext*);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long*);

struct ScratchEntry {
  unsigned long long ctx_id;
  void* addr;
};

std::mutex g_scratch_mu;
CtxGetCurrentFn g_ctx_get_current = nullptr;
CtxGetIdFn g_ctx_get_id = nullptr;
ScratchEntry g_entries[kMaxContexts] = {};
int g_n_entries = 0;
int g_next_victim = 0;

// Driver entry points (looked up once; the caller holds g_scratch_mu).
bool resolve_driver() {
  if (g_ctx_get_current && g_ctx_get_id) return true;
  void* f0 = nullptr;
  void* f1 = nullptr;
  cudaDriverEntryPointQueryResult q0 = cudaDriverEntryPointSymbolNotFound, q1 = cudaDriverEntryPointSymbolNotFound;
  if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f0, 12000, cudaEnableDefault, &q0) != cudaSuccess ||
      q0 != cudaDriverEntryPointSuccess || !f0)
    return false;
  if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f1, 12000, cudaEnableDefault, &q1) != cudaSuccess ||
      q1 != cudaDriverEntryPointSuccess || !f1)
    return false;
  g_ctx_get_current = (CtxGetCurrentFn)f0;
  g_ctx_get_id = (CtxGetIdFn)f1;
  return true;
}

// Unique id of the context current on this thread (false when none is current).
bool current_ctx_id(unsigned long long* id) {
  CUcontext ctx = nullptr;
  if (g_ctx_get_current(&ctx) != CUDA_SUCCESS || ctx == nullptr) return false;
  return g_ctx_get_id(ctx, id) == CUDA_SUCCESS;
}

// Device address of the scratch array in the current context (looked up on first use there).
int32_t scratch_for_current_context(void** out) {
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!resolve_driver()) return BNB_ERR_CUDA;
  unsigned long long id = 0;
  if (current_ctx_id(&id)) {
    for (int i = 0; i < g_n_entries; ++i)
      if (g_entries[i].ctx_id == id) {
        *out = g_entries[i].addr;
        return BNB_OK;
      }
  }
  // Not seen yet (or no context current: the runtime binds the device's primary context here).
  void* p = nullptr;
  if (cudaGetSymbolAddress(&p, g_bound_scratch) != cudaSuccess || p == nullptr) {
    cudaGetLastError();  // the lookup's error is reported as BNB_ERR_CUDA, not left for the next call
    return BNB_ERR_CUDA;
  }
  if (!current_ctx_id(&id)) return BNB_ERR_CUDA;
  int slot = g_n_entries;
  if (slot == kMaxContexts) {  // table full: reuse slots round robin (a later call looks it up again)
    slot = g_next_victim;
    g_next_victim = (g_next_victim + 1) % kMaxContexts;
  } else {
    ++g_n_entries;
  }
  g_entries[slot] = ScratchEntry{id, p};
  *out = p;
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
  const int32_t st = scratch_for_current_context(&scratch);
  if (st != BNB_OK) return st;
  // bnb_bound_tuples clears on the stream, before its first kernel, the split-queue counters (one
  // surface) or the per-cell counters and cursors of the T2 grid (two surfaces); every other part of
  // the scratch (packed triangles, grid bounds, candidate counts and offsets) is written before it
  // is read, so the previous call's contents of the shared array do not leak into this one.
  return bnb_bound_tuples(s1, s2, rec, em, cfg, out, scratch, kNoallocScratchBytes, stream);
}
