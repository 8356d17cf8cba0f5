// bnb_stream_status: reads and clears the device error words of every translation unit.
//
// Kernels report conditions that only the device can see (an output, queue or worklist too small)
// in two places: the status word of the call's output struct, which stays set until the caller
// clears it, and the device error word of the kernel's translation unit (bnb_internal.cuh).  The
// second one lets a caller that keeps no output struct around (or drives many calls on one
// stream) ask once, after the fact, whether any call failed on the device.
#include <mutex>

#include "bnb_internal.cuh"

namespace bnb {

namespace {

constexpr int kMaxUnits = 64;

struct ErrorWords {
  std::mutex mu;
  TakeErrorFn take[kMaxUnits];
  int n = 0;
};

// Constructed on first use, so units may register during static initialization in any order.
ErrorWords& error_words() {
  static ErrorWords w;
  return w;
}

}  // namespace

int register_error_word(TakeErrorFn f) {
  ErrorWords& w = error_words();
  std::lock_guard<std::mutex> lock(w.mu);
  if (w.n < kMaxUnits) w.take[w.n++] = f;
  return w.n;
}

}  // namespace bnb

extern "C" int32_t bnb_stream_status(void* stream) {
  using namespace bnb;
  cudaStream_t st = (cudaStream_t)stream;
  if (cudaStreamSynchronize(st) != cudaSuccess) return BNB_ERR_CUDA;
  ErrorWords& w = error_words();
  std::lock_guard<std::mutex> lock(w.mu);
  int32_t first = BNB_OK;
  for (int i = 0; i < w.n; ++i) {
    int32_t code = BNB_OK;
    if (w.take[i](st, &code) != cudaSuccess) return BNB_ERR_CUDA;
    if (first == BNB_OK && code != BNB_OK) first = code;
  }
  if (cudaStreamSynchronize(st) != cudaSuccess) return BNB_ERR_CUDA;
  return first;
}
