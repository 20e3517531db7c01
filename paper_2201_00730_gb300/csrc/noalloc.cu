// uot_softmin_noalloc: the softmin sweep of uot_softmin with its scratch taken
// from a fixed array compiled into this library instead of a caller workspace.
//
// For callers that cannot allocate device memory: the array below is reserved
// when the library's device code is loaded on a GPU and stays reserved until
// the process exits, so the call itself never allocates.
#include <cuda_runtime.h>
#include <stdio.h>

#include <mutex>

#include "uot_internal.cuh"

namespace {

constexpr size_t kScratchBytes = size_t(16) << 20;  // 16 MiB per GPU

// The scratch: state, log weights, sweep partials and block partials of one
// uot_softmin call.  Host code must not take its address directly (in host
// code the name is a host-side stand-in); it asks the runtime for the device
// address once per device, below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

std::mutex g_mu;
void* g_addr[64] = {nullptr};

}  // namespace

extern "C" {

// Declared in include/uot.h.
uot_status uot_softmin_noalloc(const uot_problem* prob, int32_t axis, const float* pot, float* out,
                               void* stream) {
  const size_t need = uot_workspace_size(prob);
  if (need == 0) return UOT_ERR_INVALID_ARG;  // uot_last_error() already says why
  if (need > kScratchBytes) {
    char msg[256];
    snprintf(msg, sizeof(msg),
             "uot_softmin_noalloc: this problem needs %zu bytes of scratch but the built-in scratch holds %zu "
             "bytes; use uot_softmin with a caller workspace", need, kScratchBytes);
    uot::set_last_error(msg);
    return UOT_ERR_UNSUPPORTED;
  }
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    uot::set_last_error("uot_softmin_noalloc: no usable current CUDA device");
    return UOT_ERR_CUDA;
  }
  void* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
      // One-time set-up on this device (the device is current here).
      void* p = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess || !p) {
        char msg[256];
        snprintf(msg, sizeof(msg), "uot_softmin_noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
        uot::set_last_error(msg);
        return UOT_ERR_CUDA;
      }
      g_addr[dev] = p;
    }
    scratch = g_addr[dev];
  }
  // The softmin path clears the state at the start of the call and writes every
  // partial before reading it, so stale contents of the shared scratch from an
  // earlier call are never read.
  return uot_softmin(prob, axis, pot, out, scratch, kScratchBytes, stream);
}

}  // extern "C"
