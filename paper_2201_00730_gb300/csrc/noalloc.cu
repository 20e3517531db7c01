// uot_softmin_noalloc: the softmin sweep of uot_softmin with its scratch taken
// from a fixed array compiled into this library instead of a caller workspace.
//
// For callers that cannot allocate device memory: the array below is reserved
// when this library's device code is loaded on a GPU and stays reserved until
// the process exits.  With lazy module loading (CUDA's default) that load
// happens inside the first call on each device, which is therefore the one
// call that can fail for lack of device memory; later calls allocate nothing.
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdio.h>

#include <mutex>

#include "uot_internal.cuh"

namespace {

constexpr size_t kScratchBytes = size_t(32) << 20;  // 32 MiB per GPU

// The scratch: state, log weights, sweep partials and block partials of one
// uot_softmin call.  Host code must not take its address directly (in host
// code the name is a host-side stand-in); it asks the runtime for the device
// address once per device, below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// Device address of the scratch per device, valid for the CUDA context it was
// looked up in (identified by the driver's context id, unique for the life of
// the process): after cudaDeviceReset the primary context is a new one, the
// array lives at a new address, and the look-up is redone.
struct Cached {
  void* addr = nullptr;
  unsigned long long ctx_id = 0;
};
std::mutex g_mu;
Cached g_cache[64];

typedef CUresult (*CtxGetCurrentFn)(CUcontext*);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long*);

// Id of the calling thread's current context; false if there is none yet.
bool current_ctx_id(unsigned long long* id) {
  static CtxGetCurrentFn get_current = nullptr;
  static CtxGetIdFn get_id = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_current = reinterpret_cast<CtxGetCurrentFn>(f);
    f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_id = reinterpret_cast<CtxGetIdFn>(f);
  });
  if (!get_current || !get_id) return false;
  CUcontext ctx = nullptr;
  if (get_current(&ctx) != CUDA_SUCCESS || !ctx) return false;
  return get_id(ctx, id) == CUDA_SUCCESS;
}

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
    Cached& c = g_cache[dev];
    unsigned long long id = 0;
    const bool have_ctx = current_ctx_id(&id);
    if (!c.addr || !have_ctx || id != c.ctx_id) {
      // Set-up on this device, with the device current: the first call, or the
      // first after the device's context was replaced.  Under lazy module
      // loading this loads the module and so reserves the array.
      void* p = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess || !p) {
        char msg[256];
        snprintf(msg, sizeof(msg), "uot_softmin_noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
        uot::set_last_error(msg);
        c.addr = nullptr;
        return UOT_ERR_CUDA;
      }
      c.addr = p;
      c.ctx_id = current_ctx_id(&id) ? id : 0;
    }
    scratch = c.addr;
  }
  // The softmin path clears the state at the start of the call and writes every
  // partial before reading it, so stale contents of the shared scratch from an
  // earlier call are never read.
  return uot_softmin(prob, axis, pot, out, scratch, kScratchBytes, stream);
}

}  // extern "C"
