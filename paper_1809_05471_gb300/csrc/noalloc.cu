// igasf_apply_noalloc: the apply for callers that must not allocate device
// memory. The paper has no counterpart; this is a deployment convenience.
//
// The regular apply keeps its per-tile partial results in a workspace that
// igasf_setup allocates with cudaMalloc. This entry point instead uses one
// statically sized device array, declared below at file scope, as that
// workspace. It calls no cudaMalloc, cudaFree or allocating library routine.
//
// The array occupies kStaticScratchBytes on every GPU where this library's
// module is loaded, until the process exits. Host code cannot use the array's
// name as a device address, so the first call on each device (with that device
// current) looks the address up with cudaGetSymbolAddress and caches it; make
// that first call before any stream capture. Every call on a device shares the
// same array, and its contents persist from call to call; the tile kernel
// overwrites every workspace entry the gather later reads, so nothing needs
// clearing. Calls whose kernels can overlap on the GPU (different streams, or
// different handles on the same device without ordering between them) race on
// the array and give wrong results; order them on one stream.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>

#include "igasf.h"
#include "igasf_internal.h"

static __device__ __align__(256) unsigned char g_igasf_static_scratch[IGASF_NOALLOC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
void *g_scratch_addr[kMaxDevices] = {nullptr};

}  // namespace

namespace igasf {
int apply_with_workspace(igasf_plan *h, int op, int prec, const void *u, void *v, void *ws,
                         size_t ws_bytes, void *stream);
int set_error(int code, const char *msg);
}  // namespace igasf

extern "C" int igasf_apply_noalloc(igasf_handle h, int op, int prec, const void *u, void *v,
                                   void *stream) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return igasf::set_error(IGASF_ERR_CUDA, cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return igasf::set_error(IGASF_ERR_UNSUPPORTED, "device ordinal too large");
  void *scratch = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_scratch_addr[dev]) {
      void *p = nullptr;
      e = cudaGetSymbolAddress(&p, g_igasf_static_scratch);
      if (e != cudaSuccess)
        return igasf::set_error(IGASF_ERR_CUDA, "cudaGetSymbolAddress of the static scratch failed");
      g_scratch_addr[dev] = p;
    }
    scratch = g_scratch_addr[dev];
  }
  return igasf::apply_with_workspace(h, op, prec, u, v, scratch, IGASF_NOALLOC_SCRATCH_BYTES, stream);
}
