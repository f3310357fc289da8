// igasf_apply_noalloc: the apply for callers that must not allocate device
// memory. The paper has no counterpart; this is a deployment convenience.
//
// The regular apply keeps its per-tile partial results in a workspace that
// igasf_setup allocates with cudaMalloc. This entry point instead uses one
// statically sized device array, declared below at file scope, as that
// workspace. It calls no cudaMalloc, cudaFree or allocating library routine.
//
// The array holds IGASF_NOALLOC_SCRATCH_BYTES (64 MiB). It is part of this
// translation unit's device module, which the CUDA runtime may load lazily:
// the memory is reserved when the module is loaded on a device, and stays
// reserved there until the process exits. Host code cannot use the array's
// name as a device address, so igasf_setup calls noalloc_prepare() for the
// plan's device (with that device current): it looks the address up with
// cudaGetSymbolAddress, which loads the module, and caches it. The
// reservation thus happens inside igasf_setup, next to the plan's own
// allocations, and igasf_apply_noalloc only reads the cached address. Every
// call on a device shares the same array, and its contents persist from call
// to call; the tile kernel overwrites every workspace entry the gather later
// reads, so nothing needs clearing. Calls whose kernels can overlap on the GPU
// (different streams, or different handles on the same device without
// ordering between them) race on the array and give wrong results; order
// them on one stream.
#include <cuda_runtime.h>

#include <cstdio>
#include <cstring>
#include <mutex>

#include "igasf.h"
#include "igasf_internal.h"
#include "plan.h"

static __device__ __align__(256) unsigned char g_igasf_static_scratch[IGASF_NOALLOC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
void *g_scratch_addr[kMaxDevices] = {nullptr};
cudaError_t g_scratch_err[kMaxDevices] = {cudaSuccess};

}  // namespace

namespace igasf {
int apply_with_workspace(igasf_plan *h, int op, int prec, const void *u, void *v, void *ws,
                         size_t ws_bytes, void *stream);
int set_error(int code, const char *msg);

// Called by igasf_setup with `device` current. A failed lookup (for instance
// no memory left for the module) does not fail the setup: it is remembered
// and reported by igasf_apply_noalloc on this device.
void noalloc_prepare(int device) {
  if (device < 0 || device >= kMaxDevices) return;
  std::lock_guard<std::mutex> lock(g_mutex);
  if (g_scratch_addr[device]) return;
  void *p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_igasf_static_scratch);
  if (e == cudaSuccess) {
    g_scratch_addr[device] = p;
    g_scratch_err[device] = cudaSuccess;
  } else {
    g_scratch_err[device] = e;
    cudaGetLastError();   // not sticky: leave no error for the caller's next CUDA call
  }
}
}  // namespace igasf

extern "C" int igasf_apply_noalloc(igasf_handle h, int op, int prec, const void *u, void *v,
                                   void *stream) {
  if (!h) return igasf::set_error(IGASF_ERR_INVALID_ARG, "handle is NULL");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return igasf::set_error(IGASF_ERR_CUDA, cudaGetErrorString(e));
  if (dev != h->device) {
    char msg[128];
    snprintf(msg, sizeof(msg), "device %d is current, but the plan was set up on device %d", dev,
             h->device);
    return igasf::set_error(IGASF_ERR_INVALID_ARG, msg);
  }
  if (dev < 0 || dev >= kMaxDevices)
    return igasf::set_error(IGASF_ERR_UNSUPPORTED, "device ordinal too large for the static scratch");
  void *scratch = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_mutex);
    scratch = g_scratch_addr[dev];
    e = g_scratch_err[dev];
  }
  if (!scratch) {
    char msg[192];
    snprintf(msg, sizeof(msg), "the static scratch could not be located on device %d at setup: %s",
             dev, e == cudaSuccess ? "not prepared" : cudaGetErrorString(e));
    return igasf::set_error(IGASF_ERR_CUDA, msg);
  }
  return igasf::apply_with_workspace(h, op, prec, u, v, scratch, IGASF_NOALLOC_SCRATCH_BYTES, stream);
}
