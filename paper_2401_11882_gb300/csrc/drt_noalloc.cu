// drt_forward_noalloc: the forward pass for callers that cannot allocate
// device memory.
//
// drt_forward needs a workspace for its per-chunk partial sums, which the
// caller normally allocates (cudaMalloc, or a framework's allocator).  Some
// callers cannot: plugins and callbacks that are handed only the buffers they
// must fill and have no allocator of their own, and applications that reserve
// all device memory up front under a fixed memory plan and forbid any later
// allocation.  For them this entry point uses a fixed scratch array that
// lives in the library's own device image (a file-scope __device__ array of
// DRT_NOALLOC_SCRATCH_BYTES), so it calls no allocator at all.
//
// Consequences spelled out for the user:
//  - every GPU that loads the library holds this array until the process exits;
//  - all calls on a device share it: calls that overlap on the GPU (different
//    streams without ordering between them) race on its contents;
//  - the array keeps whatever the last call left in it.  The forward pass
//    overwrites every partial sum it later reads, so nothing needs clearing.
//  - the host code must not hand the array's name to a kernel: on the host it
//    is only a stand-in symbol.  Its device address is looked up once per
//    device, on the first call made with that device current
//    (cudaGetSymbolAddress); that first call should therefore happen before
//    any stream capture begins.  The address is kept for the life of the
//    process: after cudaDeviceReset the device image is loaded anew, possibly
//    elsewhere, so this entry point (like the rest of the library, whose
//    per-device settings are lost too) must not be used on a device after it
//    has been reset.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "drt.h"
#include "drt_internal.h"

namespace drt {
namespace {

constexpr size_t kScratchFloats = DRT_NOALLOC_SCRATCH_BYTES / sizeof(float);

static __device__ __align__(256) float g_noalloc_scratch[kScratchFloats];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device (looked up once).
drt_status scratch_on_current_device(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    set_error_message((std::string("cudaGetDevice: ") + cudaGetErrorString(e)).c_str());
    return DRT_ERR_CUDA;
  }
  if (dev < 0 || dev >= kMaxDevices) {
    set_error_message("drt_forward_noalloc: device index out of range");
    return DRT_ERR_UNSUPPORTED;
  }
  std::lock_guard<std::mutex> lk(g_mu);
  if (g_scratch_ptr[dev] == nullptr) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr) {
      set_error_message((std::string("cudaGetSymbolAddress(scratch): ") +
                         cudaGetErrorString(e)).c_str());
      return DRT_ERR_CUDA;
    }
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return DRT_OK;
}

}  // namespace
}  // namespace drt

extern "C" drt_status drt_forward_noalloc(const drt_scene* scene, float* power, void* stream) {
  using namespace drt;
  if (!scene) {
    set_error_message("drt_forward_noalloc: scene is NULL");
    return DRT_ERR_INVALID_ARG;
  }
  // Validate the whole scene first (wall count, order, pointers), so that the
  // candidate count below is only computed for supported sizes.
  size_t default_need = 0;
  drt_status st = drt_forward_workspace_size(scene, nullptr, &default_need);
  if (st != DRT_OK) return st;
  if (scene->n_rx == 0) return drt_forward(scene, nullptr, power, nullptr, 0, stream);
  // One partial sum per (candidate chunk, receiver): choose the chunk so that they
  // fit beside the staged wall records of a scene with more walls than shared
  // memory holds (at most 8 float4 per wall, after the partial sums rounded up to 16
  // bytes).
  const size_t staged = scene->n_walls > DRT_MAX_WALLS ? (size_t)scene->n_walls * 128 + 16 : 0;
  const size_t room = DRT_NOALLOC_SCRATCH_BYTES > staged
                          ? (DRT_NOALLOC_SCRATCH_BYTES - staged) / sizeof(float)
                          : 0;
  const long long max_chunks = (long long)(room / (size_t)scene->n_rx);
  if (max_chunks < 1) {
    set_error_message(("drt_forward_noalloc: n_rx = " + std::to_string(scene->n_rx) +
                       " exceeds the static scratch capacity of " +
                       std::to_string(kScratchFloats) + " receivers").c_str());
    return DRT_ERR_UNSUPPORTED;
  }
  int64_t n_cand = 0;
  st = drt_num_candidates(scene->n_walls, scene->max_order, &n_cand);
  if (st != DRT_OK) return st;
  long long chunk = (n_cand + max_chunks - 1) / max_chunks;
  if (chunk < 64) chunk = 64;
  if (chunk > (1LL << 30)) {
    set_error_message("drt_forward_noalloc: too many path candidates for the scratch capacity");
    return DRT_ERR_UNSUPPORTED;
  }
  drt_tile tile = {0, (int32_t)chunk, 0, 0};
  size_t need = 0;
  st = drt_forward_workspace_size(scene, &tile, &need);
  if (st != DRT_OK) return st;
  if (need > DRT_NOALLOC_SCRATCH_BYTES) {
    set_error_message("drt_forward_noalloc: partial sums and wall records exceed the static "
                      "scratch capacity");
    return DRT_ERR_UNSUPPORTED;
  }
  void* scratch = nullptr;
  st = scratch_on_current_device(&scratch);
  if (st != DRT_OK) return st;
  return drt_forward(scene, &tile, power, scratch, DRT_NOALLOC_SCRATCH_BYTES, stream);
}
