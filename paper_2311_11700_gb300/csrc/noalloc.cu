// gs_render_forward_static: the forward render with its scratch memory in a
// fixed, statically allocated device array instead of a caller-provided
// workspace.
//
// Why it exists: some callers cannot allocate device memory at the moment they
// need a render.  Examples: a plug-in running inside a host application that
// owns the GPU's memory budget and gives plug-ins no allocator; a per-frame
// callback on a latency-critical thread, where cudaMalloc can block on a
// device-wide lock and stall the frame.  Such a caller still supplies its
// inputs (scenes, views) and its output images; everything else comes from the
// array below.
//
// Limit: kStaticScratchBytes (32 MiB) per device, reserved by every GPU that
// loads this library until the process exits.  That covers, e.g., a 640x480
// view of ~100k Gaussians.  Larger requests are rejected on the host with
// GS_ERR_INVALID_ARG.
#include <cstdio>
#include <mutex>
#include <string>

#include "gsr_internal.cuh"

namespace {

constexpr size_t kStaticScratchBytes = size_t(32) << 20;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_scratch[kStaticScratchBytes];

// Host-side names of device symbols are stand-ins, not device addresses: the
// device address of g_scratch is looked up once per device (with that device
// current) and cached here.
std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices] = {nullptr};

}  // namespace

extern "C" GS_API gs_status gs_render_forward_static(gs_ctx* ctx, const gs_scene* scenes, int n_scenes,
                                                    const gs_view* views, int n_views, int64_t max_pairs,
                                                    const gs_images* out, void* stream) {
  if (!ctx) return GS_ERR_INVALID_ARG;
  size_t need = 0;
  gs_status s = gs_workspace_query(ctx, scenes, n_scenes, views, n_views, max_pairs, &need);
  if (s != GS_OK) return s;
  if (need > kStaticScratchBytes) {
    gsr::set_ctx_error(ctx, "gs_render_forward_static: this call needs %zu bytes of scratch; the static "
                            "scratch array holds %zu bytes (use gs_render_forward with a workspace)",
                       need, kStaticScratchBytes);
    return GS_ERR_INVALID_ARG;
  }
  const int dev = gsr::ctx_device(ctx);
  if (dev < 0 || dev >= kMaxDevices) return GS_ERR_UNSUPPORTED;
  void* ptr = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    if (g_scratch_ptr[dev] == nullptr) {
      int prev = -1;
      cudaGetDevice(&prev);
      cudaError_t e = cudaSetDevice(dev);
      void* p = nullptr;
      if (e == cudaSuccess) e = cudaGetSymbolAddress(&p, g_scratch);
      if (prev >= 0) cudaSetDevice(prev);
      if (e != cudaSuccess) {
        gsr::set_ctx_error(ctx, "gs_render_forward_static: cudaGetSymbolAddress failed: %s",
                           cudaGetErrorString(e));
        return GS_ERR_CUDA;
      }
      g_scratch_ptr[dev] = p;
    }
    ptr = g_scratch_ptr[dev];
  }
  // The existing forward, pointed at the static array.  It clears the parts of
  // the scratch that must start at zero on every call.
  s = gs_render_forward(ctx, scenes, n_scenes, views, n_views, ptr, kStaticScratchBytes, max_pairs, out, stream);
  // the next call overwrites the array, so no backward may ever use this forward
  gsr::ctx_forget_forward(ctx, ptr);
  return s;
}

// The device-side status of the last gs_render_forward_static on the context's
// device: the sticky flags its kernels set in the static array's header (pair
// capacity exceeded, a bounded wait that ran out).  Synchronises `stream`.
extern "C" GS_API gs_status gs_render_forward_static_status(gs_ctx* ctx, void* stream, int64_t* pairs_needed) {
  if (!ctx) return GS_ERR_INVALID_ARG;
  const int dev = gsr::ctx_device(ctx);
  if (dev < 0 || dev >= kMaxDevices) return GS_ERR_UNSUPPORTED;
  void* ptr = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    ptr = g_scratch_ptr[dev];
  }
  if (ptr == nullptr) {
    gsr::set_ctx_error(ctx, "gs_render_forward_static_status: no static forward has run on device %d", dev);
    return GS_ERR_STATE;
  }
  return gs_workspace_status(ctx, ptr, stream, pairs_needed);
}
