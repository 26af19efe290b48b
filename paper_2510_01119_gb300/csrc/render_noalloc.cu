// i4d_render_bwd_noalloc: the backward of i4d_render_bwd with its per-(view, Gaussian) 2D-gradient
// scratch held in a fixed file-scope device array instead of a caller-supplied buffer, so that the
// call allocates nothing.
//
// Who needs it: callers that may not allocate device memory at the point where they run the
// backward -- a plain C/C++ host (an engine or viewer plugin) whose device heap is owned by its own
// memory manager, or a real-time loop that must not call cudaMalloc (it can synchronise the device
// and stall the frame).  They still pass every input and output; only the scratch moves here.
//
// Costs and rules:
//   - the array (kNoAllocMaxRecords x 9 floats = 18 MiB) is held by every GPU that loads the library,
//     until the process exits;
//   - every call shares it: calls that overlap on the GPU (different streams, or different host
//     threads without ordering) race on it and corrupt each other's gradients;
//   - it keeps the last call's contents, so each call clears it before use;
//   - each call looks up the array's device address with the caller's device current
//     (cudaGetSymbolAddress), so a context torn down and recreated between calls (cudaDeviceReset)
//     gets the array's new address; while the stream is being captured the lookup is skipped and the
//     address of the device's last uncaptured call is used, so the first call on a device must come
//     before any stream capture.
#include <mutex>

#include "kernels.cuh"

namespace i4d {

namespace {

constexpr int64_t kNoAllocMaxRecords = 1 << 19;  // n_views * n <= 524,288
constexpr int kMaxDevices = 64;

static __device__ __align__(256) float g_noalloc_grad2d[I4D_GRAD2D_FLOATS * kNoAllocMaxRecords];

std::mutex g_noalloc_mu;
void* g_noalloc_ptr[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device (host code may not use the symbol
// itself: on the host it names a stand-in, not device memory).  Looked up on every call made
// outside a stream capture; during a capture the last looked-up address of the device is used.
cudaError_t scratch_address(cudaStream_t stream, void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  e = cudaStreamIsCapturing(stream, &cap);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (cap == cudaStreamCaptureStatusNone) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_grad2d);
    if (e != cudaSuccess) return e;
    g_noalloc_ptr[dev] = p;
  } else if (!g_noalloc_ptr[dev]) {
    return cudaErrorStreamCaptureUnsupported;  // no uncaptured call on this device yet
  }
  *out = g_noalloc_ptr[dev];
  return cudaSuccess;
}

}  // namespace

}  // namespace i4d

using namespace i4d;

extern "C" {

int64_t i4d_render_bwd_noalloc_max_records(void) { return kNoAllocMaxRecords; }

int32_t i4d_render_bwd_noalloc(const i4d_gaussians* g, const i4d_views* views, const i4d_camera* cams,
                               const i4d_settings* settings, const float* proj, const uint32_t* touched,
                               const uint32_t* ids, const uint32_t* ranges, const float* T_final,
                               const uint32_t* last, const float* dL_dimg, float* grads, void* stream) {
  if (!g || g->n < 0 || g->sh_deg < 0 || g->sh_deg > 3 || g->mode < 0 || g->mode > 2) return I4D_ERR_ARG;
  if (!views || views->n_views < 1 || views->n_views > I4D_MAX_VIEWS) return I4D_ERR_ARG;
  if ((int64_t)views->n_views * g->n > kNoAllocMaxRecords) return I4D_ERR_CAPACITY;  // beyond the fixed scratch
  if (g->n == 0) return I4D_OK;
  void* scratch = nullptr;
  if (scratch_address((cudaStream_t)stream, &scratch) != cudaSuccess) return I4D_ERR_CUDA;
  // same computation as i4d_render_bwd, with the fixed array as its 2D-gradient scratch (the
  // backward clears the scratch before accumulating into it)
  return i4d_render_bwd(g, views, cams, settings, proj, touched, ids, ranges, T_final, last, dL_dimg,
                        reinterpret_cast<float*>(scratch), grads, stream);
}

}  // extern "C"
