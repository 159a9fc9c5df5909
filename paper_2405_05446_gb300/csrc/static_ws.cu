// gdgs_poisson_reconstruct_static: the Poisson reconstruction with its scratch
// in a fixed device array of the library instead of a caller workspace.
//
// It exists for callers that cannot allocate device memory when they need the
// solve: code running inside a CUDA stream capture (where cudaMalloc is not
// allowed), plug-ins that run inside a host application owning the device and
// its allocator, and real-time loops that forbid allocation after start-up.
// They pass only inputs and outputs; the scratch is a file-scope __device__
// array of kStaticBytes, held by every GPU that loads the library until the
// process exits.
#include <mutex>

#include "gdgs_internal.cuh"

namespace {

constexpr size_t kStaticBytes = 32ull << 20;  // 32 MiB

__device__ __align__(256) unsigned char g_static_ws[kStaticBytes];

std::mutex g_static_mu;
void *g_static_ptr[64] = {};

// Device address of the array on the current device. In host code the symbol
// only names a host-side stand-in, so the address is looked up once per device
// (with that device current) and remembered.
int static_workspace(void **out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return GDGS_ERR_CUDA;
  std::lock_guard<std::mutex> lk(g_static_mu);
  if (!g_static_ptr[dev]) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_static_ws) != cudaSuccess || !p) {
      cudaGetLastError();
      return GDGS_ERR_CUDA;
    }
    g_static_ptr[dev] = p;
  }
  *out = g_static_ptr[dev];
  return GDGS_OK;
}

}  // namespace

extern "C" int gdgs_poisson_reconstruct_static(const float *grad_maps, const uint8_t *tile_mask,
                                               int32_t channels, int32_t height, int32_t width,
                                               const float *mean, const gdgs_solver_opts *sopts,
                                               float *image, gdgs_solve_stats *stats,
                                               void *stream) {
  const size_t need = gdgs_workspace_size(0, channels, width, height, nullptr, sopts);
  if (need == 0) return GDGS_ERR_INVALID_ARG;
  if (need > kStaticBytes) return GDGS_ERR_WORKSPACE;  // larger than the fixed scratch
  if (stats) {
    // filling stats waits for the stream, which a stream capture does not allow:
    // refuse before anything is enqueued rather than invalidate the capture
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing((cudaStream_t)stream, &cs) != cudaSuccess) {
      cudaGetLastError();
      return GDGS_ERR_CUDA;
    }
    if (cs != cudaStreamCaptureStatusNone) return GDGS_ERR_INVALID_ARG;
  }
  void *ws = nullptr;
  int s = static_workspace(&ws);
  if (s != GDGS_OK) return s;
  s = gdgs_poisson_reconstruct(grad_maps, tile_mask, channels, height, width, mean, sopts, image,
                               ws, kStaticBytes, stream);
  if (s != GDGS_OK || !stats) return s;
  return gdgs_sync_status(ws, stats, stream);
}

extern "C" int gdgs_poisson_static_status(gdgs_solve_stats *stats, void *stream) {
  void *ws = nullptr;
  const int s = static_workspace(&ws);
  if (s != GDGS_OK) return s;
  return gdgs_sync_status(ws, stats, stream);
}
