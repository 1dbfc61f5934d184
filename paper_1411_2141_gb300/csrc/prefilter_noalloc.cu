// mreg_prefilter_noalloc: the cubic B-spline prefilter of one image for
// callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: hosts that hand every byte of device
// memory to their own pool (a framework's caching allocator, an embedding
// runtime with a fixed memory budget) and forbid allocations behind the
// pool's back, and latency-bound loops that must not pay for
// cudaMalloc/cudaFree, which synchronise the device.  For them this entry
// point runs the same two prefilter kernels as the library's set-up, but
// takes the intermediate image (the result of the row pass) from a fixed
// scratch array that is part of the library itself.
//
// The scratch is a file-scope __device__ array of kNoAllocMaxPixels floats
// (4 MiB).  Every GPU that loads the library holds it until the process
// exits.  Host code may not use the array's name as a device address: it
// stands for a host-side shadow, so the device address is looked up with
// cudaGetSymbolAddress once per device, on the first call made on that
// device, with the device current.
#include <mutex>

#include "mreg.h"
#include "mreg_internal.h"

namespace {

constexpr int64_t kNoAllocMaxPixels = MREG_NOALLOC_MAX_PIXELS;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) float g_prefilter_scratch[kNoAllocMaxPixels];

std::mutex g_mutex;
float* g_scratch_ptr[kMaxDevices] = {};

}  // namespace

namespace mreg {
// shared with api.cpp: thread-local error text of the C ABI
mreg_status set_error(mreg_status st, const char* msg);
}  // namespace mreg

namespace {

// The kernels may only be given memory that the current device can use as
// its own: device (or managed) memory of device dev.  A host pointer, or
// memory of another GPU, is rejected before anything is launched.
mreg_status check_device_pointer(const void* p, int dev, const char* what) {
  cudaPointerAttributes at{};
  const cudaError_t e = cudaPointerGetAttributes(&at, p);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();   // the query's error is not sticky; clear it
    return mreg::set_error(MREG_ERR_INVALID_ARG, what);
  }
  if ((at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged) || at.device != dev)
    return mreg::set_error(MREG_ERR_INVALID_ARG, what);
  return MREG_OK;
}

}  // namespace

extern "C" mreg_status mreg_prefilter_noalloc(const float* img_dev, int64_t row_stride,
                                              float* coef_dev, int32_t width, int32_t height,
                                              void* stream) {
  if (!img_dev || !coef_dev)
    return mreg::set_error(MREG_ERR_INVALID_ARG, "mreg_prefilter_noalloc: NULL image or output");
  if (width < 2 || height < 2)
    return mreg::set_error(MREG_ERR_INVALID_ARG,
                           "mreg_prefilter_noalloc: the image must be at least 2x2 pixels");
  if (row_stride < width)
    return mreg::set_error(MREG_ERR_INVALID_ARG, "mreg_prefilter_noalloc: row_stride < width");
  if ((int64_t)width * height > kNoAllocMaxPixels)
    return mreg::set_error(MREG_ERR_INVALID_ARG,
                           "mreg_prefilter_noalloc: width * height exceeds the fixed scratch of "
                           "MREG_NOALLOC_MAX_PIXELS (1024 * 1024) pixels");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return mreg::set_error(MREG_ERR_CUDA, cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices)
    return mreg::set_error(MREG_ERR_INVALID_ARG, "mreg_prefilter_noalloc: device index too large");
  mreg_status st = check_device_pointer(
      img_dev, dev, "mreg_prefilter_noalloc: the image is not device memory of the current device");
  if (st != MREG_OK) return st;
  st = check_device_pointer(
      coef_dev, dev, "mreg_prefilter_noalloc: the output is not device memory of the current device");
  if (st != MREG_OK) return st;
  float* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_scratch_ptr[dev]) {
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_prefilter_scratch);
      if (e != cudaSuccess) return mreg::set_error(MREG_ERR_CUDA, cudaGetErrorString(e));
      g_scratch_ptr[dev] = static_cast<float*>(p);
    }
    scratch = g_scratch_ptr[dev];
  }
  // The row pass writes every scratch element that the column pass reads, so
  // nothing needs clearing between calls.
  e = mreg::launch_prefilter(img_dev, row_stride, scratch, coef_dev, width, height,
                             (cudaStream_t)stream);
  if (e != cudaSuccess) return mreg::set_error(MREG_ERR_CUDA, cudaGetErrorString(e));
  return MREG_OK;
}
