// Copies between pinned host memory and device memory for end-to-end steps
// (inputs up, results down), through the copy engines.  An SM-driven copy
// (16-byte words, four loads in flight per thread) was measured on GB300: the
// same ~210 GB/s as the copy engines one way, and ~117 instead of ~170 GB/s
// each way with both directions busy, so the engines do the moving.  The
// entry point checks that both sides are device-addressable first, so a
// pageable host buffer is refused instead of silently staged.
#include "kernels.h"

namespace {

// Device-addressable: device or managed memory, or host memory pinned
// through the CUDA runtime (registered with the driver).
bool device_addressable(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    (void)cudaGetLastError();  // an unregistered pointer is not a sticky error
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged ||
         (a.type == cudaMemoryTypeHost && a.devicePointer == p);
}

}  // namespace

extern "C" ls_status ls_copy(void* dst, const void* src, size_t bytes, void* stream) {
  if (bytes == 0) return LS_OK;
  if (!dst || !src) return LS_ERR_INVALID_ARG;
  if (!device_addressable(dst) || !device_addressable(src)) return LS_ERR_INVALID_ARG;
  return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, static_cast<cudaStream_t>(stream)) == cudaSuccess
             ? LS_OK
             : LS_ERR_CUDA;
}
