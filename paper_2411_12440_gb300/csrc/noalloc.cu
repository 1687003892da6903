// ls_duplicate_sort_noalloc: the duplication + sort stage for callers that
// cannot allocate device memory (see include/ls.h).  Its scratch is one
// file-scope device array; this file only finds that array's device address
// and hands it to ls_duplicate_sort as the workspace.
#include <mutex>

#include "kernels.h"

namespace {

// Shared by every call on a device; holds LS_NOALLOC_SCRATCH_BYTES until exit.
static __device__ __align__(256) unsigned char g_noalloc_scratch[LS_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices] = {nullptr};

// Device address of g_noalloc_scratch on the current device.  In host code the
// array's name is only a host-side stand-in, so the address is looked up once
// per device and cached.
cudaError_t scratch_for_current_device(void** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" ls_status ls_duplicate_sort_noalloc(int64_t n_records, const void* proj, const ls_camera* cams,
                                               int32_t n_cams, const ls_params* params, int64_t key_capacity,
                                               uint32_t* keys, uint32_t* vals, int64_t* n_keys_dev,
                                               int32_t* tile_ranges, int32_t* status_dev, void* stream) {
  // the tile count under ls_duplicate_sort's own parameter and camera rules
  // (so a size that would overflow the count is rejected before it is formed)
  int64_t tiles = 0;
  if (!ls::host_total_tiles(cams, n_cams, params, &tiles) || tiles < 1) return LS_ERR_INVALID_ARG;
  if (n_records < 0 || key_capacity < 0) return LS_ERR_INVALID_ARG;
  if (n_records > LS_NOALLOC_MAX_RECORDS || key_capacity > LS_NOALLOC_MAX_KEYS) return LS_ERR_UNSUPPORTED;
  const size_t need = ls_duplicate_sort_workspace(n_records, key_capacity, (int32_t)tiles);
  if (need == 0) return LS_ERR_INVALID_ARG;
  if (need > (size_t)LS_NOALLOC_SCRATCH_BYTES) return LS_ERR_UNSUPPORTED;
  void* scratch = nullptr;
  if (scratch_for_current_device(&scratch) != cudaSuccess) return LS_ERR_CUDA;
  return ls_duplicate_sort(n_records, proj, cams, n_cams, params, key_capacity, keys, vals, n_keys_dev, tile_ranges,
                           scratch, (size_t)LS_NOALLOC_SCRATCH_BYTES, status_dev, stream);
}
