// Host-link copies and a throughput probe.
//
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
// through the CUDA runtime (page-locked and mapped for the device).
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

// ---------------------------------------------------------------- FP32 issue probe
// Dependent-free FMA throughput, the denominator of the blending rooflines
// checked by measurement: every thread runs `iters` rounds of eight
// independent FMA chains (8 FP32 lane instructions per round).
namespace {

__global__ void __launch_bounds__(256) fma_probe_kernel(int64_t iters, float seed, float* out) {
  float a[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) a[k] = seed + (float)(threadIdx.x + k);
  const float m = 0.999999f, c = 1e-7f;
  for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = __fmaf_rn(a[k], m, c);
  }
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < 8; ++k) s += a[k];
  if (s == 1234.5678f) out[0] = s;  // keeps the chains live; practically never taken
}

}  // namespace

extern "C" ls_status ls_fp32_issue_probe(int64_t iters, int32_t blocks_per_sm, float* out, int64_t* lane_ops,
                                         void* stream) {
  if (iters <= 0 || blocks_per_sm <= 0 || !out || !lane_ops) return LS_ERR_INVALID_ARG;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev))
    return LS_ERR_CUDA;
  const int64_t blocks = (int64_t)sms * blocks_per_sm;
  fma_probe_kernel<<<(unsigned)blocks, 256, 0, static_cast<cudaStream_t>(stream)>>>(iters, 1.f, out);
  *lane_ops = blocks * 256 * iters * 8;
  return cudaGetLastError() == cudaSuccess ? LS_OK : LS_ERR_CUDA;
}
