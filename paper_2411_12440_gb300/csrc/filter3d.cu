// The 3D smoothing filter of the anti-aliased variant (Sec. 4.1 evaluates
// 3DLS+AA with the technique of Mip-Splatting, whose 2D filter is the
// projection's eps2d dilation with opacity compensation).  Reading of the 3D
// filter: each primitive's highest sampling rate over the cameras that see
// its centre, nu = max fx / z (z > near, projected centre within 1.15x the
// image), bounds its frequency: the variance s2 / nu^2 is added to every
// axis of its covariance, so its scales become sqrt(scale^2 + v) and its
// opacity o prod(scale / sqrt(scale^2 + v)), which keeps o sqrt(det Sigma).
// A primitive no camera sees takes the largest variance of the others.
//
// Three small HBM-bound kernels: the variance (one pass over the means and a
// device-wide max for the unseen), the filtered parameters fed to
// ls_project, and the chain rule back to the unfiltered ones.
#include "kernels.h"

namespace ls {

namespace {

__global__ void __launch_bounds__(256) filter3d_rate_kernel(int n, const float* __restrict__ means, const CamTable cams,
                                                            float near_plane, float s2, float* __restrict__ var,
                                                            unsigned* __restrict__ max_bits) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  float v = -1.f;  // not seen by any camera (yet)
  if (i < n) {
    const float mx = means[3 * (size_t)i], my = means[3 * (size_t)i + 1], mz = means[3 * (size_t)i + 2];
    float best = 0.f;
    for (int c = 0; c < cams.n; ++c) {
      const CamDev& C = cams.c[c];
      const float tz = C.R[6] * mx + C.R[7] * my + C.R[8] * mz + C.t[2];
      if (!(tz > near_plane)) continue;
      const float tx = C.R[0] * mx + C.R[1] * my + C.R[2] * mz + C.t[0];
      const float ty = C.R[3] * mx + C.R[4] * my + C.R[5] * mz + C.t[1];
      const float x = C.fx * tx / tz + C.cx, y = C.fy * ty / tz + C.cy;
      if (x >= -0.15f * C.W && x <= 1.15f * C.W && y >= -0.15f * C.H && y <= 1.15f * C.H) best = fmaxf(best, C.fx / tz);
    }
    if (best > 0.f) v = s2 / (best * best);
    var[i] = v;
  }
  // the largest variance of the seen primitives (positive floats order as
  // their bit patterns)
  unsigned b = v > 0.f ? __float_as_uint(v) : 0u;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) b = max(b, __shfl_xor_sync(0xffffffffu, b, o));
  if ((threadIdx.x & 31) == 0 && b) atomicMax(max_bits, b);
}

__global__ void __launch_bounds__(256) filter3d_fill_kernel(int n, float* __restrict__ var,
                                                            const unsigned* __restrict__ max_bits) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && var[i] < 0.f) var[i] = __uint_as_float(*max_bits);
}

__global__ void __launch_bounds__(256) filter3d_apply_kernel(int n, const float* __restrict__ scales,
                                                             const float* __restrict__ opac,
                                                             const float* __restrict__ var, float* __restrict__ s_out,
                                                             float* __restrict__ o_out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float v = var[i];
  float ratio = 1.f;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const float s = scales[3 * (size_t)i + k];
    const float se = sqrtf(s * s + v);
    s_out[3 * (size_t)i + k] = se;
    ratio *= s / se;
  }
  o_out[i] = opac[i] * ratio;
}

// d se_k / d s_k = s_k / se_k; d oe / d o = prod(s / se);
// d oe / d s_k = oe v / (s_k se_k^2).
__global__ void __launch_bounds__(256) filter3d_apply_bwd_kernel(int n, const float* __restrict__ scales,
                                                                 const float* __restrict__ opac,
                                                                 const float* __restrict__ var,
                                                                 const float* __restrict__ g_se,
                                                                 const float* __restrict__ g_oe,
                                                                 float* __restrict__ g_s, float* __restrict__ g_o) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float v = var[i];
  float s[3], se2[3], ratio = 1.f;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    s[k] = scales[3 * (size_t)i + k];
    se2[k] = s[k] * s[k] + v;
    ratio *= s[k] * rsqrtf(se2[k]);
  }
  const float go = g_oe[i];
  const float goe = go * opac[i] * ratio;  // dL/doe times oe
#pragma unroll
  for (int k = 0; k < 3; ++k)
    g_s[3 * (size_t)i + k] = g_se[3 * (size_t)i + k] * s[k] * rsqrtf(se2[k]) + goe * v / (s[k] * se2[k]);
  g_o[i] = go * ratio;
}

}  // namespace

cudaError_t launch_filter3d_variance(int n, const float* means, const CamTable& cams, float near_plane, float s2,
                                     float* var, unsigned* max_bits, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(max_bits, 0, sizeof(unsigned), st);
  if (e != cudaSuccess || n <= 0) return e;
  filter3d_rate_kernel<<<ceil_div(n, 256), 256, 0, st>>>(n, means, cams, near_plane, s2, var, max_bits);
  filter3d_fill_kernel<<<ceil_div(n, 256), 256, 0, st>>>(n, var, max_bits);
  return cudaGetLastError();
}

cudaError_t launch_filter3d_apply(int n, const float* scales, const float* opac, const float* var, float* s_out,
                                  float* o_out, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  filter3d_apply_kernel<<<ceil_div(n, 256), 256, 0, st>>>(n, scales, opac, var, s_out, o_out);
  return cudaGetLastError();
}

cudaError_t launch_filter3d_apply_bwd(int n, const float* scales, const float* opac, const float* var,
                                      const float* g_se, const float* g_oe, float* g_s, float* g_o, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  filter3d_apply_bwd_kernel<<<ceil_div(n, 256), 256, 0, st>>>(n, scales, opac, var, g_se, g_oe, g_s, g_o);
  return cudaGetLastError();
}

}  // namespace ls
