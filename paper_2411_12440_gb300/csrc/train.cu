// Training-side consumers of the backward: the image loss of the appendix
// "Loss Functions" (L = w1 L1 + w2 L2 + w3 (1 - SSIM), 6:2:2 in the paper)
// with its gradient with respect to the rendered image, and an Adam step for
// the primitive parameters (used by the pattern fits of Sec. 5.1, Fig. 5).
//
// SSIM as 3DGS computes it (the paper only names it): per channel, an
// 11 x 11 Gaussian window (sigma 1.5, taps normalised to sum 1), zero
// outside the image, C1 = 0.01^2, C2 = 0.03^2, averaged over pixels and
// channels.  Its gradient is the adjoint of the five window sums: with P =
// dS/dmx - 2 mx dS/dsxx - my dS/dsxy, Q = dS/dsxx and R = dS/dsxy per pixel
// (the statistics mx, sxx, sxy taken as independent), dSSIM/dx = G*P +
// 2 x G*Q + y G*R, where G* is the same (symmetric) window.
//
// Both passes are tiled separable filters: a block stages a 32 x 8 output
// tile plus a 5-pixel halo of each input channel in shared memory, sums
// along rows, then along columns.  Partial sums of the loss terms are
// written per block and reduced in a fixed order (deterministic).
#include <cmath>

#include "kernels.h"

namespace ls {

namespace {

constexpr int SS_R = 5;                      // window radius (11 taps)
constexpr int SS_TX = 32, SS_TY = 8;         // output tile
constexpr int SS_HX = SS_TX + 2 * SS_R, SS_HY = SS_TY + 2 * SS_R;
constexpr int SS_THREADS = SS_TX * SS_TY;
constexpr float SS_C1 = 0.01f * 0.01f, SS_C2 = 0.03f * 0.03f;

__constant__ float c_gauss[2 * SS_R + 1];

// Block sum of three values; thread 0 gets them.
__device__ __forceinline__ void block_sum3(float& a, float& b, float& c, float (*s_red)[SS_THREADS / 32]) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
    c += __shfl_xor_sync(0xffffffffu, c, o);
  }
  if (lane == 0) {
    s_red[0][warp] = a;
    s_red[1][warp] = b;
    s_red[2][warp] = c;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    a = b = c = 0.f;
    for (int w = 0; w < SS_THREADS / 32; ++w) {
      a += s_red[0][w];
      b += s_red[1][w];
      c += s_red[2][w];
    }
  }
}

// Stage channel ch of `n` interleaved [H][W][3] images into halo tiles.
template <int NIN>
__device__ __forceinline__ void stage_halo(const float* const* img, int H, int W, int ch, int gx0, int gy0,
                                           float (*s)[SS_HY][SS_HX]) {
  for (int i = threadIdx.x; i < SS_HY * SS_HX; i += SS_THREADS) {
    const int r = i / SS_HX, c = i % SS_HX;
    const int gx = gx0 + c, gy = gy0 + r;
    const bool in = gx >= 0 && gx < W && gy >= 0 && gy < H;
    const size_t pi = 3 * ((size_t)gy * W + gx) + ch;
#pragma unroll
    for (int k = 0; k < NIN; ++k) s[k][r][c] = in ? img[k][pi] : 0.f;
  }
}

// Forward: the SSIM map, its adjoint maps P, Q, R, and per-block sums of
// SSIM, |x - y| and (x - y)^2.
__global__ void __launch_bounds__(SS_THREADS) ssim_fwd_kernel(int H, int W, const float* __restrict__ pred,
                                                              const float* __restrict__ target,
                                                              float* __restrict__ mapP, float* __restrict__ mapQ,
                                                              float* __restrict__ mapR, float* __restrict__ partial) {
  __shared__ float s_in[2][SS_HY][SS_HX];
  __shared__ float s_h[5][SS_HY][SS_TX];
  __shared__ float s_red[3][SS_THREADS / 32];
  const int tx = threadIdx.x % SS_TX, ty = threadIdx.x / SS_TX;
  const int gx0 = blockIdx.x * SS_TX - SS_R, gy0 = blockIdx.y * SS_TY - SS_R;
  const int px = blockIdx.x * SS_TX + tx, py = blockIdx.y * SS_TY + ty;
  const bool out = px < W && py < H;
  const float* imgs[2] = {pred, target};
  float acc_s = 0.f, acc_l1 = 0.f, acc_l2 = 0.f;
  for (int ch = 0; ch < 3; ++ch) {
    __syncthreads();  // the previous channel is done with shared memory
    stage_halo<2>(imgs, H, W, ch, gx0, gy0, s_in);
    __syncthreads();
    for (int i = threadIdx.x; i < SS_HY * SS_TX; i += SS_THREADS) {
      const int r = i / SS_TX, c = i % SS_TX;
      float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f, a4 = 0.f;
#pragma unroll
      for (int k = 0; k <= 2 * SS_R; ++k) {
        const float g = c_gauss[k], x = s_in[0][r][c + k], y = s_in[1][r][c + k];
        a0 += g * x;
        a1 += g * y;
        a2 += g * x * x;
        a3 += g * y * y;
        a4 += g * x * y;
      }
      s_h[0][r][c] = a0;
      s_h[1][r][c] = a1;
      s_h[2][r][c] = a2;
      s_h[3][r][c] = a3;
      s_h[4][r][c] = a4;
    }
    __syncthreads();
    float m[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int k = 0; k <= 2 * SS_R; ++k) {
      const float g = c_gauss[k];
#pragma unroll
      for (int q = 0; q < 5; ++q) m[q] += g * s_h[q][ty + k][tx];
    }
    if (out) {
      const float mx = m[0], my = m[1];
      const float sxx = m[2] - mx * mx, syy = m[3] - my * my, sxy = m[4] - mx * my;
      const float a1 = 2.f * mx * my + SS_C1, a2 = 2.f * sxy + SS_C2;
      const float b1 = mx * mx + my * my + SS_C1, b2 = sxx + syy + SS_C2;
      const float inv = 1.f / (b1 * b2);
      const float s = a1 * a2 * inv;
      const float ds_dmx = 2.f * my * a2 * inv - s * 2.f * mx / b1;
      const float ds_dsxx = -s / b2;
      const float ds_dsxy = 2.f * a1 * inv;
      const size_t pi = 3 * ((size_t)py * W + px) + ch;
      mapP[pi] = ds_dmx - 2.f * mx * ds_dsxx - my * ds_dsxy;
      mapQ[pi] = ds_dsxx;
      mapR[pi] = ds_dsxy;
      const float d = s_in[0][ty + SS_R][tx + SS_R] - s_in[1][ty + SS_R][tx + SS_R];
      acc_s += s;
      acc_l1 += fabsf(d);
      acc_l2 += d * d;
    }
  }
  block_sum3(acc_s, acc_l1, acc_l2, s_red);
  if (threadIdx.x == 0) {
    const size_t b = (size_t)blockIdx.y * gridDim.x + blockIdx.x;
    partial[3 * b] = acc_s;
    partial[3 * b + 1] = acc_l1;
    partial[3 * b + 2] = acc_l2;
  }
}

// Backward: grad = (w1 sign(x - y) + w2 2 (x - y) - w3 (G*P + 2 x G*Q + y G*R)) / N.
__global__ void __launch_bounds__(SS_THREADS) ssim_bwd_kernel(int H, int W, const float* __restrict__ pred,
                                                              const float* __restrict__ target,
                                                              const float* __restrict__ mapP,
                                                              const float* __restrict__ mapQ,
                                                              const float* __restrict__ mapR, float w1, float w2,
                                                              float w3, float inv_n, float* __restrict__ grad) {
  __shared__ float s_in[3][SS_HY][SS_HX];
  __shared__ float s_h[3][SS_HY][SS_TX];
  const int tx = threadIdx.x % SS_TX, ty = threadIdx.x / SS_TX;
  const int gx0 = blockIdx.x * SS_TX - SS_R, gy0 = blockIdx.y * SS_TY - SS_R;
  const int px = blockIdx.x * SS_TX + tx, py = blockIdx.y * SS_TY + ty;
  const bool out = px < W && py < H;
  const float* maps[3] = {mapP, mapQ, mapR};
  for (int ch = 0; ch < 3; ++ch) {
    __syncthreads();
    stage_halo<3>(maps, H, W, ch, gx0, gy0, s_in);
    __syncthreads();
    for (int i = threadIdx.x; i < SS_HY * SS_TX; i += SS_THREADS) {
      const int r = i / SS_TX, c = i % SS_TX;
      float a0 = 0.f, a1 = 0.f, a2 = 0.f;
#pragma unroll
      for (int k = 0; k <= 2 * SS_R; ++k) {
        const float g = c_gauss[k];
        a0 += g * s_in[0][r][c + k];
        a1 += g * s_in[1][r][c + k];
        a2 += g * s_in[2][r][c + k];
      }
      s_h[0][r][c] = a0;
      s_h[1][r][c] = a1;
      s_h[2][r][c] = a2;
    }
    __syncthreads();
    float bp = 0.f, bq = 0.f, br = 0.f;
#pragma unroll
    for (int k = 0; k <= 2 * SS_R; ++k) {
      const float g = c_gauss[k];
      bp += g * s_h[0][ty + k][tx];
      bq += g * s_h[1][ty + k][tx];
      br += g * s_h[2][ty + k][tx];
    }
    if (out) {
      const size_t pi = 3 * ((size_t)py * W + px) + ch;
      const float x = pred[pi], y = target[pi], d = x - y;
      const float sgn = d > 0.f ? 1.f : (d < 0.f ? -1.f : 0.f);
      const float dssim = bp + 2.f * x * bq + y * br;
      grad[pi] = (w1 * sgn + w2 * 2.f * d - w3 * dssim) * inv_n;
    }
  }
}

// out[0] = total loss, out[1] = L1, out[2] = L2, out[3] = SSIM, from the
// per-block sums (summed in double, in a fixed order).
__global__ void __launch_bounds__(256) loss_final_kernel(const float* __restrict__ partial, int blocks, float w1,
                                                         float w2, float w3, double inv_n, float* __restrict__ out) {
  __shared__ double s_red[3][256];
  double a = 0.0, b = 0.0, c = 0.0;
  for (int i = threadIdx.x; i < blocks; i += 256) {
    a += partial[3 * i];
    b += partial[3 * i + 1];
    c += partial[3 * i + 2];
  }
  s_red[0][threadIdx.x] = a;
  s_red[1][threadIdx.x] = b;
  s_red[2][threadIdx.x] = c;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o)
      for (int k = 0; k < 3; ++k) s_red[k][threadIdx.x] += s_red[k][threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double ssim = s_red[0][0] * inv_n, l1 = s_red[1][0] * inv_n, l2 = s_red[2][0] * inv_n;
    out[0] = (float)(w1 * l1 + w2 * l2 + w3 * (1.0 - ssim));
    out[1] = (float)l1;
    out[2] = (float)l2;
    out[3] = (float)ssim;
  }
}

// Adam in the unconstrained space of the parameter (mode 0: p, 1: log p,
// 2: logit p), bias-corrected.
__global__ void __launch_bounds__(256) adam_kernel(int64_t n, float* __restrict__ p, const float* __restrict__ g,
                                                   float* __restrict__ m, float* __restrict__ v, float lr, float b1,
                                                   float b2, float eps, float c1, float c2, int mode) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float pi = p[i];
    float gu = g[i];
    if (mode == 1) gu *= pi;
    else if (mode == 2) gu *= pi * (1.f - pi);
    const float mi = b1 * m[i] + (1.f - b1) * gu;
    const float vi = b2 * v[i] + (1.f - b2) * gu * gu;
    m[i] = mi;
    v[i] = vi;
    const float step = lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    if (mode == 1) {
      p[i] = pi * expf(-step);
    } else if (mode == 2) {
      const float u = logf(pi / (1.f - pi)) - step;
      p[i] = 1.f / (1.f + expf(-u));
    } else {
      p[i] = pi - step;
    }
  }
}

// Densification statistics (reading of the appendix's threshold table as the
// gsplat v1.3 default strategy applies it): per view, every primitive whose
// support box meets the image adds |(dL/dmx W/2 n, dL/dmy H/2 n)| to its
// accumulator, counts the view and keeps its largest support radius over
// max(W, H).  Binary32, each operation rounded once.
__global__ void __launch_bounds__(256) densify_accum_kernel(int n, const float* __restrict__ g2d,
                                                            const float4* __restrict__ foot,
                                                            const uint32_t* __restrict__ dkey, int W, int H,
                                                            float sx, float sy, float inv_wh,
                                                            float* __restrict__ accum, int32_t* __restrict__ count,
                                                            float* __restrict__ max_radius) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n || dkey[i] == DKEY_CULLED) return;
  const float4 f = foot[i];
  int tx0, tx1, ty0, ty1;
  if (!tile_rect(f.x, f.y, f.z, f.w, W, H, 1, 1, tx0, tx1, ty0, ty1)) return;
  const float gx = __fmul_rn(g2d[12 * (size_t)i], sx), gy = __fmul_rn(g2d[12 * (size_t)i + 1], sy);
  const float nrm = __fsqrt_rn(__fadd_rn(__fmul_rn(gx, gx), __fmul_rn(gy, gy)));
  accum[i] = __fadd_rn(accum[i], nrm);
  count[i] += 1;
  max_radius[i] = fmaxf(max_radius[i], __fmul_rn(fmaxf(f.z, f.w), inv_wh));
}

struct DensifyTh {
  float grad2d, grow2d, grow3d_ext, prune2d, prune3d_ext, prune_opac;
  int use2d, use_prune3d;
};

// Flags: bit 0 duplicate, bit 1 split, bit 2 prune; counts[3] of each.
__global__ void __launch_bounds__(256) densify_decide_kernel(int n, const float* __restrict__ accum,
                                                             const int32_t* __restrict__ count,
                                                             const float* __restrict__ max_radius,
                                                             const float* __restrict__ scales,
                                                             const float* __restrict__ opac, const DensifyTh th,
                                                             uint8_t* __restrict__ flags,
                                                             unsigned long long* __restrict__ counts) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  unsigned fl = 0u;
  if (i < n) {
    const float g = __fdiv_rn(accum[i], (float)max(count[i], 1));
    const float smax = fmaxf(fmaxf(scales[3 * (size_t)i], scales[3 * (size_t)i + 1]), scales[3 * (size_t)i + 2]);
    const bool grow = g > th.grad2d;
    const bool small = smax <= th.grow3d_ext;
    bool split = grow && !small;
    bool prune = opac[i] < th.prune_opac;
    if (th.use_prune3d) prune = prune || smax > th.prune3d_ext;
    if (th.use2d) {
      split = split || max_radius[i] > th.grow2d;
      prune = prune || max_radius[i] > th.prune2d;
    }
    fl = (grow && small ? 1u : 0u) | (split ? 2u : 0u) | (prune ? 4u : 0u);
    flags[i] = (uint8_t)fl;
  }
  if (counts) {
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      const unsigned c = __popc(__ballot_sync(FULL, (fl >> b) & 1u));
      if (lane == 0 && c) atomicAdd(&counts[b], (unsigned long long)c);
    }
  }
}

bool g_gauss_set[64] = {false};

cudaError_t ensure_gauss() {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  if (g_gauss_set[dev]) return cudaSuccess;
  float taps[2 * SS_R + 1];
  double sum = 0.0, t[2 * SS_R + 1];
  for (int k = -SS_R; k <= SS_R; ++k) sum += t[k + SS_R] = std::exp(-(double)(k * k) / (2.0 * 1.5 * 1.5));
  for (int k = 0; k <= 2 * SS_R; ++k) taps[k] = (float)(t[k] / sum);
  e = cudaMemcpyToSymbol(c_gauss, taps, sizeof(taps));
  if (e == cudaSuccess) g_gauss_set[dev] = true;
  return e;
}

}  // namespace

size_t image_loss_ws_bytes(int H, int W) {
  const size_t px = (size_t)H * W * 3;
  const size_t blocks = (size_t)ceil_div(W, SS_TX) * ceil_div(H, SS_TY);
  auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
  return 3 * al(4 * px) + al(4 * 3 * blocks);
}

cudaError_t launch_image_loss(int H, int W, const float* pred, const float* target, float w1, float w2, float w3,
                              float* loss_out, float* grad, void* ws, cudaStream_t st) {
  cudaError_t e = ensure_gauss();
  if (e != cudaSuccess) return e;
  const size_t px = (size_t)H * W * 3;
  auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
  char* b = static_cast<char*>(ws);
  float* mapP = reinterpret_cast<float*>(b);
  float* mapQ = reinterpret_cast<float*>(b + al(4 * px));
  float* mapR = reinterpret_cast<float*>(b + 2 * al(4 * px));
  float* partial = reinterpret_cast<float*>(b + 3 * al(4 * px));
  const dim3 grid(ceil_div(W, SS_TX), ceil_div(H, SS_TY));
  ssim_fwd_kernel<<<grid, SS_THREADS, 0, st>>>(H, W, pred, target, mapP, mapQ, mapR, partial);
  loss_final_kernel<<<1, 256, 0, st>>>(partial, (int)(grid.x * grid.y), w1, w2, w3, 1.0 / (double)px, loss_out);
  if (grad)
    ssim_bwd_kernel<<<grid, SS_THREADS, 0, st>>>(H, W, pred, target, mapP, mapQ, mapR, w1, w2, w3,
                                                 (float)(1.0 / (double)px), grad);
  return cudaGetLastError();
}

cudaError_t launch_densify_accum(int n, const float* g2d, const float4* foot, const uint32_t* dkey, int W, int H,
                                 int n_cams, float* accum, int32_t* count, float* max_radius, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const float sx = ((float)W * 0.5f) * (float)n_cams, sy = ((float)H * 0.5f) * (float)n_cams;
  const float inv_wh = 1.f / (float)(W > H ? W : H);
  densify_accum_kernel<<<ceil_div(n, 256), 256, 0, st>>>(n, g2d, foot, dkey, W, H, sx, sy, inv_wh, accum, count,
                                                        max_radius);
  return cudaGetLastError();
}

cudaError_t launch_densify_decide(int n, const float* accum, const int32_t* count, const float* max_radius,
                                  const float* scales, const float* opac, float extent, const ls_densify_params& p,
                                  uint8_t* flags, int64_t* counts, cudaStream_t st) {
  if (counts) {
    cudaError_t e = cudaMemsetAsync(counts, 0, 3 * sizeof(int64_t), st);
    if (e != cudaSuccess) return e;
  }
  if (n <= 0) return cudaSuccess;
  DensifyTh th;
  th.grad2d = p.grad2d;
  th.grow2d = p.grow_scale2d;
  th.grow3d_ext = p.grow_scale3d * extent;
  th.prune2d = p.prune_scale2d;
  th.prune3d_ext = p.prune_scale3d * extent;
  th.prune_opac = p.prune_opacity;
  th.use2d = p.use_scale2d;
  th.use_prune3d = p.use_prune_scale3d;
  densify_decide_kernel<<<ceil_div(n, 256), 256, 0, st>>>(n, accum, count, max_radius, scales, opac, th, flags,
                                                         reinterpret_cast<unsigned long long*>(counts));
  return cudaGetLastError();
}

cudaError_t launch_adam(int64_t n, float* p, const float* g, float* m, float* v, int step, float lr, float b1,
                        float b2, float eps, int mode, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  int sms = 0;
  cudaError_t e = current_sm_count(&sms);
  if (e != cudaSuccess) return e;
  const int64_t need = (n + 255) / 256;
  const unsigned grid = (unsigned)(need < 8 * sms ? need : 8 * sms);
  const float c1 = 1.f - (float)std::pow((double)b1, step), c2 = 1.f - (float)std::pow((double)b2, step);
  adam_kernel<<<grid, 256, 0, st>>>(n, p, g, m, v, lr, b1, b2, eps, c1, c2, mode);
  return cudaGetLastError();
}

}  // namespace ls
