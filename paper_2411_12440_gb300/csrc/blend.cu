// a4 / a5: per-tile front-to-back blending with the linear kernel and its
// adjoint (Sec. 3.1 Eq. 6; kernel of Sec. 3.2 Eq. 11 with the alignment of
// Sec. 3.3.1 Eq. 12; adaptive gradient scaling of Sec. 3.3.2 Eq. 13-14).
//
// One CTA per tile, one thread per pixel.  The tile's sorted record ids are
// walked in batches of one record per thread: each thread gathers one 48-byte
// record into shared memory, then every pixel reads the batch from shared
// memory (broadcast reads), so each record is fetched from L2/HBM once per
// tile and reused by all of the tile's pixels.
//
// Backward: each pixel restarts from its checkpoint (T_final, n_last) and
// walks its list back to front, recovering T before each entry as
// T / (1 - alpha).  Per record, a warp that has any contributing pixel sums
// the nine gradient terms with xor-shuffles, lane 0 adds them into a per-CTA
// shared-memory slot, and after the batch one set of vector atomics per
// (record, CTA) lands in global memory.
#include "kernels.h"

namespace ls {

namespace {

__device__ __forceinline__ float sqrt_approx(float x) {
  float y;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// One (pixel, record) pair, with every rounding explicit so that the forward
// and the backward take bit-identical skip decisions.  The conic is stored as
// its upper Cholesky factor L (A = L^T L), so q = d^T A d = |L d|^2 =
// (l00 dx + l01 dy)^2 + (l11 dy)^2 is a sum of squares: no cancellation even
// for needle-shaped footprints, where a dx^2 + 2 b dx dy + c dy^2 adds terms
// thousands of times larger than q.  Skip when q > rho^2; D = sqrt(q);
// alpha = min(alpha_max, o f(D / lambda)); skip when alpha < alpha_min.
struct PairEval {
  float dx, dy, e1, e2, q, D, xk, f, araw, alpha;
};

template <int KID>
__device__ __forceinline__ bool pair_alpha(float x, float y, const float4& a, const float4& bb, const ParDev& P,
                                           PairEval& e) {
  e.dx = __fsub_rn(x, a.x);
  e.dy = __fsub_rn(y, a.y);
  e.e1 = __fmaf_rn(a.z, e.dx, __fmul_rn(a.w, e.dy));
  e.e2 = __fmul_rn(bb.x, e.dy);
  e.q = __fmaf_rn(e.e1, e.e1, __fmul_rn(e.e2, e.e2));
  if (e.q > bb.z) return false;
  e.D = sqrt_approx(e.q);
  e.xk = __fmul_rn(e.D, P.inv_lambda);
  e.f = kern_f<KID>(e.xk);
  e.araw = __fmul_rn(bb.y, e.f);
  e.alpha = fminf(P.alpha_max, e.araw);
  return e.alpha >= P.alpha_min;
}

// COUNT = true also tallies the work units of the tile method: evaluated
// pairs (per tile, the pixels times the entries walked until the tile's last
// pixel finished) and composited pairs; stats[0], stats[1] (uint64).
template <int KID, bool COUNT>
__global__ void __launch_bounds__(512) blend_fwd_kernel(const float4* __restrict__ rec, const CamDev cam,
                                                        const ParDev P, const int2* __restrict__ ranges,
                                                        const uint32_t* __restrict__ vals, float* __restrict__ image,
                                                        float* __restrict__ t_final, int32_t* __restrict__ n_last,
                                                        unsigned long long* stats) {
  extern __shared__ float4 smem[];
  const int B = blockDim.x;
  float4* s_a = smem;          // {mx, my, l00, l01}
  float4* s_b = smem + B;      // {l11, o, rho2, depth}
  float4* s_c = smem + 2 * B;  // {r, g, b, -}
  const int tile = blockIdx.x;
  const int tx = tile % cam.tiles_x, ty = tile / cam.tiles_x;
  const int px = tx * P.tile_w + (int)threadIdx.x % P.tile_w;
  const int py = ty * P.tile_h + (int)threadIdx.x / P.tile_w;
  const bool inside = px < cam.W && py < cam.H;
  const float x = (float)px + 0.5f, y = (float)py + 0.5f;
  const int2 rg = ranges[cam.tile_base + tile];
  const int n = rg.y - rg.x;
  float T = 1.f, C0 = 0.f, C1 = 0.f, C2 = 0.f;
  int last = 0;
  bool done = !inside;
  int stop = n;         // COUNT: index where this pixel finished
  int composited = 0;   // COUNT
  for (int b0 = 0; b0 < n; b0 += B) {
    if (__syncthreads_and(done)) break;
    const int k = b0 + (int)threadIdx.x;
    if (k < n) {
      const uint32_t id = vals[rg.x + k];
      s_a[threadIdx.x] = rec[3 * (size_t)id];
      s_b[threadIdx.x] = rec[3 * (size_t)id + 1];
      s_c[threadIdx.x] = rec[3 * (size_t)id + 2];
    }
    __syncthreads();
    const int cnt = min(B, n - b0);
    if (!done) {
      for (int j = 0; j < cnt; ++j) {
        PairEval e;
        if (!pair_alpha<KID>(x, y, s_a[j], s_b[j], P, e)) continue;
        const float alpha = e.alpha;
        const float Tn = T * (1.f - alpha);
        if (Tn < P.t_min) {
          done = true;
          if (COUNT) stop = b0 + j;
          break;
        }
        const float4 c = s_c[j];
        const float w = alpha * T;
        C0 += c.x * w;
        C1 += c.y * w;
        C2 += c.z * w;
        T = Tn;
        last = b0 + j + 1;
        if (COUNT) ++composited;
      }
    }
  }
  if (COUNT) {
    __shared__ int s_emax, s_npix;
    __shared__ unsigned long long s_contrib;
    if (threadIdx.x == 0) {
      s_emax = 0;
      s_npix = 0;
      s_contrib = 0;
    }
    __syncthreads();
    if (inside) {
      atomicMax(&s_emax, stop < n ? stop + 1 : n);
      atomicAdd(&s_npix, 1);
      atomicAdd(&s_contrib, (unsigned long long)composited);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      atomicAdd(&stats[0], (unsigned long long)s_emax * (unsigned long long)s_npix);
      atomicAdd(&stats[1], s_contrib);
    }
  }
  if (inside) {
    const size_t p = (size_t)py * cam.W + px;
    image[3 * p] = C0 + T * P.bg[0];
    image[3 * p + 1] = C1 + T * P.bg[1];
    image[3 * p + 2] = C2 + T * P.bg[2];
    t_final[p] = T;
    n_last[p] = last;
  }
}

template <int KID>
__global__ void __launch_bounds__(512) blend_bwd_kernel(const float4* __restrict__ rec, const CamDev cam,
                                                        const ParDev P, const int2* __restrict__ ranges,
                                                        const uint32_t* __restrict__ vals,
                                                        const float* __restrict__ t_final,
                                                        const int32_t* __restrict__ n_last,
                                                        const float* __restrict__ grad_image,
                                                        const float* __restrict__ grad_t, float* __restrict__ g2d) {
  extern __shared__ float4 smem[];
  const int B = blockDim.x;
  float4* s_a = smem;
  float4* s_b = smem + B;
  float4* s_c = smem + 2 * B;
  float* s_acc = reinterpret_cast<float*>(smem + 3 * B);  // [B][9]
  uint32_t* s_id = reinterpret_cast<uint32_t*>(s_acc + 9 * B);
  int* s_touch = reinterpret_cast<int*>(s_id + B);
  __shared__ int s_max;

  const int tile = blockIdx.x;
  const int tx = tile % cam.tiles_x, ty = tile / cam.tiles_x;
  const int px = tx * P.tile_w + (int)threadIdx.x % P.tile_w;
  const int py = ty * P.tile_h + (int)threadIdx.x / P.tile_w;
  const bool inside = px < cam.W && py < cam.H;
  const float x = (float)px + 0.5f, y = (float)py + 0.5f;
  const int2 rg = ranges[cam.tile_base + tile];
  const int lane = threadIdx.x & 31;

  float T = 1.f, Tf = 1.f, gC0 = 0.f, gC1 = 0.f, gC2 = 0.f, gT = 0.f;
  int last = 0;
  if (inside) {
    const size_t p = (size_t)py * cam.W + px;
    T = Tf = t_final[p];
    last = n_last[p];
    gC0 = grad_image[3 * p];
    gC1 = grad_image[3 * p + 1];
    gC2 = grad_image[3 * p + 2];
    gT = grad_t ? grad_t[p] : 0.f;
  }
  float S0 = P.bg[0] * Tf, S1 = P.bg[1] * Tf, S2 = P.bg[2] * Tf;
  if (threadIdx.x == 0) s_max = 0;
  __syncthreads();
  if (last > 0) atomicMax(&s_max, last);
  __syncthreads();
  const int max_last = s_max;

  for (int b_end = max_last; b_end > 0; b_end -= B) {
    const int b0 = max(0, b_end - B);
    const int cnt = b_end - b0;
    __syncthreads();  // previous batch flushed
    if ((int)threadIdx.x < cnt) {
      const uint32_t id = vals[rg.x + b0 + threadIdx.x];
      s_id[threadIdx.x] = id;
      s_a[threadIdx.x] = rec[3 * (size_t)id];
      s_b[threadIdx.x] = rec[3 * (size_t)id + 1];
      s_c[threadIdx.x] = rec[3 * (size_t)id + 2];
      s_touch[threadIdx.x] = 0;
#pragma unroll
      for (int m = 0; m < 9; ++m) s_acc[9 * threadIdx.x + m] = 0.f;
    }
    __syncthreads();
    for (int jj = cnt - 1; jj >= 0; --jj) {
      const int j = b0 + jj;
      float v[9];
#pragma unroll
      for (int m = 0; m < 9; ++m) v[m] = 0.f;
      bool contrib = false;
      if (j < last) {
        const float4 a = s_a[jj];
        const float4 bb = s_b[jj];
        PairEval e;
        if (pair_alpha<KID>(x, y, a, bb, P, e)) {
          const float dx = e.dx, dy = e.dy, D = e.D, xk = e.xk, f = e.f, araw = e.araw, alpha = e.alpha;
          {
            contrib = true;
            const float4 c = s_c[jj];
            const float om = 1.f - alpha;
            const float iom = 1.f / om;
            const float Tb = T * iom;  // transmittance in front of this entry
            const float wgt = alpha * Tb;
            v[6] = wgt * gC0;
            v[7] = wgt * gC1;
            v[8] = wgt * gC2;
            const float ga = gC0 * (c.x * Tb - S0 * iom) + gC1 * (c.y * Tb - S1 * iom) +
                             gC2 * (c.z * Tb - S2 * iom) - gT * Tf * iom;
            S0 += c.x * wgt;
            S1 += c.y * wgt;
            S2 += c.z * wgt;
            T = Tb;
            if (araw <= P.alpha_max) {
              v[5] = f * ga;
              float gD = bb.y * ga * kern_df<KID>(xk) * P.inv_lambda;
              if (P.ags == 1) gD *= __expf(-D * D);
              else if (P.ags == 2) gD *= __expf(-xk * xk);
              const float gq = D > 0.f ? 0.5f * gD / D : 0.f;
              // A d = L^T (L d)
              v[0] = -2.f * gq * (a.z * e.e1);
              v[1] = -2.f * gq * (a.w * e.e1 + bb.x * e.e2);
              v[2] = gq * dx * dx;
              v[3] = 2.f * gq * dx * dy;
              v[4] = gq * dy * dy;
            }
          }
        }
      }
      if (__any_sync(0xffffffffu, contrib)) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
#pragma unroll
          for (int m = 0; m < 9; ++m) v[m] += __shfl_xor_sync(0xffffffffu, v[m], o);
        if (lane == 0) {
#pragma unroll
          for (int m = 0; m < 9; ++m) atomicAdd(&s_acc[9 * jj + m], v[m]);
          s_touch[jj] = 1;
        }
      }
    }
    __syncthreads();
    if ((int)threadIdx.x < cnt && s_touch[threadIdx.x]) {
      const float* acc = s_acc + 9 * threadIdx.x;
      float* dst = g2d + 12 * (size_t)s_id[threadIdx.x];
      atomicAdd(reinterpret_cast<float4*>(dst), make_float4(acc[0], acc[1], acc[2], acc[3]));
      atomicAdd(reinterpret_cast<float4*>(dst + 4), make_float4(acc[4], acc[5], acc[6], acc[7]));
      atomicAdd(dst + 8, acc[8]);
    }
  }
}

}  // namespace

cudaError_t launch_blend_fwd(const float4* rec, const CamDev& cam, const ParDev& P, const int2* ranges,
                             const uint32_t* vals, float* image, float* t_final, int32_t* n_last,
                             unsigned long long* stats, cudaStream_t st) {
  const int B = P.tile_w * P.tile_h;
  const unsigned grid = (unsigned)(cam.tiles_x * cam.tiles_y);
  const size_t sm = sizeof(float4) * 3 * B;
#define LS_BF(K)                                                                                           \
  do {                                                                                                     \
    if (stats)                                                                                             \
      blend_fwd_kernel<K, true><<<grid, B, sm, st>>>(rec, cam, P, ranges, vals, image, t_final, n_last, stats); \
    else                                                                                                   \
      blend_fwd_kernel<K, false><<<grid, B, sm, st>>>(rec, cam, P, ranges, vals, image, t_final, n_last,     \
                                                      nullptr);                                            \
  } while (0)
  switch (P.kernel) {
    case LS_KERNEL_GAUSSIAN: LS_BF(LS_KERNEL_GAUSSIAN); break;
    case LS_KERNEL_LAPLACIAN: LS_BF(LS_KERNEL_LAPLACIAN); break;
    case LS_KERNEL_COSINE: LS_BF(LS_KERNEL_COSINE); break;
    case LS_KERNEL_QUADRATIC: LS_BF(LS_KERNEL_QUADRATIC); break;
    default: LS_BF(LS_KERNEL_LINEAR); break;
  }
#undef LS_BF
  return cudaGetLastError();
}

cudaError_t launch_blend_bwd(const float4* rec, const CamDev& cam, const ParDev& P, const int2* ranges,
                             const uint32_t* vals, const float* t_final, const int32_t* n_last,
                             const float* grad_image, const float* grad_t, float* g2d, cudaStream_t st) {
  const int B = P.tile_w * P.tile_h;
  const unsigned grid = (unsigned)(cam.tiles_x * cam.tiles_y);
  const size_t sm = sizeof(float4) * 3 * B + sizeof(float) * 9 * B + 2 * sizeof(uint32_t) * B;
#define LS_BB(K)                                                                                        \
  blend_bwd_kernel<K><<<grid, B, sm, st>>>(rec, cam, P, ranges, vals, t_final, n_last, grad_image, grad_t, \
                                           g2d)
  switch (P.kernel) {
    case LS_KERNEL_GAUSSIAN: LS_BB(LS_KERNEL_GAUSSIAN); break;
    case LS_KERNEL_LAPLACIAN: LS_BB(LS_KERNEL_LAPLACIAN); break;
    case LS_KERNEL_COSINE: LS_BB(LS_KERNEL_COSINE); break;
    case LS_KERNEL_QUADRATIC: LS_BB(LS_KERNEL_QUADRATIC); break;
    default: LS_BB(LS_KERNEL_LINEAR); break;
  }
#undef LS_BB
  return cudaGetLastError();
}

}  // namespace ls
