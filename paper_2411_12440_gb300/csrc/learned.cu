// a8: learned per-tile termination.
//
//   tile_hist    per tile, a 32-bin log-depth histogram of the expected
//                coverage of the records whose support box covers it, and
//                their number, as 2D difference arrays (four atomics per
//                record and plane, not one per (record, tile) key) followed by
//                2D prefix sums;
//   features     log1p of the cumulative coverage in front of each bin edge
//                and the world direction of the tile's centre ray: the MLP's
//                35 inputs (fp16 rows of 48);
//   dstar        the proposed depth per tile, exp(MLP output + margin), as
//                comparable binary32 bits;
//   enum_keys    the (record, tile) keys in depth order, enumerated
//                warp-cooperatively and compacted with ballots: the kept keys
//                (depth <= proposal) and, for refuted tiles, the held-out ones
//                (depth > proposal), each in front-to-back order;
//   orchestration of ls_render_learned: kept keys are sorted and blended; a
//   tile whose pixels did not all settle and that has held-out keys is
//   refuted, its held-out keys are sorted and blending resumes from the stored
//   per-pixel state, so the image is the plain one bit for bit (t_thr =
//   t_min) or within t_thr (max rgb + bg) of it (t_thr > t_min).
#include <cuda_fp16.h>

#include <cmath>
#include <cstring>

#include "kernels.h"

namespace ls {

namespace {

constexpr int NBINS = 32;

__device__ __forceinline__ int depth_bin(float d, const DepthBins& B) {
  int b = 0;
#pragma unroll
  for (int i = 0; i < NBINS - 1; ++i) b += d >= B.edge[i] ? 1 : 0;
  return b;
}

// Each visible record adds to the tiles its support box covers: 1 to the key
// count plane, and its expected coverage of a tile to its depth bin's plane:
// o/3 (the mean of the linear profile over its support ellipse) times
// min(1, ellipse area / box area).
__global__ void __launch_bounds__(256) tile_hist_kernel(int64_t R, const float4* __restrict__ rec,
                                                        const float4* __restrict__ foot,
                                                        const uint32_t* __restrict__ dkey, const CamDev cam,
                                                        const ParDev P, const DepthBins bins, int* __restrict__ count,
                                                        float* __restrict__ mass) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= R) return;
  const uint32_t dk = dkey[r];
  if (dk == DKEY_CULLED) return;
  const float4 f = foot[r];
  int tx0, tx1, ty0, ty1;
  if (!tile_rect(f.x, f.y, f.z, f.w, cam.W, cam.H, P.tile_w, P.tile_h, tx0, tx1, ty0, ty1)) return;
  const float4 a = rec[3 * r], b = rec[3 * r + 1];  // {mx, my, l00, l01}, {l11, o, rho2, depth}
  const float ellipse = 3.14159265f * b.z / fmaxf(a.z * b.x, 1e-30f);
  const float box = (float)((tx1 - tx0 + 1) * (ty1 - ty0 + 1) * P.tile_w * P.tile_h);
  const float w = b.y * (1.f / 3.f) * fminf(1.f, ellipse / box);
  const int sx = cam.tiles_x + 1;
  atomicAdd(&count[ty0 * sx + tx0], 1);
  atomicAdd(&count[ty0 * sx + tx1 + 1], -1);
  atomicAdd(&count[(ty1 + 1) * sx + tx0], -1);
  atomicAdd(&count[(ty1 + 1) * sx + tx1 + 1], 1);
  float* d = mass + (size_t)depth_bin(__uint_as_float(dk), bins) * sx * (cam.tiles_y + 1);
  atomicAdd(&d[ty0 * sx + tx0], w);
  atomicAdd(&d[ty0 * sx + tx1 + 1], -w);
  atomicAdd(&d[(ty1 + 1) * sx + tx0], -w);
  atomicAdd(&d[(ty1 + 1) * sx + tx1 + 1], w);
}

// One block per plane (the 32 mass planes, then the count plane): prefix
// along rows, then along columns.
template <typename V>
__device__ __forceinline__ void prefix_plane(V* d, int sx, int sy) {
  for (int y = threadIdx.x; y < sy; y += blockDim.x) {
    V run = 0;
    for (int x = 0; x < sx; ++x) {
      run += d[y * sx + x];
      d[y * sx + x] = run;
    }
  }
  __syncthreads();
  for (int x = threadIdx.x; x < sx; x += blockDim.x) {
    V run = 0;
    for (int y = 0; y < sy; ++y) {
      run += d[y * sx + x];
      d[y * sx + x] = run;
    }
  }
}

__global__ void __launch_bounds__(256) hist_prefix_kernel(float* __restrict__ mass, int* __restrict__ count, int sx,
                                                          int sy) {
  if (blockIdx.x < NBINS) prefix_plane(mass + (size_t)blockIdx.x * sx * sy, sx, sy);
  else prefix_plane(count, sx, sy);
}

__global__ void __launch_bounds__(256) features_kernel(const float* __restrict__ mass, const int* __restrict__ count,
                                                       const CamDev cam, const ParDev P, __half* __restrict__ x,
                                                       int32_t* __restrict__ tile_total,
                                                       unsigned long long* key_total) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int ntiles = cam.tiles_x * cam.tiles_y;
  if (t >= ntiles) return;
  const int tx = t % cam.tiles_x, ty = t / cam.tiles_x;
  const int sx = cam.tiles_x + 1, plane = sx * (cam.tiles_y + 1);
  __half* row = x + (size_t)t * LS_MLP_IN;
  // cumulative coverage in front of each bin's upper edge
  float cum = 0.f;
  for (int b = 0; b < NBINS; ++b) {
    cum += fmaxf(mass[(size_t)b * plane + ty * sx + tx], 0.f);
    row[b] = __float2half_rn(log1pf(cum));
  }
  // direction of the ray through the tile centre, world axes
  const float u = (tx + 0.5f) * P.tile_w, v = (ty + 0.5f) * P.tile_h;
  const float rx = (u - cam.cx) / cam.fx, ry = (v - cam.cy) / cam.fy, inv = rsqrtf(rx * rx + ry * ry + 1.f);
  const float c0 = rx * inv, c1 = ry * inv, c2 = inv;
  for (int i = 0; i < 3; ++i)
    row[NBINS + i] = __float2half_rn(cam.R[i] * c0 + cam.R[3 + i] * c1 + cam.R[6 + i] * c2);
  for (int i = NBINS + 3; i < LS_MLP_IN; ++i) row[i] = __float2half_rn(0.f);
  const int total = count[ty * sx + tx];
  tile_total[t] = total;
  if (key_total) atomicAdd(key_total, (unsigned long long)total);
}

// Proposed depth per tile as comparable bits: exp(y + margin) from the MLP,
// or the caller's depths (NaN or +inf keeps everything).
__global__ void __launch_bounds__(256) dstar_kernel(int ntiles, const float* __restrict__ y, float margin,
                                                    const float* __restrict__ dstar_in, uint32_t* __restrict__ bits,
                                                    float* __restrict__ dstar_out) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= ntiles) return;
  float d = y ? expf(y[t] + margin) : dstar_in[t];
  if (!(d == d)) d = __int_as_float(0x7F800000);
  d = fmaxf(d, 0.f);
  bits[t] = __float_as_uint(d);
  if (dstar_out) dstar_out[t] = d;
}

__device__ __forceinline__ uint32_t rect_count_l(uint2 rc) {
  int x0 = rc.x & 0xFFFF, x1 = rc.x >> 16, y0 = rc.y & 0xFFFF, y1 = rc.y >> 16;
  return x1 < x0 ? 0u : (uint32_t)((x1 - x0 + 1) * (y1 - y0 + 1));
}

// Enumerate every (record, tile) key of DUP_BLOCK depth-ordered records per
// block; warp w takes records [w*128, w*128+128).  HELD = false keeps keys with
// depth bits <= the tile's proposal; HELD = true keeps keys of refuted tiles
// beyond it.  EMIT = false writes each warp's count; EMIT = true writes the
// compacted keys at the warp's scanned offset (and the tile-sort digit
// histograms).  Order is depth order inside every tile.
template <bool EMIT, bool HELD>
__global__ void __launch_bounds__(DUP_THREADS) enum_keys_kernel(
    int64_t R, const uint32_t* __restrict__ order, const uint32_t* __restrict__ dkey_sorted,
    const uint2* __restrict__ rect_sorted, int tiles_x, const uint32_t* __restrict__ dstar_bits,
    const uint8_t* __restrict__ refuted, const unsigned* __restrict__ n_refuted, uint32_t* __restrict__ warp_counts,
    const int64_t* __restrict__ n_valid, uint32_t* __restrict__ keys, uint32_t* __restrict__ vals, int key_passes,
    uint32_t* __restrict__ tile_hist) {
  __shared__ uint32_t s_off[DUP_BLOCK + 1];
  __shared__ uint2 s_rect[DUP_BLOCK];
  __shared__ uint32_t s_r[DUP_BLOCK];
  __shared__ uint32_t s_dk[DUP_BLOCK];
  __shared__ uint32_t s_hist[3][RADIX];
  __shared__ uint32_t s_warp[DUP_THREADS / 32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int wid = blockIdx.x * (DUP_THREADS / 32) + warp;
  if ((HELD && *n_refuted == 0u) || (EMIT && *n_valid == 0)) {
    if (!EMIT && lane == 0) warp_counts[wid] = 0u;
    return;  // block-uniform
  }
  if (EMIT)
    for (int i = tid; i < 3 * RADIX; i += DUP_THREADS) (&s_hist[0][0])[i] = 0;
  const int64_t base = (int64_t)blockIdx.x * DUP_BLOCK;
#pragma unroll
  for (int i = 0; i < DUP_ITEMS; ++i) {
    const int s = i * DUP_THREADS + tid;
    const int64_t j = base + s;
    uint2 rc = make_uint2(1u, 0u);
    uint32_t r = 0, dk = DKEY_CULLED;
    if (j < R) {
      rc = rect_sorted[j];
      r = order[j];
      dk = dkey_sorted[j];
    }
    s_rect[s] = rc;
    s_r[s] = r;
    s_dk[s] = dk;
  }
  __syncthreads();
  uint32_t c[DUP_ITEMS], run = 0;
#pragma unroll
  for (int i = 0; i < DUP_ITEMS; ++i) {
    c[i] = rect_count_l(s_rect[DUP_ITEMS * tid + i]);
    run += c[i];
  }
  uint32_t x = run;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t u = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += u;
  }
  if (lane == 31) s_warp[warp] = x;
  __syncthreads();
  uint32_t wpre = 0;
  for (int w = 0; w < warp; ++w) wpre += s_warp[w];
  uint32_t ex = x - run + wpre;
#pragma unroll
  for (int i = 0; i < DUP_ITEMS; ++i) {
    s_off[DUP_ITEMS * tid + i] = ex;
    ex += c[i];
  }
  if (tid == DUP_THREADS - 1) s_off[DUP_BLOCK] = ex;
  __syncthreads();
  const int s0 = warp * 32 * DUP_ITEMS, s1 = s0 + 32 * DUP_ITEMS;
  const uint32_t o0 = s_off[s0], o1 = s_off[s1];
  uint32_t out = EMIT ? warp_counts[wid] : 0u;  // EMIT: scanned offset of this warp
  uint32_t kept = 0;
  for (uint32_t cb = o0; cb < o1; cb += 32) {
    const uint32_t e = cb + lane;
    bool take = false;
    uint32_t key = 0, r = 0;
    if (e < o1) {
      int lo = s0, hi = s1 - 1;
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (s_off[mid] <= e) lo = mid;
        else hi = mid - 1;
      }
      const uint2 rc = s_rect[lo];
      const uint32_t m = e - s_off[lo];
      const uint32_t x0 = rc.x & 0xFFFF, x1 = rc.x >> 16, y0 = rc.y & 0xFFFF;
      const uint32_t w = x1 - x0 + 1;
      key = (y0 + m / w) * (uint32_t)tiles_x + x0 + m % w;
      r = s_r[lo];
      const uint32_t lim = __ldg(dstar_bits + key);
      take = HELD ? (refuted[key] && s_dk[lo] > lim) : (s_dk[lo] <= lim);
    }
    const uint32_t bal = __ballot_sync(0xffffffffu, take);
    if (EMIT && take) {
      const uint32_t pos = out + kept + __popc(bal & ((1u << lane) - 1u));
      keys[pos] = key;
      vals[pos] = r;
      for (int p = 0; p < key_passes; ++p) atomicAdd(&s_hist[p][(key >> (8 * p)) & 255u], 1u);
    }
    kept += __popc(bal);
  }
  if (!EMIT) {
    if (lane == 0) warp_counts[wid] = kept;
    return;
  }
  __syncthreads();
  for (int i = tid; i < key_passes * RADIX; i += DUP_THREADS) {
    const uint32_t v = (&s_hist[0][0])[i];
    if (v) atomicAdd(&tile_hist[i], v);
  }
}

__global__ void learned_stats_kernel(const unsigned long long* key_total, const int64_t* n_kept,
                                     const int64_t* n_held, const unsigned* n_refuted, int64_t* stats) {
  stats[0] = (int64_t)*key_total;
  stats[1] = *n_kept;
  stats[2] = *n_held;
  stats[3] = (int64_t)*n_refuted;
}

}  // namespace

DepthBins make_depth_bins() {
  // 32 bins of log depth over [0.5, 32): edge i = 0.5 * 64^((i + 1) / 32)
  DepthBins B;
  for (int i = 0; i < NBINS - 1; ++i) B.edge[i] = (float)(0.5 * std::exp(std::log(64.0) * (i + 1) / NBINS));
  return B;
}

size_t hist_planes_bytes(const CamDev& cam) {
  return (size_t)(NBINS + 1) * 4 * (cam.tiles_x + 1) * (cam.tiles_y + 1);
}

cudaError_t launch_tile_hist(int64_t R, const float4* rec, const float4* foot, const uint32_t* dkey,
                             const CamDev& cam, const ParDev& P, void* planes, cudaStream_t st) {
  if (R == 0) return cudaSuccess;
  float* mass = static_cast<float*>(planes);
  int* count = reinterpret_cast<int*>(mass + (size_t)NBINS * (cam.tiles_x + 1) * (cam.tiles_y + 1));
  tile_hist_kernel<<<ceil_div(R, 256), 256, 0, st>>>(R, rec, foot, dkey, cam, P, make_depth_bins(), count, mass);
  return cudaGetLastError();
}

cudaError_t launch_features(void* planes, const CamDev& cam, const ParDev& P, void* x, int32_t* tile_total,
                            unsigned long long* key_total, cudaStream_t st) {
  float* mass = static_cast<float*>(planes);
  int* count = reinterpret_cast<int*>(mass + (size_t)NBINS * (cam.tiles_x + 1) * (cam.tiles_y + 1));
  hist_prefix_kernel<<<NBINS + 1, 256, 0, st>>>(mass, count, cam.tiles_x + 1, cam.tiles_y + 1);
  const int ntiles = cam.tiles_x * cam.tiles_y;
  features_kernel<<<ceil_div(ntiles, 256), 256, 0, st>>>(mass, count, cam, P, static_cast<__half*>(x), tile_total,
                                                        key_total);
  return cudaGetLastError();
}

cudaError_t launch_dstar(int ntiles, const float* y, float margin, const float* dstar_in, uint32_t* bits,
                         float* dstar_out, cudaStream_t st) {
  dstar_kernel<<<ceil_div(ntiles, 256), 256, 0, st>>>(ntiles, y, margin, dstar_in, bits, dstar_out);
  return cudaGetLastError();
}

cudaError_t launch_enum_keys(bool emit, bool held, int64_t R, const uint32_t* order, const uint32_t* dkey_sorted,
                             const uint2* rect_sorted, int tiles_x, const uint32_t* dstar_bits, const uint8_t* refuted,
                             const unsigned* n_refuted, uint32_t* warp_counts, const int64_t* n_valid, uint32_t* keys,
                             uint32_t* vals, int key_passes, uint32_t* tile_hist, cudaStream_t st) {
  if (R == 0) return cudaSuccess;
  const unsigned grid = ceil_div(R, DUP_BLOCK);
#define LS_EK(E, H)                                                                                               \
  enum_keys_kernel<E, H><<<grid, DUP_THREADS, 0, st>>>(R, order, dkey_sorted, rect_sorted, tiles_x, dstar_bits, \
                                                       refuted, n_refuted, warp_counts, n_valid, keys, vals,     \
                                                       key_passes, tile_hist)
  if (emit) {
    if (held) LS_EK(true, true);
    else LS_EK(true, false);
  } else {
    if (held) LS_EK(false, true);
    else LS_EK(false, false);
  }
#undef LS_EK
  return cudaGetLastError();
}

cudaError_t launch_learned_stats(const unsigned long long* key_total, const int64_t* n_kept, const int64_t* n_held,
                                 const unsigned* n_refuted, int64_t* stats, cudaStream_t st) {
  learned_stats_kernel<<<1, 1, 0, st>>>(key_total, n_kept, n_held, n_refuted, stats);
  return cudaGetLastError();
}

}  // namespace ls
