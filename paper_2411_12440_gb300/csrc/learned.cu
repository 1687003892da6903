// a8: learned per-tile termination.
//
//   tile_hist    per tile, a 32-bin log-depth histogram of the expected
//                coverage of the records whose support box covers it, and
//                their number, as 2D difference arrays (four atomics per
//                record and plane, not one per (record, tile) key) followed by
//                2D prefix sums; tile_hist_sorted builds the same coverage
//                planes from the depth order, one bin's plane at a time in
//                shared memory (the learned render's path);
//   features     log1p of the cumulative coverage in front of each bin edge
//                and the world direction of the tile's centre ray: the MLP's
//                35 inputs (fp16 rows of 48);
//   dstar        the proposed depth per tile, exp(MLP output + margin), as
//                comparable binary32 bits, whether a tile may hold keys beyond
//                its proposal (has_held, from the coverage planes), and a max
//                pyramid of the proposals that bounds them over any support box
//                (the kept enumeration drops records beyond that bound);
//   refuted_sat  summed-area table of the refuted tiles, so that the
//                held-out enumeration (duplicate.cu, ENUM_HELD) skips records
//                whose box holds none;
//   orchestration of ls_render_learned: kept keys are sorted and blended; a
//   tile whose pixels did not all settle and that may hold held-out keys is
//   refuted, its held-out keys are sorted and blending resumes from the stored
//   per-pixel state, so the image is the plain one bit for bit (t_thr =
//   t_min) or within t_thr (max rgb + bg) of it (t_thr > t_min).
#include <cuda_fp16.h>

#include <algorithm>
#include <cmath>
#include <cstring>

#include "kernels.h"

namespace ls {

namespace {

constexpr int NBINS = 32;
// Fixed-point unit of the coverage planes: unsigned 32-bit sums are exact
// modulo 2^32 whatever the order of the atomics, and every prefix sum that is
// read (one bin's coverage of a tile, far below 2^15) fits.  Every record adds
// at least one unit, so a tile's cell of a bin is nonzero exactly when a box
// of that bin covers it.
constexpr float MASS_ONE = 65536.f;

__device__ __forceinline__ int depth_bin(float d, const DepthBins& B) {
  int b = 0;
#pragma unroll
  for (int i = 0; i < NBINS - 1; ++i) b += d >= B.edge[i] ? 1 : 0;
  return b;
}

// Each visible record adds to the tiles its support box covers: 1 to the key
// count plane, and its expected coverage of a tile to its depth bin's plane:
// o/3 (the mean of the linear profile over its support ellipse) times
// min(1, ellipse area / box area).  Every record's count corners land on a
// few thousand cells, so with COUNTS == HIST_PRIVATE the blocks are
// persistent and keep the count plane in shared memory, adding it to the
// global one once at the end; the mass corners spread over 32 planes and go
// to global memory directly.  HIST_NONE leaves the count plane out.
enum { HIST_NONE = 0, HIST_PRIVATE = 1, HIST_GLOBAL = 2 };
template <int COUNTS>
__global__ void __launch_bounds__(256) tile_hist_kernel(int64_t R, const float4* __restrict__ rec,
                                                        const float4* __restrict__ foot,
                                                        const uint32_t* __restrict__ dkey, const CamDev cam,
                                                        const ParDev P, const DepthBins bins, int* __restrict__ count,
                                                        unsigned* __restrict__ mass) {
  extern __shared__ int s_count[];
  const int sx = cam.tiles_x + 1, cells = sx * (cam.tiles_y + 1);
  int* cnt = count;
  if (COUNTS == HIST_PRIVATE) {
    for (int i = threadIdx.x; i < cells; i += blockDim.x) s_count[i] = 0;
    __syncthreads();
    cnt = s_count;
  }
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < R; r += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t dk = dkey[r];
    if (dk == DKEY_CULLED) continue;
    const float4 f = foot[r];
    int tx0, tx1, ty0, ty1;
    if (!tile_rect(f.x, f.y, f.z, f.w, cam.W, cam.H, P.tile_w, P.tile_h, tx0, tx1, ty0, ty1)) continue;
    const float4 a = rec[3 * r], b = rec[3 * r + 1];  // {mx, my, l00, l01}, {l11, o, rho2, depth}
    const float ellipse = 3.14159265f * b.z / fmaxf(a.z * b.x, 1e-30f);
    const float box = (float)((tx1 - tx0 + 1) * (ty1 - ty0 + 1) * P.tile_w * P.tile_h);
    const float w = b.y * (1.f / 3.f) * fminf(1.f, ellipse / box);
    // fixed point: integer sums do not depend on the order of the atomics
    const unsigned wq = (unsigned)max(1, __float2int_rn(w * MASS_ONE));  // >= 1: a covered cell is never 0
    if (COUNTS != HIST_NONE) {
      atomicAdd(&cnt[ty0 * sx + tx0], 1);
      atomicAdd(&cnt[ty0 * sx + tx1 + 1], -1);
      atomicAdd(&cnt[(ty1 + 1) * sx + tx0], -1);
      atomicAdd(&cnt[(ty1 + 1) * sx + tx1 + 1], 1);
    }
    unsigned* d = mass + (size_t)depth_bin(__uint_as_float(dk), bins) * cells;
    atomicAdd(&d[ty0 * sx + tx0], wq);
    atomicAdd(&d[ty0 * sx + tx1 + 1], 0u - wq);
    atomicAdd(&d[(ty1 + 1) * sx + tx0], 0u - wq);
    atomicAdd(&d[(ty1 + 1) * sx + tx1 + 1], wq);
  }
  if (COUNTS == HIST_PRIVATE) {
    __syncthreads();
    for (int i = threadIdx.x; i < cells; i += blockDim.x)
      if (s_count[i]) atomicAdd(&count[i], s_count[i]);
  }
}

// The coverage planes from the depth order: records of one depth bin are
// contiguous there, so each block takes a contiguous range of the sorted
// records, accumulates the plane of the bin at hand in shared memory, and
// adds it to the global plane (nonzero cells only) when the bin changes and
// at the end: shared-memory atomics per record, a few plane flushes per
// block.  Same weights and fixed point as tile_hist_kernel, so the planes are
// the same bit for bit.  Dynamic shared memory: one plane of unsigned cells.
constexpr int HIST_SORTED_THREADS = 1024, HIST_SORTED_ITEMS = 4;

__device__ __forceinline__ void flush_plane(unsigned* __restrict__ s_plane, unsigned* __restrict__ g_plane,
                                            int cells) {
  for (int i = threadIdx.x; i < cells; i += blockDim.x) {
    const unsigned v = s_plane[i];
    if (v) {
      atomicAdd(&g_plane[i], v);
      s_plane[i] = 0u;
    }
  }
}

__global__ void __launch_bounds__(HIST_SORTED_THREADS) tile_hist_sorted_kernel(
    int64_t R, const uint32_t* __restrict__ order, const uint32_t* __restrict__ dkey_sorted,
    const uint2* __restrict__ rect_sorted, const float4* __restrict__ rec, const CamDev cam, const ParDev P,
    const DepthBins bins, unsigned* __restrict__ mass) {
  constexpr int CHUNK = HIST_SORTED_THREADS * HIST_SORTED_ITEMS;
  extern __shared__ unsigned s_plane[];
  __shared__ int s_bin[2];
  const int sx = cam.tiles_x + 1, cells = sx * (cam.tiles_y + 1);
  for (int i = threadIdx.x; i < cells; i += blockDim.x) s_plane[i] = 0u;
  const int64_t per = (R + gridDim.x - 1) / gridDim.x;
  const int64_t lo = (int64_t)blockIdx.x * per, hi = lo + per < R ? lo + per : R;
  int cur = -1;  // bin of the shared plane (block-uniform)
  for (int64_t c0 = lo; c0 < hi; c0 += CHUNK) {
    int bin[HIST_SORTED_ITEMS];
    unsigned wq[HIST_SORTED_ITEMS];
    uint2 rc[HIST_SORTED_ITEMS];
    uint32_t r[HIST_SORTED_ITEMS];
#pragma unroll
    for (int i = 0; i < HIST_SORTED_ITEMS; ++i) {  // loads of all items first
      const int64_t j = c0 + i * HIST_SORTED_THREADS + threadIdx.x;
      bin[i] = -1;
      rc[i] = make_uint2(1u, 0u);
      r[i] = 0;
      if (j < hi) {
        const uint32_t dk = dkey_sorted[j];
        rc[i] = rect_sorted[j];
        if (dk != DKEY_CULLED && (rc[i].x >> 16) >= (rc[i].x & 0xFFFFu)) {  // a non-empty box
          r[i] = order[j];
          bin[i] = depth_bin(__uint_as_float(dk), bins);
        }
      }
    }
    int bmin = NBINS, bmax = -1;
#pragma unroll
    for (int i = 0; i < HIST_SORTED_ITEMS; ++i) {
      wq[i] = 0u;
      if (bin[i] >= 0) {
        const float4 a = rec[3 * (size_t)r[i]], b = rec[3 * (size_t)r[i] + 1];  // {mx, my, l00, l01}, {l11, o, rho2, depth}
        const int tx0 = rc[i].x & 0xFFFF, tx1 = rc[i].x >> 16, ty0 = rc[i].y & 0xFFFF, ty1 = rc[i].y >> 16;
        const float ellipse = 3.14159265f * b.z / fmaxf(a.z * b.x, 1e-30f);
        const float box = (float)((tx1 - tx0 + 1) * (ty1 - ty0 + 1) * P.tile_w * P.tile_h);
        const float w = b.y * (1.f / 3.f) * fminf(1.f, ellipse / box);
        wq[i] = (unsigned)max(1, __float2int_rn(w * MASS_ONE));
        bmin = min(bmin, bin[i]);
        bmax = max(bmax, bin[i]);
      }
    }
    // bins rise with the depth order: the chunk's bins are [first, last] of
    // its binned records
    if (threadIdx.x == 0) s_bin[0] = NBINS, s_bin[1] = -1;
    __syncthreads();
    if (bmax >= 0) {
      atomicMin(&s_bin[0], bmin);
      atomicMax(&s_bin[1], bmax);
    }
    __syncthreads();
    const int b_first = s_bin[0], b_last = s_bin[1];
    __syncthreads();  // s_bin is read before the next chunk resets it
    for (int b = b_first; b <= b_last; ++b) {
      if (b != cur) {
        if (cur >= 0) {
          flush_plane(s_plane, mass + (size_t)cur * cells, cells);
          __syncthreads();
        }
        cur = b;
      }
#pragma unroll
      for (int i = 0; i < HIST_SORTED_ITEMS; ++i) {
        if (bin[i] == b) {
          const int tx0 = rc[i].x & 0xFFFF, tx1 = rc[i].x >> 16, ty0 = rc[i].y & 0xFFFF, ty1 = rc[i].y >> 16;
          atomicAdd(&s_plane[ty0 * sx + tx0], wq[i]);
          atomicAdd(&s_plane[ty0 * sx + tx1 + 1], 0u - wq[i]);
          atomicAdd(&s_plane[(ty1 + 1) * sx + tx0], 0u - wq[i]);
          atomicAdd(&s_plane[(ty1 + 1) * sx + tx1 + 1], wq[i]);
        }
      }
      __syncthreads();
    }
  }
  if (cur >= 0) flush_plane(s_plane, mass + (size_t)cur * cells, cells);
}

// One block per plane (the 32 mass planes, then the count plane): prefix
// along rows (a warp per row, coalesced warp scans), then along columns (a
// thread per column, loads batched eight rows at a time).
template <typename V>
__device__ __forceinline__ void prefix_plane(V* d, int sx, int sy) {
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int y = warp; y < sy; y += nw) {
    V carry = 0;
    for (int x0 = 0; x0 < sx; x0 += 32) {
      const int x = x0 + lane;
      V v = x < sx ? d[y * sx + x] : V(0);
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const V u = __shfl_up_sync(FULL, v, o);
        if (lane >= o) v += u;
      }
      v += carry;
      if (x < sx) d[y * sx + x] = v;
      carry = __shfl_sync(FULL, v, 31);
    }
  }
  __syncthreads();
  for (int x = threadIdx.x; x < sx; x += blockDim.x) {
    V run = 0;
    int y = 0;
    for (; y + 8 <= sy; y += 8) {
      V t[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) t[i] = d[(y + i) * sx + x];
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        run += t[i];
        d[(y + i) * sx + x] = run;
      }
    }
    for (; y < sy; ++y) {
      run += d[y * sx + x];
      d[y * sx + x] = run;
    }
  }
}

__global__ void __launch_bounds__(256) hist_prefix_kernel(unsigned* __restrict__ mass, int* __restrict__ count, int sx,
                                                          int sy) {
  if (blockIdx.x < NBINS) prefix_plane(mass + (size_t)blockIdx.x * sx * sy, sx, sy);
  else prefix_plane(count, sx, sy);
}

__global__ void __launch_bounds__(256) features_kernel(const unsigned* __restrict__ mass, const int* __restrict__ count,
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
    const int m = (int)mass[(size_t)b * plane + ty * sx + tx];  // exact: the true sum fits
    cum += m > 0 ? (float)m * (1.f / MASS_ONE) : 0.f;
    row[b] = __float2half_rn(log1pf(cum));
  }
  // direction of the ray through the tile centre, world axes
  const float u = (tx + 0.5f) * P.tile_w, v = (ty + 0.5f) * P.tile_h;
  const float rx = (u - cam.cx) / cam.fx, ry = (v - cam.cy) / cam.fy, inv = rsqrtf(rx * rx + ry * ry + 1.f);
  const float c0 = rx * inv, c1 = ry * inv, c2 = inv;
  for (int i = 0; i < 3; ++i)
    row[NBINS + i] = __float2half_rn(cam.R[i] * c0 + cam.R[3 + i] * c1 + cam.R[6 + i] * c2);
  for (int i = NBINS + 3; i < LS_MLP_IN; ++i) row[i] = __float2half_rn(0.f);
  if (tile_total) {
    const int total = count[ty * sx + tx];
    tile_total[t] = total;
    if (key_total) atomicAdd(key_total, (unsigned long long)total);
  }
}

// Proposed depth per tile as comparable bits: exp(y + margin) from the MLP,
// or the caller's depths (NaN or +inf keeps everything); and has_held from the
// prefixed coverage planes: records of bin b have depths below its upper
// edge, so only bins whose upper edge exceeds the proposal can hold records
// beyond it.
__global__ void __launch_bounds__(256) dstar_kernel(const CamDev cam, const float* __restrict__ y, float margin,
                                                    const float* __restrict__ dstar_in, uint32_t* __restrict__ bits,
                                                    float* __restrict__ dstar_out, const unsigned* __restrict__ mass,
                                                    const DepthBins B, uint8_t* __restrict__ has_held) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int ntiles = cam.tiles_x * cam.tiles_y;
  if (t >= ntiles) return;
  float d = y ? expf(y[t] + margin) : dstar_in[t];
  if (!(d == d)) d = __int_as_float(0x7F800000);
  d = fmaxf(d, 0.f);
  bits[t] = __float_as_uint(d);
  if (dstar_out) dstar_out[t] = d;
  const int tx = t % cam.tiles_x, ty = t / cam.tiles_x, sx = cam.tiles_x + 1;
  const size_t plane = (size_t)sx * (cam.tiles_y + 1);
  bool held = false;
  for (int b = NBINS - 1; b >= 0 && !held; --b) {
    const float upper = b < NBINS - 1 ? B.edge[b] : __int_as_float(0x7F800000);
    if (!(upper > d)) break;  // this bin and all below end at or before the proposal
    held = mass[(size_t)b * plane + ty * sx + tx] != 0u;
  }
  has_held[t] = held ? 1 : 0;
}

// Upper levels of the proposal pyramid (level 0 written by dstar_kernel).
// One block.
__global__ void __launch_bounds__(1024) dstar_pyramid_kernel(uint32_t* __restrict__ pyr, const DstarPyramid D) {
  for (int k = 1; k < D.levels; ++k) {
    const int w = D.w[k], h = D.h[k], pw = D.w[k - 1], ph = D.h[k - 1];
    const uint32_t* lo = pyr + D.off[k - 1];
    uint32_t* hi = pyr + D.off[k];
    for (int i = threadIdx.x; i < w * h; i += blockDim.x) {
      const int cx = i % w, cy = i / w, x0 = 2 * cx, y0 = 2 * cy;
      const int x1 = min(x0 + 1, pw - 1), y1 = min(y0 + 1, ph - 1);
      hi[i] = max(max(lo[y0 * pw + x0], lo[y0 * pw + x1]), max(lo[y1 * pw + x0], lo[y1 * pw + x1]));
    }
    __syncthreads();
  }
}

// Summed-area table of the refuted flags over the tile grid, with a zero
// first row and column: sat[(y + 1) * (tiles_x + 1) + x + 1] counts the
// refuted tiles in [0, x] x [0, y].  One block.
__global__ void __launch_bounds__(1024) refuted_sat_kernel(const uint8_t* __restrict__ refuted,
                                                           const unsigned* __restrict__ n_refuted, int tiles_x,
                                                           int tiles_y, int* __restrict__ sat) {
  if (*n_refuted == 0u) return;  // the held-out passes return at once
  const int sx = tiles_x + 1, sy = tiles_y + 1;
  for (int i = threadIdx.x; i < sx * sy; i += blockDim.x) {
    const int x = i % sx, y = i / sx;
    sat[i] = (x > 0 && y > 0) ? (int)refuted[(y - 1) * tiles_x + x - 1] : 0;
  }
  __syncthreads();
  prefix_plane(sat, sx, sy);
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
                             const CamDev& cam, const ParDev& P, void* planes, bool counts, cudaStream_t st) {
  if (R == 0) return cudaSuccess;
  unsigned* mass = static_cast<unsigned*>(planes);
  int* count = reinterpret_cast<int*>(mass + (size_t)NBINS * (cam.tiles_x + 1) * (cam.tiles_y + 1));
  const size_t plane = sizeof(int) * (size_t)(cam.tiles_x + 1) * (cam.tiles_y + 1);
  if (!counts) {
    tile_hist_kernel<HIST_NONE><<<ceil_div(R, 256), 256, 0, st>>>(R, rec, foot, dkey, cam, P, make_depth_bins(),
                                                                  count, mass);
  } else if (plane <= 96 * 1024) {
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess && plane > 48 * 1024)
      e = cudaFuncSetAttribute(tile_hist_kernel<HIST_PRIVATE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)plane);
    if (e != cudaSuccess) return e;
    const unsigned grid = (unsigned)std::min<int64_t>(ceil_div(R, 256), (int64_t)sms * 4);
    tile_hist_kernel<HIST_PRIVATE><<<grid, 256, plane, st>>>(R, rec, foot, dkey, cam, P, make_depth_bins(), count,
                                                             mass);
  } else {
    tile_hist_kernel<HIST_GLOBAL><<<ceil_div(R, 256), 256, 0, st>>>(R, rec, foot, dkey, cam, P, make_depth_bins(),
                                                                    count, mass);
  }
  return cudaGetLastError();
}

size_t tile_hist_sorted_smem(const CamDev& cam) {
  return sizeof(unsigned) * (size_t)(cam.tiles_x + 1) * (cam.tiles_y + 1);
}

cudaError_t launch_tile_hist_sorted(int64_t R, const uint32_t* order, const uint32_t* dkey_sorted,
                                    const uint2* rect_sorted, const float4* rec, const CamDev& cam, const ParDev& P,
                                    void* planes, cudaStream_t st) {
  if (R == 0) return cudaSuccess;
  const size_t sm = tile_hist_sorted_smem(cam);
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess && sm > 48 * 1024)
    e = cudaFuncSetAttribute(tile_hist_sorted_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  // one block per SM: every block flushes each plane it touched once, so the
  // global atomics grow with the number of blocks
  const int64_t grid = std::max<int64_t>(
      1, std::min<int64_t>((int64_t)sms, ceil_div(R, 4 * HIST_SORTED_THREADS * HIST_SORTED_ITEMS)));
  tile_hist_sorted_kernel<<<(unsigned)grid, HIST_SORTED_THREADS, sm, st>>>(
      R, order, dkey_sorted, rect_sorted, rec, cam, P, make_depth_bins(), static_cast<unsigned*>(planes));
  return cudaGetLastError();
}

cudaError_t launch_features(void* planes, const CamDev& cam, const ParDev& P, void* x, int32_t* tile_total,
                            unsigned long long* key_total, cudaStream_t st) {
  unsigned* mass = static_cast<unsigned*>(planes);
  int* count = reinterpret_cast<int*>(mass + (size_t)NBINS * (cam.tiles_x + 1) * (cam.tiles_y + 1));
  // the count plane is prefixed only when its totals are wanted
  hist_prefix_kernel<<<tile_total ? NBINS + 1 : NBINS, 256, 0, st>>>(mass, count, cam.tiles_x + 1, cam.tiles_y + 1);
  const int ntiles = cam.tiles_x * cam.tiles_y;
  features_kernel<<<ceil_div(ntiles, 256), 256, 0, st>>>(mass, count, cam, P, static_cast<__half*>(x), tile_total,
                                                        key_total);
  return cudaGetLastError();
}

cudaError_t launch_dstar(const CamDev& cam, const float* y, float margin, const float* dstar_in, uint32_t* pyr,
                         float* dstar_out, const void* planes, uint8_t* has_held, cudaStream_t st) {
  const int ntiles = cam.tiles_x * cam.tiles_y;
  dstar_kernel<<<ceil_div(ntiles, 256), 256, 0, st>>>(cam, y, margin, dstar_in, pyr, dstar_out,
                                                      static_cast<const unsigned*>(planes), make_depth_bins(),
                                                      has_held);
  const DstarPyramid D = make_dstar_pyramid(cam.tiles_x, cam.tiles_y);
  if (D.levels > 1) dstar_pyramid_kernel<<<1, 1024, 0, st>>>(pyr, D);
  return cudaGetLastError();
}

cudaError_t launch_refuted_sat(const uint8_t* refuted, const unsigned* n_refuted, int tiles_x, int tiles_y, int* sat,
                               cudaStream_t st) {
  refuted_sat_kernel<<<1, 1024, 0, st>>>(refuted, n_refuted, tiles_x, tiles_y, sat);
  return cudaGetLastError();
}

cudaError_t launch_learned_stats(const unsigned long long* key_total, const int64_t* n_kept, const int64_t* n_held,
                                 const unsigned* n_refuted, int64_t* stats, cudaStream_t st) {
  learned_stats_kernel<<<1, 1, 0, st>>>(key_total, n_kept, n_held, n_refuted, stats);
  return cudaGetLastError();
}

}  // namespace ls
