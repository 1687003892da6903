// a2: duplication of records into per-tile keys, in front-to-back order.
//
// Records arrive already sorted by (depth bits, record id).  Emitting their
// tile keys in that order and then sorting the keys stably by tile id alone
// gives each tile's list in (depth, id) order, so the 64-bit (tile, depth)
// key of the classic pipeline is never built: the tile sort moves 8 bytes per
// key per pass over ceil(tile bits / 8) passes instead of 12 bytes over six.
//
//   dup_count : support box in tiles per record (binary32 tile rule), packed
//               and stored in depth order; block sums of the tile counts.
//   dup_scan  : exclusive scan of the block sums, total key count K and the
//               capacity check.
//   dup_emit  : block-level prefix of the counts, then each warp writes the
//               keys of its 128 records cooperatively (lane e of the warp's
//               output range finds its record by binary search), so stores
//               are coalesced whatever the footprint sizes; the digit
//               histograms of the tile sort are gathered on the way.
#include "kernels.h"

namespace ls {

namespace {

struct CamLite {
  int W, H, tiles_x, tile_base;
};

__device__ __forceinline__ uint32_t rect_count(uint2 rc) {
  int x0 = rc.x & 0xFFFF, x1 = rc.x >> 16, y0 = rc.y & 0xFFFF, y1 = rc.y >> 16;
  return x1 < x0 ? 0u : (uint32_t)((x1 - x0 + 1) * (y1 - y0 + 1));
}

__global__ void __launch_bounds__(DUP_THREADS) dup_count_kernel(int64_t R, const uint32_t* __restrict__ order,
                                                                const uint32_t* __restrict__ dkey_sorted,
                                                                const float4* __restrict__ foot, const CamTable cams,
                                                                int n_per_cam, const ParDev P,
                                                                uint2* __restrict__ rect_sorted,
                                                                uint32_t* __restrict__ block_sums) {
  __shared__ CamLite s_cam[LS_MAX_CAMS];
  __shared__ uint32_t s_red[DUP_THREADS / 32];
  for (int c = threadIdx.x; c < cams.n; c += blockDim.x)
    s_cam[c] = CamLite{cams.c[c].W, cams.c[c].H, cams.c[c].tiles_x, cams.c[c].tile_base};
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * DUP_BLOCK;
  uint32_t sum = 0;
#pragma unroll
  for (int i = 0; i < DUP_ITEMS; ++i) {
    const int64_t j = base + i * DUP_THREADS + threadIdx.x;
    if (j >= R) break;
    uint2 rc = make_uint2(1u, 0u);  // empty: x1 < x0
    if (dkey_sorted[j] != DKEY_CULLED) {
      const uint32_t r = order[j];
      const CamLite cm = s_cam[r / (uint32_t)n_per_cam];
      const float4 f = foot[r];
      int tx0, tx1, ty0, ty1;
      if (tile_rect(f.x, f.y, f.z, f.w, cm.W, cm.H, P.tile_w, P.tile_h, tx0, tx1, ty0, ty1))
        rc = make_uint2((uint32_t)tx0 | ((uint32_t)tx1 << 16), (uint32_t)ty0 | ((uint32_t)ty1 << 16));
    }
    rect_sorted[j] = rc;
    sum += rect_count(rc);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
  if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = sum;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t t = 0;
    for (int w = 0; w < DUP_THREADS / 32; ++w) t += s_red[w];
    block_sums[blockIdx.x] = t;
  }
}

// One block scans all block sums in chunks of 1024 (exclusive, in place).
__global__ void __launch_bounds__(1024) dup_scan_kernel(int64_t nb, uint32_t* sums, int64_t cap, int64_t* n_keys,
                                                        int64_t* n_valid, int32_t* status) {
  __shared__ uint64_t s_warp[32];
  __shared__ uint64_t s_carry;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) s_carry = 0;
  __syncthreads();
  for (int64_t b0 = 0; b0 < nb; b0 += 1024) {
    const int64_t i = b0 + threadIdx.x;
    uint64_t v = i < nb ? sums[i] : 0;
    uint64_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint64_t u = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += u;
    }
    if (lane == 31) s_warp[warp] = x;
    __syncthreads();
    if (warp == 0) {
      uint64_t w = s_warp[lane];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        uint64_t u = __shfl_up_sync(0xffffffffu, w, o);
        if (lane >= o) w += u;
      }
      s_warp[lane] = w;
    }
    __syncthreads();
    const uint64_t incl = x + (warp > 0 ? s_warp[warp - 1] : 0) + s_carry;
    if (i < nb) sums[i] = (uint32_t)(incl - v);
    __syncthreads();
    if (threadIdx.x == 1023) s_carry = incl;
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const uint64_t K = s_carry;
    *n_keys = (int64_t)K;
    const bool fits = (int64_t)K <= cap;
    *n_valid = fits ? (int64_t)K : 0;
    if (!fits) set_status(status, LS_ERR_CAPACITY);
  }
}

__global__ void __launch_bounds__(DUP_THREADS) dup_emit_kernel(int64_t R, const uint32_t* __restrict__ order,
                                                               const uint2* __restrict__ rect_sorted,
                                                               const uint32_t* __restrict__ block_offs,
                                                               const CamTable cams, int n_per_cam,
                                                               const int64_t* n_valid, uint32_t* __restrict__ keys,
                                                               uint32_t* __restrict__ vals, int key_passes,
                                                               uint32_t* __restrict__ tile_hist) {
  __shared__ uint32_t s_off[DUP_BLOCK + 1];
  __shared__ uint2 s_rect[DUP_BLOCK];
  __shared__ uint32_t s_r[DUP_BLOCK];
  __shared__ uint32_t s_hist[3][RADIX];
  __shared__ uint32_t s_warp[DUP_THREADS / 32];
  __shared__ CamLite s_cam[LS_MAX_CAMS];
  if (*n_valid == 0) return;  // nothing to emit, or over capacity
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int c = tid; c < cams.n; c += DUP_THREADS)
    s_cam[c] = CamLite{cams.c[c].W, cams.c[c].H, cams.c[c].tiles_x, cams.c[c].tile_base};
  for (int i = tid; i < 3 * RADIX; i += DUP_THREADS) (&s_hist[0][0])[i] = 0;
  const int64_t base = (int64_t)blockIdx.x * DUP_BLOCK;
  // coalesced load of the block's records
#pragma unroll
  for (int i = 0; i < DUP_ITEMS; ++i) {
    const int s = i * DUP_THREADS + tid;
    const int64_t j = base + s;
    uint2 rc = make_uint2(1u, 0u);
    uint32_t r = 0;
    if (j < R) {
      rc = rect_sorted[j];
      r = order[j];
    }
    s_rect[s] = rc;
    s_r[s] = r;
  }
  __syncthreads();
  // block exclusive scan of the counts: thread t owns slots 4t..4t+3
  uint32_t c[DUP_ITEMS], run = 0;
#pragma unroll
  for (int i = 0; i < DUP_ITEMS; ++i) {
    c[i] = rect_count(s_rect[DUP_ITEMS * tid + i]);
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
  // warp w emits slots [w*128, w*128+128)
  const int s0 = warp * 32 * DUP_ITEMS, s1 = s0 + 32 * DUP_ITEMS;
  const uint32_t o0 = s_off[s0], o1 = s_off[s1];
  const uint64_t gbase = (uint64_t)block_offs[blockIdx.x];
  for (uint32_t e = o0 + lane; e < o1; e += 32) {
    // last slot in [s0, s1) whose offset is <= e
    int lo = s0, hi = s1 - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (s_off[mid] <= e) lo = mid;
      else hi = mid - 1;
    }
    const uint2 rc = s_rect[lo];
    const uint32_t r = s_r[lo];
    const uint32_t m = e - s_off[lo];
    const uint32_t x0 = rc.x & 0xFFFF, x1 = rc.x >> 16, y0 = rc.y & 0xFFFF;
    const uint32_t w = x1 - x0 + 1;
    const CamLite cm = s_cam[r / (uint32_t)n_per_cam];
    const uint32_t key = (uint32_t)cm.tile_base + (y0 + m / w) * (uint32_t)cm.tiles_x + x0 + m % w;
    keys[gbase + e] = key;
    vals[gbase + e] = r;
    for (int p = 0; p < key_passes; ++p) atomicAdd(&s_hist[p][(key >> (8 * p)) & 255u], 1u);
  }
  __syncthreads();
  for (int i = tid; i < key_passes * RADIX; i += DUP_THREADS) {
    const uint32_t v = (&s_hist[0][0])[i];
    if (v) atomicAdd(&tile_hist[i], v);
  }
}

}  // namespace

cudaError_t launch_dup_count(int64_t R, const uint32_t* order, const uint32_t* dkey_sorted, const float4* foot,
                             const CamTable& cams, int n_per_cam, const ParDev& P, uint2* rect_sorted,
                             uint32_t* block_sums, cudaStream_t st) {
  if (R == 0) return cudaSuccess;
  dup_count_kernel<<<ceil_div(R, DUP_BLOCK), DUP_THREADS, 0, st>>>(R, order, dkey_sorted, foot, cams, n_per_cam, P,
                                                                  rect_sorted, block_sums);
  return cudaGetLastError();
}

cudaError_t launch_dup_scan(int64_t R, uint32_t* block_sums, int64_t cap, int64_t* n_keys_dev, int64_t* n_valid_dev,
                            int32_t* status, cudaStream_t st) {
  dup_scan_kernel<<<1, 1024, 0, st>>>(R > 0 ? (int64_t)ceil_div(R, DUP_BLOCK) : 0, block_sums, cap, n_keys_dev,
                                      n_valid_dev, status);
  return cudaGetLastError();
}

cudaError_t launch_dup_emit(int64_t R, const uint32_t* order, const uint2* rect_sorted, const uint32_t* block_offs,
                            const CamTable& cams, int n_per_cam, const int64_t* n_valid_dev, uint32_t* keys,
                            uint32_t* vals, int key_passes, uint32_t* tile_hist, cudaStream_t st) {
  if (R == 0) return cudaSuccess;
  dup_emit_kernel<<<ceil_div(R, DUP_BLOCK), DUP_THREADS, 0, st>>>(R, order, rect_sorted, block_offs, cams, n_per_cam,
                                                                 n_valid_dev, keys, vals, key_passes, tile_hist);
  return cudaGetLastError();
}

}  // namespace ls
