// a2: duplication of records into per-tile keys, in front-to-back order.
//
// Records arrive already sorted by (depth bits, record id).  Emitting their
// tile keys in that order and then sorting the keys stably by tile id alone
// gives each tile's list in (depth, id) order, so the 64-bit (tile, depth)
// key of the classic pipeline is never built: the tile sort moves 8 bytes per
// key per pass over ceil(tile bits / 8) passes instead of 12 bytes over six.
//
// A record gets a key for a tile of its support box only when its support
// ellipse reaches one of the tile's pixel centres (emit.cuh, tile_touched):
// the pairs the blend can composite are all kept, and the ~40 % of box tiles
// that only the box corners reach are never sorted or blended.
//
//   dup_count : support box in tiles per record (binary32 tile rule), packed
//               and stored in depth order.
//   enum_keys : per warp of 64 depth-ordered records, the box tiles the
//               ellipse reaches, counted (first launch) and then, after
//               dup_scan has turned the warp counts into offsets, written
//               (second launch) with the digit histograms of the tile sort.
//               The learned path (learned.cu) uses the same kernel with the
//               proposal depth (kept keys) and the refuted tiles (held-out
//               keys) as extra conditions.
//   dup_reduce, dup_scan : exclusive scan of the warp counts, total key count
//               K and the capacity check.
#include "emit.cuh"
#include "kernels.h"

namespace ls {

namespace {


__global__ void __launch_bounds__(DUP_THREADS) dup_count_kernel(int64_t R, const uint32_t* __restrict__ order,
                                                                const uint32_t* __restrict__ dkey_sorted,
                                                                const float4* __restrict__ foot, const CamTable cams,
                                                                int n_per_cam, const ParDev P,
                                                                uint2* __restrict__ rect_sorted) {
  chain_enter();
  __shared__ CamLite s_cam[LS_MAX_CAMS];
  for (int c = threadIdx.x; c < cams.n; c += blockDim.x)
    s_cam[c] = CamLite{cams.c[c].W, cams.c[c].H, cams.c[c].tiles_x, cams.c[c].tile_base};
  __syncthreads();
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= R) return;
  uint2 rc = make_uint2(1u, 0u);  // empty: x1 < x0
  if (dkey_sorted[j] != DKEY_CULLED) {
    const uint32_t r = order[j];
    const CamLite cm = s_cam[cams.n > 1 ? r / (uint32_t)n_per_cam : 0u];
    const float4 f = foot[r];
    int tx0, tx1, ty0, ty1;
    if (tile_rect(f.x, f.y, f.z, f.w, cm.W, cm.H, P.tile_w, P.tile_h, tx0, tx1, ty0, ty1))
      rc = make_uint2((uint32_t)tx0 | ((uint32_t)tx1 << 16), (uint32_t)ty0 | ((uint32_t)ty1 << 16));
  }
  rect_sorted[j] = rc;
}

// The scan of the warp counts in two launches over chunks of SCAN_CHUNK
// counts, a block per chunk: dup_reduce sums each chunk; dup_scan adds up the
// sums of the chunks before its own (the carry) and scans its chunk in place
// (exclusive), 8 consecutive counts per thread.  The chunk sums sit behind
// the counts, in the same buffer (enum_count_words).
constexpr int SCAN_THREADS = 1024, SCAN_PER = 8, SCAN_CHUNK = SCAN_THREADS * SCAN_PER;

__device__ __forceinline__ uint64_t* scan_parts(uint32_t* counts, int64_t n) {
  return reinterpret_cast<uint64_t*>(counts + ((n + 1) & ~(int64_t)1));
}

// The 8 counts of this thread in its chunk (zero past n).
__device__ __forceinline__ void scan_load(const uint32_t* counts, int64_t n, int64_t b0, uint32_t (&v)[SCAN_PER]) {
  const int64_t i0 = b0 + (int64_t)SCAN_PER * threadIdx.x;
  if (i0 + SCAN_PER <= n) {  // 32-byte aligned: b0 and SCAN_PER * tid are multiples of 8 counts
    const uint4* g = reinterpret_cast<const uint4*>(counts + i0);
    const uint4 a = g[0], b = g[1];
    v[0] = a.x, v[1] = a.y, v[2] = a.z, v[3] = a.w, v[4] = b.x, v[5] = b.y, v[6] = b.z, v[7] = b.w;
  } else {
#pragma unroll
    for (int k = 0; k < SCAN_PER; ++k) v[k] = i0 + k < n ? counts[i0 + k] : 0u;
  }
}

// Block sum of x (every thread gets it); s_warp holds 32 entries.
__device__ __forceinline__ uint64_t block_sum(uint64_t x, uint64_t* s_warp) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  if (lane == 0) s_warp[warp] = x;
  __syncthreads();
  uint64_t t = lane < (int)(blockDim.x >> 5) ? s_warp[lane] : 0;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  __syncthreads();
  return t;
}

__global__ void __launch_bounds__(SCAN_THREADS) dup_reduce_kernel(int64_t n, uint32_t* counts) {
  chain_enter();
  __shared__ uint64_t s_warp[32];
  uint32_t v[SCAN_PER];
  scan_load(counts, n, (int64_t)blockIdx.x * SCAN_CHUNK, v);
  uint64_t x = 0;
#pragma unroll
  for (int k = 0; k < SCAN_PER; ++k) x += v[k];
  x = block_sum(x, s_warp);
  if (threadIdx.x == 0) scan_parts(counts, n)[blockIdx.x] = x;
}

__global__ void __launch_bounds__(SCAN_THREADS) dup_scan_kernel(int64_t n, uint32_t* counts, int64_t cap,
                                                                int64_t* n_keys, int64_t* n_valid, int32_t* status) {
  chain_enter();
  __shared__ uint64_t s_warp[32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t b0 = (int64_t)blockIdx.x * SCAN_CHUNK;
  uint64_t carry = 0;
  if (blockIdx.x > 0) {
    const uint64_t* part = scan_parts(counts, n);
    for (int i = tid; i < (int)blockIdx.x; i += SCAN_THREADS) carry += part[i];
    carry = block_sum(carry, s_warp);
  }
  uint32_t v[SCAN_PER];
  scan_load(counts, n, b0, v);
  uint64_t run = 0;
#pragma unroll
  for (int k = 0; k < SCAN_PER; ++k) run += v[k];
  uint64_t x = run;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint64_t u = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += u;
  }
  if (lane == 31) s_warp[warp] = x;
  __syncthreads();
  if (warp == 0) {
    uint64_t w = s_warp[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint64_t u = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += u;
    }
    s_warp[lane] = w;
  }
  __syncthreads();
  uint64_t ex = x - run + (warp > 0 ? s_warp[warp - 1] : 0) + carry;
  const int64_t i0 = b0 + (int64_t)SCAN_PER * tid;
  if (i0 + SCAN_PER <= n) {
    uint32_t o[SCAN_PER];
#pragma unroll
    for (int k = 0; k < SCAN_PER; ++k) {
      o[k] = (uint32_t)ex;
      ex += v[k];
    }
    uint4* g = reinterpret_cast<uint4*>(counts + i0);
    g[0] = make_uint4(o[0], o[1], o[2], o[3]);
    g[1] = make_uint4(o[4], o[5], o[6], o[7]);
  } else {
#pragma unroll
    for (int k = 0; k < SCAN_PER; ++k) {
      if (i0 + k < n) counts[i0 + k] = (uint32_t)ex;
      ex += v[k];
    }
  }
  if (blockIdx.x == gridDim.x - 1 && tid == SCAN_THREADS - 1) {  // ex is now the total
    const uint64_t K = ex;
    *n_keys = (int64_t)K;
    const bool fits = (int64_t)K <= cap;
    *n_valid = fits ? (int64_t)K : 0;
    if (!fits) set_status(status, LS_ERR_CAPACITY);
  }
}

// The condition of each mode on a key its record reaches (depth bits dk):
// ENUM_ALL none; ENUM_KEPT depth bits <= the tile's proposal; ENUM_HELD the
// tile is refuted and the depth is beyond its proposal.
template <int MODE>
__device__ __forceinline__ bool key_taken(const EnumArgs& A, uint32_t dk, uint32_t key) {
  if (MODE == ENUM_ALL) return true;
  const uint32_t lim = __ldg(A.dstar_bits + key);
  if (MODE == ENUM_KEPT) return dk <= lim;
  return A.refuted[key] && dk > lim;
}

constexpr uint32_t NO_STASH = 0xFFFFFFFFu;

// Keys of ENUM_WARP_RECS depth-ordered records per warp (emit.cuh).
//
// Count launch (EMIT = false): each warp walks its records' rows and keys,
// counts the taken keys (warp_counts) and, when the whole box-tile count of
// its records fits in the stash (tmp_*, bump-allocated per warp), also
// writes them there, compacted (warp_tbase; NO_STASH otherwise), with their
// tile-sort digits.  ENUM_KEPT takes no key of a record that lies beyond the
// proposal bound of its whole box; when key_total is given, it adds every
// reached key to it (walking such a record's rows for the count only),
// else it drops such records up front.  Emit launch (EMIT =
// true), after the counts are scanned into offsets: a stashed warp copies
// its keys to its offset; any other warp walks again and writes them (and
// their digits).  ENUM_HELD drops up front every record whose box holds no
// refuted tile (summed-area table `sat`).
template <bool EMIT, int MODE>
__global__ void __launch_bounds__(ENUM_THREADS) enum_keys_kernel(EnumArgs A) {
  chain_enter();
  __shared__ EnumRec S[ENUM_WARPS][ENUM_WARP_RECS];
  __shared__ uint4 SR[ENUM_WARPS][32];  // a step's rows with keys: {first key, first index, record, depth bits}
  __shared__ CamLite s_cam[LS_MAX_CAMS];
  __shared__ uint32_t s_hist[3][RADIX];
  const unsigned FULL = 0xffffffffu;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const unsigned lt = (1u << lane) - 1u;
  const int64_t gw = (int64_t)blockIdx.x * ENUM_WARPS + warp;
  // ENUM_HELD: a record at or in front of the smallest proposal of a refuted
  // tile has no held-out key; depth order puts all such records first
  const uint32_t held_lim = MODE == ENUM_HELD ? ~*A.refuted_floor : 0u;
  bool none_here = false;
  if (MODE == ENUM_HELD) {
    const int64_t jl = min(A.R, (int64_t)(blockIdx.x + 1) * ENUM_BLOCK_RECS) - 1;
    none_here = A.dkey_sorted[jl] <= held_lim;
  }
  if ((MODE == ENUM_HELD && (*A.n_refuted == 0u || none_here)) || (EMIT && *A.n_valid == 0)) {
    if (!EMIT && lane == 0) {
      A.warp_counts[gw] = 0u;
      A.warp_tbase[gw] = NO_STASH;
    }
    return;  // block-uniform: nothing to do, or over capacity
  }
  if (EMIT) {  // a block whose warps took no key has nothing to write
    const int64_t g0 = (int64_t)blockIdx.x * ENUM_WARPS, g1 = g0 + ENUM_WARPS;
    const uint64_t first = A.warp_counts[g0];
    const uint64_t last = g1 < A.n_warps ? (uint64_t)A.warp_counts[g1] : (uint64_t)*A.n_valid;
    if (last == first) return;  // block-uniform
  }
  for (int c = tid; c < A.cams.n; c += ENUM_THREADS)
    s_cam[c] = CamLite{A.cams.c[c].W, A.cams.c[c].H, A.cams.c[c].tiles_x, A.cams.c[c].tile_base};
  const bool hist = A.tile_hist != nullptr;
  for (int i = tid; i < 3 * RADIX; i += ENUM_THREADS) (&s_hist[0][0])[i] = 0;
  __syncthreads();
  uint64_t out = 0;
  bool walk = true, counted = false;  // counted: digits of keys written by this warp were counted
  if (EMIT) {
    out = A.out_base + (uint64_t)A.warp_counts[gw];
    const uint32_t tb = A.warp_tbase[gw];
    if (tb != NO_STASH) {  // copy the stashed keys (their digits were counted then)
      walk = false;
      const uint64_t end = gw + 1 < A.n_warps ? A.out_base + (uint64_t)A.warp_counts[gw + 1]
                                              : A.out_base + (uint64_t)*A.n_valid;
      const uint32_t n = (uint32_t)(end - out);
      // sixteen 32-key chunks in flight per lane (most warps copy theirs in
      // one round; four per lane took 7 us longer per frame)
      for (uint32_t i0 = 0; i0 < n; i0 += 512) {
        uint32_t k[16], v[16];
#pragma unroll
        for (int u = 0; u < 16; ++u) {
          const uint32_t i = i0 + 32 * u + lane;
          if (i < n) {
            k[u] = A.tmp_keys[tb + i];
            v[u] = A.tmp_vals[tb + i];
          }
        }
#pragma unroll
        for (int u = 0; u < 16; ++u) {
          const uint32_t i = i0 + 32 * u + lane;
          if (i < n) {
            A.keys[out + i] = k[u];
            A.vals[out + i] = v[u];
          }
        }
      }
    }
  }
  if (walk) {
    // the warp's records with a non-empty box, compacted, with the offsets of their rows
    EnumRec* W = S[warp];
    uint4* SRw = SR[warp];
    int n_nz = 0;
    uint32_t total = 0, box_total = 0;
    const int sx = s_cam[0].tiles_x + 1;
#pragma unroll
    for (int i = 0; i < ENUM_WARP_RECS / 32; ++i) {
      const int64_t j = (int64_t)blockIdx.x * ENUM_BLOCK_RECS + warp * ENUM_WARP_RECS + i * 32 + lane;
      uint2 rc = make_uint2(1u, 0u);
      uint32_t r = 0, dk = DKEY_CULLED;
      if (j < A.R) {
        rc = A.rect_sorted[j];
        r = A.order[j];
        if (MODE != ENUM_ALL) dk = A.dkey_sorted[j];
      }
      if (MODE == ENUM_HELD && dk <= held_lim) rc = make_uint2(1u, 0u);
      if (MODE == ENUM_HELD && box_rows(rc)) {
        const int x0 = rc.x & 0xFFFF, x1 = rc.x >> 16, y0 = rc.y & 0xFFFF, y1 = rc.y >> 16;
        const int* sat = A.sat;
        if (sat[(y1 + 1) * sx + x1 + 1] - sat[y0 * sx + x1 + 1] - sat[(y1 + 1) * sx + x0] + sat[y0 * sx + x0] == 0)
          rc = make_uint2(1u, 0u);
      }
      // ENUM_KEPT: a record beyond the proposal bound of its whole box takes
      // no key; it is walked only to count its reached keys (*key_total)
      bool beyond = false;
      if (MODE == ENUM_KEPT && box_rows(rc)) {
        beyond = dk > box_dstar_bound(A.dstar_pyr, A.pyr, (int)(rc.x & 0xFFFF), (int)(rc.x >> 16),
                                      (int)(rc.y & 0xFFFF), (int)(rc.y >> 16));
        if (beyond && (EMIT || !A.key_total)) rc = make_uint2(1u, 0u);
      }
      const uint32_t rows = box_rows(rc);
      uint32_t x = rows, bx = beyond ? 0u : box_count(rc);
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t u = __shfl_up_sync(FULL, x, o);
        if (lane >= o) x += u;
        bx += __shfl_xor_sync(FULL, bx, o);
      }
      const unsigned nz = __ballot_sync(FULL, rows > 0);
      if (rows) {
        const CamLite cm = s_cam[A.cams.n > 1 ? r / (uint32_t)A.n_per_cam : 0u];
        EnumRec& t = W[n_nz + __popc(nz & lt)];
        enum_rec(t, total + x - rows, rc, r, dk, cm, A.rec);
        if (MODE == ENUM_KEPT) t.beyond = beyond;
      }
      n_nz += __popc(nz);
      total += __shfl_sync(FULL, x, 31);
      box_total += bx;
    }
    __syncwarp();
    // count launch: a stash region for every box tile of the warp's records
    uint32_t tb = NO_STASH;
    if (!EMIT) {
      if (lane == 0 && box_total > 0) {
        const unsigned long long b = atomicAdd(A.tmp_ctr, (unsigned long long)box_total);
        if (b + box_total <= (unsigned long long)A.tmp_cap) tb = (uint32_t)b;
      }
      tb = __shfl_sync(FULL, tb, 0);
    }
    const bool store = EMIT || tb != NO_STASH;
    counted = store;
    uint32_t kept = 0, reached = 0;
    int sp = 0;  // record of the step's first row
    for (uint32_t cb = 0; cb < total; cb += 32) {
      // lane i marks where record sp + 1 + i starts, when inside this step;
      // lane l's record is sp plus the number of marks at or below l
      const int ns = sp + 1 + lane;
      uint32_t mark = 0;
      if (ns < n_nz) {
        const uint32_t d = W[ns].off - cb;
        if (d < 32u) mark = 1u << d;
      }
      const int sl = sp + __popc(__reduce_or_sync(FULL, mark) & ((2u << lane) - 1u));
      const uint32_t e = cb + lane;
      uint32_t n = 0, key0 = 0, r = 0, dk = 0;
      if (e < total) {
        const uint4* q = reinterpret_cast<const uint4*>(&W[sl]);
        const uint4 g0 = q[0], g3 = q[3];
        const float4 g1 = reinterpret_cast<const float4*>(q)[1], g2 = reinterpret_cast<const float4*>(q)[2];
        const int row = (int)(e - g0.x), x0 = (int)(g0.w & 0xFFFFu), y0 = (int)(g0.w >> 16);
        int tx_a, tx_b;
        row_range(g1, g2, y0 + row, A.tile_w, A.tile_h, x0, x0 + (int)(g0.z & 0xFFFFu) - 1, tx_a, tx_b);
        if (tx_b >= tx_a) {
          n = (uint32_t)(tx_b - tx_a + 1);
          key0 = g0.y + (uint32_t)row * (g0.z >> 16) + (uint32_t)(tx_a - x0);
        }
        r = g3.x;
        dk = g3.y;
        if (MODE == ENUM_KEPT && g3.z) {  // beyond every proposal of its box: reached, none taken
          reached += n;
          n = 0;
        }
      }
      sp = __shfl_sync(FULL, sl, 31);
      // this step's rows with keys to walk, compacted, and the walk over their keys
      uint32_t xs = n;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t u = __shfl_up_sync(FULL, xs, o);
        if (lane >= o) xs += u;
      }
      const unsigned rz = __ballot_sync(FULL, n > 0);
      if (n) SRw[__popc(rz & lt)] = make_uint4(key0, xs - n, r, dk);
      const uint32_t keys_here = __shfl_sync(FULL, xs, 31);
      const int n_rows = __popc(rz);
      reached += n;
      __syncwarp();
      int sq = 0;
      for (uint32_t c2 = 0; c2 < keys_here; c2 += 32) {
        const int ms = sq + 1 + lane;
        uint32_t mk = 0;
        if (ms < n_rows) {
          const uint32_t d = SRw[ms].y - c2;
          if (d < 32u) mk = 1u << d;
        }
        const int sj = sq + __popc(__reduce_or_sync(FULL, mk) & ((2u << lane) - 1u));
        const uint32_t e2 = c2 + lane;
        bool take = false;
        uint32_t key = 0, rr = 0;
        if (e2 < keys_here) {
          const uint4 rw = SRw[sj];
          key = rw.x + (e2 - rw.y);
          rr = rw.z;
          take = key_taken<MODE>(A, rw.w, key);
        }
        sq = __shfl_sync(FULL, sj, 31);
        const unsigned bal = __ballot_sync(FULL, take);
        if (take && store) {
          const uint32_t rank = kept + __popc(bal & lt);
          if (EMIT) {
            A.keys[out + rank] = key;
            A.vals[out + rank] = rr;
          } else {
            A.tmp_keys[tb + rank] = key;
            A.tmp_vals[tb + rank] = rr;
          }
        }
        if (hist && store && bal) {
          // low digit: consecutive tiles, distinct per lane; higher digits:
          // usually one value for the whole step, added once
          if (take) atomicAdd(&s_hist[0][(key >> A.dshift[0]) & A.dmask[0]], 1u);
          const int first = __ffs(bal) - 1;
          for (int p = 1; p < A.key_passes; ++p) {
            const uint32_t d = (key >> A.dshift[p]) & A.dmask[p];
            const uint32_t d0 = __shfl_sync(FULL, d, first);
            if (__all_sync(FULL, !take || d == d0)) {
              if (lane == first) atomicAdd(&s_hist[p][d0], (uint32_t)__popc(bal));
            } else if (take) {
              atomicAdd(&s_hist[p][d], 1u);
            }
          }
        }
        kept += __popc(bal);
      }
      __syncwarp();  // the rows of this step are read before the next step rewrites them
    }
    if (!EMIT) {
      if (MODE == ENUM_KEPT && A.key_total) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) reached += __shfl_xor_sync(FULL, reached, o);
      }
      if (lane == 0) {
        A.warp_counts[gw] = kept;
        A.warp_tbase[gw] = tb;
        if (MODE == ENUM_KEPT && A.key_total && reached) atomicAdd(A.key_total, (unsigned long long)reached);
      }
    }
  }
  if (!hist) return;
  // digits were counted only where keys were written here
  if (!__syncthreads_or(counted)) return;
  for (int i = tid; i < A.key_passes * RADIX; i += ENUM_THREADS) {
    const uint32_t v = (&s_hist[0][0])[i];
    if (v) atomicAdd(&A.tile_hist[i], v);
  }
}

}  // namespace

cudaError_t launch_dup_count(int64_t R, const uint32_t* order, const uint32_t* dkey_sorted, const float4* foot,
                             const CamTable& cams, int n_per_cam, const ParDev& P, uint2* rect_sorted, cudaStream_t st) {
  if (R == 0) return cudaSuccess;
  return launch_chain(dup_count_kernel, dim3(ceil_div(R, DUP_THREADS)), dim3(DUP_THREADS), 0, st, R, order,
                      dkey_sorted, foot, cams, n_per_cam, P, rect_sorted);
}

cudaError_t launch_dup_scan(int64_t n, uint32_t* counts, int64_t cap, int64_t* n_keys_dev, int64_t* n_valid_dev,
                            int32_t* status, cudaStream_t st) {
  const int64_t nb = n > 0 ? ceil_div(n, SCAN_CHUNK) : 1;
  if (nb > 1) {
    const cudaError_t e = launch_chain(dup_reduce_kernel, dim3((unsigned)nb), dim3(SCAN_THREADS), 0, st, n, counts);
    if (e != cudaSuccess) return e;
  }
  return launch_chain(dup_scan_kernel, dim3((unsigned)nb), dim3(SCAN_THREADS), 0, st, n, counts, cap, n_keys_dev,
                      n_valid_dev, status);
}

int64_t enum_count_words(int64_t R) {
  const int64_t n = enum_warps(R);
  return ((n + 1) & ~(int64_t)1) + 2 * (n > 0 ? ceil_div(n, SCAN_CHUNK) : 1);
}

int64_t enum_warps(int64_t R) { return R > 0 ? (int64_t)ceil_div(R, ENUM_BLOCK_RECS) * ENUM_WARPS : 0; }

cudaError_t launch_enum_keys(bool emit, int mode, const EnumArgs& A, cudaStream_t st) {
  if (A.R == 0) return cudaSuccess;
  const unsigned grid = ceil_div(A.R, ENUM_BLOCK_RECS);
#define LS_EK(E, M) launch_chain(enum_keys_kernel<E, M>, dim3(grid), dim3(ENUM_THREADS), 0, st, A)
  if (emit) {
    if (mode == ENUM_ALL) return LS_EK(true, ENUM_ALL);
    if (mode == ENUM_KEPT) return LS_EK(true, ENUM_KEPT);
    return LS_EK(true, ENUM_HELD);
  }
  if (mode == ENUM_ALL) return LS_EK(false, ENUM_ALL);
  if (mode == ENUM_KEPT) return LS_EK(false, ENUM_KEPT);
  return LS_EK(false, ENUM_HELD);
#undef LS_EK
}

}  // namespace ls
