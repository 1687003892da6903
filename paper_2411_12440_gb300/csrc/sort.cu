// a3: onesweep LSD radix sort of (uint32 key, uint32 value) pairs with digits
// of up to 8 bits (single-pass prefix by decoupled look-back); the tile sort
// splits the tile-id bits evenly over its passes (13 bits: 7 + 6), so each
// pass ranks with as few ballots and digits as the keys need.  Stable, so sorting the
// duplication output by tile id keeps each tile's entries in the depth order
// they were emitted in: the front-to-back order of Sec. 3.1 Eq. 6.
//
// Per pass a persistent grid claims the partitions of SORT_PART keys with an
// atomic ticket (so a partition only ever waits on partitions that are
// already running, and no block is launched for capacity that holds no keys),
// ranked in registers with warp ballots, published as a per-digit aggregate,
// completed by looking back over its predecessors, staged in shared memory in
// sorted order and written out in digit runs.  Every wait on a predecessor is
// bounded: after a host-set number of polls (about a second at the default)
// the kernel records LS_ERR_TIMEOUT and finishes with in-bounds writes only.
#include "kernels.h"

namespace ls {

namespace {

constexpr uint64_t LB_AGG = 1ull << 62;
constexpr uint64_t LB_INC = 1ull << 63;
constexpr uint64_t LB_VAL = (1ull << 62) - 1;
// Bounded waits of the look-back (ls_debug_set_sort_wait): polls before a
// wait gives up, and a partition of the last tile-sort pass that publishes
// nothing (-1: none), so that the wait of the partition after it runs out.
constexpr int SPIN_LIMIT_DEFAULT = 1 << 21;
int g_spin_limit = SPIN_LIMIT_DEFAULT;
int g_hold_part = -1;
// Threads of a onesweep CTA, its warps and the CTAs an SM holds.
constexpr int OS_THREADS = SORT_THREADS;
constexpr int SORT_WARPS = OS_THREADS / 32;
constexpr int OS_CTAS_PER_SM = 1024 / OS_THREADS;
// Predecessor states a look-back step loads at once.  On the 3M-primitive
// 1080p frame a partition's look-back reads 15-33 predecessors and is
// its longest phase; 4 at once took 4 us off the duplicate + sort stage,
// 8 and 16 added 10 and 37 us (more polling traffic).
constexpr int LB_WINDOW = 4;
static_assert(OS_THREADS >= RADIX && OS_THREADS % RADIX == 0, "a thread for every digit");

__device__ __forceinline__ uint64_t ld_relaxed_u64(const uint64_t* p) {
  uint64_t v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_relaxed_u64(uint64_t* p, uint64_t v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Inclusive scan of one value per thread over a block of WARPS warps.
template <int WARPS>
__device__ __forceinline__ uint32_t block_incl_scan(uint32_t v, uint32_t* s_warp) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t u = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += u;
  }
  if (lane == 31) s_warp[warp] = v;
  __syncthreads();
  if (warp == 0) {
    uint32_t w = lane < WARPS ? s_warp[lane] : 0;
#pragma unroll
    for (int o = 1; o < WARPS; o <<= 1) {
      uint32_t u = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += u;
    }
    if (lane < WARPS) s_warp[lane] = w;
  }
  __syncthreads();
  return v + (warp > 0 ? s_warp[warp - 1] : 0);
}

__global__ void __launch_bounds__(256) radix_hist_kernel(const uint32_t* __restrict__ keys, const int64_t* n_dev,
                                                         int64_t n_host, int begin_bit, int passes,
                                                         uint32_t* __restrict__ hist) {
  chain_enter();
  __shared__ uint32_t s_h[4][RADIX];
  for (int i = threadIdx.x; i < 4 * RADIX; i += blockDim.x) (&s_h[0][0])[i] = 0;
  __syncthreads();
  const int64_t n = n_dev ? *n_dev : n_host;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    uint32_t k = keys[i];
    for (int p = 0; p < passes; ++p) atomicAdd(&s_h[p][(k >> (begin_bit + 8 * p)) & 255u], 1u);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < passes * RADIX; i += blockDim.x) {
    uint32_t v = (&s_h[0][0])[i];
    if (v) atomicAdd(&hist[i], v);
  }
}

__global__ void __launch_bounds__(RADIX) radix_scan_kernel(uint32_t* hist) {
  chain_enter();
  __shared__ uint32_t s_warp[RADIX / 32];
  uint32_t* h = hist + (size_t)blockIdx.x * RADIX;
  uint32_t v = h[threadIdx.x];
  uint32_t incl = block_incl_scan<RADIX / 32>(v, s_warp);
  h[threadIdx.x] = incl - v;
}

__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Dynamic shared memory of one onesweep block.
template <int PART>
struct OnesweepSmem {
  uint32_t keys[PART];           // keys in block-sorted order
  uint32_t vin[PART];            // the partition's values in input order (cp.async)
  uint16_t src[PART];            // input position of the key at each sorted slot
  uint32_t whist[SORT_WARPS][RADIX];
  uint32_t local[RADIX];
  uint32_t glob[RADIX];
  uint32_t warp[SORT_WARPS];
  uint32_t part;
};

// BITS: digit width of the pass (<= 8); digits are (key >> shift) & (2^BITS - 1).
// ITEMS: keys per thread; a partition holds OS_THREADS * ITEMS keys.
template <int BITS, int ITEMS>
__global__ void __launch_bounds__(OS_THREADS, OS_CTAS_PER_SM) onesweep_kernel(
    const uint32_t* __restrict__ keys_in, const uint32_t* __restrict__ vals_in, uint32_t* __restrict__ keys_out,
    uint32_t* __restrict__ vals_out, const int64_t* n_dev, int64_t n_host, int shift,
    const uint32_t* __restrict__ digit_base, uint64_t* lookback, uint32_t* part_ctr, uint2* ranges,
    int32_t* status, int spin_limit, int hold_part) {
  chain_enter();
  constexpr uint32_t MASK = (1u << BITS) - 1u;
  constexpr int PART = OS_THREADS * ITEMS;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  OnesweepSmem<PART>& S = *reinterpret_cast<OnesweepSmem<PART>*>(smem_raw);

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t n = n_dev ? *n_dev : n_host;
  // persistent: the block takes partitions by ticket until none is left
  for (;;) {
  __syncthreads();  // the previous partition is done with shared memory
  for (int i = tid; i < SORT_WARPS * RADIX; i += OS_THREADS) (&S.whist[0][0])[i] = 0;
  if (tid == 0) S.part = atomicAdd(part_ctr, 1u);
  __syncthreads();
  const uint32_t part = S.part;
  const int64_t base = (int64_t)part * PART;
  if (base >= n) break;  // block-uniform
  const int n_in = (int)(n - base < PART ? n - base : PART);

  // values: asynchronous copy into shared memory, in flight during ranking
  if (vals_in) {
    for (int i = tid; i < n_in; i += OS_THREADS) cp_async4(&S.vin[i], vals_in + base + i);
    asm volatile("cp.async.commit_group;" ::: "memory");
  }
  // keys: warp-striped, warp w holds positions w*32*ITEMS + i*32 + lane
  const int wofs = warp * 32 * ITEMS;
  uint32_t k[ITEMS];
#pragma unroll
  for (int i = 0; i < ITEMS; ++i) {
    const int li = wofs + i * 32 + lane;
    k[i] = li < n_in ? keys_in[base + li] : 0xFFFFFFFFu;
  }
  // rank inside the warp: peers with the same digit from 8 ballots; items are
  // visited in position order, so ranks are stable.  Ranks fit 16 bits.
  uint32_t rk[(ITEMS + 1) / 2];
#pragma unroll
  for (int i = 0; i < (ITEMS + 1) / 2; ++i) rk[i] = 0;
  const uint32_t lt = (1u << lane) - 1u;
#pragma unroll
  for (int i = 0; i < ITEMS; ++i) {
    const bool valid = wofs + i * 32 + lane < n_in;
    const uint32_t d = (k[i] >> shift) & MASK;
    uint32_t peers = __ballot_sync(0xffffffffu, valid);
#pragma unroll
    for (int b = 0; b < BITS; ++b) {
      const uint32_t bit = (d >> b) & 1u;
      const uint32_t bal = __ballot_sync(0xffffffffu, bit);
      peers &= bit ? bal : ~bal;
    }
    const uint32_t before = S.whist[warp][d];
    __syncwarp();
    rk[i / 2] |= (before + __popc(peers & lt)) << (16 * (i & 1));
    if (valid && lane == 31 - __clz(peers)) S.whist[warp][d] = before + __popc(peers);
    __syncwarp();
  }
  __syncthreads();

  // one thread per digit (the first RADIX threads): warp-exclusive offsets,
  // block count, look-back
  {
    const int d = tid;
    const bool digit = d < RADIX;
    uint32_t run = 0;
    if (digit) {
#pragma unroll
      for (int w = 0; w < SORT_WARPS; ++w) {
        uint32_t c = S.whist[w][d];
        S.whist[w][d] = run;
        run += c;
      }
    }
    uint64_t* my = lookback + (size_t)part * RADIX + d;
    const bool used = digit && d <= (int)MASK;  // digits beyond the pass's width never occur
    const bool publish = (int)part != hold_part;
    if (used && publish) st_relaxed_u64(my, (part == 0 ? LB_INC : LB_AGG) | (uint64_t)run);
    const uint32_t incl = block_incl_scan<SORT_WARPS>(run, S.warp);  // threads past RADIX add 0
    if (digit) S.local[d] = incl - run;
    uint64_t prefix = 0;
    if (used && part > 0) {
      // Walk back over the predecessors LB_WINDOW at a time (their states
      // loaded together), summing aggregates up to the first inclusive
      // prefix.  A window stops at its first unpublished state; when that
      // is the nearest one, only it is polled until it is published.
      int64_t p = (int64_t)part - 1;
      int spins = 0;
      bool done = false;
      while (!done && p >= 0) {
        uint64_t w[LB_WINDOW];
#pragma unroll
        for (int i = 0; i < LB_WINDOW; ++i)
          w[i] = p - i >= 0 ? ld_relaxed_u64(lookback + (size_t)(p - i) * RADIX + d) : 0ull;
        int took = 0;
#pragma unroll
        for (int i = 0; i < LB_WINDOW; ++i) {
          if (done || p - i < 0) break;
          uint64_t v = w[i];
          if ((v & (LB_AGG | LB_INC)) == 0) {
            if (i > 0) break;  // the next window starts here
            while ((v & (LB_AGG | LB_INC)) == 0) {
              if (++spins > spin_limit) break;
              v = ld_relaxed_u64(lookback + (size_t)p * RADIX + d);
            }
            if ((v & (LB_AGG | LB_INC)) == 0) {
              set_status(status, LS_ERR_TIMEOUT);
              done = true;
              break;
            }
          }
          prefix += v & LB_VAL;
          if (v & LB_INC) done = true;
          took = i + 1;
        }
        p -= took;
      }
      if (publish) st_relaxed_u64(my, LB_INC | (prefix + run));
    }
    if (digit) S.glob[d] = digit_base[d] + (uint32_t)prefix - S.local[d];
  }
  __syncthreads();

  // stage the keys (and where each came from) in block-sorted order
#pragma unroll
  for (int i = 0; i < ITEMS; ++i) {
    const int li = wofs + i * 32 + lane;
    if (li < n_in) {
      const uint32_t d = (k[i] >> shift) & MASK;
      const uint32_t pos = S.local[d] + S.whist[warp][d] + ((rk[i / 2] >> (16 * (i & 1))) & 0xFFFFu);
      S.keys[pos] = k[i];
      S.src[pos] = (uint16_t)li;
    }
  }
  if (vals_in) cp_async_wait_all();
  __syncthreads();
  // digit runs go to consecutive global positions
  for (int s = tid; s < n_in; s += OS_THREADS) {
    const uint32_t key = S.keys[s];
    const uint32_t dst = S.glob[(key >> shift) & MASK] + (uint32_t)s;
    if (dst < (uint64_t)n) {
      keys_out[dst] = key;
      vals_out[dst] = vals_in ? S.vin[S.src[s]] : (uint32_t)(base + S.src[s]);
      if (ranges) {
        // last pass of a tile sort: the block's keys are fully sorted, so a
        // tile's entries here form one run; record its ends
        if (s == 0 || S.keys[s - 1] != key) atomicMin(&ranges[key].x, dst);
        if (s == n_in - 1 || S.keys[s + 1] != key) atomicMin(&ranges[key].y, ~(dst + 1u));
      }
    }
  }
  }  // partitions
}

// Ranges were accumulated as (min start, ~max end) from 0xFFFFFFFF; empty
// tiles become [0, 0).
__global__ void __launch_bounds__(256) ranges_fixup_kernel(uint2* ranges, int total_tiles) {
  chain_enter();
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= total_tiles) return;
  uint2 r = ranges[t];
  ranges[t] = (r.x == 0xFFFFFFFFu) ? make_uint2(0u, 0u) : make_uint2(r.x, ~r.y);
}

inline size_t al256(size_t b) { return (b + 255) & ~(size_t)255; }

}  // namespace

size_t sort_scratch_bytes(int64_t cap, int passes, int items) {
  const int64_t part = (int64_t)OS_THREADS * items;
  int64_t parts = cap > 0 ? (cap + part - 1) / part : 1;
  return al256((size_t)passes * RADIX * 4) + al256((size_t)passes * 4) +
         al256((size_t)passes * parts * RADIX * 8);
}

SortScratch sort_scratch_carve(void* base, int64_t cap, int passes, int items) {
  SortScratch s;
  const int64_t part = (int64_t)OS_THREADS * items;
  s.items = items;
  s.parts = cap > 0 ? (cap + part - 1) / part : 1;
  char* p = static_cast<char*>(base);
  s.hist = reinterpret_cast<uint32_t*>(p);
  p += al256((size_t)passes * RADIX * 4);
  s.part_ctr = reinterpret_cast<uint32_t*>(p);
  p += al256((size_t)passes * 4);
  s.lookback = reinterpret_cast<uint64_t*>(p);
  return s;
}

cudaError_t launch_radix_hist(const uint32_t* keys, const int64_t* n_dev, int64_t n_host, int begin_bit,
                              int passes, uint32_t* hist, cudaStream_t st) {
  int sms = 0;
  cudaError_t e = current_sm_count(&sms);
  if (e != cudaSuccess) return e;
  const int blocks = 4 * sms;
  return launch_chain(radix_hist_kernel, dim3(blocks), dim3(256), 0, st, keys, n_dev, n_host, begin_bit, passes, hist);
}

cudaError_t launch_radix_scan(uint32_t* hist, int passes, cudaStream_t st) {
  return launch_chain(radix_scan_kernel, dim3(passes), dim3(RADIX), 0, st, hist);
}

template <int BITS, int ITEMS>
static cudaError_t onesweep_launch(const uint32_t* keys_in, const uint32_t* vals_in, uint32_t* keys_out,
                                   uint32_t* vals_out, const int64_t* n_dev, int64_t n_host, int64_t cap, int shift,
                                   int pass, const SortScratch& s, int32_t* ranges, int32_t* status, cudaStream_t st) {
  // the dynamic shared memory limit is a per-device attribute of the kernel
  static bool attr_set[64] = {false};
  constexpr int PART = OS_THREADS * ITEMS;
  const size_t sm = sizeof(OnesweepSmem<PART>);
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64 || !attr_set[dev]) {
    e = cudaFuncSetAttribute(onesweep_kernel<BITS, ITEMS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev < 64) attr_set[dev] = true;
  }
  // persistent grid: as many blocks as fit at once (OS_CTAS_PER_SM per SM), or fewer
  // when the capacity needs fewer partitions
  int sms = 0;
  e = current_sm_count(&sms);
  if (e != cudaSuccess) return e;
  const int64_t parts = (cap > 0 ? cap + PART - 1 : PART) / PART;
  const int64_t resident = (int64_t)sms * OS_CTAS_PER_SM;
  const unsigned grid = (unsigned)(parts < resident ? parts : resident);
  return launch_chain(onesweep_kernel<BITS, ITEMS>, dim3(grid), dim3(OS_THREADS), sm, st, keys_in, vals_in, keys_out,
                      vals_out, n_dev, n_host, shift, (const uint32_t*)(s.hist + (size_t)pass * RADIX),
                      s.lookback + (size_t)pass * s.parts * RADIX, s.part_ctr + pass,
                      reinterpret_cast<uint2*>(ranges), status, g_spin_limit, ranges ? g_hold_part : -1);
}

cudaError_t launch_onesweep_pass(const uint32_t* keys_in, const uint32_t* vals_in, uint32_t* keys_out,
                                 uint32_t* vals_out, const int64_t* n_dev, int64_t n_host, int64_t cap, int shift,
                                 int bits, int pass, const SortScratch& s, int32_t* ranges, int32_t* status,
                                 cudaStream_t st) {
#define LS_OS(B, I)                                                                                        \
  onesweep_launch<B, I>(keys_in, vals_in, keys_out, vals_out, n_dev, n_host, cap, shift, pass, s, ranges, status, \
                        st)
  switch (bits) {
    case 4: return LS_OS(4, SORT_ITEMS);
    case 5: return LS_OS(5, SORT_ITEMS);
    case 6: return LS_OS(6, SORT_ITEMS);
    case 7: return LS_OS(7, SORT_ITEMS);
    default: return LS_OS(8, SORT_ITEMS);
  }
#undef LS_OS
}

void set_sort_wait(int spin_limit, int hold_part) {
  g_spin_limit = spin_limit > 0 ? spin_limit : SPIN_LIMIT_DEFAULT;
  g_hold_part = hold_part;
}

cudaError_t launch_ranges_fixup(int32_t* ranges, int total_tiles, cudaStream_t st) {
  return launch_chain(ranges_fixup_kernel, dim3(ceil_div(total_tiles, 256)), dim3(256), 0, st,
                      reinterpret_cast<uint2*>(ranges), total_tiles);
}

}  // namespace ls
