// Host-side launchers of the sm_103a kernels (internal to libls.so).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace ls {

// Multiprocessor count of the current device, read once per device.
inline cudaError_t current_sm_count(int* out) {
  static int cache[64] = {0};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  if (cache[dev] == 0) {
    e = cudaDeviceGetAttribute(&cache[dev], cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
  }
  *out = cache[dev];
  return cudaSuccess;
}

// Launch of a kernel of the frame's chain (every kernel launched this way
// starts with chain_enter()): with programmatic stream serialisation when it
// is on (the default; ls_set_dependent_launch) and the stream is not being
// captured into a CUDA graph, else a plain launch.  On the 3M-primitive
// 1080p frame the attribute took 0.8 % off the frame launched call by call
// but added 1.5 % to the same frame replayed from a graph.
bool chain_launch_on();
void set_chain_launch(bool on);
inline bool chain_attr_for(cudaStream_t st) {
  if (!chain_launch_on()) return false;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) {
    (void)cudaGetLastError();  // the query's own error is not a launch error
    return false;
  }
  return cs == cudaStreamCaptureStatusNone;
}
template <typename... KArgs, typename... Args>
inline cudaError_t launch_chain(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                                Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = chain_attr_for(st) ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

// Total tiles of a camera set under the host-side rules of the ABI (valid
// parameters, camera sizes up to 16384, at most 2^24 tiles); false when a
// rule is broken.
bool host_total_tiles(const ls_camera* cams, int n_cams, const ls_params* p, int64_t* total_tiles);

// Bounded waits of the onesweep look-back (ls_debug_set_sort_wait).
void set_sort_wait(int spin_limit, int hold_part);

// ---- projection (project.cu)
cudaError_t launch_project_fwd(int n, const float* means, const float* scales, const float* quats,
                               const float* opac, const float* sh, const CamTable& cams, const ParDev& P,
                               ProjPtr out, int32_t* tile_counts, cudaStream_t st);
cudaError_t launch_project_bwd(int n, const float* means, const float* scales, const float* quats,
                               const float* opac, const float* sh, const CamTable& cams, const ParDev& P,
                               ProjCPtr proj, const float* g2d, float* g_means, float* g_scales, float* g_quats,
                               float* g_opac, float* g_sh, cudaStream_t st);

// ---- onesweep radix sort (sort.cu)
// Threads of a onesweep CTA: two CTAs of 512 per SM (0.599 ms for the
// duplicate + sort stage of the 3M-primitive 1080p frame, against 0.605 for
// four of 256 and 0.657 for one of 1024).
constexpr int SORT_THREADS = 512;
// Keys per thread of a partition: 9216-key partitions take 110 KB of shared
// memory, so two CTAs still fit an SM.  With 256-thread CTAs, 8, 11, 13,
// 15, 16 and 17 were slower on the bench frame (more partitions to look back
// over), 19 and 24 too (three CTAs per SM).
constexpr int SORT_ITEMS = 18;
constexpr int SORT_PART = SORT_THREADS * SORT_ITEMS;  // keys per partition
constexpr int RADIX = 256;

// Scratch of one sort of up to `cap` keys over `passes` 8-bit digits.
struct SortScratch {
  uint32_t* hist;      // [passes][RADIX] digit counts, scanned in place
  uint32_t* part_ctr;  // [passes] partition tickets
  uint64_t* lookback;  // [passes][parts][RADIX]
  int64_t parts;
  int items;           // keys per thread of a partition
};
size_t sort_scratch_bytes(int64_t cap, int passes, int items = SORT_ITEMS);
SortScratch sort_scratch_carve(void* base, int64_t cap, int passes, int items = SORT_ITEMS);

// Digit histograms of all passes in one read (skipped when the caller has
// filled `hist` itself); then the exclusive scans.
cudaError_t launch_radix_hist(const uint32_t* keys, const int64_t* n_dev, int64_t n_host, int begin_bit,
                              int passes, uint32_t* hist, cudaStream_t st);
cudaError_t launch_radix_scan(uint32_t* hist, int passes, cudaStream_t st);
// One onesweep pass over digit (key >> shift) & (2^bits - 1), bits in 4..8,
// using the scratch of pass index `pass`.
// vals_in == nullptr means the identity values 0..n-1.  n is read from
// n_dev when not null, else n_host; the grid covers `cap` keys.
// ranges != nullptr on the last pass of a tile sort: the pass also records
// each tile's [start, end) (prefilled with 0xFF bytes, finished by
// launch_ranges_fixup).
cudaError_t launch_onesweep_pass(const uint32_t* keys_in, const uint32_t* vals_in, uint32_t* keys_out,
                                 uint32_t* vals_out, const int64_t* n_dev, int64_t n_host, int64_t cap, int shift,
                                 int bits, int pass, const SortScratch& s, int32_t* ranges, int32_t* status,
                                 cudaStream_t st);
// Digits of a tile sort: the bits of the largest tile id split evenly over
// ceil(bits / 8) passes (the earlier passes take the remainder).
struct TileDigits {
  int passes;
  int shift[3], bits[3];
};
inline TileDigits tile_digits(int64_t total_tiles) {
  int nb = 1;
  while ((1ll << nb) < total_tiles) ++nb;
  TileDigits d{};
  d.passes = (nb + 7) / 8;
  int at = 0;
  for (int p = 0; p < d.passes; ++p) {
    const int b = (nb - at + (d.passes - p) - 1) / (d.passes - p);
    d.shift[p] = at;
    d.bits[p] = b < 4 ? 4 : b;
    at += b;
  }
  return d;
}
cudaError_t launch_ranges_fixup(int32_t* ranges, int total_tiles, cudaStream_t st);

// ---- duplication and tile ranges (duplicate.cu)
constexpr int DUP_THREADS = 256;
cudaError_t launch_dup_count(int64_t R, const uint32_t* order, const uint32_t* dkey_sorted, const float4* foot,
                             const CamTable& cams, int n_per_cam, const ParDev& P, uint2* rect_sorted, cudaStream_t st);
// Exclusive scan of n = enum_warps(R) counts in place (the buffer holds
// enum_count_words(R) words); *n_keys_dev = total, *n_valid_dev = total when
// it fits cap (else 0, and LS_ERR_CAPACITY in *status).
cudaError_t launch_dup_scan(int64_t n, uint32_t* counts, int64_t cap, int64_t* n_keys_dev, int64_t* n_valid_dev,
                            int32_t* status, cudaStream_t st);

// Key enumeration (duplicate.cu): which keys of the depth-ordered records'
// support boxes are taken.
enum { ENUM_ALL = 0, ENUM_KEPT = 1, ENUM_HELD = 2 };
// Max pyramid of the per-tile proposal depth bits: level 0 is the tiles,
// each next level the max over 2 x 2 cells of the one below (ceil halves), up
// to one cell; levels are stored one after another in one array.
constexpr int PYR_MAX = 24;
struct DstarPyramid {
  int levels;
  int w[PYR_MAX], h[PYR_MAX];
  int off[PYR_MAX];  // first word of each level
};
inline DstarPyramid make_dstar_pyramid(int tiles_x, int tiles_y) {
  DstarPyramid d{};
  int w = tiles_x, h = tiles_y, off = 0, k = 0;
  for (;;) {
    d.w[k] = w, d.h[k] = h, d.off[k] = off;
    off += w * h;
    ++k;
    if ((w == 1 && h == 1) || k == PYR_MAX) break;
    w = (w + 1) / 2, h = (h + 1) / 2;
  }
  d.levels = k;
  return d;
}
inline int64_t dstar_pyramid_words(int tiles_x, int tiles_y) {
  const DstarPyramid d = make_dstar_pyramid(tiles_x, tiles_y);
  return (int64_t)d.off[d.levels - 1] + (int64_t)d.w[d.levels - 1] * d.h[d.levels - 1];
}

struct EnumArgs {
  int64_t R;                      // records in depth order
  const uint32_t* order;          // [R] record id at each depth rank
  const uint32_t* dkey_sorted;    // [R] depth bits (ENUM_KEPT, ENUM_HELD)
  const uint2* rect_sorted;       // [R] packed tile box, empty when x1 < x0
  const float4* rec;              // [R][3] projected records (ellipse of each)
  CamTable cams;                  // tile_base / tiles_x of each camera
  int n_per_cam;
  int tile_w, tile_h;
  const uint32_t* dstar_bits;     // [tiles] proposal depth bits (ENUM_KEPT, ENUM_HELD)
  const uint8_t* refuted;         // [tiles] (ENUM_HELD)
  const int* sat;                 // summed-area table of refuted (ENUM_HELD)
  const unsigned* n_refuted;      // (ENUM_HELD)
  const unsigned* refuted_floor;  // (ENUM_HELD) ~(smallest proposal bits of a refuted tile)
  uint32_t* warp_counts;          // [n_warps] taken keys per warp, then scanned offsets
  uint32_t* warp_tbase;           // [n_warps] stash offset of each warp's keys (0xFFFFFFFF: none)
  int64_t n_warps;                // enum_warps(R)
  uint32_t *tmp_keys, *tmp_vals;  // stash of the count launch, tmp_cap entries
  int64_t tmp_cap;
  unsigned long long* tmp_ctr;    // stash bump allocator, zeroed before the count launch
  const int64_t* n_valid;         // total that fits the capacity (emit)
  uint64_t out_base;              // emit: first output position
  uint32_t *keys, *vals;          // emit outputs
  int key_passes;
  int dshift[3];                  // digit p of a key: (key >> dshift[p]) & dmask[p]
  uint32_t dmask[3];
  uint32_t* tile_hist;            // [key_passes][RADIX] digit counts (emit)
  unsigned long long* key_total;  // ENUM_KEPT count launch: all keys reached
  const uint32_t* dstar_pyr;      // ENUM_KEPT: max pyramid of dstar_bits (level 0 is dstar_bits itself)
  DstarPyramid pyr;
};
int64_t enum_warps(int64_t R);
// 32-bit words of a warp-count buffer for R records: the counts, then the
// chunk sums of their scan.
int64_t enum_count_words(int64_t R);
cudaError_t launch_enum_keys(bool emit, int mode, const EnumArgs& A, cudaStream_t st);

// ---- blending (blend.cu)
// Pixel offset of each camera's image in a batched render's packed output.
struct BatchPix {
  size_t base[LS_MAX_CAMS];
};
cudaError_t launch_build_queue(const int32_t* ranges, int total_tiles, uint32_t* queue, unsigned* job_ctr,
                               cudaStream_t st);
cudaError_t launch_blend_batch(const float4* rec, const uint32_t* vals, const int32_t* ranges, const CamTable& cams,
                              const BatchPix& pix, const ParDev& P, const uint32_t* queue, int n_jobs,
                              unsigned* job_ctr, float* images, float* t_final, int batch, cudaStream_t st);
// Extra inputs/outputs of the truncated, resumed and labelled forwards.
struct TruncArgs {
  float t_thr;                // a pixel with T < t_thr counts as settled
  const uint8_t* has_held;    // [tiles] set when the tile has keys beyond its proposal
  uint8_t* refuted;           // [tiles] set for refuted tiles
  unsigned* n_refuted;
  const uint32_t* dstar_bits;  // [tiles] proposal bits
  unsigned* refuted_floor;     // ~(smallest proposal bits of a refuted tile); zero before the pass
  const int2* kept_ranges;    // resume: the kept list of each tile
  float* labels;              // counting forward: per-tile termination depth
};
// labels != nullptr (with stats) also writes each tile's termination depth.
cudaError_t launch_blend_fwd(const float4* rec, const CamDev& cam, const ParDev& P, const int2* ranges,
                             const uint32_t* vals, float* image, float* t_final, int32_t* n_last,
                             unsigned long long* stats, cudaStream_t st, float* labels = nullptr);
// mode 1: truncated forward over the kept lists; mode 2: resume of refuted tiles
// over their held-out lists (ranges = held-out ranges).
cudaError_t launch_blend_trunc(int mode, const float4* rec, const CamDev& cam, const ParDev& P, const int2* ranges,
                               const uint32_t* vals, float* image, float* t_final, int32_t* n_last,
                               const TruncArgs& ta, cudaStream_t st);
// order != nullptr: CTA b blends tile order[b] (a permutation of the
// camera's tiles, from launch_tile_order); else tile b.
cudaError_t launch_blend_bwd(const float4* rec, const CamDev& cam, const ParDev& P, const int2* ranges,
                             const uint32_t* vals, const float* t_final, const int32_t* n_last,
                             const float* grad_image, const float* grad_t, float* g2d, cudaStream_t st,
                             const uint32_t* order = nullptr);
// Longest-first order of a camera's tiles for the backward blend: each
// tile's work is the largest n_last over its pixels, bucketed by
// quarter-octaves (TILE_ORDER_BUCKETS counts in `hist`, zero before the
// call; `bkt` holds each tile's bucket), and `order` lists the tiles from
// the heaviest bucket down.
constexpr int TILE_ORDER_BUCKETS = 132;
cudaError_t launch_tile_order(const int32_t* n_last, const CamDev& cam, const ParDev& P, unsigned* hist,
                              uint32_t* bkt, uint32_t* order, cudaStream_t st);

// ---- learned termination (learned.cu)
struct DepthBins {
  float edge[31];  // binary32 lower edges of bins 1..31 of log depth
};
DepthBins make_depth_bins();
// Scratch planes of the per-tile histograms (32 float coverage planes and one
// int count plane of (tiles_x + 1) x (tiles_y + 1)), zeroed by the caller.
size_t hist_planes_bytes(const CamDev& cam);
// counts = false leaves out the plane of box counts (no tile totals wanted).
cudaError_t launch_tile_hist(int64_t R, const float4* rec, const float4* foot, const uint32_t* dkey,
                             const CamDev& cam, const ParDev& P, void* planes, bool counts, cudaStream_t st);
// The coverage planes only (no count plane) from the depth order: order,
// sorted depth keys and the support boxes of dup_count (rect_sorted).  The
// shared plane of tile_hist_sorted_smem(cam) bytes must fit one block.
size_t tile_hist_sorted_smem(const CamDev& cam);
cudaError_t launch_tile_hist_sorted(int64_t R, const uint32_t* order, const uint32_t* dkey_sorted,
                                    const uint2* rect_sorted, const float4* rec, const CamDev& cam, const ParDev& P,
                                    void* planes, cudaStream_t st);
cudaError_t launch_features(void* planes, const CamDev& cam, const ParDev& P, void* x, int32_t* tile_total,
                            unsigned long long* key_total, cudaStream_t st);
// Proposal bits per tile (level 0 of the pyramid `pyr`, then its upper
// levels) and has_held: whether any record of a depth bin that can lie beyond
// the proposal has a support box covering the tile (from the prefixed
// coverage planes, where every such record adds at least one unit): a
// superset of the tiles with keys beyond their proposal.
cudaError_t launch_dstar(const CamDev& cam, const float* y, float margin, const float* dstar_in, uint32_t* pyr,
                         float* dstar_out, const void* planes, uint8_t* has_held, cudaStream_t st);
// Summed-area table of the refuted flags, (tiles_x + 1) x (tiles_y + 1) ints.
cudaError_t launch_refuted_sat(const uint8_t* refuted, const unsigned* n_refuted, int tiles_x, int tiles_y, int* sat,
                               cudaStream_t st);
cudaError_t launch_learned_stats(const unsigned long long* key_total, const int64_t* n_kept, const int64_t* n_held,
                                 const unsigned* n_refuted, int64_t* stats, cudaStream_t st);

// ---- training-side consumers of the backward (train.cu)
size_t image_loss_ws_bytes(int H, int W);
// loss_out[4] = total, L1, L2, SSIM; grad (nullable) = dL/dpred [H][W][3]
cudaError_t launch_image_loss(int H, int W, const float* pred, const float* target, float w1, float w2, float w3,
                              float* loss_out, float* grad, void* ws, cudaStream_t st);
cudaError_t launch_adam(int64_t n, float* p, const float* g, float* m, float* v, int step, float lr, float b1,
                        float b2, float eps, int mode, cudaStream_t st);
cudaError_t launch_densify_accum(int n, const float* g2d, const float4* foot, const uint32_t* dkey, int W, int H,
                                 int n_cams, float* accum, int32_t* count, float* max_radius, cudaStream_t st);
cudaError_t launch_densify_decide(int n, const float* accum, const int32_t* count, const float* max_radius,
                                  const float* scales, const float* opac, float extent, const ls_densify_params& p,
                                  uint8_t* flags, int64_t* counts, cudaStream_t st);

// ---- 3D smoothing filter of the anti-aliased variant (filter3d.cu)
cudaError_t launch_filter3d_variance(int n, const float* means, const CamTable& cams, float near_plane, float s2,
                                     float* var, unsigned* max_bits, cudaStream_t st);
cudaError_t launch_filter3d_apply(int n, const float* scales, const float* opac, const float* var, float* s_out,
                                  float* o_out, cudaStream_t st);
cudaError_t launch_filter3d_apply_bwd(int n, const float* scales, const float* opac, const float* var,
                                      const float* g_se, const float* g_oe, float* g_s, float* g_o, cudaStream_t st);

// ---- termination MLP (mlp.cu)
struct MlpDev {
  const void* w1t;
  const float* b1;
  const void* w2t;
  const float* b2;
  const void* w3;
  const float* b3;
};
struct MlpMut {
  void* w1t;
  float* b1;
  void* w2t;
  float* b2;
  void* w3;
  float* b3;
};
cudaError_t launch_mlp_forward(int64_t m, const void* x, const MlpDev& net, float* y, cudaStream_t st);
cudaError_t launch_mlp_backward(int64_t m, const void* x, const MlpDev& net, const float* target, float under_weight,
                                float* grad, float* loss, cudaStream_t st);
cudaError_t launch_mlp_adam(int step, float lr, float beta1, float beta2, float eps, float* master, const float* grad,
                            float* m1, float* m2, const MlpMut& net, cudaStream_t st);

}  // namespace ls
