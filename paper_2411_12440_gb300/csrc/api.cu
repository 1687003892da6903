// C ABI of libls.so (declared in include/ls.h): argument checks, camera and
// parameter tables, workspace layout, and the launch sequence of each stage.
#include <cmath>
#include <cstring>

#include "kernels.h"

using namespace ls;

namespace {

inline size_t al256(size_t b) { return (b + 255) & ~(size_t)255; }

bool tile_ok(int tw, int th) { return (tw == 8 && th == 8) || (tw == 16 && th == 16) || (tw == 32 && th == 16); }

bool params_ok(const ls_params* p) {
  if (!p) return false;
  if (!(p->lambda > 0.f) || p->kernel < 0 || p->kernel > 4 || p->ags < 0 || p->ags > 2) return false;
  if (!(p->eps2d >= 0.f) || !(p->alpha_min >= 0.f) || !(p->alpha_max > 0.f && p->alpha_max < 1.f)) return false;
  if (!(p->t_min >= 0.f) || !tile_ok(p->tile_w, p->tile_h)) return false;
  if (p->sh_degree < 0 || p->sh_degree > 3) return false;
  if (!(p->near_plane > 0.f && p->far_plane > p->near_plane)) return false;
  return true;
}

bool cam_ok(const ls_camera& c) {
  if (c.width <= 0 || c.height <= 0 || c.width > 16384 || c.height > 16384) return false;
  if (!(c.fx > 0.f) || !(c.fy > 0.f)) return false;
  for (int i = 0; i < 16; ++i)
    if (!std::isfinite(c.viewmat[i])) return false;
  return true;
}

ParDev make_par(const ls_params* p) {
  ParDev P;
  P.lambda = p->lambda;
  P.inv_lambda = 1.f / p->lambda;
  P.kernel = p->kernel;
  P.ags = p->ags;
  P.antialias = p->antialias;
  P.eps2d = p->eps2d;
  P.alpha_min = p->alpha_min;
  P.alpha_max = p->alpha_max;
  P.t_min = p->t_min;
  P.tile_w = p->tile_w;
  P.tile_h = p->tile_h;
  for (int i = 0; i < 3; ++i) P.bg[i] = p->bg[i];
  P.near_plane = p->near_plane;
  P.far_plane = p->far_plane;
  P.sh_degree = p->sh_degree;
  return P;
}

// Returns false on a bad camera.  Tile ids are global: camera c's tiles start
// after those of cameras 0..c-1.
bool make_cams(const ls_camera* cams, int n_cams, const ls_params* p, CamTable& T, int64_t* total_tiles) {
  if (!cams || n_cams < 1 || n_cams > LS_MAX_CAMS) return false;
  std::memset(&T, 0, sizeof(T));
  T.n = n_cams;
  int64_t base = 0;
  for (int c = 0; c < n_cams; ++c) {
    const ls_camera& s = cams[c];
    if (!cam_ok(s)) return false;
    CamDev& d = T.c[c];
    for (int i = 0; i < 3; ++i) {
      for (int j = 0; j < 3; ++j) d.R[3 * i + j] = s.viewmat[4 * i + j];
      d.t[i] = s.viewmat[4 * i + 3];
    }
    for (int j = 0; j < 3; ++j) {
      double v = 0.0;
      for (int i = 0; i < 3; ++i) v -= (double)s.viewmat[4 * i + j] * (double)s.viewmat[4 * i + 3];
      d.campos[j] = (float)v;
    }
    d.fx = s.fx;
    d.fy = s.fy;
    d.cx = s.cx;
    d.cy = s.cy;
    d.W = s.width;
    d.H = s.height;
    d.lim_xl = (float)((s.cx + 0.15 * s.width) / s.fx);
    d.lim_xh = (float)((s.width - s.cx + 0.15 * s.width) / s.fx);
    d.lim_yl = (float)((s.cy + 0.15 * s.height) / s.fy);
    d.lim_yh = (float)((s.height - s.cy + 0.15 * s.height) / s.fy);
    d.tiles_x = (s.width + p->tile_w - 1) / p->tile_w;
    d.tiles_y = (s.height + p->tile_h - 1) / p->tile_h;
    d.tile_base = (int)base;
    base += (int64_t)d.tiles_x * d.tiles_y;
  }
  if (base > (1 << 24)) return false;
  if (total_tiles) *total_tiles = base;
  return true;
}

int key_passes_for(int64_t total_tiles) {
  int bits = 1;
  while ((1ll << bits) < total_tiles) ++bits;
  return (bits + 7) / 8;
}

ProjPtr proj_planes(void* proj, int64_t R) {
  char* b = static_cast<char*>(proj);
  return ProjPtr{reinterpret_cast<float4*>(b), reinterpret_cast<float4*>(b + 48 * (size_t)R),
                 reinterpret_cast<uint32_t*>(b + 64 * (size_t)R)};
}
ProjCPtr proj_cplanes(const void* proj, int64_t R) {
  const char* b = static_cast<const char*>(proj);
  return ProjCPtr{reinterpret_cast<const float4*>(b), reinterpret_cast<const float4*>(b + 48 * (size_t)R),
                  reinterpret_cast<const uint32_t*>(b + 64 * (size_t)R)};
}

// Workspace of ls_duplicate_sort, in carve order.
struct DupWs {
  uint32_t *dk_a, *dv_a, *dk_b, *dv_b;  // depth sort ping-pong [R]
  uint2* rect;                          // [R]
  uint32_t* warp_counts;                // [enum warps]
  uint32_t* warp_tbase;                 // [enum warps]
  int64_t* n_valid;
  unsigned long long* tmp_ctr;          // stash allocator (zeroed)
  uint32_t *k_alt, *v_alt;              // tile sort ping-pong [cap]
  void* depth_scratch;
  void* tile_scratch;
  size_t zero_begin, zero_bytes;        // byte range cleared before every call
  size_t total;
};

DupWs dup_layout(char* base, int64_t R, int64_t cap, int key_passes) {
  DupWs w;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    char* p = base + off;
    off += al256(bytes);
    return p;
  };
  const size_t Rz = (size_t)(R > 0 ? R : 1), Cz = (size_t)(cap > 0 ? cap : 1);
  w.dk_a = reinterpret_cast<uint32_t*>(take(4 * Rz));
  w.dv_a = reinterpret_cast<uint32_t*>(take(4 * Rz));
  w.dk_b = reinterpret_cast<uint32_t*>(take(4 * Rz));
  w.dv_b = reinterpret_cast<uint32_t*>(take(4 * Rz));
  w.rect = reinterpret_cast<uint2*>(take(8 * Rz));
  w.warp_counts = reinterpret_cast<uint32_t*>(take(4 * (size_t)enum_count_words((int64_t)Rz)));
  w.warp_tbase = reinterpret_cast<uint32_t*>(take(4 * (size_t)enum_warps((int64_t)Rz)));
  w.n_valid = reinterpret_cast<int64_t*>(take(8));
  w.k_alt = reinterpret_cast<uint32_t*>(take(4 * Cz));
  w.v_alt = reinterpret_cast<uint32_t*>(take(4 * Cz));
  w.zero_begin = off;
  w.tmp_ctr = reinterpret_cast<unsigned long long*>(take(8));
  w.depth_scratch = take(sort_scratch_bytes((int64_t)Rz, 4));
  w.tile_scratch = take(sort_scratch_bytes((int64_t)Cz, key_passes));
  w.zero_bytes = off - w.zero_begin;
  w.total = off;
  return w;
}

#define LS_TRY(expr)                          \
  do {                                        \
    if ((expr) != cudaSuccess) return LS_ERR_CUDA; \
  } while (0)

}  // namespace

namespace {
bool g_chain_launch = true;
}
bool ls::chain_launch_on() { return g_chain_launch; }
void ls::set_chain_launch(bool on) { g_chain_launch = on; }

bool ls::host_total_tiles(const ls_camera* cams, int n_cams, const ls_params* p, int64_t* total_tiles) {
  if (!params_ok(p)) return false;
  CamTable T;
  return make_cams(cams, n_cams, p, T, total_tiles);
}

extern "C" {

int32_t ls_version(void) { return 1; }

ls_status ls_debug_set_sort_wait(int32_t spin_limit, int32_t hold_partition) {
  if (spin_limit < 0 || hold_partition < -1) return LS_ERR_INVALID_ARG;
  set_sort_wait(spin_limit, hold_partition);
  return LS_OK;
}

ls_status ls_set_dependent_launch(int32_t on) {
  if (on != 0 && on != 1) return LS_ERR_INVALID_ARG;
  set_chain_launch(on == 1);
  return LS_OK;
}

const char* ls_status_string(int32_t s) {
  switch (s) {
    case LS_OK: return "ok";
    case LS_ERR_INVALID_ARG: return "invalid argument";
    case LS_ERR_CUDA: return "CUDA launch error";
    case LS_ERR_CAPACITY: return "tile-key capacity exceeded";
    case LS_ERR_TIMEOUT: return "device-side wait timed out";
    case LS_ERR_UNSUPPORTED: return "unsupported configuration";
    default: return "unknown status";
  }
}

size_t ls_proj_bytes(int64_t n_records) { return n_records > 0 ? (size_t)n_records * 68 : 0; }

ls_status ls_project(int32_t n, const float* means, const float* scales, const float* quats,
                     const float* opacities, const float* sh, const ls_camera* cams, int32_t n_cams,
                     const ls_params* params, void* proj, int32_t* tile_counts, int32_t* status_dev,
                     void* stream) {
  if (n < 0 || !params_ok(params)) return LS_ERR_INVALID_ARG;
  CamTable T;
  if (!make_cams(cams, n_cams, params, T, nullptr)) return LS_ERR_INVALID_ARG;
  if ((int64_t)n * n_cams > 0x7FFFFFFFll) return LS_ERR_INVALID_ARG;
  if (n == 0) return LS_OK;
  if (!means || !scales || !quats || !opacities || !sh || !proj) return LS_ERR_INVALID_ARG;
  if (reinterpret_cast<uintptr_t>(quats) % 16 || reinterpret_cast<uintptr_t>(proj) % 16) return LS_ERR_INVALID_ARG;
  ParDev P = make_par(params);
  LS_TRY(launch_project_fwd(n, means, scales, quats, opacities, sh, T, P, proj_planes(proj, (int64_t)n * n_cams),
                            tile_counts, static_cast<cudaStream_t>(stream)));
  return LS_OK;
}

size_t ls_duplicate_sort_workspace(int64_t n_records, int64_t key_capacity, int32_t total_tiles) {
  if (n_records < 0 || key_capacity < 0 || total_tiles < 1) return 0;
  return dup_layout(nullptr, n_records, key_capacity, key_passes_for(total_tiles)).total;
}

ls_status ls_duplicate_sort(int64_t n_records, const void* proj, const ls_camera* cams, int32_t n_cams,
                            const ls_params* params, int64_t key_capacity, uint32_t* keys, uint32_t* vals,
                            int64_t* n_keys_dev, int32_t* tile_ranges, void* workspace, size_t ws_bytes,
                            int32_t* status_dev, void* stream) {
  if (n_records < 0 || !params_ok(params)) return LS_ERR_INVALID_ARG;
  if (key_capacity < 0 || key_capacity > 0x7FFFFFFFll || n_records > 0xFFFFFFFFll) return LS_ERR_INVALID_ARG;
  CamTable T;
  int64_t total_tiles = 0;
  if (!make_cams(cams, n_cams, params, T, &total_tiles)) return LS_ERR_INVALID_ARG;
  if (n_records % n_cams) return LS_ERR_INVALID_ARG;
  if (!n_keys_dev || !tile_ranges || !workspace) return LS_ERR_INVALID_ARG;
  if (key_capacity > 0 && (!keys || !vals)) return LS_ERR_INVALID_ARG;
  if (n_records > 0 && !proj) return LS_ERR_INVALID_ARG;
  if (reinterpret_cast<uintptr_t>(workspace) % 256) return LS_ERR_INVALID_ARG;
  const int kp = key_passes_for(total_tiles);
  const TileDigits td = tile_digits(total_tiles);
  DupWs w = dup_layout(static_cast<char*>(workspace), n_records, key_capacity, kp);
  if (ws_bytes < w.total) return LS_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const ParDev P = make_par(params);
  const int64_t R = n_records;
  const int n_per_cam = (int)(R / n_cams);
  ProjCPtr pp = proj_cplanes(proj, R);

  LS_TRY(cudaMemsetAsync(static_cast<char*>(workspace) + w.zero_begin, 0, w.zero_bytes, st));
  // depth sort of the records: key = binary32 depth bits (0xFFFFFFFF when
  // culled), value = record id; four 8-bit passes, the last lands in (dk_a, dv_a)
  SortScratch ds = sort_scratch_carve(w.depth_scratch, R > 0 ? R : 1, 4);
  if (R > 0) {
    LS_TRY(launch_radix_hist(pp.dkey, nullptr, R, 0, 4, ds.hist, st));
    LS_TRY(launch_radix_scan(ds.hist, 4, st));
    LS_TRY(launch_onesweep_pass(pp.dkey, nullptr, w.dk_b, w.dv_b, nullptr, R, R, 0, 8, 0, ds, nullptr, status_dev, st));
    LS_TRY(launch_onesweep_pass(w.dk_b, w.dv_b, w.dk_a, w.dv_a, nullptr, R, R, 8, 8, 1, ds, nullptr, status_dev, st));
    LS_TRY(launch_onesweep_pass(w.dk_a, w.dv_a, w.dk_b, w.dv_b, nullptr, R, R, 16, 8, 2, ds, nullptr, status_dev, st));
    LS_TRY(launch_onesweep_pass(w.dk_b, w.dv_b, w.dk_a, w.dv_a, nullptr, R, R, 24, 8, 3, ds, nullptr, status_dev, st));
    LS_TRY(launch_dup_count(R, w.dv_a, w.dk_a, pp.foot, T, n_per_cam, P, w.rect, st));
  }
  // keys of the tiles each support ellipse reaches: count per warp (and
  // stash them), scan (total K and the capacity check), then write in depth
  // order.  Emission goes to the buffer that makes the last tile-sort pass
  // end in the caller's keys/vals; the stash is the other one.
  uint32_t* ek = (kp % 2 == 0) ? keys : w.k_alt;
  uint32_t* ev = (kp % 2 == 0) ? vals : w.v_alt;
  uint32_t* ok = (kp % 2 == 0) ? w.k_alt : keys;
  uint32_t* ov = (kp % 2 == 0) ? w.v_alt : vals;
  EnumArgs ea{};
  ea.R = R;
  ea.order = w.dv_a;
  ea.dkey_sorted = w.dk_a;
  ea.rect_sorted = w.rect;
  ea.rec = pp.rec;
  ea.cams = T;
  ea.n_per_cam = n_per_cam;
  ea.tile_w = P.tile_w;
  ea.tile_h = P.tile_h;
  ea.warp_counts = w.warp_counts;
  ea.warp_tbase = w.warp_tbase;
  ea.n_warps = enum_warps(R);
  ea.tmp_keys = ok;
  ea.tmp_vals = ov;
  ea.tmp_cap = (ok && ov) ? key_capacity : 0;
  ea.tmp_ctr = w.tmp_ctr;
  ea.n_valid = w.n_valid;
  ea.key_passes = kp;
  for (int p = 0; p < kp; ++p) {
    ea.dshift[p] = td.shift[p];
    ea.dmask[p] = (1u << td.bits[p]) - 1u;
  }
  SortScratch ts = sort_scratch_carve(w.tile_scratch, key_capacity > 0 ? key_capacity : 1, kp);
  ea.tile_hist = ts.hist;  // digits of the keys are counted where they are written
  LS_TRY(launch_enum_keys(false, ENUM_ALL, ea, st));
  LS_TRY(launch_dup_scan(enum_warps(R), w.warp_counts, key_capacity, n_keys_dev, w.n_valid, status_dev, st));
  // ranges: accumulated by the last tile pass as (min start, ~max end)
  LS_TRY(cudaMemsetAsync(tile_ranges, 0xFF, sizeof(int32_t) * 2 * (size_t)total_tiles, st));
  if (R > 0 && key_capacity > 0) {
    ea.keys = ek;
    ea.vals = ev;
    LS_TRY(launch_enum_keys(true, ENUM_ALL, ea, st));
    LS_TRY(launch_radix_scan(ts.hist, kp, st));
    for (int p = 0; p < kp; ++p) {
      LS_TRY(launch_onesweep_pass(ek, ev, ok, ov, w.n_valid, 0, key_capacity, td.shift[p], td.bits[p], p, ts,
                                  p == kp - 1 ? tile_ranges : nullptr, status_dev, st));
      std::swap(ek, ok);
      std::swap(ev, ov);
    }
  }
  LS_TRY(launch_ranges_fixup(tile_ranges, (int)total_tiles, st));
  return LS_OK;
}

ls_status ls_render_fwd(const void* proj, int64_t n_records, const ls_camera* cam, const ls_params* params,
                        const int32_t* tile_ranges, const uint32_t* vals, float* image, float* t_final,
                        int32_t* n_last, int32_t* status_dev, void* stream) {
  if (!params_ok(params) || n_records < 0) return LS_ERR_INVALID_ARG;
  CamTable T;
  if (!make_cams(cam, 1, params, T, nullptr)) return LS_ERR_INVALID_ARG;
  if (!tile_ranges || !image || !t_final || !n_last) return LS_ERR_INVALID_ARG;
  if (n_records > 0 && (!proj || !vals)) return LS_ERR_INVALID_ARG;
  (void)status_dev;
  ProjCPtr pp = proj_cplanes(proj, n_records);
  LS_TRY(launch_blend_fwd(pp.rec, T.c[0], make_par(params), reinterpret_cast<const int2*>(tile_ranges), vals, image,
                          t_final, n_last, nullptr, static_cast<cudaStream_t>(stream)));
  return LS_OK;
}

ls_status ls_render_stats(const void* proj, int64_t n_records, const ls_camera* cam, const ls_params* params,
                          const int32_t* tile_ranges, const uint32_t* vals, float* image, float* t_final,
                          int32_t* n_last, uint64_t* stats_dev, float* tile_labels, int32_t* status_dev,
                          void* stream) {
  if (!params_ok(params) || n_records < 0) return LS_ERR_INVALID_ARG;
  CamTable T;
  if (!make_cams(cam, 1, params, T, nullptr)) return LS_ERR_INVALID_ARG;
  if (!tile_ranges || !image || !t_final || !n_last || !stats_dev) return LS_ERR_INVALID_ARG;
  if (n_records > 0 && (!proj || !vals)) return LS_ERR_INVALID_ARG;
  (void)status_dev;
  ProjCPtr pp = proj_cplanes(proj, n_records);
  LS_TRY(launch_blend_fwd(pp.rec, T.c[0], make_par(params), reinterpret_cast<const int2*>(tile_ranges), vals, image,
                          t_final, n_last, reinterpret_cast<unsigned long long*>(stats_dev),
                          static_cast<cudaStream_t>(stream), tile_labels));
  return LS_OK;
}

}  // extern "C"

namespace {

// ls_blend_bwd with an optional tile order (CTA b blends tile order[b]).
ls_status blend_bwd_impl(const void* proj, int64_t n_records, const ls_camera* cam, const ls_params* params,
                         const int32_t* tile_ranges, const uint32_t* vals, const float* t_final,
                         const int32_t* n_last, const float* grad_image, const float* grad_t, float* g2d,
                         const uint32_t* order, cudaStream_t st) {
  if (!params_ok(params) || n_records < 0) return LS_ERR_INVALID_ARG;
  CamTable T;
  if (!make_cams(cam, 1, params, T, nullptr)) return LS_ERR_INVALID_ARG;
  if (!tile_ranges || !t_final || !n_last || !grad_image) return LS_ERR_INVALID_ARG;
  if (n_records > 0 && (!proj || !vals || !g2d)) return LS_ERR_INVALID_ARG;
  if (reinterpret_cast<uintptr_t>(g2d) % 16) return LS_ERR_INVALID_ARG;
  ProjCPtr pp = proj_cplanes(proj, n_records);
  LS_TRY(launch_blend_bwd(pp.rec, T.c[0], make_par(params), reinterpret_cast<const int2*>(tile_ranges), vals,
                          t_final, n_last, grad_image, grad_t, g2d, st, order));
  return LS_OK;
}

// Tiles of a valid single camera, else 0.
int64_t cam_tiles(const ls_camera* cam, const ls_params* params, CamTable* out = nullptr) {
  if (!params_ok(params)) return 0;
  CamTable T;
  if (!make_cams(cam, 1, params, T, nullptr)) return 0;
  if (out) *out = T;
  return (int64_t)T.c[0].tiles_x * T.c[0].tiles_y;
}

// Scratch of a tile order: bucket counts, then each tile's bucket.
size_t order_scratch_bytes(int64_t tiles) { return al256(4 * (size_t)TILE_ORDER_BUCKETS) + al256(4 * (size_t)tiles); }

// The longest-first order of the camera's tiles into `order` (launch_tile_order);
// `scratch` holds order_scratch_bytes, its bucket counts already zero.
ls_status tile_order_impl(const int32_t* n_last, const ls_camera* cam, const ls_params* params, uint32_t* order,
                          char* scratch, cudaStream_t st) {
  CamTable T;
  const int64_t tiles = cam_tiles(cam, params, &T);
  if (tiles == 0 || !n_last || !order || !scratch) return LS_ERR_INVALID_ARG;
  unsigned* hist = reinterpret_cast<unsigned*>(scratch);
  uint32_t* bkt = reinterpret_cast<uint32_t*>(scratch + al256(4 * (size_t)TILE_ORDER_BUCKETS));
  LS_TRY(launch_tile_order(n_last, T.c[0], make_par(params), hist, bkt, order, st));
  return LS_OK;
}

// Bytes of the tile-order part of an ordered backward workspace (scratch and
// the order; 0 when the camera or the parameters are invalid).
size_t order_ws_bytes(const ls_camera* cam, const ls_params* params) {
  const int64_t tiles = cam_tiles(cam, params);
  return tiles == 0 ? 0 : order_scratch_bytes(tiles) + al256(4 * (size_t)tiles);
}

}  // namespace

extern "C" {

ls_status ls_blend_bwd(const void* proj, int64_t n_records, const ls_camera* cam, const ls_params* params,
                       const int32_t* tile_ranges, const uint32_t* vals, const float* t_final,
                       const int32_t* n_last, const float* grad_image, const float* grad_t, float* g2d,
                       int32_t* status_dev, void* stream) {
  (void)status_dev;
  return blend_bwd_impl(proj, n_records, cam, params, tile_ranges, vals, t_final, n_last, grad_image, grad_t, g2d,
                        nullptr, static_cast<cudaStream_t>(stream));
}

size_t ls_tile_order_workspace(const ls_camera* cam, const ls_params* params) {
  const int64_t tiles = cam_tiles(cam, params);
  return tiles == 0 ? 0 : order_scratch_bytes(tiles);
}

ls_status ls_tile_order(const int32_t* n_last, const ls_camera* cam, const ls_params* params, uint32_t* tile_order,
                        void* workspace, size_t ws_bytes, void* stream) {
  const size_t need = ls_tile_order_workspace(cam, params);
  if (need == 0 || !workspace || ws_bytes < need || reinterpret_cast<uintptr_t>(workspace) % 256)
    return LS_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  LS_TRY(cudaMemsetAsync(workspace, 0, 4 * (size_t)TILE_ORDER_BUCKETS, st));
  return tile_order_impl(n_last, cam, params, tile_order, static_cast<char*>(workspace), st);
}

ls_status ls_blend_bwd_ordered(const void* proj, int64_t n_records, const ls_camera* cam, const ls_params* params,
                               const int32_t* tile_ranges, const uint32_t* tile_order, const uint32_t* vals,
                               const float* t_final, const int32_t* n_last, const float* grad_image,
                               const float* grad_t, float* g2d, int32_t* status_dev, void* stream) {
  (void)status_dev;
  if (!tile_order) return LS_ERR_INVALID_ARG;
  return blend_bwd_impl(proj, n_records, cam, params, tile_ranges, vals, t_final, n_last, grad_image, grad_t, g2d,
                        tile_order, static_cast<cudaStream_t>(stream));
}

ls_status ls_project_bwd(int32_t n, const float* means, const float* scales, const float* quats,
                         const float* opacities, const float* sh, const ls_camera* cams, int32_t n_cams,
                         const ls_params* params, const void* proj, const float* g2d, float* g_means,
                         float* g_scales, float* g_quats, float* g_opac, float* g_sh, int32_t* status_dev,
                         void* stream) {
  if (n < 0 || !params_ok(params)) return LS_ERR_INVALID_ARG;
  CamTable T;
  if (!make_cams(cams, n_cams, params, T, nullptr)) return LS_ERR_INVALID_ARG;
  if (n == 0) return LS_OK;
  if (!means || !scales || !quats || !opacities || !sh || !proj || !g2d || !g_means || !g_scales || !g_quats ||
      !g_opac || !g_sh)
    return LS_ERR_INVALID_ARG;
  if (reinterpret_cast<uintptr_t>(quats) % 16 || reinterpret_cast<uintptr_t>(g_quats) % 16 ||
      reinterpret_cast<uintptr_t>(g2d) % 16)
    return LS_ERR_INVALID_ARG;
  (void)status_dev;
  LS_TRY(launch_project_bwd(n, means, scales, quats, opacities, sh, T, make_par(params),
                            proj_cplanes(proj, (int64_t)n * n_cams), g2d, g_means, g_scales, g_quats, g_opac, g_sh,
                            static_cast<cudaStream_t>(stream)));
  return LS_OK;
}

size_t ls_render_bwd_workspace(int64_t n_records) { return n_records > 0 ? al256((size_t)n_records * 48) : 256; }

size_t ls_render_bwd_workspace_ordered(int64_t n_records, const ls_camera* cam, const ls_params* params) {
  const size_t o = order_ws_bytes(cam, params);
  return n_records < 0 || o == 0 ? 0 : ls_render_bwd_workspace(n_records) + o;
}

ls_status ls_render_bwd(int32_t n, const float* means, const float* scales, const float* quats,
                        const float* opacities, const float* sh, const ls_camera* cam, const ls_params* params,
                        const void* proj, const int32_t* tile_ranges, const uint32_t* vals,
                        const float* t_final, const int32_t* n_last, const float* grad_image,
                        const float* grad_t, float* g_means, float* g_scales, float* g_quats, float* g_opac,
                        float* g_sh, float* g2d_out, void* workspace, size_t ws_bytes, int32_t* status_dev,
                        void* stream) {
  if (n < 0 || !params_ok(params)) return LS_ERR_INVALID_ARG;
  if (!workspace || ws_bytes < ls_render_bwd_workspace(n)) return LS_ERR_INVALID_ARG;
  if (reinterpret_cast<uintptr_t>(workspace) % 256) return LS_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  float* g2d = static_cast<float*>(workspace);
  // a workspace with room for the tile order blends the tiles longest first
  const size_t plain = ls_render_bwd_workspace(n), ord = order_ws_bytes(cam, params);
  char* order_ws = ord > 0 && ws_bytes >= plain + ord ? static_cast<char*>(workspace) + plain : nullptr;
  // one clear for the 2D gradients and the order's bucket counts behind them
  const size_t zero = order_ws ? plain + al256(4 * (size_t)TILE_ORDER_BUCKETS) : (size_t)n * 48;
  if (zero > 0) LS_TRY(cudaMemsetAsync(g2d, 0, zero, st));
  const uint32_t* order = nullptr;
  if (order_ws) {
    uint32_t* ord = reinterpret_cast<uint32_t*>(order_ws + order_scratch_bytes(cam_tiles(cam, params)));
    const ls_status so = tile_order_impl(n_last, cam, params, ord, order_ws, st);
    if (so != LS_OK) return so;
    order = ord;
  }
  ls_status s = blend_bwd_impl(proj, n, cam, params, tile_ranges, vals, t_final, n_last, grad_image, grad_t, g2d,
                               order, st);
  if (s != LS_OK) return s;
  s = ls_project_bwd(n, means, scales, quats, opacities, sh, cam, 1, params, proj, g2d, g_means, g_scales, g_quats,
                     g_opac, g_sh, status_dev, stream);
  if (s != LS_OK) return s;
  if (g2d_out && n > 0) LS_TRY(cudaMemcpyAsync(g2d_out, g2d, (size_t)n * 48, cudaMemcpyDeviceToDevice, st));
  return LS_OK;
}

// ---------------------------------------------------------------- batched render
namespace {

struct BatchWs {
  char* proj;
  uint32_t *keys, *vals;
  int32_t* ranges;
  uint32_t* queue;
  unsigned* job_ctr;
  char* dup;
  size_t dup_bytes, total;
};

BatchWs batch_layout(char* base, int64_t R, int64_t cap, int64_t total_tiles) {
  BatchWs w;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    char* p = base + off;
    off += al256(bytes);
    return p;
  };
  const size_t Cz = (size_t)(cap > 0 ? cap : 1);
  w.proj = take(ls_proj_bytes(R > 0 ? R : 1));
  w.keys = reinterpret_cast<uint32_t*>(take(4 * Cz));
  w.vals = reinterpret_cast<uint32_t*>(take(4 * Cz));
  w.ranges = reinterpret_cast<int32_t*>(take(8 * (size_t)total_tiles));
  w.queue = reinterpret_cast<uint32_t*>(take(4 * (size_t)total_tiles));
  w.job_ctr = reinterpret_cast<unsigned*>(take(4));
  w.dup_bytes = ls_duplicate_sort_workspace(R, cap, (int32_t)total_tiles);
  w.dup = take(w.dup_bytes);
  w.total = off;
  return w;
}

}  // namespace

size_t ls_render_batch_workspace(int32_t n, const ls_camera* cams, int32_t n_cams, const ls_params* params,
                                 int64_t key_capacity) {
  if (n < 0 || key_capacity < 0 || !params_ok(params)) return 0;
  CamTable T;
  int64_t total_tiles = 0;
  if (!make_cams(cams, n_cams, params, T, &total_tiles)) return 0;
  return batch_layout(nullptr, (int64_t)n * n_cams, key_capacity, total_tiles).total;
}

ls_status ls_render_batch(int32_t n, const float* means, const float* scales, const float* quats,
                          const float* opacities, const float* sh, const ls_camera* cams, int32_t n_cams,
                          const ls_params* params, int32_t blend_batch, int64_t key_capacity, float* images,
                          float* t_final, int64_t* n_keys_dev, void* workspace, size_t ws_bytes,
                          int32_t* status_dev, void* stream) {
  if (n < 0 || !params_ok(params)) return LS_ERR_INVALID_ARG;
  if (blend_batch != 0 && (blend_batch < 16 || blend_batch > 1024)) return LS_ERR_INVALID_ARG;
  CamTable T;
  int64_t total_tiles = 0;
  if (!make_cams(cams, n_cams, params, T, &total_tiles)) return LS_ERR_INVALID_ARG;
  const int64_t R = (int64_t)n * n_cams;
  if (R > 0x7FFFFFFFll || key_capacity < 0 || key_capacity > 0x7FFFFFFFll) return LS_ERR_INVALID_ARG;
  if (!images || !n_keys_dev || !workspace) return LS_ERR_INVALID_ARG;
  if (n > 0 && (!means || !scales || !quats || !opacities || !sh)) return LS_ERR_INVALID_ARG;
  if (reinterpret_cast<uintptr_t>(quats) % 16 || reinterpret_cast<uintptr_t>(workspace) % 256)
    return LS_ERR_INVALID_ARG;
  BatchWs w = batch_layout(static_cast<char*>(workspace), R, key_capacity, total_tiles);
  if (ws_bytes < w.total) return LS_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const ParDev P = make_par(params);
  BatchPix pix;
  size_t acc = 0;
  for (int c = 0; c < n_cams; ++c) {
    pix.base[c] = acc;
    acc += (size_t)cams[c].width * cams[c].height;
  }
  if (n > 0) {
    LS_TRY(launch_project_fwd(n, means, scales, quats, opacities, sh, T, P, proj_planes(w.proj, R), nullptr, st));
  }
  ls_status s = ls_duplicate_sort(R, w.proj, cams, n_cams, params, key_capacity, w.keys, w.vals, n_keys_dev,
                                  w.ranges, w.dup, w.dup_bytes, status_dev, stream);
  if (s != LS_OK) return s;
  LS_TRY(launch_build_queue(w.ranges, (int)total_tiles, w.queue, w.job_ctr, st));
  LS_TRY(launch_blend_batch(proj_cplanes(w.proj, R).rec, w.vals, w.ranges, T, pix, P, w.queue, (int)total_tiles,
                            w.job_ctr, images, t_final, blend_batch, st));
  return LS_OK;
}

ls_status ls_render_batch_blend(int32_t n, const ls_camera* cams, int32_t n_cams, const ls_params* params,
                                int32_t blend_batch, int64_t key_capacity, float* images, float* t_final,
                                void* workspace, size_t ws_bytes, int32_t* status_dev, void* stream) {
  (void)status_dev;
  if (n < 0 || !params_ok(params)) return LS_ERR_INVALID_ARG;
  if (blend_batch != 0 && (blend_batch < 16 || blend_batch > 1024)) return LS_ERR_INVALID_ARG;
  CamTable T;
  int64_t total_tiles = 0;
  if (!make_cams(cams, n_cams, params, T, &total_tiles)) return LS_ERR_INVALID_ARG;
  const int64_t R = (int64_t)n * n_cams;
  if (R > 0x7FFFFFFFll || key_capacity < 0 || key_capacity > 0x7FFFFFFFll) return LS_ERR_INVALID_ARG;
  if (!images || !workspace || reinterpret_cast<uintptr_t>(workspace) % 256) return LS_ERR_INVALID_ARG;
  BatchWs w = batch_layout(static_cast<char*>(workspace), R, key_capacity, total_tiles);
  if (ws_bytes < w.total) return LS_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  BatchPix pix;
  size_t acc = 0;
  for (int c = 0; c < n_cams; ++c) {
    pix.base[c] = acc;
    acc += (size_t)cams[c].width * cams[c].height;
  }
  LS_TRY(launch_build_queue(w.ranges, (int)total_tiles, w.queue, w.job_ctr, st));
  LS_TRY(launch_blend_batch(proj_cplanes(w.proj, R).rec, w.vals, w.ranges, T, pix, make_par(params), w.queue,
                            (int)total_tiles, w.job_ctr, images, t_final, blend_batch, st));
  return LS_OK;
}

// ---------------------------------------------------------------- training-side consumers
size_t ls_image_loss_workspace(int32_t height, int32_t width) {
  if (height <= 0 || width <= 0 || height > 16384 || width > 16384) return 0;
  return image_loss_ws_bytes(height, width);
}

ls_status ls_image_loss(int32_t height, int32_t width, const float* pred, const float* target, float w_l1,
                        float w_l2, float w_ssim, float* loss_dev, float* grad, void* workspace, size_t ws_bytes,
                        void* stream) {
  if (height <= 0 || width <= 0 || height > 16384 || width > 16384) return LS_ERR_INVALID_ARG;
  if (!pred || !target || !loss_dev || !workspace) return LS_ERR_INVALID_ARG;
  if (!std::isfinite(w_l1) || !std::isfinite(w_l2) || !std::isfinite(w_ssim)) return LS_ERR_INVALID_ARG;
  if (ws_bytes < image_loss_ws_bytes(height, width) || reinterpret_cast<uintptr_t>(workspace) % 256)
    return LS_ERR_INVALID_ARG;
  LS_TRY(launch_image_loss(height, width, pred, target, w_l1, w_l2, w_ssim, loss_dev, grad, workspace,
                           static_cast<cudaStream_t>(stream)));
  return LS_OK;
}

ls_status ls_adam(int64_t n, float* param, const float* grad, float* m1, float* m2, int32_t step, float lr,
                  float beta1, float beta2, float eps, int32_t mode, void* stream) {
  if (n < 0 || step < 1 || mode < 0 || mode > 2) return LS_ERR_INVALID_ARG;
  if (!(lr >= 0.f) || !(beta1 >= 0.f && beta1 < 1.f) || !(beta2 >= 0.f && beta2 < 1.f) || !(eps >= 0.f))
    return LS_ERR_INVALID_ARG;
  if (n > 0 && (!param || !grad || !m1 || !m2)) return LS_ERR_INVALID_ARG;
  LS_TRY(launch_adam(n, param, grad, m1, m2, step, lr, beta1, beta2, eps, mode, static_cast<cudaStream_t>(stream)));
  return LS_OK;
}

ls_status ls_densify_accumulate(int32_t n, const float* g2d, const void* proj, const ls_camera* cam, int32_t n_cams,
                                float* grad_accum, int32_t* count, float* max_radius, void* stream) {
  if (n < 0 || n_cams < 1 || !cam || !cam_ok(*cam)) return LS_ERR_INVALID_ARG;
  if (n > 0 && (!g2d || !proj || !grad_accum || !count || !max_radius)) return LS_ERR_INVALID_ARG;
  if (reinterpret_cast<uintptr_t>(proj) % 16) return LS_ERR_INVALID_ARG;
  ProjCPtr pp = proj_cplanes(proj, n);
  LS_TRY(launch_densify_accum(n, g2d, pp.foot, pp.dkey, cam->width, cam->height, n_cams, grad_accum, count,
                              max_radius, static_cast<cudaStream_t>(stream)));
  return LS_OK;
}

ls_status ls_densify_decide(int32_t n, const float* grad_accum, const int32_t* count, const float* max_radius,
                            const float* scales, const float* opacities, float scene_extent,
                            const ls_densify_params* params, uint8_t* flags, int64_t* counts_dev, void* stream) {
  if (n < 0 || !params || !(scene_extent > 0.f) || !std::isfinite(scene_extent)) return LS_ERR_INVALID_ARG;
  if (n > 0 && (!grad_accum || !count || !max_radius || !scales || !opacities || !flags)) return LS_ERR_INVALID_ARG;
  LS_TRY(launch_densify_decide(n, grad_accum, count, max_radius, scales, opacities, scene_extent, *params, flags,
                               counts_dev, static_cast<cudaStream_t>(stream)));
  return LS_OK;
}

size_t ls_filter3d_workspace(void) { return 256; }

ls_status ls_filter3d_variance(int32_t n, const float* means, const ls_camera* cams, int32_t n_cams, float near_plane,
                               float s2, float* filter_var, void* workspace, size_t ws_bytes, void* stream) {
  if (n < 0 || !(near_plane > 0.f) || !(s2 >= 0.f) || !std::isfinite(s2)) return LS_ERR_INVALID_ARG;
  if (!workspace || ws_bytes < ls_filter3d_workspace() || reinterpret_cast<uintptr_t>(workspace) % 256)
    return LS_ERR_INVALID_ARG;
  ls_params p{};
  p.lambda = 1.f;
  p.alpha_max = 0.5f;
  p.tile_w = p.tile_h = 16;
  p.near_plane = near_plane;
  p.far_plane = 2.f * near_plane + 1.f;
  CamTable T;
  if (!make_cams(cams, n_cams, &p, T, nullptr)) return LS_ERR_INVALID_ARG;
  if (n > 0 && (!means || !filter_var)) return LS_ERR_INVALID_ARG;
  LS_TRY(launch_filter3d_variance(n, means, T, near_plane, s2, filter_var, static_cast<unsigned*>(workspace),
                                  static_cast<cudaStream_t>(stream)));
  return LS_OK;
}

ls_status ls_filter3d_apply(int32_t n, const float* scales, const float* opacities, const float* filter_var,
                            float* scales_out, float* opacities_out, void* stream) {
  if (n < 0) return LS_ERR_INVALID_ARG;
  if (n > 0 && (!scales || !opacities || !filter_var || !scales_out || !opacities_out)) return LS_ERR_INVALID_ARG;
  LS_TRY(launch_filter3d_apply(n, scales, opacities, filter_var, scales_out, opacities_out,
                               static_cast<cudaStream_t>(stream)));
  return LS_OK;
}

ls_status ls_filter3d_apply_bwd(int32_t n, const float* scales, const float* opacities, const float* filter_var,
                                const float* g_scales_out, const float* g_opacities_out, float* g_scales,
                                float* g_opacities, void* stream) {
  if (n < 0) return LS_ERR_INVALID_ARG;
  if (n > 0 && (!scales || !opacities || !filter_var || !g_scales_out || !g_opacities_out || !g_scales ||
                !g_opacities))
    return LS_ERR_INVALID_ARG;
  LS_TRY(launch_filter3d_apply_bwd(n, scales, opacities, filter_var, g_scales_out, g_opacities_out, g_scales,
                                   g_opacities, static_cast<cudaStream_t>(stream)));
  return LS_OK;
}

// ---------------------------------------------------------------- termination MLP
namespace {
bool mlp_ok(const ls_mlp* n) { return n && n->w1t && n->b1 && n->w2t && n->b2 && n->w3 && n->b3; }
MlpDev mlp_dev(const ls_mlp* n) { return MlpDev{n->w1t, n->b1, n->w2t, n->b2, n->w3, n->b3}; }
}  // namespace

ls_status ls_mlp_forward(int64_t m, const void* x, const ls_mlp* net, float* y, void* stream) {
  if (m < 0 || !mlp_ok(net)) return LS_ERR_INVALID_ARG;
  if (m > 0 && (!x || !y)) return LS_ERR_INVALID_ARG;
  if (reinterpret_cast<uintptr_t>(x) % 16) return LS_ERR_INVALID_ARG;
  LS_TRY(launch_mlp_forward(m, x, mlp_dev(net), y, static_cast<cudaStream_t>(stream)));
  return LS_OK;
}

ls_status ls_mlp_backward(int64_t m, const void* x, const ls_mlp* net, const float* target, float under_weight,
                          float* grad, float* loss, void* stream) {
  if (m < 0 || !mlp_ok(net) || !grad || !(under_weight > 0.f)) return LS_ERR_INVALID_ARG;
  if (m > 0 && (!x || !target)) return LS_ERR_INVALID_ARG;
  if (reinterpret_cast<uintptr_t>(x) % 16) return LS_ERR_INVALID_ARG;
  LS_TRY(launch_mlp_backward(m, x, mlp_dev(net), target, under_weight, grad, loss, static_cast<cudaStream_t>(stream)));
  return LS_OK;
}

ls_status ls_mlp_adam(int32_t step, float lr, float beta1, float beta2, float eps, float* master, const float* grad,
                      float* m1, float* m2, const ls_mlp* net, void* stream) {
  if (step < 1 || !mlp_ok(net) || !master || !grad || !m1 || !m2) return LS_ERR_INVALID_ARG;
  MlpMut w{const_cast<void*>(net->w1t), const_cast<float*>(net->b1), const_cast<void*>(net->w2t),
           const_cast<float*>(net->b2), const_cast<void*>(net->w3), const_cast<float*>(net->b3)};
  LS_TRY(launch_mlp_adam(step, lr, beta1, beta2, eps, master, grad, m1, m2, w, static_cast<cudaStream_t>(stream)));
  return LS_OK;
}

// ---------------------------------------------------------------- learned termination
namespace {

struct LearnedWs {
  char* proj;
  uint32_t *dk_a, *dv_a, *dk_b, *dv_b;
  uint2* rect;
  int* diff;
  void* x16;
  float* y;
  uint32_t* dstar_bits;
  uint8_t* refuted;
  uint8_t* has_held;
  uint32_t* warp_tbase;
  unsigned long long *tmp_ctr_kept, *tmp_ctr_held;
  uint32_t *wc_kept, *wc_held;
  uint32_t *k_keys, *k_vals, *k_alt_keys, *k_alt_vals;
  uint32_t *h_keys, *h_vals, *h_alt_keys, *h_alt_vals;
  int32_t *k_ranges, *h_ranges;
  int* sat;
  int64_t *n_kept, *n_kept_valid, *n_held, *n_held_valid;
  unsigned* n_refuted;
  unsigned* refuted_floor;
  unsigned long long* key_total;
  size_t zero_begin, zero_bytes;
  char *depth_scratch, *kept_scratch, *held_scratch;
  size_t total;
};

LearnedWs learned_layout(char* base, int64_t R, int64_t cap, int tiles_x, int tiles_y, int kp) {
  LearnedWs w;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    char* p = base + off;
    off += al256(bytes);
    return p;
  };
  const size_t Rz = (size_t)(R > 0 ? R : 1), Cz = (size_t)(cap > 0 ? cap : 1);
  const size_t tiles = (size_t)tiles_x * tiles_y;
  w.proj = take(ls_proj_bytes((int64_t)Rz));
  w.dk_a = reinterpret_cast<uint32_t*>(take(4 * Rz));
  w.dv_a = reinterpret_cast<uint32_t*>(take(4 * Rz));
  w.dk_b = reinterpret_cast<uint32_t*>(take(4 * Rz));
  w.dv_b = reinterpret_cast<uint32_t*>(take(4 * Rz));
  w.rect = reinterpret_cast<uint2*>(take(8 * Rz));
  w.x16 = take(2 * LS_MLP_IN * tiles);
  w.y = reinterpret_cast<float*>(take(4 * tiles));
  w.dstar_bits = reinterpret_cast<uint32_t*>(take(4 * (size_t)dstar_pyramid_words(tiles_x, tiles_y)));  // + pyramid
  w.wc_kept = reinterpret_cast<uint32_t*>(take(4 * (size_t)enum_count_words((int64_t)Rz)));
  w.wc_held = reinterpret_cast<uint32_t*>(take(4 * (size_t)enum_count_words((int64_t)Rz)));
  w.warp_tbase = reinterpret_cast<uint32_t*>(take(4 * (size_t)enum_warps((int64_t)Rz)));
  w.k_keys = reinterpret_cast<uint32_t*>(take(4 * Cz));
  w.k_vals = reinterpret_cast<uint32_t*>(take(4 * Cz));
  w.k_alt_keys = reinterpret_cast<uint32_t*>(take(4 * Cz));
  w.k_alt_vals = reinterpret_cast<uint32_t*>(take(4 * Cz));
  w.h_keys = reinterpret_cast<uint32_t*>(take(4 * Cz));
  w.h_vals = reinterpret_cast<uint32_t*>(take(4 * Cz));
  w.h_alt_keys = reinterpret_cast<uint32_t*>(take(4 * Cz));
  w.h_alt_vals = reinterpret_cast<uint32_t*>(take(4 * Cz));
  w.sat = reinterpret_cast<int*>(take(4 * (size_t)(tiles_x + 1) * (tiles_y + 1)));
  w.k_ranges = reinterpret_cast<int32_t*>(take(8 * tiles));
  w.h_ranges = reinterpret_cast<int32_t*>(take(8 * tiles));
  // cleared before every call
  w.zero_begin = off;
  w.diff = reinterpret_cast<int*>(take(33 * 4 * (size_t)(tiles_x + 1) * (tiles_y + 1)));  // coverage planes
  w.refuted = reinterpret_cast<uint8_t*>(take(tiles));
  w.has_held = reinterpret_cast<uint8_t*>(take(tiles));
  w.tmp_ctr_kept = reinterpret_cast<unsigned long long*>(take(8));
  w.tmp_ctr_held = reinterpret_cast<unsigned long long*>(take(8));
  w.n_kept = reinterpret_cast<int64_t*>(take(8));
  w.n_kept_valid = reinterpret_cast<int64_t*>(take(8));
  w.n_held = reinterpret_cast<int64_t*>(take(8));
  w.n_held_valid = reinterpret_cast<int64_t*>(take(8));
  w.n_refuted = reinterpret_cast<unsigned*>(take(4));
  w.refuted_floor = reinterpret_cast<unsigned*>(take(4));
  w.key_total = reinterpret_cast<unsigned long long*>(take(8));
  w.depth_scratch = take(sort_scratch_bytes((int64_t)Rz, 4));
  w.kept_scratch = take(sort_scratch_bytes((int64_t)Cz, kp));
  w.held_scratch = take(sort_scratch_bytes((int64_t)Cz, kp));
  w.zero_bytes = off - w.zero_begin;
  w.total = off;
  return w;
}

// Sort `n_dev` keys (ek, ev) by tile in kp passes so that the result lands in
// (keys, vals); the last pass records the ranges.
ls_status tile_sort(uint32_t* ek, uint32_t* ev, uint32_t* ok, uint32_t* ov, const int64_t* n_dev, int64_t cap, int kp,
                    const SortScratch& ss, int32_t* ranges, int tiles, int32_t* status, cudaStream_t st) {
  const TileDigits td = tile_digits(tiles);
  LS_TRY(launch_radix_scan(ss.hist, kp, st));
  for (int p = 0; p < kp; ++p) {
    LS_TRY(launch_onesweep_pass(ek, ev, ok, ov, n_dev, 0, cap, td.shift[p], td.bits[p], p, ss,
                                p == kp - 1 ? ranges : nullptr, status, st));
    std::swap(ek, ok);
    std::swap(ev, ov);
  }
  LS_TRY(launch_ranges_fixup(ranges, tiles, st));
  return LS_OK;
}

}  // namespace

size_t ls_tile_features_workspace(const ls_camera* cam, const ls_params* params) {
  if (!params_ok(params)) return 0;
  CamTable T;
  if (!make_cams(cam, 1, params, T, nullptr)) return 0;
  return al256(hist_planes_bytes(T.c[0]));
}

ls_status ls_tile_features(const void* proj, int64_t n_records, const ls_camera* cam, const ls_params* params,
                           void* features, int32_t* tile_total, void* workspace, size_t ws_bytes, void* stream) {
  if (!params_ok(params) || n_records < 0) return LS_ERR_INVALID_ARG;
  CamTable T;
  if (!make_cams(cam, 1, params, T, nullptr)) return LS_ERR_INVALID_ARG;
  if (!features || !tile_total || !workspace || ws_bytes < ls_tile_features_workspace(cam, params))
    return LS_ERR_INVALID_ARG;
  if (n_records > 0 && !proj) return LS_ERR_INVALID_ARG;
  if (reinterpret_cast<uintptr_t>(workspace) % 256) return LS_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const ParDev P = make_par(params);
  LS_TRY(cudaMemsetAsync(workspace, 0, ls_tile_features_workspace(cam, params), st));
  ProjCPtr pp = proj_cplanes(proj, n_records);
  LS_TRY(launch_tile_hist(n_records, pp.rec, pp.foot, pp.dkey, T.c[0], P, workspace, true, st));
  LS_TRY(launch_features(workspace, T.c[0], P, features, tile_total, nullptr, st));
  return LS_OK;
}

size_t ls_render_learned_workspace(int32_t n, const ls_camera* cam, const ls_params* params, int64_t key_capacity) {
  if (n < 0 || key_capacity < 0 || !params_ok(params)) return 0;
  CamTable T;
  int64_t tiles = 0;
  if (!make_cams(cam, 1, params, T, &tiles)) return 0;
  return learned_layout(nullptr, n, key_capacity, T.c[0].tiles_x, T.c[0].tiles_y, key_passes_for(tiles)).total;
}

ls_status ls_render_learned(int32_t n, const float* means, const float* scales, const float* quats,
                            const float* opacities, const float* sh, const ls_camera* cam, const ls_params* params,
                            const ls_mlp* mlp, float margin, const float* dstar_in, float t_thr, int64_t key_capacity,
                            float* image, float* t_final, int32_t* n_last, float* dstar_out, int64_t* stats_dev,
                            void* workspace, size_t ws_bytes, int32_t* status_dev, void* stream) {
  if (n < 0 || !params_ok(params) || !(t_thr >= 0.f)) return LS_ERR_INVALID_ARG;
  CamTable T;
  int64_t tiles64 = 0;
  if (!make_cams(cam, 1, params, T, &tiles64)) return LS_ERR_INVALID_ARG;
  if (key_capacity < 0 || key_capacity > 0x7FFFFFFFll) return LS_ERR_INVALID_ARG;
  if (!image || !t_final || !n_last || !workspace) return LS_ERR_INVALID_ARG;
  if (mlp ? !mlp_ok(mlp) : !dstar_in) return LS_ERR_INVALID_ARG;
  if (n > 0 && (!means || !scales || !quats || !opacities || !sh)) return LS_ERR_INVALID_ARG;
  if (reinterpret_cast<uintptr_t>(quats) % 16 || reinterpret_cast<uintptr_t>(workspace) % 256)
    return LS_ERR_INVALID_ARG;
  const CamDev& C = T.c[0];
  const int tiles = (int)tiles64, kp = key_passes_for(tiles64);
  const TileDigits td = tile_digits(tiles64);
  const int64_t R = n;
  LearnedWs w = learned_layout(static_cast<char*>(workspace), R, key_capacity, C.tiles_x, C.tiles_y, kp);
  if (ws_bytes < w.total) return LS_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const ParDev P = make_par(params);
  ProjPtr pw = proj_planes(w.proj, R);
  ProjCPtr pp = proj_cplanes(w.proj, R);
  LS_TRY(cudaMemsetAsync(static_cast<char*>(workspace) + w.zero_begin, 0, w.zero_bytes, st));
  // projection and depth order (as the plain path)
  if (R > 0) {
    LS_TRY(launch_project_fwd(n, means, scales, quats, opacities, sh, T, P, pw, nullptr, st));
    SortScratch ds = sort_scratch_carve(w.depth_scratch, R, 4);
    LS_TRY(launch_radix_hist(pp.dkey, nullptr, R, 0, 4, ds.hist, st));
    LS_TRY(launch_radix_scan(ds.hist, 4, st));
    LS_TRY(launch_onesweep_pass(pp.dkey, nullptr, w.dk_b, w.dv_b, nullptr, R, R, 0, 8, 0, ds, nullptr, status_dev, st));
    LS_TRY(launch_onesweep_pass(w.dk_b, w.dv_b, w.dk_a, w.dv_a, nullptr, R, R, 8, 8, 1, ds, nullptr, status_dev, st));
    LS_TRY(launch_onesweep_pass(w.dk_a, w.dv_a, w.dk_b, w.dv_b, nullptr, R, R, 16, 8, 2, ds, nullptr, status_dev, st));
    LS_TRY(launch_onesweep_pass(w.dk_b, w.dv_b, w.dk_a, w.dv_a, nullptr, R, R, 24, 8, 3, ds, nullptr, status_dev, st));
    LS_TRY(launch_dup_count(R, w.dv_a, w.dk_a, pp.foot, T, n, P, w.rect, st));
  }
  // per-tile features and the proposal
  if (tile_hist_sorted_smem(C) <= 160 * 1024)
    LS_TRY(launch_tile_hist_sorted(R, w.dv_a, w.dk_a, w.rect, pp.rec, C, P, w.diff, st));
  else
    LS_TRY(launch_tile_hist(R, pp.rec, pp.foot, pp.dkey, C, P, w.diff, false, st));
  LS_TRY(launch_features(w.diff, C, P, w.x16, nullptr, nullptr, st));
  if (mlp) LS_TRY(launch_mlp_forward(tiles, w.x16, mlp_dev(mlp), w.y, st));
  LS_TRY(launch_dstar(C, mlp ? w.y : nullptr, margin, dstar_in, w.dstar_bits, dstar_out, w.diff, w.has_held, st));
  // kept keys: count per warp (and every key the ellipses reach), scan,
  // emit, sort, blend
  SortScratch ks = sort_scratch_carve(w.kept_scratch, key_capacity > 0 ? key_capacity : 1, kp);
  SortScratch hs = sort_scratch_carve(w.held_scratch, key_capacity > 0 ? key_capacity : 1, kp);
  LS_TRY(cudaMemsetAsync(w.k_ranges, 0xFF, 8 * (size_t)tiles, st));
  LS_TRY(cudaMemsetAsync(w.h_ranges, 0xFF, 8 * (size_t)tiles, st));
  uint32_t *ek = kp % 2 == 0 ? w.k_keys : w.k_alt_keys, *ev = kp % 2 == 0 ? w.k_vals : w.k_alt_vals;
  uint32_t *ok = kp % 2 == 0 ? w.k_alt_keys : w.k_keys, *ov = kp % 2 == 0 ? w.k_alt_vals : w.k_vals;
  EnumArgs ea{};
  ea.R = R;
  ea.order = w.dv_a;
  ea.dkey_sorted = w.dk_a;
  ea.rect_sorted = w.rect;
  ea.rec = pp.rec;
  ea.cams = T;
  ea.n_per_cam = n;
  ea.tile_w = P.tile_w;
  ea.tile_h = P.tile_h;
  ea.dstar_bits = w.dstar_bits;
  ea.refuted = w.refuted;
  ea.sat = w.sat;
  ea.n_refuted = w.n_refuted;
  ea.refuted_floor = w.refuted_floor;
  ea.key_passes = kp;
  for (int p = 0; p < kp; ++p) {
    ea.dshift[p] = td.shift[p];
    ea.dmask[p] = (1u << td.bits[p]) - 1u;
  }
  ea.key_total = stats_dev ? w.key_total : nullptr;  // counting every reached key only for the stats
  ea.dstar_pyr = w.dstar_bits;
  ea.pyr = make_dstar_pyramid(C.tiles_x, C.tiles_y);
  ea.warp_counts = w.wc_kept;
  ea.warp_tbase = w.warp_tbase;
  ea.n_warps = enum_warps(R);
  ea.tmp_keys = ok;
  ea.tmp_vals = ov;
  ea.tmp_cap = key_capacity;
  ea.tmp_ctr = w.tmp_ctr_kept;
  ea.n_valid = w.n_kept_valid;
  ea.tile_hist = ks.hist;
  LS_TRY(launch_enum_keys(false, ENUM_KEPT, ea, st));
  LS_TRY(launch_dup_scan(enum_warps(R), w.wc_kept, key_capacity, w.n_kept, w.n_kept_valid, status_dev, st));
  if (R > 0 && key_capacity > 0) {
    ea.keys = ek;
    ea.vals = ev;
    LS_TRY(launch_enum_keys(true, ENUM_KEPT, ea, st));
    ls_status s = tile_sort(ek, ev, ok, ov, w.n_kept_valid, key_capacity, kp, ks, w.k_ranges, tiles, status_dev, st);
    if (s != LS_OK) return s;
  } else {
    LS_TRY(launch_ranges_fixup(w.k_ranges, tiles, st));
  }
  TruncArgs ta{};
  ta.t_thr = t_thr;
  ta.has_held = w.has_held;
  ta.refuted = w.refuted;
  ta.n_refuted = w.n_refuted;
  ta.dstar_bits = w.dstar_bits;
  ta.refuted_floor = w.refuted_floor;
  ta.kept_ranges = reinterpret_cast<const int2*>(w.k_ranges);
  LS_TRY(launch_blend_trunc(1, pp.rec, C, P, reinterpret_cast<const int2*>(w.k_ranges), w.k_vals, image, t_final,
                            n_last, ta, st));
  // held-out keys of refuted tiles (every kernel returns at once when none)
  LS_TRY(launch_refuted_sat(w.refuted, w.n_refuted, C.tiles_x, C.tiles_y, w.sat, st));
  uint32_t *hk = kp % 2 == 0 ? w.h_keys : w.h_alt_keys, *hv = kp % 2 == 0 ? w.h_vals : w.h_alt_vals;
  uint32_t *hok = kp % 2 == 0 ? w.h_alt_keys : w.h_keys, *hov = kp % 2 == 0 ? w.h_alt_vals : w.h_vals;
  ea.warp_counts = w.wc_held;
  ea.tmp_keys = hok;
  ea.tmp_vals = hov;
  ea.tmp_ctr = w.tmp_ctr_held;
  ea.n_valid = w.n_held_valid;
  ea.keys = ea.vals = nullptr;
  ea.tile_hist = hs.hist;
  LS_TRY(launch_enum_keys(false, ENUM_HELD, ea, st));
  LS_TRY(launch_dup_scan(enum_warps(R), w.wc_held, key_capacity, w.n_held, w.n_held_valid, status_dev, st));
  if (R > 0 && key_capacity > 0) {
    ea.keys = hk;
    ea.vals = hv;
    LS_TRY(launch_enum_keys(true, ENUM_HELD, ea, st));
    ls_status s = tile_sort(hk, hv, hok, hov, w.n_held_valid, key_capacity, kp, hs, w.h_ranges, tiles, status_dev, st);
    if (s != LS_OK) return s;
  } else {
    LS_TRY(launch_ranges_fixup(w.h_ranges, tiles, st));
  }
  LS_TRY(launch_blend_trunc(2, pp.rec, C, P, reinterpret_cast<const int2*>(w.h_ranges), w.h_vals, image, t_final,
                            n_last, ta, st));
  if (stats_dev) LS_TRY(launch_learned_stats(w.key_total, w.n_kept, w.n_held, w.n_refuted, stats_dev, st));
  return LS_OK;
}

}  // extern "C"
