/*
 * ls.h -- C ABI of the GB300 (sm_103a) rasterizer for 3D Linear Splatting
 * (arxiv 2411.12440, "Beyond Gaussians: Fast and High-Fidelity 3D Splatting
 * with Linear Kernels").
 *
 * Every entry point takes plain pointers and sizes.  Unless a parameter says
 * otherwise:
 *   - array pointers are DEVICE memory owned by the caller; the library never
 *     allocates, frees or keeps them after the call returns;
 *   - structs passed by pointer (ls_params, ls_camera) are HOST memory, read
 *     during the call only;
 *   - work is enqueued asynchronously on `stream` (a cudaStream_t, NULL = the
 *     legacy default stream); the call returns before it runs;
 *   - the return value reports argument checks and launch errors only:
 *     LS_ERR_INVALID_ARG before anything is enqueued, LS_ERR_CUDA when a
 *     launch fails (cudaGetLastError);
 *   - errors found while the kernels run (key capacity exceeded, a bounded
 *     device-side wait that gave up) are written to *status_dev, an int32 in
 *     device memory that the caller zeroes beforehand and reads after
 *     synchronising; the first error written wins;
 *   - all floating point is IEEE binary32, row-major.
 *
 * Pipeline (one frame): ls_project -> ls_duplicate_sort -> ls_render_fwd,
 * and for training ls_render_bwd with the forward's T_final / n_last.
 * ls_render_batch runs the same pipeline for many cameras over one shared
 * sort and one persistent blending launch.
 */
#ifndef LS_H_
#define LS_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  LS_OK = 0,
  LS_ERR_INVALID_ARG = 1,
  LS_ERR_CUDA = 2,
  LS_ERR_CAPACITY = 3,   /* more tile keys than key_capacity (device-detected) */
  LS_ERR_TIMEOUT = 4,    /* a bounded device-side wait gave up (device-detected) */
  LS_ERR_UNSUPPORTED = 5
} ls_status;

/* Attenuation f(D / lambda) of the Mahalanobis distance D.  Linear is the
 * paper's kernel (Sec. 3.2 Eq. 9-11 with the alignment of Sec. 3.3.1 Eq. 12);
 * the others are the family of Appendix B Eq. 21-24. */
typedef enum {
  LS_KERNEL_LINEAR = 0,     /* max(0, 1 - x)                 */
  LS_KERNEL_GAUSSIAN = 1,   /* exp(-x^2 / 2)                 */
  LS_KERNEL_LAPLACIAN = 2,  /* exp(-x)                       */
  LS_KERNEL_COSINE = 3,     /* (1 + cos(pi x)) / 2, 0 for x>1 */
  LS_KERNEL_QUADRATIC = 4   /* max(0, 1 - x^2)               */
} ls_kernel;

/* Rendering parameters.  Defaults in brackets. */
typedef struct {
  float lambda;      /* distribution-alignment factor, Eq. 12 [2.5]; > 0 */
  int32_t kernel;    /* ls_kernel [LS_KERNEL_LINEAR] */
  int32_t ags;       /* adaptive gradient scaling, Eq. 13-14: 0 off, 1 w = exp(-D^2),
                        2 w = exp(-(D/lambda)^2) [0] */
  int32_t antialias; /* 1: scale opacity by sqrt(det Sigma_2D / det(Sigma_2D + eps2d I))
                        (Mip-Splatting 2D filter, named in Sec. 4.1) [0] */
  float eps2d;       /* screen-space dilation added to Sigma_2D [0.3]; >= 0 */
  float alpha_min;   /* pairs with alpha below this are skipped [1/255]; >= 0 */
  float alpha_max;   /* alpha clamp [0.999]; in (0, 1) */
  float t_min;       /* a pixel stops before T would fall below this [1e-4]; >= 0 */
  int32_t tile_w, tile_h; /* tile shape: 8x8, 16x16 or 32x16 [16x16] */
  float bg[3];       /* background colour composited behind [0,0,0] */
  float near_plane, far_plane; /* depth cull (near, far) [0.2, 1e4] */
  int32_t sh_degree; /* spherical-harmonic degree 0..3 */
} ls_params;

/* Pinhole camera, OpenCV axes (x right, y down, z forward).  viewmat is the
 * world-to-camera matrix W of Sec. 3.1 Eq. 3, row-major [R t; 0 0 0 1]. */
typedef struct {
  float viewmat[16];
  float fx, fy, cx, cy;
  int32_t width, height;
} ls_camera;

#define LS_MAX_CAMS 64

/* Projected-record buffer.  For n primitives seen by n_cams cameras there are
 * R = n_cams * n records; record r = cam * n + i.  The buffer holds three
 * consecutive planes, 68 bytes per record (ls_proj_bytes):
 *   rec  [R][12] float at byte 0:        {mx, my, l00, l01}, {l11, o_eff, rho^2, depth}, {r, g, b, 0}
 *        screen centre mu' (pixel units, pixel (px,py) covers [px,px+1)x[py,py+1)),
 *        the conic A = (Sigma_2D + eps2d I)^-1 = [[a, b], [b, c]] as its upper
 *        Cholesky factor L = [[l00, l01], [0, l11]], A = L^T L (so D^2 = |L d|^2
 *        is a sum of squares), effective opacity, squared support radius in
 *        Mahalanobis units, camera depth, colour;
 *   foot [R][4] float at byte 48*R:      {mx, my, ex, ey} half extents of the support box;
 *   dkey [R] uint32 at byte 64*R:        binary32 bits of depth, 0xFFFFFFFF when culled.
 * Fields of culled records other than dkey are unspecified. */
size_t ls_proj_bytes(int64_t n_records);

/* a1: projection (Sec. 3.1 Eq. 1-4; support of Eq. 12; view-dependent colour).
 * means [n][3], scales [n][3] (positive, activated), quats [n][4] (w,x,y,z, any
 * non-zero norm), opacities [n] (activated, in [0,1]), sh [(deg+1)^2][3][n]
 * (coefficient-major: sh[(k*3+ch)*n + i]); cams: host array of n_cams
 * (1..LS_MAX_CAMS).  Writes proj (ls_proj_bytes(n_cams*n) bytes) and, when not
 * NULL, tile_counts [n_cams*n] (tiles each record touches, 0 when culled). */
ls_status ls_project(int32_t n, const float* means, const float* scales, const float* quats,
                     const float* opacities, const float* sh, const ls_camera* cams, int32_t n_cams,
                     const ls_params* params, void* proj, int32_t* tile_counts, int32_t* status_dev,
                     void* stream);

/* Workspace of ls_duplicate_sort in bytes. */
size_t ls_duplicate_sort_workspace(int64_t n_records, int64_t key_capacity, int32_t total_tiles);

/* a2+a3: duplication of every visible record into the tiles of its support
 * box that its support ellipse reaches, and a stable radix sort into
 * front-to-back order per tile (compositing order of Sec. 3.1 Eq. 6, kept
 * "without alteration", Sec. 3.2).  Reach rule, binary32 with every operation
 * rounded once: per box row, the ellipse D^2 <= 1.02 rho^2 + 1e-3 cut by the
 * band of the row's pixel-centre heights has an x-extent (from its left and
 * right boundary points), and the tiles whose pixel-centre columns meet it
 * (0.01 px slack) are listed; boxes of at most 2 tiles are listed whole.
 * Every pair the blend can composite is listed.  K is at most the sum of the
 * tile_counts of ls_project (the box tiles), which therefore bounds the
 * capacity a caller needs.
 * Tile ids are global over the cameras: camera c's tiles follow those of
 * cameras 0..c-1, row-major within a camera.  Output, for K keys:
 *   keys [K] tile ids ascending; vals [K] record ids, ordered inside a tile by
 *   (depth bits, record id); *n_keys_dev = K (int64, device);
 *   tile_ranges [total_tiles][2] = [start, end) of each tile in keys/vals.
 * key_capacity bounds K (<= 2^31-1); when K > key_capacity nothing past the
 * count is written, ranges are empty and LS_ERR_CAPACITY goes to status_dev.
 * workspace: device scratch of at least ls_duplicate_sort_workspace bytes,
 * 256-byte aligned. */
ls_status ls_duplicate_sort(int64_t n_records, const void* proj, const ls_camera* cams, int32_t n_cams,
                            const ls_params* params, int64_t key_capacity, uint32_t* keys, uint32_t* vals,
                            int64_t* n_keys_dev, int32_t* tile_ranges, void* workspace, size_t ws_bytes,
                            int32_t* status_dev, void* stream);

/* a4: front-to-back blending of one camera's tiles (Sec. 3.1 Eq. 6 with
 * alpha = o_eff * f(D/lambda), Eq. 11-12): per pixel centre x', over its
 * tile's records in order, skip when D^2 > rho^2, alpha = min(alpha_max, .),
 * skip when alpha < alpha_min, stop before T would drop below t_min.
 * proj/vals/tile_ranges as produced above for n_cams = 1.  Writes image
 * [H][W][3] (colour + T * bg), t_final [H][W] and n_last [H][W] (number of
 * leading entries of the pixel's tile list up to and including the last one
 * composited: the checkpoint the backward pass resumes from). */
ls_status ls_render_fwd(const void* proj, int64_t n_records, const ls_camera* cam, const ls_params* params,
                        const int32_t* tile_ranges, const uint32_t* vals, float* image, float* t_final,
                        int32_t* n_last, int32_t* status_dev, void* stream);

/* ls_render_fwd that also counts the work units of the tile method into
 * stats_dev[2] (uint64, device, accumulated: zero it first): [0] evaluated
 * (pixel, record) pairs -- per tile, its pixels times the entries walked until
 * the tile's last pixel finished -- and [1] composited pairs (alpha >=
 * alpha_min, before the stop).  Same outputs as ls_render_fwd; slower (used
 * to size the roofline of the blending kernels, not on the hot path). */
ls_status ls_render_stats(const void* proj, int64_t n_records, const ls_camera* cam, const ls_params* params,
                          const int32_t* tile_ranges, const uint32_t* vals, float* image, float* t_final,
                          int32_t* n_last, uint64_t* stats_dev, float* tile_labels, int32_t* status_dev,
                          void* stream);
/* tile_labels [tiles] (or NULL): per tile, the camera depth of the list entry
 * at which its last pixel stopped (every later entry is never needed), +inf
 * when some pixel never stops, 0 for an empty tile: the target of the
 * learned termination. */

/* a5: adjoint of ls_render_fwd with respect to each record's (mx, my, a, b,
 * c, o_eff, r, g, b), recomputing T back to front from t_final / n_last
 * (Eq. 6); with params->ags the kernel-derivative path is scaled by w(D)
 * (Eq. 13-14).  grad_image [H][W][3]; grad_t [H][W] or NULL.  g2d [R][12]
 * float is ACCUMULATED into (zero it first): {gmx, gmy, ga, gb}, {gc, go,
 * gr, gg}, {gb, 0, 0, 0}, where ga, gb, gc are the gradients with respect to
 * the conic entries a, b, c of A (b counted once, as in d^T A d =
 * a dx^2 + 2 b dx dy + c dy^2), whatever factor the record stores. */
ls_status ls_blend_bwd(const void* proj, int64_t n_records, const ls_camera* cam, const ls_params* params,
                       const int32_t* tile_ranges, const uint32_t* vals, const float* t_final,
                       const int32_t* n_last, const float* grad_image, const float* grad_t, float* g2d,
                       int32_t* status_dev, void* stream);

/* a6: chain rule from g2d [n_cams*n][12] (summed over cameras) to the 3D
 * parameters of ls_project (Eq. 1-4 and the colour).  Outputs are OVERWRITTEN:
 * g_means [n][3], g_scales [n][3], g_quats [n][4], g_opac [n],
 * g_sh [(deg+1)^2][3][n]. */
ls_status ls_project_bwd(int32_t n, const float* means, const float* scales, const float* quats,
                         const float* opacities, const float* sh, const ls_camera* cams, int32_t n_cams,
                         const ls_params* params, const void* proj, const float* g2d, float* g_means,
                         float* g_scales, float* g_quats, float* g_opac, float* g_sh, int32_t* status_dev,
                         void* stream);

/* Longest-first order of a camera's tiles for the backward blend (the
 * order ls_render_bwd uses with its ordered workspace): each tile's work is
 * the largest n_last over its pixels (n_last [H][W] as written by
 * ls_render_fwd), the tiles go into quarter-octave buckets of it and
 * tile_order [tiles_x * tiles_y] (caller-owned, device) lists them from the
 * heaviest bucket down, in no particular order within a bucket.  workspace:
 * device scratch of at least ls_tile_order_workspace bytes, 256-byte
 * aligned.  LS_ERR_INVALID_ARG for an invalid camera or parameters, null
 * pointers or a short workspace. */
size_t ls_tile_order_workspace(const ls_camera* cam, const ls_params* params);
ls_status ls_tile_order(const int32_t* n_last, const ls_camera* cam, const ls_params* params, uint32_t* tile_order,
                        void* workspace, size_t ws_bytes, void* stream);

/* ls_blend_bwd with CTA b blending tile tile_order[b] (a permutation of the
 * camera's tiles, e.g. from ls_tile_order; not NULL).  Results as
 * ls_blend_bwd up to the order of the floating-point atomic additions. */
ls_status ls_blend_bwd_ordered(const void* proj, int64_t n_records, const ls_camera* cam, const ls_params* params,
                               const int32_t* tile_ranges, const uint32_t* tile_order, const uint32_t* vals,
                               const float* t_final, const int32_t* n_last, const float* grad_image,
                               const float* grad_t, float* g2d, int32_t* status_dev, void* stream);

/* Workspace of ls_render_bwd in bytes (the g2d buffer). */
size_t ls_render_bwd_workspace(int64_t n_records);

/* Workspace of ls_render_bwd with room behind the g2d buffer for a tile
 * order of the given camera (bucket counts, buckets and order, 4 bytes per
 * tile each); 0 for an invalid camera or parameters or n_records < 0. */
size_t ls_render_bwd_workspace_ordered(int64_t n_records, const ls_camera* cam, const ls_params* params);

/* a5+a6 in one call for one camera: zeroes a g2d buffer in `workspace`, runs
 * ls_blend_bwd then ls_project_bwd.  When g2d_out is not NULL the 2D
 * gradients are also copied there ([n][12] float).  With ws_bytes at least
 * ls_render_bwd_workspace_ordered(n, cam, params), the backward blend takes
 * its tiles longest first: each tile's work is the largest n_last over its
 * pixels, and two small kernels order the tiles by it (in quarter-octave
 * buckets) so that the longest lists do not finish last.  The results are
 * those of the plain order up to the order of the floating-point atomic
 * additions into the 2D gradients. */
ls_status ls_render_bwd(int32_t n, const float* means, const float* scales, const float* quats,
                        const float* opacities, const float* sh, const ls_camera* cam, const ls_params* params,
                        const void* proj, const int32_t* tile_ranges, const uint32_t* vals,
                        const float* t_final, const int32_t* n_last, const float* grad_image,
                        const float* grad_t, float* g_means, float* g_scales, float* g_quats, float* g_opac,
                        float* g_sh, float* g2d_out, void* workspace, size_t ws_bytes, int32_t* status_dev,
                        void* stream);

/* ---- a8: learned termination --------------------------------------------
 * A per-tile MLP 48 -> 64 -> 64 -> 1 (ReLU) with FP16 inputs and weights and
 * FP32 accumulation (tensor cores) predicts the log camera depth at which
 * every pixel of the tile has stopped.  Inputs: LS_MLP_FEATURES = 35 used
 * features of a 48-wide FP16 row (the rest zero).  Parameters, packed FP32
 * (master copy and gradients, LS_MLP_NPARAM floats):
 *   w1t [64][48] | b1 [64] | w2t [64][64] | b2 [64] | w3 [64] | b3 [1]
 * (w1t, w2t are [out][in]).  The forward reads FP16 copies of w1t, w2t, w3
 * and FP32 biases through ls_mlp (device pointers). */
#define LS_MLP_IN 48
#define LS_MLP_HID 64
#define LS_MLP_FEATURES 35
#define LS_MLP_NPARAM 7361
typedef struct {
  const void* w1t;  /* fp16 [64][48] */
  const float* b1;  /* [64] */
  const void* w2t;  /* fp16 [64][64] */
  const float* b2;  /* [64] */
  const void* w3;   /* fp16 [64] */
  const float* b3;  /* [1] */
} ls_mlp;

/* y [m] = MLP(x [m][48] fp16).  Tensor-core forward. */
ls_status ls_mlp_forward(int64_t m, const void* x, const ls_mlp* net, float* y, void* stream);

/* Gradient of the mean asymmetric squared error
 *   (1/m) sum_r w_r (y_r - target_r)^2,  w_r = under_weight if y_r < target_r else 1,
 * ACCUMULATED into grad [LS_MLP_NPARAM] (packed layout) and, when not NULL,
 * the loss into *loss.  Tensor-core backward (layer inputs rounded to fp16 as
 * in the forward; the rounding is passed through as identity). */
ls_status ls_mlp_backward(int64_t m, const void* x, const ls_mlp* net, const float* target, float under_weight,
                          float* grad, float* loss, void* stream);

/* One Adam step (bias-corrected, step >= 1) on the packed FP32 master
 * parameters with moments m1, m2, then refresh of the FP16 weights and FP32
 * biases pointed to by net (which must be writable device memory). */
ls_status ls_mlp_adam(int32_t step, float lr, float beta1, float beta2, float eps, float* master, const float* grad,
                      float* m1, float* m2, const ls_mlp* net, void* stream);

/* Per-tile inputs of the termination MLP for one camera, from projected
 * records.  Each visible record whose support box covers the tile adds its
 * expected coverage w = (o_eff / 3) min(1, ellipse area / box area) to its
 * log-depth bin (32 bins, edges 0.5 * 64^(i/32), i = 1..31).  features
 * [tiles][48] fp16 = log1p of the coverage summed over bins 0..b (b = 0..31),
 * then the world direction of the ray through the tile centre (3), then
 * zeros; tile_total [tiles] = number of records covering the tile.
 * workspace: ls_tile_features_workspace bytes. */
size_t ls_tile_features_workspace(const ls_camera* cam, const ls_params* params);
ls_status ls_tile_features(const void* proj, int64_t n_records, const ls_camera* cam, const ls_params* params,
                           void* features, int32_t* tile_total, void* workspace, size_t ws_bytes, void* stream);

/* a8: forward render of one camera with learned termination.  The MLP (or,
 * when mlp is NULL, the caller's per-tile depths dstar_in [tiles]) proposes
 * per tile a depth d* = exp(MLP + margin); only keys with depth <= d* are
 * sorted and blended.  A tile is final when every pixel stopped or has
 * T < t_thr, or when no record of a depth bin reaching beyond d* has a
 * support box covering it (so it has no held-out keys); otherwise it is
 * refuted and blending resumes over its held-out keys (possibly none) from
 * the stored per-pixel state.
 * With t_thr <= params->t_min the image equals ls_render_fwd's bit for bit;
 * with a larger t_thr each pixel is within t_thr (max rgb + bg) of it.
 * Outputs as ls_render_fwd (n_last continues into the held-out lists),
 * dstar_out [tiles] (or NULL), stats_dev [4] (int64, device, or NULL): keys
 * before truncation, kept keys, held-out keys sorted for refuted tiles,
 * refuted tiles (counting the keys before truncation walks the rows of
 * records that lie beyond every proposal of their box, which NULL skips).
 * key_capacity bounds both the kept and the held-out keys. */
size_t ls_render_learned_workspace(int32_t n, const ls_camera* cam, const ls_params* params, int64_t key_capacity);
ls_status ls_render_learned(int32_t n, const float* means, const float* scales, const float* quats,
                            const float* opacities, const float* sh, const ls_camera* cam, const ls_params* params,
                            const ls_mlp* mlp, float margin, const float* dstar_in, float t_thr, int64_t key_capacity,
                            float* image, float* t_final, int32_t* n_last, float* dstar_out, int64_t* stats_dev,
                            void* workspace, size_t ws_bytes, int32_t* status_dev, void* stream);

/* Workspace of ls_render_batch in bytes (projected records, keys, ranges,
 * job queue and the duplicate/sort scratch). */
size_t ls_render_batch_workspace(int32_t n, const ls_camera* cams, int32_t n_cams, const ls_params* params,
                                 int64_t key_capacity);

/* a7: forward render of n_cams cameras (1..LS_MAX_CAMS, sizes may differ)
 * in one pass: projection of all (camera, primitive) records, one shared
 * duplicate/sort over global tile ids, a queue of every (camera, tile) job
 * with the longest lists first, and one persistent blending launch whose
 * CTAs take jobs until the queue is empty.  Per pixel the result is exactly
 * ls_render_fwd's for that camera.  Parameters as ls_project; blend_batch =
 * records staged per shared-memory batch (16..1024, 0 = default).  Outputs:
 * images [sum_c H_c W_c][3] float, camera c's image starting at pixel
 * sum_{c'<c} H_c' W_c'; t_final (same pixel layout) or NULL; *n_keys_dev = K.
 * key_capacity and LS_ERR_CAPACITY as for ls_duplicate_sort.  Nothing in the
 * call synchronises with the host, so a caller can capture it in a CUDA graph
 * once the dynamic-shared-memory attributes are set (any earlier call). */
ls_status ls_render_batch(int32_t n, const float* means, const float* scales, const float* quats,
                          const float* opacities, const float* sh, const ls_camera* cams, int32_t n_cams,
                          const ls_params* params, int32_t blend_batch, int64_t key_capacity, float* images,
                          float* t_final, int64_t* n_keys_dev, void* workspace, size_t ws_bytes,
                          int32_t* status_dev, void* stream);

/* The blending stage of ls_render_batch alone (its job queue and persistent
 * blend), on what the last ls_render_batch call with the same workspace and
 * the same n, cams, n_cams, params and key_capacity left in the workspace
 * (projected records, sorted keys, tile ranges): the images equal that
 * call's.  For timing the stage by itself.  Arguments as ls_render_batch;
 * LS_ERR_INVALID_ARG for invalid ones or a short workspace. */
ls_status ls_render_batch_blend(int32_t n, const ls_camera* cams, int32_t n_cams, const ls_params* params,
                                int32_t blend_batch, int64_t key_capacity, float* images, float* t_final,
                                void* workspace, size_t ws_bytes, int32_t* status_dev, void* stream);

/* ls_duplicate_sort without a caller-supplied workspace, for callers that
 * cannot allocate device memory themselves: a plugin running inside a host
 * application that owns every device allocation, a real-time loop that must
 * not allocate, or a small C program that links only this library and keeps
 * no allocator of its own.  The paper has no counterpart; this is a packaging
 * choice.
 *
 * The scratch lives in one file-scope device array of LS_NOALLOC_SCRATCH_BYTES
 * that every GPU which loads the library holds until the process exits.  The
 * caller still passes (and owns) proj, keys, vals, n_keys_dev, tile_ranges and
 * status_dev, exactly as for ls_duplicate_sort, and gets the same results.
 * Limits: n_records <= LS_NOALLOC_MAX_RECORDS, key_capacity <=
 * LS_NOALLOC_MAX_KEYS, and the scratch that ls_duplicate_sort_workspace asks
 * for must fit the array; anything larger returns LS_ERR_UNSUPPORTED before
 * any work is enqueued.  Other argument errors are those of ls_duplicate_sort.
 * The first call on a device looks up the array's device address (once per
 * device, with that device current); make that first call before any stream
 * capture begins.  Every call uses the same array: the call clears what must
 * start at zero, and calls whose work overlaps on the GPU (other streams,
 * other threads) race on it, so serialise them.  No cudaMalloc or cudaFree,
 * and no allocating library routine, is called. */
#define LS_NOALLOC_MAX_RECORDS 65536
#define LS_NOALLOC_MAX_KEYS 524288
#define LS_NOALLOC_SCRATCH_BYTES (8u << 20)
ls_status ls_duplicate_sort_noalloc(int64_t n_records, const void* proj, const ls_camera* cams, int32_t n_cams,
                                    const ls_params* params, int64_t key_capacity, uint32_t* keys, uint32_t* vals,
                                    int64_t* n_keys_dev, int32_t* tile_ranges, int32_t* status_dev, void* stream);

/* Copy of `bytes` bytes from src to dst where each side is device memory or
 * host memory pinned through the CUDA runtime (cudaHostAlloc /
 * cudaHostRegister), in either direction, on the copy engines.  For the
 * host<->device moves of an end-to-end step.  LS_ERR_INVALID_ARG when a
 * pointer is NULL or not device-addressable (pageable host memory): nothing
 * is enqueued. */
ls_status ls_copy(void* dst, const void* src, size_t bytes, void* stream);

/* Throughput probe of dependent-free FP32 FMAs (the denominator of the
 * blending rooflines, checked by measurement): blocks_per_sm x SMs blocks of
 * 256 threads, each running `iters` rounds of eight independent FMA chains.
 * *lane_ops (host) receives the FP32 lane instructions the launch executes;
 * time it with events on `stream`.  out: one float of device memory (written
 * only to keep the chains live). */
ls_status ls_fp32_issue_probe(int64_t iters, int32_t blocks_per_sm, float* out, int64_t* lane_ops, void* stream);

/* ---- training-side consumers of the backward ---------------------------
 * Image loss of the appendix "Loss Functions": L = w_l1 L1 + w_l2 L2 +
 * w_ssim (1 - SSIM) of a rendered image pred and a target, both [H][W][3]
 * float (the paper's weights are 0.6, 0.2, 0.2).  L1 and L2 are means over
 * the H W 3 values; SSIM (only named by the paper) is read as 3DGS computes
 * it: per channel, 11 x 11 Gaussian window of standard deviation 1.5 (taps
 * normalised to sum 1), zero outside the image, C1 = 0.01^2, C2 = 0.03^2,
 * averaged over pixels and channels.  loss_dev [4] (device) receives total,
 * L1, L2 and SSIM; grad (device [H][W][3], or NULL) is OVERWRITTEN with
 * dL/dpred (the L1 term's derivative at a zero difference taken as 0).
 * workspace: ls_image_loss_workspace bytes, 256-byte aligned.  Deterministic
 * (fixed reduction order).  LS_ERR_INVALID_ARG for sizes outside 1..16384,
 * NULL inputs, non-finite weights or a short workspace. */
size_t ls_image_loss_workspace(int32_t height, int32_t width);
ls_status ls_image_loss(int32_t height, int32_t width, const float* pred, const float* target, float w_l1,
                        float w_l2, float w_ssim, float* loss_dev, float* grad, void* workspace, size_t ws_bytes,
                        void* stream);

/* One bias-corrected Adam step (step >= 1) of n parameters in place, with
 * first and second moments m1, m2 (device, n floats each, zero before step
 * 1), in the parameter's unconstrained space: mode 0 the value itself, 1 its
 * log (for positive values such as scales; the gradient is taken times p),
 * 2 its logit (for values in (0, 1) such as opacities; times p (1 - p)).
 * The optimiser of the pattern fits (Sec. 5.1).  LS_ERR_INVALID_ARG for a
 * bad step, mode, rate or NULL pointer. */
ls_status ls_adam(int64_t n, float* param, const float* grad, float* m1, float* m2, int32_t step, float lr,
                  float beta1, float beta2, float eps, int32_t mode, void* stream);

/* Densification statistics, the thresholds of the appendix's densification
 * table (3DLS row in brackets).  The paper builds on gsplat v1.3 and gives
 * only the six values; they are read as that library's default strategy
 * applies them:
 *   ls_densify_accumulate, after each backward of one view: every primitive
 *   whose support box meets the image adds the norm of its screen-mean
 *   gradient in normalised device units, |(g_mx W/2 n_cams, g_my H/2
 *   n_cams)|, to grad_accum [n], adds 1 to count [n] and raises max_radius
 *   [n] to max(ex, ey) / max(W, H).  g2d [n][12] as ls_render_bwd's g2d_out
 *   (g_mx, g_my first), proj the view's records (n_cams = 1 at projection;
 *   n_cams here is the number of views averaged into one step's loss).
 *   ACCUMULATED (zero the three arrays at a refinement step).
 *   ls_densify_decide, at a refinement step, with g = grad_accum / max(count,
 *   1) and s = the largest of a primitive's three scales: flags [n] (uint8)
 *   bit 0 duplicate (g > grad2d and s <= grow_scale3d * extent), bit 1 split
 *   (g > grad2d and s above it, or max_radius > grow_scale2d when
 *   use_scale2d), bit 2 prune (opacity < prune_opacity, or s >
 *   prune_scale3d * extent when use_prune_scale3d, or max_radius >
 *   prune_scale2d when use_scale2d); counts_dev [3] (int64, device, or NULL)
 *   receives how many primitives carry each bit.  Binary32, every operation
 *   rounded once (decisions reproducible bit for bit). */
typedef struct {
  float grad2d;              /* [0.0002] */
  float grow_scale2d;        /* [0.05] */
  float grow_scale3d;        /* times the scene extent [0.006] */
  float prune_scale2d;       /* [0.15] */
  float prune_scale3d;       /* times the scene extent [0.4] */
  float prune_opacity;       /* [0.025] */
  int32_t use_scale2d;       /* the two 2D-radius rules [0] */
  int32_t use_prune_scale3d; /* the 3D-scale prune [0] */
} ls_densify_params;
ls_status ls_densify_accumulate(int32_t n, const float* g2d, const void* proj, const ls_camera* cam, int32_t n_cams,
                                float* grad_accum, int32_t* count, float* max_radius, void* stream);
ls_status ls_densify_decide(int32_t n, const float* grad_accum, const int32_t* count, const float* max_radius,
                            const float* scales, const float* opacities, float scene_extent,
                            const ls_densify_params* params, uint8_t* flags, int64_t* counts_dev, void* stream);

/* ---- 3D smoothing filter of the anti-aliased variant ---------------------
 * Sec. 4.1 evaluates 3DLS+AA with the anti-aliasing of Mip-Splatting; its
 * 2D filter is ls_params.antialias.  Its 3D filter, read (the paper gives no
 * formula): each primitive's highest sampling rate over the training cameras
 * that see its centre, nu = max fx / z (camera depth z > near_plane, the
 * projected centre within 1.15x the image: x in [-0.15 W, 1.15 W], y in
 * [-0.15 H, 1.15 H]), bounds its frequency; the variance v = s2 / nu^2
 * (s2 = 0.2 in Mip-Splatting) is added to all three axes.
 *   ls_filter3d_variance: filter_var [n] from means [n][3] and the cameras
 *     (host array, 1..LS_MAX_CAMS); a primitive no camera sees takes the
 *     largest v of the others (0 when none is seen).  workspace:
 *     ls_filter3d_workspace() bytes of device scratch, 256-byte aligned.
 *   ls_filter3d_apply: scales_out = sqrt(scales^2 + v) per axis and
 *     opacities_out = o prod_k scales_k / scales_out_k (keeps o sqrt(det
 *     Sigma)); feed them to ls_project.
 *   ls_filter3d_apply_bwd: gradients with respect to the unfiltered scales
 *     and opacities from those of the filtered ones (OVERWRITTEN). */
size_t ls_filter3d_workspace(void);
ls_status ls_filter3d_variance(int32_t n, const float* means, const ls_camera* cams, int32_t n_cams, float near_plane,
                               float s2, float* filter_var, void* workspace, size_t ws_bytes, void* stream);
ls_status ls_filter3d_apply(int32_t n, const float* scales, const float* opacities, const float* filter_var,
                            float* scales_out, float* opacities_out, void* stream);
ls_status ls_filter3d_apply_bwd(int32_t n, const float* scales, const float* opacities, const float* filter_var,
                                const float* g_scales_out, const float* g_opacities_out, float* g_scales,
                                float* g_opacities, void* stream);

/* For tests of failure detection: the onesweep radix sort's look-back waits
 * on its predecessor partitions, each wait bounded by spin_limit polls (0
 * restores the default, about a second); after that it writes
 * LS_ERR_TIMEOUT to status_dev and the pass finishes with in-bounds writes
 * (its output order is then unspecified).  hold_partition >= 0 makes that
 * partition of the last pass of every tile sort publish nothing, so the
 * wait of the partition after it runs out on purpose; -1 turns that off.
 * Process-wide, not thread-safe; LS_ERR_INVALID_ARG for spin_limit < 0 or
 * hold_partition < -1. */
ls_status ls_debug_set_sort_wait(int32_t spin_limit, int32_t hold_partition);

/* Launch mode of the kernels of a frame (ls_project, ls_duplicate_sort,
 * ls_render_fwd, ls_render_bwd and their parts): on = 1 (the default) lets
 * each kernel be scheduled while the one before it in the stream finishes
 * (programmatic dependent launch; each kernel still waits for its
 * predecessor's results before it reads or writes anything), except while
 * the stream is being captured into a CUDA graph, where launches stay plain;
 * on = 0 launches them plainly always.  Results are the same either way.
 * Process-wide, not thread-safe; LS_ERR_INVALID_ARG for other values of
 * on. */
ls_status ls_set_dependent_launch(int32_t on);

/* Text of a status code (static storage). */
const char* ls_status_string(int32_t status);

/* ABI version, bumped on any incompatible change. */
int32_t ls_version(void);

#ifdef __cplusplus
}
#endif

#endif /* LS_H_ */
