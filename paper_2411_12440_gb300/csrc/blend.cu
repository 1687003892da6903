// a4 / a5: per-tile front-to-back blending with the linear kernel and its
// adjoint (Sec. 3.1 Eq. 6; kernel of Sec. 3.2 Eq. 11 with the alignment of
// Sec. 3.3.1 Eq. 12; adaptive gradient scaling of Sec. 3.3.2 Eq. 13-14).
//
// One CTA per tile; each thread owns PPT pixels of one row, tile_w / PPT
// apart, so one shared-memory read of a record serves PPT pixels and the
// per-record terms that depend only on the row (dy, l01 dy, l11 dy) are
// computed once.  A warp's p-th pixels then form a compact block (8 x 4 for
// 16 x 16 tiles at 4 pixels per thread, 4 x 8 at 2), so the per-pixel work,
// which runs once per p for the lanes whose p-th pixel takes the record,
// wastes fewer lanes than with contiguous strips (whose p-th pixels are PPT
// columns apart).  Both passes run 4 pixels per thread on 16 x 16 tiles (64
// threads), 2 on 8 x 8 (one warp).
// The tile's sorted record ids are walked in batches: the threads gather the
// batch's 48-byte records into shared memory (each record is fetched from
// L2/HBM once per tile), then every thread reads them as broadcasts.
//
// Backward: each pixel restarts from its checkpoint (T_final, n_last) and
// walks its list back to front, recovering T before each entry as
// T / (1 - alpha).  The per-pixel adjoint is predicated (a pixel slot that
// some lane of the warp takes runs as one straight line for every lane), and
// the AGS reading is a template argument, not a branch per pair.  Each
// thread first sums its pixels' nine gradient terms; a warp with any
// contributing pixel then reduce-scatters the nine sums
// (14 shuffles instead of 45: eight values end in eight lane groups), those
// lanes add into a per-CTA shared-memory slot, and after the batch one set of
// float4 atomics per (record, CTA) lands in global memory.
#include "kernels.h"

namespace ls {

namespace {

__device__ __forceinline__ float sqrt_approx(float x) {
  float y;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// The squared Mahalanobis distance of pixel (x, y) to record (a, bb), with
// every rounding explicit so that the forward and the backward compute the
// same bits.  The conic is stored as its upper Cholesky factor L (A = L^T L),
// so q = |L d|^2 = (l00 dx + l01 dy)^2 + (l11 dy)^2 is a sum of squares: no
// cancellation even for needle-shaped footprints.  Row terms (depending on y
// only) are passed in: l01dy = l01 dy, e2s = (l11 dy)^2.
__device__ __forceinline__ float pair_q(float x, float mx, float l00, float l01dy, float e2s, float& dx, float& e1) {
  dx = __fsub_rn(x, mx);
  e1 = __fmaf_rn(l00, dx, l01dy);
  return __fmaf_rn(e1, e1, e2s);
}

__device__ __forceinline__ float rsqrt_approx(float x) {
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// alpha of a pair inside the support: min(alpha_max, o f(D / lambda)).  The
// linear profile is one fused 1 - D / lambda: inside the support
// D / lambda <= x_s < 1, so its clamp at 0 never acts on a pair that is
// composited (a pair just past the support by rounding gets f <= 0 and is
// skipped as alpha < alpha_min).
template <int KID>
__device__ __forceinline__ void pair_alpha(float q, float o, const ParDev& P, float& D, float& xk, float& f,
                                           float& araw, float& alpha) {
  D = sqrt_approx(q);
  xk = __fmul_rn(D, P.inv_lambda);
  f = KID == LS_KERNEL_LINEAR ? __fmaf_rn(-D, P.inv_lambda, 1.f) : kern_f<KID>(xk);
  araw = __fmul_rn(o, f);
  alpha = fminf(P.alpha_max, araw);
}

// Where a tile lives: pixel origin, image size, its key range, and the base of
// its camera's image in the output arrays.
struct TileJob {
  int x0, y0, W, H;
  int2 rg;
  size_t pix_base;
};


// ---------------------------------------------------------------- forward
// Modes of the per-tile forward:
//   FWD_PLAIN   one pass over the tile's list;
//   FWD_TRUNC   the list holds only the keys in front of a proposed depth; a
//               tile whose pixels are not all settled afterwards (stopped, or
//               T < t_thr) and that has held-out keys is refuted: it stores
//               its raw per-pixel state (C without background, T with the
//               sign bit marking a stopped pixel, n_last) and is flagged;
//   FWD_RESUME  a refuted tile continues over its held-out list (the rest of
//               the same front-to-back list) from that state, so the result is
//               the plain one bit for bit.
enum { FWD_PLAIN = 0, FWD_TRUNC = 1, FWD_RESUME = 2 };

template <int KID, int PPT, bool COUNT, int MODE>
__device__ __forceinline__ void fwd_tile(const float4* __restrict__ rec, const uint32_t* __restrict__ vals,
                                         const ParDev& P, const TileJob& J, float4* s_a, float4* s_b, float4* s_c,
                                         int B, float* __restrict__ image, float* __restrict__ t_final,
                                         int32_t* __restrict__ n_last, unsigned long long* stats,
                                         const TruncArgs& ta, int tile_gid) {
  const int sx = P.tile_w / PPT;
  const int lr = (int)threadIdx.x / sx, lc = (int)threadIdx.x % sx;
  const int py = J.y0 + lr, px0 = J.x0 + lc;
  const float y = (float)py + 0.5f;
  float xs[PPT], T[PPT], C0[PPT], C1[PPT], C2[PPT];
  int last[PPT], stop[PPT], comp[PPT];
  unsigned done = 0;
  int ofs = 0;  // FWD_RESUME: entries of the tile already composited (kept list)
  if (MODE == FWD_RESUME) ofs = ta.kept_ranges[tile_gid].y - ta.kept_ranges[tile_gid].x;
#pragma unroll
  for (int p = 0; p < PPT; ++p) {
    xs[p] = (float)(px0 + p * sx) + 0.5f;
    T[p] = 1.f;
    C0[p] = C1[p] = C2[p] = 0.f;
    last[p] = 0;
    comp[p] = 0;
    const bool inside = px0 + p * sx < J.W && py < J.H;
    // a pixel that is done sits at x = +inf: its q is +inf, above every
    // support, so the support test alone skips it
    if (!inside) {
      done |= 1u << p;
      xs[p] = __int_as_float(0x7F800000);
    }
    if (MODE == FWD_RESUME && inside) {
      const size_t pi = J.pix_base + (size_t)py * J.W + px0 + p * sx;
      C0[p] = image[3 * pi];
      C1[p] = image[3 * pi + 1];
      C2[p] = image[3 * pi + 2];
      const float tv = t_final[pi];
      T[p] = fabsf(tv);
      if (signbit(tv)) {
        done |= 1u << p;
        xs[p] = __int_as_float(0x7F800000);
      }
      last[p] = n_last[pi];
    }
  }
  const unsigned all = (1u << PPT) - 1u;
  const int n = J.rg.y - J.rg.x;
#pragma unroll
  for (int p = 0; p < PPT; ++p) stop[p] = n;
  for (int b0 = 0; b0 < n; b0 += B) {
    if (__syncthreads_and(done == all)) break;
    const int cnt = min(B, n - b0);
    for (int k = threadIdx.x; k < cnt; k += blockDim.x) {
      const uint32_t id = vals[J.rg.x + b0 + k];
      s_a[k] = rec[3 * (size_t)id];
      s_b[k] = rec[3 * (size_t)id + 1];
      s_c[k] = rec[3 * (size_t)id + 2];
    }
    __syncthreads();
    if (done != all) {
      for (int j = 0; j < cnt; ++j) {
        const float4 a = s_a[j];   // {mx, my, l00, l01}
        const float4 bb = s_b[j];  // {l11, o, rho2, depth}
        const float dy = __fsub_rn(y, a.y);
        const float l01dy = __fmul_rn(a.w, dy);
        const float e2 = __fmul_rn(bb.x, dy);
        const float e2s = __fmul_rn(e2, e2);
        // q = fma(e1, e1, e2s) >= e2s for every pixel of the row: all of the
        // thread's pixels are outside the support when the row term alone is
        if (e2s > bb.z) continue;
#pragma unroll
        for (int p = 0; p < PPT; ++p) {
          float dx, e1;
          const float q = pair_q(xs[p], a.x, a.z, l01dy, e2s, dx, e1);
          if (q > bb.z) continue;  // outside the support, or the pixel is done
          float D, xk, f, araw, alpha;
          pair_alpha<KID>(q, bb.y, P, D, xk, f, araw, alpha);
          if (alpha < P.alpha_min) continue;
          const float Tn = T[p] * (1.f - alpha);
          if (Tn < P.t_min) {
            done |= 1u << p;
            xs[p] = __int_as_float(0x7F800000);
            if (COUNT) stop[p] = b0 + j;
            continue;
          }
          const float4 c = s_c[j];
          const float w = alpha * T[p];
          C0[p] += c.x * w;
          C1[p] += c.y * w;
          C2[p] += c.z * w;
          T[p] = Tn;
          last[p] = ofs + b0 + j + 1;
          if (COUNT) ++comp[p];
        }
        if (done == all) break;
      }
    }
  }
  bool raw = false;  // FWD_TRUNC: store the state instead of the final colour
  if (MODE == FWD_TRUNC) {
    bool settled = true;
#pragma unroll
    for (int p = 0; p < PPT; ++p) settled = settled && (((done >> p) & 1u) || T[p] < ta.t_thr);
    const bool all_settled = __syncthreads_and(settled);
    raw = !all_settled && ta.has_held[tile_gid];
    if (raw && threadIdx.x == 0) {
      ta.refuted[tile_gid] = 1;
      atomicAdd(ta.n_refuted, 1u);
      atomicMax(ta.refuted_floor, ~ta.dstar_bits[tile_gid]);
    }
  }
#pragma unroll
  for (int p = 0; p < PPT; ++p) {
    if (px0 + p * sx < J.W && py < J.H) {
      const size_t pi = J.pix_base + (size_t)py * J.W + px0 + p * sx;
      if (raw) {
        image[3 * pi] = C0[p];
        image[3 * pi + 1] = C1[p];
        image[3 * pi + 2] = C2[p];
        t_final[pi] = ((done >> p) & 1u) ? -T[p] : T[p];
        n_last[pi] = last[p];
        continue;
      }
      image[3 * pi] = C0[p] + T[p] * P.bg[0];
      image[3 * pi + 1] = C1[p] + T[p] * P.bg[1];
      image[3 * pi + 2] = C2[p] + T[p] * P.bg[2];
      if (t_final) t_final[pi] = T[p];
      if (n_last) n_last[pi] = last[p];
    }
  }
  if (COUNT) {
    __shared__ int s_emax, s_npix;
    __shared__ unsigned long long s_contrib;
    __syncthreads();
    if (threadIdx.x == 0) {
      s_emax = 0;
      s_npix = 0;
      s_contrib = 0;
    }
    __syncthreads();
    int emax = 0, npix = 0, cc = 0;
#pragma unroll
    for (int p = 0; p < PPT; ++p) {
      if (px0 + p * sx < J.W && py < J.H) {
        emax = max(emax, stop[p] < n ? stop[p] + 1 : n);
        ++npix;
        cc += comp[p];
      }
    }
    int never = 0;  // a pixel that never stopped
#pragma unroll
    for (int p = 0; p < PPT; ++p)
      if (px0 + p * sx < J.W && py < J.H && stop[p] >= n) never = 1;
    atomicMax(&s_emax, emax);
    atomicAdd(&s_npix, npix);
    atomicAdd(&s_contrib, (unsigned long long)cc);
    const int any_never = __syncthreads_or(never);
    if (threadIdx.x == 0) {
      atomicAdd(&stats[0], (unsigned long long)s_emax * (unsigned long long)s_npix);
      atomicAdd(&stats[1], s_contrib);
      if (ta.labels) {
        // termination depth: depth of the entry at which the tile's last pixel
        // stopped; +inf when some pixel never stops; 0 for an empty tile
        float lab = 0.f;
        if (any_never && n > 0) lab = __int_as_float(0x7F800000);
        else if (s_npix > 0 && s_emax > 0) lab = rec[3 * (size_t)vals[J.rg.x + s_emax - 1] + 1].w;
        ta.labels[tile_gid] = lab;
      }
    }
  }
}

template <int KID, int PPT, bool COUNT>
__global__ void __launch_bounds__(128) blend_fwd_kernel(const float4* __restrict__ rec, const CamDev cam,
                                                        const ParDev P, const int2* __restrict__ ranges,
                                                        const uint32_t* __restrict__ vals, float* __restrict__ image,
                                                        float* __restrict__ t_final, int32_t* __restrict__ n_last,
                                                        unsigned long long* stats, const TruncArgs ta) {
  chain_enter();
  extern __shared__ float4 smem[];
  // two records per thread per batch: tiles of dense scenes stop within a
  // few hundred entries, and a smaller batch gathers fewer records that no
  // pixel reads (measured 5 % faster than four per thread)
  const int B = 2 * blockDim.x;
  const int tile = blockIdx.x;
  TileJob J;
  J.x0 = (tile % cam.tiles_x) * P.tile_w;
  J.y0 = (tile / cam.tiles_x) * P.tile_h;
  J.W = cam.W;
  J.H = cam.H;
  J.rg = ranges[cam.tile_base + tile];
  J.pix_base = 0;
  fwd_tile<KID, PPT, COUNT, FWD_PLAIN>(rec, vals, P, J, smem, smem + B, smem + 2 * B, B, image, t_final, n_last,
                                       stats, ta, cam.tile_base + tile);
}

// Truncated (MODE 1) and resumed (MODE 2) forwards of one camera; a resume
// CTA whose tile was not refuted returns at once.
template <int KID, int PPT, int MODE>
__global__ void __launch_bounds__(128) blend_trunc_kernel(const float4* __restrict__ rec, const CamDev cam,
                                                          const ParDev P, const int2* __restrict__ ranges,
                                                          const uint32_t* __restrict__ vals, float* __restrict__ image,
                                                          float* __restrict__ t_final, int32_t* __restrict__ n_last,
                                                          const TruncArgs ta) {
  extern __shared__ float4 smem[];
  const int B = 2 * blockDim.x;
  const int tile = blockIdx.x;
  if (MODE == FWD_RESUME && !ta.refuted[tile]) return;
  TileJob J;
  J.x0 = (tile % cam.tiles_x) * P.tile_w;
  J.y0 = (tile / cam.tiles_x) * P.tile_h;
  J.W = cam.W;
  J.H = cam.H;
  J.rg = ranges[tile];
  J.pix_base = 0;
  fwd_tile<KID, PPT, false, MODE>(rec, vals, P, J, smem, smem + B, smem + 2 * B, B, image, t_final, n_last, nullptr, ta,
                                  tile);
}

// ---------------------------------------------------------------- backward
// Reduce-scatter of nine per-lane values over a warp.  Afterwards the warp
// sum of value (lane >> 2) & 7 is in `mine` of every lane, and the sum of
// v[8] in `ninth` of every lane.
__device__ __forceinline__ void warp_reduce9(const float v[9], float& mine, float& ninth) {
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const bool b4 = lane & 16, b3 = lane & 8, b2 = lane & 4;
  float w4[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const float send = b4 ? v[i] : v[i + 4];
    const float keep = b4 ? v[i + 4] : v[i];
    w4[i] = keep + __shfl_xor_sync(FULL, send, 16);
  }
  float w2[2];
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const float send = b3 ? w4[i] : w4[i + 2];
    const float keep = b3 ? w4[i + 2] : w4[i];
    w2[i] = keep + __shfl_xor_sync(FULL, send, 8);
  }
  {
    const float send = b2 ? w2[0] : w2[1];
    const float keep = b2 ? w2[1] : w2[0];
    mine = keep + __shfl_xor_sync(FULL, send, 4);
  }
  mine += __shfl_xor_sync(FULL, mine, 2);
  mine += __shfl_xor_sync(FULL, mine, 1);
  float u = v[8];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) u += __shfl_xor_sync(FULL, u, o);
  ninth = u;
}

// One thread owns RPT rows x PPR pixels of a tile: rows lr + r sy, columns
// lc + c sx (sx = tile_w / PPR threads across, sy = tile_h / RPT down), so
// that the p-th pixels of a warp form a compact block.
template <int KID, int AGS, int PPR, int RPT>
__device__ __forceinline__ void bwd_tile(const float4* __restrict__ rec, const uint32_t* __restrict__ vals,
                                         const ParDev& P, const TileJob& J, float4* s_a, float4* s_b, float4* s_c,
                                         float* s_acc, uint32_t* s_id, int* s_touch, int* s_max, int B,
                                         const float* __restrict__ t_final, const int32_t* __restrict__ n_last,
                                         const float* __restrict__ grad_image, const float* __restrict__ grad_t,
                                         float* __restrict__ g2d) {
  constexpr int NPX = PPR * RPT;
  const unsigned FULL = 0xffffffffu;
  const int sx = P.tile_w / PPR, sy = P.tile_h / RPT;
  const int lr = (int)threadIdx.x / sx, lc = (int)threadIdx.x % sx;
  const int px0 = J.x0 + lc, py0 = J.y0 + lr;
  const int lane = threadIdx.x & 31;
  // GS = dL/dC . S + dL/dT_final T_final, where S is the colour composited
  // behind the current entry (background included): the part of dL/dalpha
  // that the entries behind contribute, kept as one running scalar
  float T[NPX], gC0[NPX], gC1[NPX], gC2[NPX], GS[NPX];
  int last[NPX];
  int row_max[RPT];
  float xs[PPR], ys[RPT];
#pragma unroll
  for (int c = 0; c < PPR; ++c) xs[c] = (float)(px0 + c * sx) + 0.5f;
#pragma unroll
  for (int r = 0; r < RPT; ++r) ys[r] = (float)(py0 + r * sy) + 0.5f;
  int my_max = 0;
#pragma unroll
  for (int r = 0; r < RPT; ++r) {
    row_max[r] = 0;
#pragma unroll
    for (int c = 0; c < PPR; ++c) {
      const int p = r * PPR + c;
      const int px = px0 + c * sx, py = py0 + r * sy;
      T[p] = 1.f;
      float Tf = 1.f, gTT = 0.f;
      gC0[p] = gC1[p] = gC2[p] = 0.f;
      last[p] = 0;
      if (px < J.W && py < J.H) {
        const size_t pi = J.pix_base + (size_t)py * J.W + px;
        T[p] = Tf = t_final[pi];
        last[p] = n_last[pi];
        gC0[p] = grad_image[3 * pi];
        gC1[p] = grad_image[3 * pi + 1];
        gC2[p] = grad_image[3 * pi + 2];
        gTT = grad_t ? grad_t[pi] * Tf : 0.f;  // dL/dT_final times T_final
      }
      GS[p] = (gC0[p] * P.bg[0] + gC1[p] * P.bg[1] + gC2[p] * P.bg[2]) * Tf + gTT;
      row_max[r] = max(row_max[r], last[p]);
    }
    my_max = max(my_max, row_max[r]);
  }
  if (threadIdx.x == 0) *s_max = 0;
  __syncthreads();
  if (my_max > 0) atomicMax(s_max, my_max);
  __syncthreads();
  const int max_last = *s_max;
  const int warp_max = __reduce_max_sync(FULL, my_max);  // entries at or past it touch none of the warp's pixels

  for (int b_end = max_last; b_end > 0; b_end -= B) {
    const int b0 = max(0, b_end - B);
    const int cnt = b_end - b0;
    __syncthreads();  // previous batch flushed
    for (int k = threadIdx.x; k < cnt; k += blockDim.x) {
      const uint32_t id = vals[J.rg.x + b0 + k];
      s_id[k] = id;
      s_a[k] = rec[3 * (size_t)id];
      s_b[k] = rec[3 * (size_t)id + 1];
      s_c[k] = rec[3 * (size_t)id + 2];
      s_touch[k] = 0;
#pragma unroll
      for (int m = 0; m < 9; ++m) s_acc[9 * k + m] = 0.f;
    }
    __syncthreads();
    for (int jj = min(cnt, warp_max - b0) - 1; jj >= 0; --jj) {
      const int j = b0 + jj;
      const float4 a = s_a[jj];   // {mx, my, l00, l01}
      const float4 bb = s_b[jj];  // {l11, o, rho2, depth}
      // row terms: dy, l01 dy and (l11 dy)^2 for each of the thread's rows;
      // q >= (l11 dy)^2, so a row whose term alone exceeds rho^2 takes nothing
      float dy[RPT], l01dy[RPT], e2[RPT], e2s[RPT];
      bool row_in[RPT];
      bool any_row = false;
#pragma unroll
      for (int r = 0; r < RPT; ++r) {
        dy[r] = __fsub_rn(ys[r], a.y);
        l01dy[r] = __fmul_rn(a.w, dy[r]);
        e2[r] = __fmul_rn(bb.x, dy[r]);
        e2s[r] = __fmul_rn(e2[r], e2[r]);
        row_in[r] = e2s[r] <= bb.z && j < row_max[r];
        any_row = any_row || row_in[r];
      }
      if (!__any_sync(FULL, any_row)) continue;  // nothing for the warp
      // per-thread sums: the geometric terms are gathered as sums over the
      // thread's pixels of gq e1, gq dx, gq dx^2 and, per row, gq and gq dx
      // (dy and l11 dy are the same along a row) and expanded once below
      float s_e1 = 0.f, s_dx2 = 0.f, v5 = 0.f, v6 = 0.f, v7 = 0.f, v8 = 0.f;
      float s_q[RPT], s_dx[RPT];
      bool any = false;
      const float kq = (KID == LS_KERNEL_LINEAR ? -0.5f : 0.5f) * bb.y * P.inv_lambda;
      // The per-pixel work is predicated rather than branched: once any lane
      // of the warp takes pixel slot p, every lane runs the same straight
      // line and a lane that does not take it contributes zeros.
#pragma unroll
      for (int r = 0; r < RPT; ++r) {
        s_q[r] = 0.f;
        s_dx[r] = 0.f;
#pragma unroll
        for (int c = 0; c < PPR; ++c) {
          const int p = r * PPR + c;
          float dx, e1;
          const float q = pair_q(xs[c], a.x, a.z, l01dy[r], e2s[r], dx, e1);
          bool take = row_in[r] && j < last[p] && q <= bb.z;
          if (!__any_sync(FULL, take)) continue;  // warp-uniform
          // a lane outside the support runs on finite stand-ins (q = 0 and
          // e1 = 0; dx is a difference of two finite coordinates), so that
          // its zero weights never meet an infinity
          const float qa = take ? q : 0.f;
          e1 = take ? e1 : 0.f;
          float D, xk, f, araw, alpha;
          pair_alpha<KID>(qa, bb.y, P, D, xk, f, araw, alpha);
          take = take && alpha >= P.alpha_min;
          any = any || take;
          const float4 cc = s_c[jj];
          // a lane that does not take the pair passes through it with alpha
          // 0: its reciprocal is exactly 1 (the approximate reciprocal is
          // exact at powers of two), so T and the weights need no select
          const float at = take ? alpha : 0.f;
          const float iom = __fdividef(1.f, 1.f - at);  // 1 - alpha >= 1 - alpha_max
          const float Tb = T[p] * iom;  // transmittance in front of this entry
          const float wgt = at * Tb;
          v6 += wgt * gC0[p];
          v7 += wgt * gC1[p];
          v8 += wgt * gC2[p];
          // dL/dalpha = Tb dL/dC . c - (dL/dC . S + dL/dT_final T_final) / (1 - alpha)
          const float gcd = gC0[p] * cc.x + gC1[p] * cc.y + gC2[p] * cc.z;
          const float ga = Tb * gcd - iom * GS[p];
          GS[p] += wgt * gcd;
          T[p] = Tb;
          // a clamped alpha passes no gradient to o or D
          const float gat = (take && araw <= P.alpha_max) ? ga : 0.f;
          v5 += f * gat;
          // dL/dq = dL/dalpha o f'(x) / (lambda 2 D); the record's factor
          // o / (2 lambda) (and the linear profile's slope, -1 wherever
          // alpha > 0) multiplies the sums once per entry, below.  1 / D from
          // rsqrt(max(q, FLT_MIN)): exact where q is a normal number, and at
          // the mean (q = 0) the huge gq meets dx = dy = e1 = 0
          float gD = KID == LS_KERNEL_LINEAR ? gat : gat * kern_df<KID>(xk);
          if (AGS == 1) gD *= __expf(-D * D);
          else if (AGS == 2) gD *= __expf(-xk * xk);
          const float gq = gD * rsqrt_approx(fmaxf(qa, 1.17549435e-38f));
          const float gdx = gq * dx;
          s_e1 += gq * e1;
          s_dx[r] += gdx;
          s_dx2 += gdx * dx;
          s_q[r] += gq;
        }
      }
      const unsigned bal = __ballot_sync(FULL, any);
      if (bal == 0u) continue;
      // A d = L^T (L d) = (l00 e1, l01 e1 + l11 e2): the conic-space mean
      // gradient and the conic-entry gradients (b counted once)
      float v[9];
      float t1 = a.w * s_e1, t3 = 0.f, t4 = 0.f;
#pragma unroll
      for (int r = 0; r < RPT; ++r) {
        t1 += bb.x * e2[r] * s_q[r];
        t3 += dy[r] * s_dx[r];
        t4 += dy[r] * dy[r] * s_q[r];
      }
      v[0] = -2.f * kq * a.z * s_e1;
      v[1] = -2.f * kq * t1;
      v[2] = kq * s_dx2;
      v[3] = 2.f * kq * t3;
      v[4] = kq * t4;
      v[5] = v5;
      v[6] = v6;
      v[7] = v7;
      v[8] = v8;
      if (__popc(bal) == 1) {
        if (any) {
#pragma unroll
          for (int m = 0; m < 9; ++m) atomicAdd(&s_acc[9 * jj + m], v[m]);
          s_touch[jj] = 1;
        }
      } else {
        float mine, ninth;
        warp_reduce9(v, mine, ninth);
        if ((lane & 3) == 0) atomicAdd(&s_acc[9 * jj + (lane >> 2)], mine);
        if (lane == 1) {
          atomicAdd(&s_acc[9 * jj + 8], ninth);
          s_touch[jj] = 1;
        }
      }
    }
    __syncthreads();
    for (int k = threadIdx.x; k < cnt; k += blockDim.x) {
      if (!s_touch[k]) continue;
      const float* acc = s_acc + 9 * k;
      float* dst = g2d + 12 * (size_t)s_id[k];
      atomicAdd(reinterpret_cast<float4*>(dst), make_float4(acc[0], acc[1], acc[2], acc[3]));
      atomicAdd(reinterpret_cast<float4*>(dst + 4), make_float4(acc[4], acc[5], acc[6], acc[7]));
      atomicAdd(dst + 8, acc[8]);
    }
  }
}

template <int KID, int AGS, int PPR, int RPT>
__global__ void __launch_bounds__(128) blend_bwd_kernel(const float4* __restrict__ rec, const CamDev cam,
                                                        const ParDev P, const int2* __restrict__ ranges,
                                                        const uint32_t* __restrict__ vals,
                                                        const float* __restrict__ t_final,
                                                        const int32_t* __restrict__ n_last,
                                                        const float* __restrict__ grad_image,
                                                        const float* __restrict__ grad_t, float* __restrict__ g2d,
                                                        int B, const uint32_t* __restrict__ order) {
  chain_enter();
  extern __shared__ float4 smem[];
  __shared__ int s_max;
  float* s_acc = reinterpret_cast<float*>(smem + 3 * B);
  uint32_t* s_id = reinterpret_cast<uint32_t*>(s_acc + 9 * B);
  int* s_touch = reinterpret_cast<int*>(s_id + B);
  const int tile = order ? (int)order[blockIdx.x] : (int)blockIdx.x;
  TileJob J;
  J.x0 = (tile % cam.tiles_x) * P.tile_w;
  J.y0 = (tile / cam.tiles_x) * P.tile_h;
  J.W = cam.W;
  J.H = cam.H;
  J.rg = ranges[cam.tile_base + tile];
  J.pix_base = 0;
  bwd_tile<KID, AGS, PPR, RPT>(rec, vals, P, J, smem, smem + B, smem + 2 * B, s_acc, s_id, s_touch, &s_max, B, t_final,
                          n_last, grad_image, grad_t, g2d);
}

// ---------------------------------------------------------------- tile order
// Bucket of a tile's work m (its largest n_last): 0 for none, else
// 1 + 4 floor(log2 m) + the next two bits of m (quarter-octaves, 1..128).
__device__ __forceinline__ int work_bucket(uint32_t m) {
  if (m == 0) return 0;
  const int l = 31 - __clz(m);
  const int f = l >= 2 ? (int)((m >> (l - 2)) & 3u) : (int)((m << (2 - l)) & 3u);
  return 1 + 4 * l + f;
}

// One warp per tile: the largest n_last over its pixels, bucketed.
__global__ void __launch_bounds__(256) tile_work_kernel(const int32_t* __restrict__ n_last, const CamDev cam, int tw,
                                                        int th, unsigned* hist, uint32_t* bkt) {
  chain_enter();
  const int tiles = cam.tiles_x * cam.tiles_y;
  const int t = (int)blockIdx.x * 8 + ((int)threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (t >= tiles) return;  // warp-uniform
  const int x0 = (t % cam.tiles_x) * tw, y0 = (t / cam.tiles_x) * th;
  int m = 0;
  for (int i = lane; i < tw * th; i += 32) {
    const int x = x0 + i % tw, y = y0 + i / tw;
    if (x < cam.W && y < cam.H) m = max(m, n_last[(size_t)y * cam.W + x]);
  }
  m = __reduce_max_sync(0xffffffffu, m);
  if (lane == 0) {
    const int b = work_bucket((uint32_t)m);
    bkt[t] = (uint32_t)b;
    atomicAdd(&hist[b], 1u);
  }
}

// One block: the buckets' offsets from the heaviest down, then every tile
// placed in its bucket (in no particular order within it).
__global__ void __launch_bounds__(1024) tile_order_kernel(const uint32_t* __restrict__ bkt, int tiles,
                                                          const unsigned* __restrict__ hist,
                                                          uint32_t* __restrict__ order) {
  chain_enter();
  __shared__ unsigned s_cnt[TILE_ORDER_BUCKETS], s_off[TILE_ORDER_BUCKETS];
  const int tid = threadIdx.x;
  if (tid < TILE_ORDER_BUCKETS) s_cnt[tid] = hist[tid];
  __syncthreads();
  if (tid < TILE_ORDER_BUCKETS) {  // tiles in heavier buckets come first
    unsigned run = 0;
    for (int b = TILE_ORDER_BUCKETS - 1; b > tid; --b) run += s_cnt[b];
    s_off[tid] = run;
  }
  __syncthreads();
  for (int t = tid; t < tiles; t += blockDim.x) order[atomicAdd(&s_off[bkt[t]], 1u)] = (uint32_t)t;
}

// ---------------------------------------------------------------- batched
// Work queue of a batched render: every (camera, tile) job, the longest
// lists first (log2 buckets), so the persistent blend finishes on short jobs.
__global__ void __launch_bounds__(1024) build_queue_kernel(const int2* __restrict__ ranges, int total_tiles,
                                                           uint32_t* __restrict__ queue, unsigned* job_ctr) {
  __shared__ unsigned s_cnt[33];
  __shared__ unsigned s_off[33];
  if (threadIdx.x < 33) s_cnt[threadIdx.x] = 0;
  if (threadIdx.x == 0) *job_ctr = 0;
  __syncthreads();
  for (int t = threadIdx.x; t < total_tiles; t += blockDim.x) {
    const int2 rg = ranges[t];
    const unsigned len = (unsigned)max(rg.y - rg.x, 0);
    atomicAdd(&s_cnt[__clz(len)], 1u);  // bucket 0 holds the longest lists
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned run = 0;
    for (int b = 0; b < 33; ++b) {
      s_off[b] = run;
      run += s_cnt[b];
    }
  }
  __syncthreads();
  for (int t = threadIdx.x; t < total_tiles; t += blockDim.x) {
    const int2 rg = ranges[t];
    const unsigned len = (unsigned)max(rg.y - rg.x, 0);
    queue[atomicAdd(&s_off[__clz(len)], 1u)] = (uint32_t)t;
  }
}

// Persistent forward blend over the job queue of all cameras: each CTA takes
// the next job with an atomic ticket until the queue is empty.
template <int KID, int PPT>
__global__ void __launch_bounds__(128) blend_batch_kernel(const float4* __restrict__ rec, const uint32_t* __restrict__ vals,
                                                          const int2* __restrict__ ranges, const CamTable cams,
                                                          const BatchPix pix, const ParDev P,
                                                          const uint32_t* __restrict__ queue, int n_jobs,
                                                          unsigned* job_ctr, float* __restrict__ images,
                                                          float* __restrict__ t_final, int B) {
  extern __shared__ float4 smem[];
  __shared__ int s_job;
  __shared__ int s_base[LS_MAX_CAMS];
  const int nc = cams.n;
  for (int c = threadIdx.x; c < nc; c += blockDim.x) s_base[c] = cams.c[c].tile_base;
  for (;;) {
    __syncthreads();  // the previous job is done with shared memory and s_job
    if (threadIdx.x == 0) s_job = (int)atomicAdd(job_ctr, 1u);
    __syncthreads();
    const int job = s_job;
    if (job >= n_jobs) break;
    const int gt = (int)queue[job];
    int lo = 0, hi = nc - 1;  // camera: last tile_base <= gt
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (s_base[mid] <= gt) lo = mid;
      else hi = mid - 1;
    }
    const CamDev& cam = cams.c[lo];
    const int tile = gt - cam.tile_base;
    TileJob J;
    J.x0 = (tile % cam.tiles_x) * P.tile_w;
    J.y0 = (tile / cam.tiles_x) * P.tile_h;
    J.W = cam.W;
    J.H = cam.H;
    J.rg = ranges[gt];
    J.pix_base = pix.base[lo];
    fwd_tile<KID, PPT, false, FWD_PLAIN>(rec, vals, P, J, smem, smem + B, smem + 2 * B, B, images, t_final, nullptr,
                                         nullptr, TruncArgs{}, gt);
  }
}

}  // namespace

// Pixels per thread: 4 for tiles of 256+ pixels, 2 for 8x8 (one warp).
static inline int ppt_for(const ParDev& P) { return P.tile_w * P.tile_h >= 256 ? 4 : 2; }

cudaError_t launch_blend_fwd(const float4* rec, const CamDev& cam, const ParDev& P, const int2* ranges,
                             const uint32_t* vals, float* image, float* t_final, int32_t* n_last,
                             unsigned long long* stats, cudaStream_t st, float* labels) {
  TruncArgs labels_ta{};
  labels_ta.labels = labels;
  // 4 pixels per thread from 16x16 tiles up (64 threads on 16x16: 0.195
  // against 0.199 ms for 2 pixels per thread), 2 on 8x8 (one warp)
  const int ppt = P.tile_w * P.tile_h < 256 ? 2 : 4;
  const int threads = P.tile_w * P.tile_h / ppt;
  const unsigned grid = (unsigned)(cam.tiles_x * cam.tiles_y);
  const size_t sm = sizeof(float4) * 3 * 2 * threads;
  cudaError_t e = cudaSuccess;
#define LS_BF3(K, PP, C)                                                                                     \
  e = launch_chain(blend_fwd_kernel<K, PP, C>, dim3(grid), dim3(threads), sm, st, rec, cam, P, ranges, vals, image, \
                   t_final, n_last, stats, labels_ta)
#define LS_BF2(K, PP)               \
  do {                              \
    if (stats) LS_BF3(K, PP, true); \
    else LS_BF3(K, PP, false);      \
  } while (0)
#define LS_BF(K)                \
  do {                          \
    if (ppt == 4) LS_BF2(K, 4); \
    else LS_BF2(K, 2);          \
  } while (0)
  switch (P.kernel) {
    case LS_KERNEL_GAUSSIAN: LS_BF(LS_KERNEL_GAUSSIAN); break;
    case LS_KERNEL_LAPLACIAN: LS_BF(LS_KERNEL_LAPLACIAN); break;
    case LS_KERNEL_COSINE: LS_BF(LS_KERNEL_COSINE); break;
    case LS_KERNEL_QUADRATIC: LS_BF(LS_KERNEL_QUADRATIC); break;
    default: LS_BF(LS_KERNEL_LINEAR); break;
  }
#undef LS_BF
#undef LS_BF2
#undef LS_BF3
  return e;
}

cudaError_t launch_blend_bwd(const float4* rec, const CamDev& cam, const ParDev& P, const int2* ranges,
                             const uint32_t* vals, const float* t_final, const int32_t* n_last,
                             const float* grad_image, const float* grad_t, float* g2d, cudaStream_t st,
                             const uint32_t* order) {
  // 4 pixels per row per thread; one row per thread (64 threads per 16x16
  // tile), 8x8 tiles: 2 pixels of one row
  const int ppr = P.tile_w * P.tile_h >= 256 ? 4 : 2;
  const int rpt = 1;
  const int threads = P.tile_w * P.tile_h / (ppr * rpt);
  const int B = threads;  // one record per thread per batch (2.5 % faster than two)
  const unsigned grid = (unsigned)(cam.tiles_x * cam.tiles_y);
  const size_t sm = sizeof(float4) * 3 * B + sizeof(float) * 9 * B + 2 * sizeof(uint32_t) * B;
  cudaError_t e = cudaSuccess;
#define LS_BB3(K, A, PR, RT)                                                                                  \
  e = launch_chain(blend_bwd_kernel<K, A, PR, RT>, dim3(grid), dim3(threads), sm, st, rec, cam, P, ranges, vals, \
                   t_final, n_last, grad_image, grad_t, g2d, B, order)
#define LS_BB2(K, A)                \
  do {                              \
    if (ppr == 4) LS_BB3(K, A, 4, 1); \
    else LS_BB3(K, A, 2, 1);          \
  } while (0)
  // the AGS reading is a template argument: a branch on it per pair cost 9 %
#define LS_BB(K)                   \
  do {                             \
    if (P.ags == 1) LS_BB2(K, 1);  \
    else if (P.ags == 2) LS_BB2(K, 2); \
    else LS_BB2(K, 0);             \
  } while (0)
  switch (P.kernel) {
    case LS_KERNEL_GAUSSIAN: LS_BB(LS_KERNEL_GAUSSIAN); break;
    case LS_KERNEL_LAPLACIAN: LS_BB(LS_KERNEL_LAPLACIAN); break;
    case LS_KERNEL_COSINE: LS_BB(LS_KERNEL_COSINE); break;
    case LS_KERNEL_QUADRATIC: LS_BB(LS_KERNEL_QUADRATIC); break;
    default: LS_BB(LS_KERNEL_LINEAR); break;
  }
#undef LS_BB
#undef LS_BB2
#undef LS_BB3
  return e;
}

cudaError_t launch_tile_order(const int32_t* n_last, const CamDev& cam, const ParDev& P, unsigned* hist,
                              uint32_t* bkt, uint32_t* order, cudaStream_t st) {
  const int tiles = cam.tiles_x * cam.tiles_y;
  if (tiles <= 0) return cudaSuccess;
  const cudaError_t e = launch_chain(tile_work_kernel, dim3(ceil_div(tiles, 8)), dim3(256), 0, st, n_last, cam,
                                     P.tile_w, P.tile_h, hist, bkt);
  if (e != cudaSuccess) return e;
  return launch_chain(tile_order_kernel, dim3(1), dim3(1024), 0, st, (const uint32_t*)bkt, tiles,
                      (const unsigned*)hist, order);
}

}  // namespace ls

namespace ls {

cudaError_t launch_blend_trunc(int mode, const float4* rec, const CamDev& cam, const ParDev& P, const int2* ranges,
                               const uint32_t* vals, float* image, float* t_final, int32_t* n_last,
                               const TruncArgs& ta, cudaStream_t st) {
  const int ppt = ppt_for(P);
  const int threads = P.tile_w * P.tile_h / ppt;
  const unsigned grid = (unsigned)(cam.tiles_x * cam.tiles_y);
  const size_t sm = sizeof(float4) * 3 * 2 * threads;
#define LS_BT3(K, PP, M) \
  blend_trunc_kernel<K, PP, M><<<grid, threads, sm, st>>>(rec, cam, P, ranges, vals, image, t_final, n_last, ta)
#define LS_BT2(K, PP)                        \
  do {                                       \
    if (mode == 1) LS_BT3(K, PP, FWD_TRUNC); \
    else LS_BT3(K, PP, FWD_RESUME);          \
  } while (0)
#define LS_BT(K)                \
  do {                          \
    if (ppt == 4) LS_BT2(K, 4); \
    else LS_BT2(K, 2);          \
  } while (0)
  switch (P.kernel) {
    case LS_KERNEL_GAUSSIAN: LS_BT(LS_KERNEL_GAUSSIAN); break;
    case LS_KERNEL_LAPLACIAN: LS_BT(LS_KERNEL_LAPLACIAN); break;
    case LS_KERNEL_COSINE: LS_BT(LS_KERNEL_COSINE); break;
    case LS_KERNEL_QUADRATIC: LS_BT(LS_KERNEL_QUADRATIC); break;
    default: LS_BT(LS_KERNEL_LINEAR); break;
  }
#undef LS_BT
#undef LS_BT2
#undef LS_BT3
  return cudaGetLastError();
}

cudaError_t launch_build_queue(const int32_t* ranges, int total_tiles, uint32_t* queue, unsigned* job_ctr,
                               cudaStream_t st) {
  build_queue_kernel<<<1, 1024, 0, st>>>(reinterpret_cast<const int2*>(ranges), total_tiles, queue, job_ctr);
  return cudaGetLastError();
}

// Persistent grid: as many CTAs as fit on the device at once.
cudaError_t launch_blend_batch(const float4* rec, const uint32_t* vals, const int32_t* ranges, const CamTable& cams,
                              const BatchPix& pix, const ParDev& P, const uint32_t* queue, int n_jobs,
                              unsigned* job_ctr, float* images, float* t_final, int batch, cudaStream_t st) {
  const int ppt = ppt_for(P);
  const int threads = P.tile_w * P.tile_h / ppt;
  const int B = batch > 0 ? batch : 4 * threads;
  const size_t sm = sizeof(float4) * 3 * B;
  int dev = 0, sms = 0, per_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
#define LS_BB3(K, PP)                                                                                               \
  do {                                                                                                              \
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, blend_batch_kernel<K, PP>, threads, sm);             \
    if (e != cudaSuccess) return e;                                                                                 \
    blend_batch_kernel<K, PP><<<(unsigned)(sms * (per_sm > 0 ? per_sm : 1)), threads, sm, st>>>(                    \
        rec, vals, reinterpret_cast<const int2*>(ranges), cams, pix, P, queue, n_jobs, job_ctr, images, t_final, B); \
  } while (0)
#define LS_BB(K)                \
  do {                          \
    if (ppt == 4) LS_BB3(K, 4); \
    else LS_BB3(K, 2);          \
  } while (0)
  switch (P.kernel) {
    case LS_KERNEL_GAUSSIAN: LS_BB(LS_KERNEL_GAUSSIAN); break;
    case LS_KERNEL_LAPLACIAN: LS_BB(LS_KERNEL_LAPLACIAN); break;
    case LS_KERNEL_COSINE: LS_BB(LS_KERNEL_COSINE); break;
    case LS_KERNEL_QUADRATIC: LS_BB(LS_KERNEL_QUADRATIC); break;
    default: LS_BB(LS_KERNEL_LINEAR); break;
  }
#undef LS_BB
#undef LS_BB3
  return cudaGetLastError();
}

}  // namespace ls
