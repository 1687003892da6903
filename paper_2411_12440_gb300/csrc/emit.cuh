// Enumeration of (record, tile) keys, shared by the plain duplication and the
// learned path's kept / held-out enumerations (duplicate.cu).
//
// A warp takes ENUM_WARP_RECS consecutive records of the depth order and
// keeps those with a non-empty support box (ballot compaction into shared
// memory, with the constants of their row ranges).  It then walks their box
// rows 32 at a time: lane l takes row e = step + l; the lanes holding the
// next records' first rows mark them in one warp OR-reduction, so lane l's
// record is the step's first record plus the number of marks at or below l
// (no search).  Each row gives, in closed form, the contiguous run of tiles
// the support ellipse reaches in it (row_range); the rows with tiles are
// compacted and their keys walked 32 at a time with the same marking, the
// mode's condition applied per key, and the taken keys compacted with a
// ballot.  A count launch records each warp's total (and stashes its keys
// in a spare buffer); after a scan of the totals, the emit launch copies or
// writes them from the warp's offset, so keys come out in depth order and
// every tile's keys in (depth, id) order.
#pragma once

#include "kernels.h"

namespace ls {

constexpr int ENUM_THREADS = 256;
constexpr int ENUM_WARPS = ENUM_THREADS / 32;
constexpr int ENUM_WARP_RECS = 64;  // records per warp (two per lane)
constexpr int ENUM_BLOCK_RECS = ENUM_WARPS * ENUM_WARP_RECS;

struct CamLite {
  int W, H, tiles_x, tile_base;
};

// One compacted record of a warp, as four 16-byte words (one shared load
// each): where its box rows start in the warp's row list, its box, and the
// constants of its row ranges.
struct __align__(16) EnumRec {
  uint32_t off;          // warp-exclusive offset of its first box row
  uint32_t kb;           // key of its first box tile
  uint32_t wt;           // box width in tiles | camera tiles_x << 16
  uint32_t xy;           // first tile column | first tile row << 16
  float mx, my;          // centre
  float a01;             // l01 / l00
  float inv_l00;         // 1 / l00
  float l11;
  float lim;             // accepted bound L on D^2
  float dyl;             // dy of the leftmost point of D^2 = L
  float ext_y;           // half height of D^2 = L: sqrt(L) / l11
  uint32_t r, dk;        // record id, depth bits
  uint32_t beyond;       // ENUM_KEPT: the record lies beyond every proposal of its box (takes no key)
  uint32_t pad1;
};

__device__ __forceinline__ uint32_t box_count(uint2 rc) {
  const int x0 = rc.x & 0xFFFF, x1 = rc.x >> 16, y0 = rc.y & 0xFFFF, y1 = rc.y >> 16;
  return x1 < x0 ? 0u : (uint32_t)((x1 - x0 + 1) * (y1 - y0 + 1));
}
__device__ __forceinline__ uint32_t box_rows(uint2 rc) {
  const int x0 = rc.x & 0xFFFF, x1 = rc.x >> 16, y0 = rc.y & 0xFFFF, y1 = rc.y >> 16;
  return x1 < x0 ? 0u : (uint32_t)(y1 - y0 + 1);
}

// The support ellipse, loosened so that binary32 rounding of D^2 in the
// blend can never composite a pair in a tile left out: D^2 <= L with
// L = 1.02 rho^2 + 1e-3 (D^2 = |L d|^2 for the upper Cholesky factor
// [[l00, l01], [0, l11]] of the conic), and every range below widened by
// RANGE_EPS pixels.
constexpr float RANGE_EPS = 0.01f;

// Boxes of at most WHOLE_BOX tiles are listed whole: the ellipse reaches
// nearly all of their tiles, and their records skip the gather of the
// ellipse.
constexpr uint32_t WHOLE_BOX = 2;

// Every operation below is rounded explicitly (no contraction), so the
// lists can be reproduced bit for bit in binary32 elsewhere.
__device__ __forceinline__ void enum_rec(EnumRec& t, uint32_t off, uint2 rc, uint32_t r, uint32_t dk,
                                         const CamLite& cm, const float4* __restrict__ rec) {
  const uint32_t x0 = rc.x & 0xFFFF, x1 = rc.x >> 16, y0 = rc.y & 0xFFFF;
  const uint32_t w = x1 - x0 + 1;
  uint4* q = reinterpret_cast<uint4*>(&t);
  q[0] = make_uint4(off, (uint32_t)cm.tile_base + y0 * (uint32_t)cm.tiles_x + x0, w | ((uint32_t)cm.tiles_x << 16),
                    x0 | (y0 << 16));
  q[3] = make_uint4(r, dk, 0u, 0u);
  if (box_count(rc) <= WHOLE_BOX) {
    reinterpret_cast<float4*>(&t)[2] = make_float4(0.f, 0.f, 0.f, -1.f);  // ext_y < 0: the whole box
    return;
  }
  const float4 a = rec[3 * (size_t)r], b = rec[3 * (size_t)r + 1];  // {mx, my, l00, l01}, {l11, o, rho2, depth}
  const float L = __fmaf_rn(b.z, 1.02f, 1e-3f), sL = __fsqrt_rn(L);
  const float inv_l00 = __fdiv_rn(1.f, a.z);
  reinterpret_cast<float4*>(&t)[1] = make_float4(a.x, a.y, __fmul_rn(a.w, inv_l00), inv_l00);
  // leftmost point of the ellipse: dy = sqrt(L) l01 / (l11 sqrt(l11^2 + l01^2))
  const float nrm = __fsqrt_rn(__fmaf_rn(b.x, b.x, __fmul_rn(a.w, a.w)));
  reinterpret_cast<float4*>(&t)[2] =
      make_float4(b.x, L, __fdiv_rn(__fmul_rn(sL, a.w), __fmul_rn(b.x, nrm)), __fdiv_rn(sL, b.x));
}

// An upper bound of the proposal bits over the tile box [x0, x1] x [y0, y1]:
// the max of the (at most 2 x 2) cells of the first pyramid level at which
// the box spans at most two cells each way.
__device__ __forceinline__ uint32_t box_dstar_bound(const uint32_t* __restrict__ pyr, const DstarPyramid& D, int x0,
                                                    int x1, int y0, int y1) {
  int k = 0;
  while (k + 1 < D.levels && ((x1 >> k) - (x0 >> k) > 1 || (y1 >> k) - (y0 >> k) > 1)) ++k;
  const int w = D.w[k];
  const uint32_t* L = pyr + D.off[k];
  const int ax = x0 >> k, bx = x1 >> k, ay = y0 >> k, by = y1 >> k;
  return max(max(__ldg(L + ay * w + ax), __ldg(L + ay * w + bx)), max(__ldg(L + by * w + ax), __ldg(L + by * w + bx)));
}

// The tiles of box row ty that the ellipse reaches: [tx_a, tx_b] (empty when
// tx_b < tx_a), clamped to the box columns [x0, x1].  The ellipse cut by the
// row's band of pixel-centre heights [Y0, Y1] is convex, so the tiles it
// reaches are those whose pixel-centre columns meet its x-extent
// [X_lo, X_hi]; X_lo is the convex left boundary
// x(dy) = mx - (sqrt(L - (l11 dy)^2) + l01 dy) / l00 minimised over the band
// (at the leftmost point's dy, clamped into the band), X_hi the mirror.
__device__ __forceinline__ void row_range(const float4& g1, const float4& g2, int ty, int TW, int TH, int x0, int x1,
                                          int& tx_a, int& tx_b) {
  const float mx = g1.x, my = g1.y, a01 = g1.z, inv_l00 = g1.w, l11 = g2.x, L = g2.y, dyl = g2.z, ext = g2.w;
  if (ext < 0.f) {  // a small box, listed whole
    tx_a = x0;
    tx_b = x1;
    return;
  }
  const float Y0 = __fadd_rn((float)(ty * TH), 0.5f), Y1 = __fadd_rn(Y0, (float)(TH - 1));
  const float lo = fmaxf(__fsub_rn(__fsub_rn(Y0, my), RANGE_EPS), -ext);
  const float hi = fminf(__fadd_rn(__fsub_rn(Y1, my), RANGE_EPS), ext);
  tx_a = x0;
  tx_b = x0 - 1;
  if (!(lo <= hi)) return;
  const float d1 = fminf(fmaxf(dyl, lo), hi), d2 = fminf(fmaxf(-dyl, lo), hi);
  const float e1 = __fmul_rn(l11, d1), e2 = __fmul_rn(l11, d2);
  const float s1 = __fsqrt_rn(fmaxf(__fmaf_rn(-e1, e1, L), 0.f)), s2 = __fsqrt_rn(fmaxf(__fmaf_rn(-e2, e2, L), 0.f));
  const float xlo = __fsub_rn(__fsub_rn(mx, __fmaf_rn(s1, inv_l00, __fmul_rn(a01, d1))), RANGE_EPS);
  const float xhi = __fadd_rn(__fadd_rn(mx, __fmaf_rn(s2, inv_l00, -__fmul_rn(a01, d2))), RANGE_EPS);
  // tile tx holds pixel-centre columns [tx TW + 0.5, tx TW + TW - 0.5]
  const float inv_tw = 1.f / (float)TW;  // exact: TW is a power of two
  const float fa = ceilf(__fmaf_rn(__fadd_rn(xlo, 0.5f), inv_tw, -1.f));
  const float fb = floorf(__fmul_rn(__fsub_rn(xhi, 0.5f), inv_tw));
  tx_a = fa <= (float)x0 ? x0 : (fa > (float)x1 ? x1 + 1 : (int)fa);
  tx_b = fb >= (float)x1 ? x1 : (fb < (float)x0 ? x0 - 1 : (int)fb);
}

}  // namespace ls
