// Enumeration of (record, tile) keys, shared by the plain duplication and the
// learned path's kept / held-out enumerations (duplicate.cu).
//
// A warp takes ENUM_WARP_RECS consecutive records of the depth order.  Their
// candidates are the tiles of their binary32 support boxes; a candidate is
// taken when the support ellipse reaches the tile (tile_reached) and the
// mode's condition holds.  The warp first keeps only the records with
// candidates (ballot compaction into shared memory, with the per-record
// constants of the reach test) and scans their candidate counts.  Then it
// walks the candidates 32 at a time: lane l takes candidate e = step + l;
// the lanes holding the next records' first candidates mark them in one
// warp OR-reduction, so lane l's record is the step's first record plus the
// number of marks at or below l (no search), and its tile follows from one
// division done in binary32 and corrected to the exact quotient.  Taken
// candidates are compacted with a ballot.  A count launch records each
// warp's total; after a scan of the totals, the emit launch walks the same
// candidates in the same order and writes the taken keys from the warp's
// offset, so keys come out in depth order and every tile's keys in
// (depth, id) order.
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

// One compacted record of a warp: its candidates and the reach-test constants.
struct EnumRec {
  uint32_t off;          // warp-exclusive offset of its first candidate
  uint32_t kb;           // key of its first box tile
  uint32_t wt;           // box width in tiles | camera tiles_x << 16
  uint32_t xy;           // first tile column | first tile row << 16
  uint32_t r, dk;        // record id, depth bits
  float rw;              // 1 / box width
  float mx, my, l00, l01, l11;
  float inv_l00;         // 1 / l00
  float kq;              // l00 l01 / (l01^2 + l11^2)
  float lim;             // accepted bound on D^2
};

__device__ __forceinline__ uint32_t box_count(uint2 rc) {
  const int x0 = rc.x & 0xFFFF, x1 = rc.x >> 16, y0 = rc.y & 0xFFFF, y1 = rc.y >> 16;
  return x1 < x0 ? 0u : (uint32_t)((x1 - x0 + 1) * (y1 - y0 + 1));
}

__device__ __forceinline__ void enum_rec(EnumRec& t, uint2 rc, uint32_t r, uint32_t dk, const CamLite& cm,
                                         const float4* __restrict__ rec) {
  const uint32_t x0 = rc.x & 0xFFFF, x1 = rc.x >> 16, y0 = rc.y & 0xFFFF;
  const uint32_t w = x1 - x0 + 1;
  t.kb = (uint32_t)cm.tile_base + y0 * (uint32_t)cm.tiles_x + x0;
  t.wt = w | ((uint32_t)cm.tiles_x << 16);
  t.xy = x0 | (y0 << 16);
  t.r = r;
  t.dk = dk;
  t.rw = 1.f / (float)w;
  const float4 a = rec[3 * (size_t)r], b = rec[3 * (size_t)r + 1];  // {mx, my, l00, l01}, {l11, o, rho2, depth}
  t.mx = a.x;
  t.my = a.y;
  t.l00 = a.z;
  t.l01 = a.w;
  t.l11 = b.x;
  t.inv_l00 = 1.f / a.z;
  t.kq = a.z * a.w / fmaf(a.w, a.w, b.x * b.x);
  t.lim = fmaf(b.z, 1.02f, 1e-3f);
}

// Whether the support ellipse q(p - mu) <= rho^2, q = |L d|^2 for the upper
// Cholesky factor L = [[l00, l01], [0, l11]] of the conic, reaches the
// rectangle spanned by the pixel centres of tile (tx, ty).  A convex q whose
// minimum lies outside the rectangle attains its minimum over it on a side
// that faces the centre, so at most two sides are tried, each by clamping
// the 1D minimiser.  The bound is loosened by 2 % (+1e-3) so that binary32
// rounding of q in the blend can never composite a pair in a tile this test
// left out.
__device__ __forceinline__ bool tile_reached(const EnumRec& t, int tx, int ty, int TW, int TH) {
  const float X0 = (float)(tx * TW) + 0.5f, X1 = X0 + (float)(TW - 1);
  const float Y0 = (float)(ty * TH) + 0.5f, Y1 = Y0 + (float)(TH - 1);
  const bool inx = t.mx >= X0 && t.mx <= X1, iny = t.my >= Y0 && t.my <= Y1;
  if (inx && iny) return true;
  float best = __int_as_float(0x7F800000);
  if (!iny) {  // the row of pixel centres facing the centre: dx* = -l01 dy / l00
    const float dy = (t.my < Y0 ? Y0 : Y1) - t.my;
    const float dx = fminf(fmaxf(-t.l01 * dy * t.inv_l00, X0 - t.mx), X1 - t.mx);
    const float e1 = fmaf(t.l00, dx, t.l01 * dy), e2 = t.l11 * dy;
    best = fmaf(e1, e1, e2 * e2);
  }
  if (!inx) {  // the column facing it: dy* = -l00 l01 dx / (l01^2 + l11^2)
    const float dx = (t.mx < X0 ? X0 : X1) - t.mx;
    const float dy = fminf(fmaxf(-t.kq * dx, Y0 - t.my), Y1 - t.my);
    const float e1 = fmaf(t.l00, dx, t.l01 * dy), e2 = t.l11 * dy;
    best = fminf(best, fmaf(e1, e1, e2 * e2));
  }
  return best <= t.lim;
}

// Candidate m (row-major in the box) of record t: its key and tile.  m < 2^24,
// so float(m) is exact and the binary32 quotient is within one of m / w.
__device__ __forceinline__ uint32_t cand_key(const EnumRec& t, uint32_t m, int& tx, int& ty) {
  const int w = (int)(t.wt & 0xFFFFu);
  int q = (int)__float2uint_rz(__uint2float_rn(m) * t.rw);
  int rem = (int)m - q * w;
  if (rem < 0) {
    --q;
    rem += w;
  } else if (rem >= w) {
    ++q;
    rem -= w;
  }
  tx = (int)(t.xy & 0xFFFFu) + rem;
  ty = (int)(t.xy >> 16) + q;
  return t.kb + (uint32_t)q * (t.wt >> 16) + (uint32_t)rem;
}

}  // namespace ls
