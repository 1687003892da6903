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

// One compacted record of a warp: its candidates and the reach-test
// constants, as four 16-byte words (one shared load each).
struct __align__(16) EnumRec {
  uint32_t off;          // warp-exclusive offset of its first candidate
  uint32_t kb;           // key of its first box tile
  uint32_t wt;           // box width in tiles | camera tiles_x << 16
  uint32_t xy;           // first tile column | first tile row << 16
  float mx, my, l00, l01;
  float l11;
  float inv_l00;         // 1 / l00
  float kq;              // l00 l01 / (l01^2 + l11^2)
  float lim;             // accepted bound on D^2
  uint32_t r, dk;        // record id, depth bits
  float rw;              // 1 / box width
  uint32_t pad;
};

__device__ __forceinline__ uint32_t box_count(uint2 rc) {
  const int x0 = rc.x & 0xFFFF, x1 = rc.x >> 16, y0 = rc.y & 0xFFFF, y1 = rc.y >> 16;
  return x1 < x0 ? 0u : (uint32_t)((x1 - x0 + 1) * (y1 - y0 + 1));
}

__device__ __forceinline__ void enum_rec(EnumRec& t, uint32_t off, uint2 rc, uint32_t r, uint32_t dk,
                                         const CamLite& cm, const float4* __restrict__ rec) {
  const uint32_t x0 = rc.x & 0xFFFF, x1 = rc.x >> 16, y0 = rc.y & 0xFFFF;
  const uint32_t w = x1 - x0 + 1;
  const float4 a = rec[3 * (size_t)r], b = rec[3 * (size_t)r + 1];  // {mx, my, l00, l01}, {l11, o, rho2, depth}
  uint4* q = reinterpret_cast<uint4*>(&t);
  q[0] = make_uint4(off, (uint32_t)cm.tile_base + y0 * (uint32_t)cm.tiles_x + x0, w | ((uint32_t)cm.tiles_x << 16),
                    x0 | (y0 << 16));
  reinterpret_cast<float4*>(&t)[1] = a;
  reinterpret_cast<float4*>(&t)[2] =
      make_float4(b.x, 1.f / a.z, a.z * a.w / fmaf(a.w, a.w, b.x * b.x), fmaf(b.z, 1.02f, 1e-3f));
  q[3] = make_uint4(r, dk, __float_as_uint(1.f / (float)w), 0u);
}

// The reach test of one candidate: a record's geometry words g1 = {mx, my,
// l00, l01} and g2 = {l11, 1/l00, l00 l01 / (l01^2 + l11^2), bound}.
//
// Whether the support ellipse q(p - mu) <= rho^2, q = |L d|^2 for the upper
// Cholesky factor L = [[l00, l01], [0, l11]] of the conic, reaches the
// rectangle spanned by the pixel centres of tile (tx, ty).  A convex q whose
// minimum lies outside the rectangle attains its minimum over it on a side
// that faces the centre; the minimum along the facing row and along the
// facing column are both taken (each by clamping the 1D minimiser; a side
// that does not face the centre still gives a point of the rectangle, so the
// smaller value is the minimum), and the centre itself when inside.  The
// bound is loosened by 2 % (+1e-3) so that binary32 rounding of q in the
// blend can never composite a pair in a tile this test left out.
__device__ __forceinline__ bool tile_reached(const float4& g1, const float4& g2, int tx, int ty, int TW, int TH) {
  const float mx = g1.x, my = g1.y, l00 = g1.z, l01 = g1.w, l11 = g2.x;
  const float X0 = (float)(tx * TW) + 0.5f, X1 = X0 + (float)(TW - 1);
  const float Y0 = (float)(ty * TH) + 0.5f, Y1 = Y0 + (float)(TH - 1);
  const bool inside = mx >= X0 && mx <= X1 && my >= Y0 && my <= Y1;
  // facing row: dx* = -l01 dy / l00
  const float dyr = (my < Y0 ? Y0 : Y1) - my;
  const float dxr = fminf(fmaxf(-l01 * dyr * g2.y, X0 - mx), X1 - mx);
  const float e1r = fmaf(l00, dxr, l01 * dyr), e2r = l11 * dyr;
  // facing column: dy* = -l00 l01 dx / (l01^2 + l11^2)
  const float dxc = (mx < X0 ? X0 : X1) - mx;
  const float dyc = fminf(fmaxf(-g2.z * dxc, Y0 - my), Y1 - my);
  const float e1c = fmaf(l00, dxc, l01 * dyc), e2c = l11 * dyc;
  const float best = fminf(fmaf(e1r, e1r, e2r * e2r), fmaf(e1c, e1c, e2c * e2c));
  return inside || best <= g2.w;
}

// Candidate m (row-major in the box) of a record with words g0 = {off, kb,
// wt, xy} and 1 / width rw: its key and tile.  m < 2^24, so float(m) is exact
// and the binary32 quotient is within one of m / w.
__device__ __forceinline__ uint32_t cand_key(const uint4& g0, float rw, uint32_t m, int& tx, int& ty) {
  const int w = (int)(g0.z & 0xFFFFu);
  int q = (int)__float2uint_rz(__uint2float_rn(m) * rw);
  int rem = (int)m - q * w;
  if (rem < 0) {
    --q;
    rem += w;
  } else if (rem >= w) {
    ++q;
    rem -= w;
  }
  tx = (int)(g0.w & 0xFFFFu) + rem;
  ty = (int)(g0.w >> 16) + q;
  return g0.y + (uint32_t)q * (g0.z >> 16) + (uint32_t)rem;
}

}  // namespace ls
