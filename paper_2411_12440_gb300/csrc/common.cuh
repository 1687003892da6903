// Device-side definitions shared by the sm_103a kernels of the linear-splatting
// rasterizer (camera table, parameters, tile rule, kernel family, status).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "ls.h"

namespace ls {

constexpr uint32_t DKEY_CULLED = 0xFFFFFFFFu;

// Camera as the kernels read it: rotation/translation of W, intrinsics, the
// clamp of t_x/t_z, t_y/t_z (1.3x the half field of view), the camera centre
// -R^T t (for view-dependent colour) and the tile grid.
struct CamDev {
  float R[9];
  float t[3];
  float fx, fy, cx, cy;
  float campos[3];
  float lim_xl, lim_xh, lim_yl, lim_yh;
  int W, H, tiles_x, tiles_y, tile_base;
};

struct CamTable {
  CamDev c[LS_MAX_CAMS];
  int n;
};

struct ParDev {
  float lambda, inv_lambda;
  int kernel, ags, antialias;
  float eps2d, alpha_min, alpha_max, t_min;
  int tile_w, tile_h;
  float bg[3];
  float near_plane, far_plane;
  int sh_degree;
};

// Record planes of the projected buffer (see ls.h).
struct ProjPtr {
  float4* rec;     // [R][3] float4
  float4* foot;    // [R]
  uint32_t* dkey;  // [R]
};
struct ProjCPtr {
  const float4* rec;
  const float4* foot;
  const uint32_t* dkey;
};

__device__ __forceinline__ void set_status(int32_t* st, int code) {
  if (st) atomicCAS(st, 0, code);
}

// Support box of a footprint in tiles, in binary32 with every operation
// rounded as written (no contraction): pixel centres at +0.5, so the pixel
// range is [ceil(mx - ex - 0.5), floor(mx + ex - 0.5)] clipped to the image.
// Returns false when the box holds no pixel centre of the image.
__device__ __forceinline__ bool tile_rect(float mx, float my, float ex, float ey, int W, int H, int TW, int TH,
                                          int& tx0, int& tx1, int& ty0, int& ty1) {
  float xl = ceilf(__fsub_rn(__fsub_rn(mx, ex), 0.5f));
  float xh = floorf(__fsub_rn(__fadd_rn(mx, ex), 0.5f));
  float yl = ceilf(__fsub_rn(__fsub_rn(my, ey), 0.5f));
  float yh = floorf(__fsub_rn(__fadd_rn(my, ey), 0.5f));
  if (!(xl <= xh && yl <= yh) || xh < 0.f || yh < 0.f || xl > (float)(W - 1) || yl > (float)(H - 1)) return false;
  int x0 = (int)fmaxf(xl, 0.f), x1 = (int)fminf(xh, (float)(W - 1));
  int y0 = (int)fmaxf(yl, 0.f), y1 = (int)fminf(yh, (float)(H - 1));
  tx0 = x0 / TW;
  tx1 = x1 / TW;
  ty0 = y0 / TH;
  ty1 = y1 / TH;
  return true;
}

// Kernel family f(x), x = D / lambda (Sec. 3.2 Eq. 9; Appendix B Eq. 21-25)
// and df/dx inside the support.
template <int KID>
__device__ __forceinline__ float kern_f(float x) {
  if (KID == LS_KERNEL_GAUSSIAN) return __expf(__fmul_rn(__fmul_rn(-0.5f, x), x));
  if (KID == LS_KERNEL_LAPLACIAN) return __expf(-x);
  if (KID == LS_KERNEL_COSINE)
    return x <= 1.f ? __fmul_rn(0.5f, __fadd_rn(1.f, __cosf(__fmul_rn(3.14159265358979f, x)))) : 0.f;
  if (KID == LS_KERNEL_QUADRATIC) return fmaxf(0.f, __fsub_rn(1.f, __fmul_rn(x, x)));
  return fmaxf(0.f, __fsub_rn(1.f, x));
}
template <int KID>
__device__ __forceinline__ float kern_df(float x) {
  if (KID == LS_KERNEL_GAUSSIAN) return -x * __expf(-0.5f * x * x);
  if (KID == LS_KERNEL_LAPLACIAN) return -__expf(-x);
  if (KID == LS_KERNEL_COSINE) return x <= 1.f ? -0.5f * 3.14159265358979f * __sinf(3.14159265358979f * x) : 0.f;
  if (KID == LS_KERNEL_QUADRATIC) return x < 1.f ? -2.f * x : 0.f;
  return x < 1.f ? -1.f : 0.f;
}

// Support end x_s: largest x with o f(x) >= alpha_min (0 when o < alpha_min);
// without an alpha threshold compact kernels end at 1, infinite tails at 3.
__device__ __forceinline__ float kern_support(int kid, float o, float amin) {
  float m = amin / o;
  if (m > 1.f) return 0.f;
  if (m <= 0.f) return (kid == LS_KERNEL_GAUSSIAN || kid == LS_KERNEL_LAPLACIAN) ? 3.f : 1.f;
  switch (kid) {
    case LS_KERNEL_GAUSSIAN: return sqrtf(2.f * logf(1.f / m));
    case LS_KERNEL_LAPLACIAN: return logf(1.f / m);
    case LS_KERNEL_COSINE: return acosf(2.f * m - 1.f) * 0.318309886183791f;
    case LS_KERNEL_QUADRATIC: return sqrtf(1.f - m);
    default: return 1.f - m;
  }
}

// Programmatic dependent launch.  A kernel of the frame's chain is launched
// with programmatic stream serialisation (launch_chain in kernels.h), so the
// next kernel of the stream may be scheduled before this one has finished.
// Every such kernel therefore starts with chain_enter(): it first waits until
// the kernel before it in the stream has completed and its writes are
// visible (so nothing is read or written early, and a kernel's completion
// still implies that of every kernel before it), then allows the kernel
// after it to be scheduled onto the SMs as they free up.  Both instructions
// are no-ops for a kernel launched without the attribute.
__device__ __forceinline__ void chain_enter() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// Launch helpers shared by the host-side launchers.
inline unsigned ceil_div(int64_t a, int64_t b) { return (unsigned)((a + b - 1) / b); }

}  // namespace ls
