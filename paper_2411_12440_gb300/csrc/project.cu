// a1 / a6: projection of 3D primitives to screen-space footprints and its
// adjoint (Sec. 3.1 Eq. 1-4; support radius from Sec. 3.3.1 Eq. 12).
//
// One thread per (camera, primitive); blockIdx.y is the camera so every
// camera read is warp-uniform.  Inputs are structure-of-arrays: means /
// scales [n][3], quats [n][4] (one 16-byte load), opacities [n] and SH
// coefficient-major [K*3][n], so each coefficient load is coalesced across
// the warp and culled primitives skip their SH bytes entirely.
#include "common.cuh"
#include "kernels.h"

namespace ls {

// Real spherical harmonics to degree 3, with the Condon-Shortley phase:
// Y_l,m in order m = -l..l, each written as a polynomial of the unit
// direction (x, y, z) times its normalisation constant.
#define SH_C0 0.28209479177387814f   // 1/(2 sqrt(pi))
#define SH_C1 0.48860251190291992f   // sqrt(3/(4 pi))
#define SH_C2A 1.0925484305920792f   // sqrt(15/(4 pi))
#define SH_C2B 0.31539156525252005f  // sqrt(5/(16 pi))
#define SH_C2C 0.54627421529603959f  // sqrt(15/(16 pi))
#define SH_C3A 0.59004358992664352f  // sqrt(35/(32 pi))
#define SH_C3B 2.8906114426405538f   // sqrt(105/(4 pi))
#define SH_C3C 0.45704579946446572f  // sqrt(21/(32 pi))
#define SH_C3D 0.37317633259011540f  // sqrt(7/(16 pi))
#define SH_C3E 1.4453057213202769f   // sqrt(105/(16 pi))

template <int DEG>
__device__ __forceinline__ void sh_basis(float x, float y, float z, float* Y) {
  Y[0] = SH_C0;
  if (DEG >= 1) {
    Y[1] = -SH_C1 * y;
    Y[2] = SH_C1 * z;
    Y[3] = -SH_C1 * x;
  }
  if (DEG >= 2) {
    float xx = x * x, yy = y * y, zz = z * z;
    Y[4] = SH_C2A * x * y;
    Y[5] = -SH_C2A * y * z;
    Y[6] = SH_C2B * (2.f * zz - xx - yy);
    Y[7] = -SH_C2A * x * z;
    Y[8] = SH_C2C * (xx - yy);
    if (DEG >= 3) {
      Y[9] = -SH_C3A * y * (3.f * xx - yy);
      Y[10] = SH_C3B * x * y * z;
      Y[11] = -SH_C3C * y * (4.f * zz - xx - yy);
      Y[12] = SH_C3D * z * (2.f * zz - 3.f * xx - 3.f * yy);
      Y[13] = -SH_C3C * x * (4.f * zz - xx - yy);
      Y[14] = SH_C3E * z * (xx - yy);
      Y[15] = -SH_C3A * x * (xx - 3.f * yy);
    }
  }
}

// Gradient of sum_k w_k Y_k with respect to the (unnormalised) polynomial
// arguments (x, y, z).
template <int DEG>
__device__ __forceinline__ void sh_basis_grad(float x, float y, float z, const float* w, float& gx, float& gy,
                                              float& gz) {
  gx = gy = gz = 0.f;
  if (DEG >= 1) {
    gy += -SH_C1 * w[1];
    gz += SH_C1 * w[2];
    gx += -SH_C1 * w[3];
  }
  if (DEG >= 2) {
    float xx = x * x, yy = y * y, zz = z * z;
    gx += SH_C2A * y * w[4];
    gy += SH_C2A * x * w[4];
    gy += -SH_C2A * z * w[5];
    gz += -SH_C2A * y * w[5];
    gx += -2.f * SH_C2B * x * w[6];
    gy += -2.f * SH_C2B * y * w[6];
    gz += 4.f * SH_C2B * z * w[6];
    gx += -SH_C2A * z * w[7];
    gz += -SH_C2A * x * w[7];
    gx += 2.f * SH_C2C * x * w[8];
    gy += -2.f * SH_C2C * y * w[8];
    if (DEG >= 3) {
      gx += -SH_C3A * 6.f * x * y * w[9];
      gy += -SH_C3A * (3.f * xx - 3.f * yy) * w[9];
      gx += SH_C3B * y * z * w[10];
      gy += SH_C3B * x * z * w[10];
      gz += SH_C3B * x * y * w[10];
      gx += SH_C3C * 2.f * x * y * w[11];
      gy += -SH_C3C * (4.f * zz - xx - 3.f * yy) * w[11];
      gz += -SH_C3C * 8.f * y * z * w[11];
      gx += -SH_C3D * 6.f * x * z * w[12];
      gy += -SH_C3D * 6.f * y * z * w[12];
      gz += SH_C3D * (6.f * zz - 3.f * xx - 3.f * yy) * w[12];
      gx += -SH_C3C * (4.f * zz - 3.f * xx - yy) * w[13];
      gy += SH_C3C * 2.f * x * y * w[13];
      gz += -SH_C3C * 8.f * x * z * w[13];
      gx += SH_C3E * 2.f * x * z * w[14];
      gy += -SH_C3E * 2.f * y * z * w[14];
      gz += SH_C3E * (xx - yy) * w[14];
      gx += -SH_C3A * (3.f * xx - 3.f * yy) * w[15];
      gy += SH_C3A * 6.f * x * y * w[15];
    }
  }
}

// Rotation matrix of a unit quaternion (w, x, y, z), row-major.
__device__ __forceinline__ void quat_to_rot(float w, float x, float y, float z, float* R) {
  R[0] = 1.f - 2.f * (y * y + z * z);
  R[1] = 2.f * (x * y - w * z);
  R[2] = 2.f * (x * z + w * y);
  R[3] = 2.f * (x * y + w * z);
  R[4] = 1.f - 2.f * (x * x + z * z);
  R[5] = 2.f * (y * z - w * x);
  R[6] = 2.f * (x * z - w * y);
  R[7] = 2.f * (y * z + w * x);
  R[8] = 1.f - 2.f * (x * x + y * y);
}

// Forward intermediates shared by the forward kernel and the adjoint.
//
// Sigma_2D = J W Sigma W^T J^T is formed as r r^T with the 2x3 factor
// r = J W Rq diag(s), so det(Sigma_2D) = |r1 x r2|^2 and
// det(Sigma_2D + eps I) = det0 + eps (tr) + eps^2 are sums of non-negative
// terms: no cancellation for needle-like footprints, where the usual
// sxx syy - sxy^2 loses most of its binary32 digits.
struct ProjState {
  float t[3];
  float qn, q[4];  // norm and normalised quaternion
  float Rq[9];
  float Wm[9];     // Rc Rq diag(s)
  float r1[3], r2[3];
  float ux, uy;
  bool cx_free, cy_free;  // t_x/t_z, t_y/t_z inside the clamp
  float S2[3];     // Sigma_2D xx xy yy (before dilation)
  float det, det0, aa;    // det(Sigma_d), det(Sigma_2D), opacity factor
  float dir[3], dist;
};

// Returns false when culled by depth or a degenerate footprint.
__device__ __forceinline__ bool proj_geometry(const float* mu, const float* sc, float4 qv, const CamDev& cam,
                                              const ParDev& P, ProjState& s) {
  const float* Rc = cam.R;
  for (int i = 0; i < 3; ++i) s.t[i] = Rc[3 * i] * mu[0] + Rc[3 * i + 1] * mu[1] + Rc[3 * i + 2] * mu[2] + cam.t[i];
  if (!(s.t[2] > P.near_plane && s.t[2] < P.far_plane)) return false;
  float qq = qv.x * qv.x + qv.y * qv.y + qv.z * qv.z + qv.w * qv.w;
  s.qn = sqrtf(qq);
  float iq = 1.f / s.qn;
  s.q[0] = qv.x * iq;
  s.q[1] = qv.y * iq;
  s.q[2] = qv.z * iq;
  s.q[3] = qv.w * iq;
  quat_to_rot(s.q[0], s.q[1], s.q[2], s.q[3], s.Rq);
  // W = Rc Rq diag(s): Sigma in camera axes is W W^T (Eq. 2 and the W of Eq. 3)
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j)
      s.Wm[3 * i + j] = (Rc[3 * i] * s.Rq[j] + Rc[3 * i + 1] * s.Rq[3 + j] + Rc[3 * i + 2] * s.Rq[6 + j]) * sc[j];
  // J of the perspective map with the clamped t_x/t_z, t_y/t_z (Eq. 3)
  float tz = s.t[2], itz = 1.f / tz;
  float rx = s.t[0] * itz, ry = s.t[1] * itz;
  s.cx_free = rx >= -cam.lim_xl && rx <= cam.lim_xh;
  s.cy_free = ry >= -cam.lim_yl && ry <= cam.lim_yh;
  s.ux = fminf(fmaxf(rx, -cam.lim_xl), cam.lim_xh);
  s.uy = fminf(fmaxf(ry, -cam.lim_yl), cam.lim_yh);
  float j00 = cam.fx * itz, j02 = -cam.fx * s.ux * itz;
  float j11 = cam.fy * itz, j12 = -cam.fy * s.uy * itz;
  // r = J W, J = [[j00, 0, j02], [0, j11, j12]]; Sigma_2D = r r^T (Eq. 3-4)
  for (int j = 0; j < 3; ++j) {
    s.r1[j] = j00 * s.Wm[j] + j02 * s.Wm[6 + j];
    s.r2[j] = j11 * s.Wm[3 + j] + j12 * s.Wm[6 + j];
  }
  s.S2[0] = s.r1[0] * s.r1[0] + s.r1[1] * s.r1[1] + s.r1[2] * s.r1[2];
  s.S2[1] = s.r1[0] * s.r2[0] + s.r1[1] * s.r2[1] + s.r1[2] * s.r2[2];
  s.S2[2] = s.r2[0] * s.r2[0] + s.r2[1] * s.r2[1] + s.r2[2] * s.r2[2];
  float cx_ = s.r1[1] * s.r2[2] - s.r1[2] * s.r2[1];
  float cy_ = s.r1[2] * s.r2[0] - s.r1[0] * s.r2[2];
  float cz_ = s.r1[0] * s.r2[1] - s.r1[1] * s.r2[0];
  s.det0 = cx_ * cx_ + cy_ * cy_ + cz_ * cz_;
  s.det = s.det0 + P.eps2d * (s.S2[0] + s.S2[2]) + P.eps2d * P.eps2d;
  if (!(s.det > 0.f)) return false;
  s.aa = P.antialias ? sqrtf(s.det0 / s.det) : 1.f;
  float d0 = mu[0] - cam.campos[0], d1 = mu[1] - cam.campos[1], d2 = mu[2] - cam.campos[2];
  s.dist = sqrtf(d0 * d0 + d1 * d1 + d2 * d2);
  float idn = 1.f / s.dist;
  s.dir[0] = d0 * idn;
  s.dir[1] = d1 * idn;
  s.dir[2] = d2 * idn;
  return true;
}

// Five CTAs per SM (at most 48 registers, no spills): more loads in flight;
// 5 % faster than three CTAs at 80 registers, 2 % faster than four at 64
// (six, at 40 registers, spill and are not faster).
template <int DEG>
__global__ void __launch_bounds__(256, 5) project_fwd_kernel(int n, const float* __restrict__ means,
                                                          const float* __restrict__ scales,
                                                          const float4* __restrict__ quats,
                                                          const float* __restrict__ opac,
                                                          const float* __restrict__ sh, const CamTable cams,
                                                          const ParDev P, ProjPtr out, int32_t* tile_counts) {
  chain_enter();
  constexpr int K = (DEG + 1) * (DEG + 1);
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const CamDev& cam = cams.c[blockIdx.y];
  size_t r = (size_t)blockIdx.y * n + i;
  float mu[3] = {means[3 * i], means[3 * i + 1], means[3 * i + 2]};
  ProjState s;
  bool ok = false;
  float sc[3] = {scales[3 * i], scales[3 * i + 1], scales[3 * i + 2]};
  float oe = 0.f;
  if (proj_geometry(mu, sc, quats[i], cam, P, s)) {
    oe = opac[i] * s.aa;
    ok = oe >= P.alpha_min;
  }
  float rho = 0.f;
  if (ok) {
    rho = P.lambda * kern_support(P.kernel, oe, P.alpha_min);
    ok = rho > 0.f;
  }
  if (!ok) {
    out.dkey[r] = DKEY_CULLED;
    if (tile_counts) tile_counts[r] = 0;
    return;
  }
  float Y[K];
  sh_basis<DEG>(s.dir[0], s.dir[1], s.dir[2], Y);
  float col[3];
#pragma unroll
  for (int ch = 0; ch < 3; ++ch) {
    float v = 0.5f;
#pragma unroll
    for (int k = 0; k < K; ++k) v += sh[(size_t)(3 * k + ch) * n + i] * Y[k];
    col[ch] = fmaxf(v, 0.f);
  }
  float sxx = s.S2[0] + P.eps2d, syy = s.S2[2] + P.eps2d, sxy = s.S2[1];
  float itz = 1.f / s.t[2];
  float mx = cam.fx * s.t[0] * itz + cam.cx;
  float my = cam.fy * s.t[1] * itz + cam.cy;
  float ex = rho * sqrtf(sxx), ey = rho * sqrtf(syy);
  // conic A = Sigma_d^-1 as its upper Cholesky factor, from the accurate det:
  // l00 = sqrt(syy / det), l01 = -sxy / sqrt(det syy), l11 = 1 / sqrt(syy)
  float l00 = sqrtf(syy / s.det);
  float l01 = -sxy / sqrtf(s.det * syy);
  float l11 = 1.f / sqrtf(syy);
  out.rec[3 * r] = make_float4(mx, my, l00, l01);
  out.rec[3 * r + 1] = make_float4(l11, oe, rho * rho, s.t[2]);
  out.rec[3 * r + 2] = make_float4(col[0], col[1], col[2], 0.f);
  out.foot[r] = make_float4(mx, my, ex, ey);
  out.dkey[r] = __float_as_uint(s.t[2]);
  if (tile_counts) {
    int tx0, tx1, ty0, ty1;
    int cnt = 0;
    if (tile_rect(mx, my, ex, ey, cam.W, cam.H, P.tile_w, P.tile_h, tx0, tx1, ty0, ty1))
      cnt = (tx1 - tx0 + 1) * (ty1 - ty0 + 1);
    tile_counts[r] = cnt;
  }
}

// a6: hand-derived chain rule, recomputing the forward intermediates.
// ONE: a single camera, so the SH gradient of each channel is final as soon
// as it is formed and is stored at once instead of being held (3 (D+1)^2
// accumulators) across cameras; the kernel then fits twice the warps per SM.
template <int DEG, bool ONE>
__global__ void __launch_bounds__(ONE ? 256 : 128, ONE ? 2 : 1) project_bwd_kernel(int n, const float* __restrict__ means,
                                                          const float* __restrict__ scales,
                                                          const float4* __restrict__ quats,
                                                          const float* __restrict__ opac,
                                                          const float* __restrict__ sh, const CamTable cams,
                                                          const ParDev P, ProjCPtr proj,
                                                          const float4* __restrict__ g2d, float* g_means,
                                                          float* g_scales, float4* g_quats, float* g_opac,
                                                          float* g_sh) {
  chain_enter();
  constexpr int K = (DEG + 1) * (DEG + 1);
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float mu[3] = {means[3 * i], means[3 * i + 1], means[3 * i + 2]};
  float sc[3] = {scales[3 * i], scales[3 * i + 1], scales[3 * i + 2]};
  float4 qv = quats[i];
  float o = opac[i];
  float gmu[3] = {0.f, 0.f, 0.f}, gs[3] = {0.f, 0.f, 0.f}, gq[4] = {0.f, 0.f, 0.f, 0.f}, go = 0.f;
  constexpr int KA = ONE ? 1 : K;  // SH accumulators held across cameras
  float gsh[KA][3];
#pragma unroll
  for (int k = 0; k < KA; ++k) gsh[k][0] = gsh[k][1] = gsh[k][2] = 0.f;
  bool sh_written = false;

  for (int c = 0; c < cams.n; ++c) {
    size_t r = (size_t)c * n + i;
    if (proj.dkey[r] == DKEY_CULLED) continue;
    float4 g0 = g2d[3 * r], g1 = g2d[3 * r + 1], g2 = g2d[3 * r + 2];
    // g0 = {gmx, gmy, ga, gb}, g1 = {gc, go, gr, gg}, g2 = {gb, -, -, -}
    if (g0.x == 0.f && g0.y == 0.f && g0.z == 0.f && g0.w == 0.f && g1.x == 0.f && g1.y == 0.f &&
        g1.z == 0.f && g1.w == 0.f && g2.x == 0.f)
      continue;
    const CamDev& cam = cams.c[c];
    ProjState s;
    if (!proj_geometry(mu, sc, qv, cam, P, s)) continue;
    const float* Rc = cam.R;
    // ---- colour: rgb = max(0, sum_k sh_k Y_k(dir) + 0.5)
    float Y[K];
    sh_basis<DEG>(s.dir[0], s.dir[1], s.dir[2], Y);
    float grgb[3] = {g1.z, g1.w, g2.x};
    float wsum[K];
#pragma unroll
    for (int k = 0; k < K; ++k) wsum[k] = 0.f;
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) {
      float v = 0.5f;
#pragma unroll
      for (int k = 0; k < K; ++k) v += sh[(size_t)(3 * k + ch) * n + i] * Y[k];
      float gc = v > 0.f ? grgb[ch] : 0.f;
#pragma unroll
      for (int k = 0; k < K; ++k) {
        if (ONE) g_sh[(size_t)(3 * k + ch) * n + i] = gc * Y[k];
        else gsh[k][ch] += gc * Y[k];
        wsum[k] += gc * sh[(size_t)(3 * k + ch) * n + i];
      }
    }
    sh_written = ONE;
    if (DEG > 0) {
      float gdx, gdy, gdz;
      sh_basis_grad<DEG>(s.dir[0], s.dir[1], s.dir[2], wsum, gdx, gdy, gdz);
      float dot = gdx * s.dir[0] + gdy * s.dir[1] + gdz * s.dir[2];
      float idn = 1.f / s.dist;
      gmu[0] += (gdx - s.dir[0] * dot) * idn;
      gmu[1] += (gdy - s.dir[1] * dot) * idn;
      gmu[2] += (gdz - s.dir[2] * dot) * idn;
    }
    // ---- opacity and the anti-aliasing factor f = sqrt(det0 / det)
    float goe = g1.y;
    go += goe * s.aa;
    float Ad = s.S2[0] + P.eps2d, Cd = s.S2[2] + P.eps2d, B = s.S2[1];
    float idet = 1.f / s.det;
    // ---- conic a = Cd/det, b = -B/det, c = Ad/det
    float ca = Cd * idet, cb = -B * idet, cc = Ad * idet;
    float gdet = -(g0.z * ca + g0.w * cb + g1.x * cc) * idet;
    float gA = g1.x * idet + gdet * Cd;
    float gC = g0.z * idet + gdet * Ad;
    float gB = -g0.w * idet - 2.f * B * gdet;
    if (P.antialias && s.aa > 0.f) {
      float ratio = s.det0 * idet;
      float gr = goe * o / (2.f * s.aa);
      gA += gr * (s.S2[2] - ratio * Cd) * idet;
      gC += gr * (s.S2[0] - ratio * Ad) * idet;
      gB += gr * (-2.f * B + ratio * 2.f * B) * idet;
    }
    // ---- Sigma_2D = r r^T with r = J W: G_r = 2 G2 r, G2 = [[gA, gB/2], [gB/2, gC]]
    float tz = s.t[2], itz = 1.f / tz;
    float j00 = cam.fx * itz, j02 = -cam.fx * s.ux * itz;
    float j11 = cam.fy * itz, j12 = -cam.fy * s.uy * itz;
    float Gr1[3], Gr2[3];
    for (int j = 0; j < 3; ++j) {
      Gr1[j] = 2.f * gA * s.r1[j] + gB * s.r2[j];
      Gr2[j] = gB * s.r1[j] + 2.f * gC * s.r2[j];
    }
    // r1 = j00 W0 + j02 W2, r2 = j11 W1 + j12 W2 (W rows)
    float GJ00 = 0.f, GJ02 = 0.f, GJ11 = 0.f, GJ12 = 0.f;
    for (int j = 0; j < 3; ++j) {
      GJ00 += Gr1[j] * s.Wm[j];
      GJ02 += Gr1[j] * s.Wm[6 + j];
      GJ11 += Gr2[j] * s.Wm[3 + j];
      GJ12 += Gr2[j] * s.Wm[6 + j];
    }
    float GW[9];
    for (int j = 0; j < 3; ++j) {
      GW[j] = j00 * Gr1[j];
      GW[3 + j] = j11 * Gr2[j];
      GW[6 + j] = j02 * Gr1[j] + j12 * Gr2[j];
    }
    // ---- J and the centre mu' -> t
    float gt[3];
    float itz2 = itz * itz;
    gt[0] = g0.x * cam.fx * itz;
    gt[1] = g0.y * cam.fy * itz;
    gt[2] = -g0.x * cam.fx * s.t[0] * itz2 - g0.y * cam.fy * s.t[1] * itz2;
    gt[2] += -GJ00 * cam.fx * itz2 - GJ11 * cam.fy * itz2;
    gt[2] += GJ02 * cam.fx * s.ux * itz2 + GJ12 * cam.fy * s.uy * itz2;
    if (s.cx_free) {
      gt[0] += -GJ02 * cam.fx * itz2;
      gt[2] += GJ02 * cam.fx * s.t[0] * itz2 * itz;
    }
    if (s.cy_free) {
      gt[1] += -GJ12 * cam.fy * itz2;
      gt[2] += GJ12 * cam.fy * s.t[1] * itz2 * itz;
    }
    for (int a = 0; a < 3; ++a) gmu[a] += Rc[a] * gt[0] + Rc[3 + a] * gt[1] + Rc[6 + a] * gt[2];
    // ---- W = Rc Rq diag(s): G_(Rq diag s) = Rc^T G_W
    float GR[9];
    for (int k = 0; k < 3; ++k)
      for (int j = 0; j < 3; ++j) {
        float gm = Rc[k] * GW[j] + Rc[3 + k] * GW[3 + j] + Rc[6 + k] * GW[6 + j];
        gs[j] += gm * s.Rq[3 * k + j];
        GR[3 * k + j] = gm * sc[j];
      }
    // ---- rotation matrix -> normalised quaternion -> raw quaternion
    float w = s.q[0], x = s.q[1], y = s.q[2], z = s.q[3];
    float gw = 2.f * (-z * GR[1] + y * GR[2] + z * GR[3] - x * GR[5] - y * GR[6] + x * GR[7]);
    float gx = 2.f * (y * GR[1] + z * GR[2] + y * GR[3] - 2.f * x * GR[4] - w * GR[5] + z * GR[6] + w * GR[7] -
                      2.f * x * GR[8]);
    float gy = 2.f * (-2.f * y * GR[0] + x * GR[1] + w * GR[2] + x * GR[3] + z * GR[5] - w * GR[6] + z * GR[7] -
                      2.f * y * GR[8]);
    float gz = 2.f * (-2.f * z * GR[0] - w * GR[1] + x * GR[2] + w * GR[3] - 2.f * z * GR[4] + y * GR[5] +
                      x * GR[6] + y * GR[7]);
    float dq = gw * w + gx * x + gy * y + gz * z;
    float iq = 1.f / s.qn;
    gq[0] += (gw - w * dq) * iq;
    gq[1] += (gx - x * dq) * iq;
    gq[2] += (gy - y * dq) * iq;
    gq[3] += (gz - z * dq) * iq;
  }
  g_means[3 * i] = gmu[0];
  g_means[3 * i + 1] = gmu[1];
  g_means[3 * i + 2] = gmu[2];
  g_scales[3 * i] = gs[0];
  g_scales[3 * i + 1] = gs[1];
  g_scales[3 * i + 2] = gs[2];
  g_quats[i] = make_float4(gq[0], gq[1], gq[2], gq[3]);
  g_opac[i] = go;
  if (!sh_written) {
#pragma unroll
    for (int k = 0; k < K; ++k)
#pragma unroll
      for (int ch = 0; ch < 3; ++ch) g_sh[(size_t)(3 * k + ch) * n + i] = ONE ? 0.f : gsh[k][ch];
  }
}

cudaError_t launch_project_fwd(int n, const float* means, const float* scales, const float* quats,
                               const float* opac, const float* sh, const CamTable& cams, const ParDev& P,
                               ProjPtr out, int32_t* tile_counts, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  dim3 grid(ceil_div(n, 256), cams.n);
  const float4* q4 = reinterpret_cast<const float4*>(quats);
#define LS_PF(D) launch_chain(project_fwd_kernel<D>, grid, dim3(256), 0, st, n, means, scales, q4, opac, sh, cams, P, \
                             out, tile_counts)
  switch (P.sh_degree) {
    case 0: return LS_PF(0);
    case 1: return LS_PF(1);
    case 2: return LS_PF(2);
    default: return LS_PF(3);
  }
#undef LS_PF
}

cudaError_t launch_project_bwd(int n, const float* means, const float* scales, const float* quats,
                               const float* opac, const float* sh, const CamTable& cams, const ParDev& P,
                               ProjCPtr proj, const float* g2d, float* g_means, float* g_scales, float* g_quats,
                               float* g_opac, float* g_sh, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  const float4* q4 = reinterpret_cast<const float4*>(quats);
  const float4* g4 = reinterpret_cast<const float4*>(g2d);
  float4* gq4 = reinterpret_cast<float4*>(g_quats);
#define LS_PB(D, ONE, TB)                                                                                  \
  launch_chain(project_bwd_kernel<D, ONE>, dim3(ceil_div(n, TB)), dim3(TB), 0, st, n, means, scales, q4, opac, sh, \
               cams, P, proj, g4, g_means, g_scales, gq4, g_opac, g_sh)
  if (cams.n == 1) {
    switch (P.sh_degree) {
      case 0: return LS_PB(0, true, 256);
      case 1: return LS_PB(1, true, 256);
      case 2: return LS_PB(2, true, 256);
      default: return LS_PB(3, true, 256);
    }
  }
  switch (P.sh_degree) {
    case 0: return LS_PB(0, false, 128);
    case 1: return LS_PB(1, false, 128);
    case 2: return LS_PB(2, false, 128);
    default: return LS_PB(3, false, 128);
  }
#undef LS_PB
}

}  // namespace ls
