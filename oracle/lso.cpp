// FP64 CPU oracle for 3D Linear Splatting (arxiv 2411.12440).
//
// TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
// call this file; only tests/, the package smoke check and the benchmark's
// CPU-baseline leg do.  It shares no code with the CUDA implementation.
//
// What it computes, and where the paper defines it:
//   * primitive covariance  Sigma = R S S^T R^T                 Sec. 3.1, Eq. 2
//   * EWA projection  Sigma' = J W Sigma W^T J^T, Sigma_2D = top-left 2x2
//                                                               Sec. 3.1, Eq. 3-4
//   * Mahalanobis distance D'_M of a pixel to the projected centre
//                                                               Sec. 3.2, Eq. 8, 11
//   * linear kernel with distribution alignment  max(0, 1 - D/lambda)
//                                                               Sec. 3.3.1, Eq. 12
//   * kernel family f(D/lambda) (Gaussian, Laplacian, raised cosine,
//     quadratic, linear)                                        Appendix B, Eq. 19-25
//   * front-to-back compositing  C = sum c_i a_i prod_{j<i}(1 - a_j),
//     a_i = o_i K_i(x')                                          Sec. 3.1, Eq. 6
//   * adaptive gradient scaling  w(D) = exp(-D^2) on the kernel-derivative
//     path of the adjoint                                       Sec. 3.3.2, Eq. 13-14
//
// Readings where the paper is silent (3DGS conventions the paper says it keeps
// unchanged, Sec. 3.2): near/far cull, Jacobian clamp at 1.3x the half field of
// view, a 2D dilation eps2d*I, the Mip-Splatting opacity compensation when
// anti-aliasing is on, pixel centre at (px+0.5, py+0.5), alpha clamp
// alpha_max, alpha skip below alpha_min, stop when T would fall below T_min
// (that entry excluded), ties in depth broken by primitive id, real SH basis
// with the Condon-Shortley phase (3DGS sign table), colour = SH + 0.5 clamped
// at 0.  The anti-aliasing compensation o * sqrt(det Sigma_2D / det(Sigma_2D +
// eps2d I)) is a reading of the Mip-Splatting 2D filter named in Sec. 4.1;
// the tests pin the factor itself (closed forms, and the footprint integral
// that it keeps independent of eps2d).
//
// Design: slow and plain.  The projection is written once as a template over
// the scalar type; instantiated with forward-mode dual numbers it yields exact
// projection derivatives (no hand-derived chain rule).  The blend adjoint keeps
// the forward transmittances instead of recomputing them.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

const double PI = 3.14159265358979323846;

// ---------------------------------------------------------------- dual numbers
struct Dual {
  double v, d;
  Dual(double x = 0.0, double dx = 0.0) : v(x), d(dx) {}
};
inline Dual operator+(Dual a, Dual b) { return Dual(a.v + b.v, a.d + b.d); }
inline Dual operator-(Dual a, Dual b) { return Dual(a.v - b.v, a.d - b.d); }
inline Dual operator-(Dual a) { return Dual(-a.v, -a.d); }
inline Dual operator*(Dual a, Dual b) { return Dual(a.v * b.v, a.d * b.v + a.v * b.d); }
inline Dual operator/(Dual a, Dual b) { return Dual(a.v / b.v, (a.d * b.v - a.v * b.d) / (b.v * b.v)); }
inline Dual operator+(Dual a, double b) { return Dual(a.v + b, a.d); }
inline Dual operator+(double a, Dual b) { return Dual(a + b.v, b.d); }
inline Dual operator-(Dual a, double b) { return Dual(a.v - b, a.d); }
inline Dual operator-(double a, Dual b) { return Dual(a - b.v, -b.d); }
inline Dual operator*(Dual a, double b) { return Dual(a.v * b, a.d * b); }
inline Dual operator*(double a, Dual b) { return Dual(a * b.v, a * b.d); }
inline Dual operator/(Dual a, double b) { return Dual(a.v / b, a.d / b); }
inline Dual operator/(double a, Dual b) { return Dual(a / b.v, -a * b.d / (b.v * b.v)); }
inline Dual sqrt(Dual a) {
  double s = std::sqrt(a.v);
  return Dual(s, s > 0 ? a.d / (2.0 * s) : 0.0);
}
inline double val(double x) { return x; }
inline double val(Dual x) { return x.v; }
inline double dsqrt(double x) { return std::sqrt(x); }
inline Dual dsqrt(Dual x) { return sqrt(x); }
// max(0, x) and clamp keep the derivative only on the active branch.
template <class T> T relu(T x) { return val(x) > 0 ? x : T(0.0); }
template <class T> T clampv(T x, double lo, double hi) {
  if (val(x) < lo) return T(lo);
  if (val(x) > hi) return T(hi);
  return x;
}

// ---------------------------------------------------------------- parameters
struct Par {
  double lambda;
  int kernel;  // 0 linear, 1 gaussian, 2 laplacian, 3 raised cosine, 4 quadratic
  int ags;     // 0 off, 1 w = exp(-D^2), 2 w = exp(-(D/lambda)^2)
  int antialias;
  double eps2d, alpha_min, alpha_max, t_min;
  int tile_w, tile_h;
  double bg[3];
  double near_plane, far_plane;
  int sh_degree;
};
Par unpack_par(const double* p) {
  Par P;
  P.lambda = p[0];
  P.kernel = (int)p[1];
  P.ags = (int)p[2];
  P.antialias = (int)p[3];
  P.eps2d = p[4];
  P.alpha_min = p[5];
  P.alpha_max = p[6];
  P.t_min = p[7];
  P.tile_w = (int)p[8];
  P.tile_h = (int)p[9];
  P.bg[0] = p[10];
  P.bg[1] = p[11];
  P.bg[2] = p[12];
  P.near_plane = p[13];
  P.far_plane = p[14];
  P.sh_degree = (int)p[15];
  return P;
}

struct Cam {
  double R[3][3], t[3];
  double fx, fy, cx, cy;
  int W, H;
};
Cam unpack_cam(const double* c) {
  Cam C;
  for (int i = 0; i < 3; ++i) {
    for (int j = 0; j < 3; ++j) C.R[i][j] = c[4 * i + j];
    C.t[i] = c[4 * i + 3];
  }
  C.fx = c[16];
  C.fy = c[17];
  C.cx = c[18];
  C.cy = c[19];
  C.W = (int)c[20];
  C.H = (int)c[21];
  return C;
}

// ---------------------------------------------------------------- kernel family
// f(x) with x = D / lambda (Appendix B, Eq. 20-25 with the alignment of Eq. 26).
double kern_f(int k, double x) {
  switch (k) {
    case 1: return std::exp(-0.5 * x * x);
    case 2: return std::exp(-x);
    case 3: return x <= 1.0 ? 0.5 * (1.0 + std::cos(PI * x)) : 0.0;
    case 4: return std::max(0.0, 1.0 - x * x);
    default: return std::max(0.0, 1.0 - x);
  }
}
double kern_df(int k, double x) {  // df/dx inside the support
  switch (k) {
    case 1: return -x * std::exp(-0.5 * x * x);
    case 2: return -std::exp(-x);
    case 3: return x <= 1.0 ? -0.5 * PI * std::sin(PI * x) : 0.0;
    case 4: return x < 1.0 ? -2.0 * x : 0.0;
    default: return x < 1.0 ? -1.0 : 0.0;
  }
}
// Largest x with o * f(x) >= alpha_min (0 when o < alpha_min).
double kern_support(int k, double o, double amin) {
  double m = amin / o;
  if (m > 1.0) return 0.0;
  if (m <= 0.0) {
    // no alpha threshold: compact kernels end at x = 1; infinite tails use 3.
    return (k == 1 || k == 2) ? 3.0 : 1.0;
  }
  switch (k) {
    case 1: return std::sqrt(2.0 * std::log(1.0 / m));
    case 2: return std::log(1.0 / m);
    case 3: return std::acos(2.0 * m - 1.0) / PI;
    case 4: return std::sqrt(1.0 - m);
    default: return 1.0 - m;
  }
}

// ---------------------------------------------------------------- real SH basis
// Built from the Legendre polynomials (Bonnet recursion) and
// Re/Im (x + i y)^m, so no trigonometry and no tabulated products:
//   Y_l0 = K_l0 P_l(z),
//   Y_l,+m = sqrt2 K_lm (-1)^m P_l^(m)(z) Re (x+iy)^m,
//   Y_l,-m = sqrt2 K_lm (-1)^m P_l^(m)(z) Im (x+iy)^m,
//   K_lm = sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!); index l^2 + l + m.
struct ShTables {
  double dleg[4][4][4];  // [l][m][k]: coefficient of z^k in d^m P_l / dz^m
  double K[4][4];
  ShTables() {
    double leg[4][4] = {{0}};
    leg[0][0] = 1.0;
    leg[1][1] = 1.0;
    for (int n = 1; n < 3; ++n)
      for (int k = 0; k < 4; ++k) {
        double zp = k > 0 ? leg[n][k - 1] : 0.0;
        leg[n + 1][k] = ((2 * n + 1) * zp - n * leg[n - 1][k]) / (n + 1);
      }
    std::memset(dleg, 0, sizeof(dleg));
    for (int l = 0; l < 4; ++l) {
      for (int k = 0; k < 4; ++k) dleg[l][0][k] = leg[l][k];
      for (int m = 1; m < 4; ++m)
        for (int k = 0; k < 3; ++k) dleg[l][m][k] = (k + 1) * dleg[l][m - 1][k + 1];
    }
    auto fact = [](int n) { double f = 1; for (int i = 2; i <= n; ++i) f *= i; return f; };
    for (int l = 0; l < 4; ++l)
      for (int m = 0; m <= l; ++m)
        K[l][m] = std::sqrt((2 * l + 1) / (4 * PI) * fact(l - m) / fact(l + m));
  }
};
const ShTables& sht() {
  static ShTables t;
  return t;
}

template <class T> void sh_basis(int deg, T x, T y, T z, T* out) {
  const ShTables& S = sht();
  // powers of (x + i y)
  T re[4], im[4];
  re[0] = T(1.0);
  im[0] = T(0.0);
  for (int m = 1; m < 4; ++m) {
    re[m] = re[m - 1] * x - im[m - 1] * y;
    im[m] = re[m - 1] * y + im[m - 1] * x;
  }
  for (int l = 0; l <= deg; ++l) {
    for (int m = 0; m <= l; ++m) {
      T p(0.0);
      for (int k = 3; k >= 0; --k) p = p * z + S.dleg[l][m][k];
      double sgn = (m % 2) ? -1.0 : 1.0;
      if (m == 0) {
        out[l * l + l] = S.K[l][0] * p;
      } else {
        double c = std::sqrt(2.0) * S.K[l][m] * sgn;
        out[l * l + l + m] = c * p * re[m];
        out[l * l + l - m] = c * p * im[m];
      }
    }
  }
}

// ---------------------------------------------------------------- projection
// Projected record, doubles: see NP_* indices.
enum { P_MX, P_MY, P_A, P_B, P_C, P_O, P_RHO2, P_DEPTH, P_R, P_G, P_BL, P_EX, P_EY, P_SXX, P_SXY, P_SYY, NP };

// Sec. 3.1, Eq. 1-4 and Sec. 3.3.1, Eq. 12; returns false when culled.
template <class T>
bool project_one(const T mu[3], const T sc[3], const T qv[4], T o, const T* sh, int deg,
                 const Cam& cam, const Par& P, T out[NP]) {
  // camera-space centre t = W mu
  T t[3];
  for (int i = 0; i < 3; ++i)
    t[i] = cam.R[i][0] * mu[0] + cam.R[i][1] * mu[1] + cam.R[i][2] * mu[2] + cam.t[i];
  if (!(val(t[2]) > P.near_plane && val(t[2]) < P.far_plane)) return false;
  // rotation from the normalised quaternion (w, x, y, z)
  T qn = dsqrt(qv[0] * qv[0] + qv[1] * qv[1] + qv[2] * qv[2] + qv[3] * qv[3]);
  T w = qv[0] / qn, x = qv[1] / qn, y = qv[2] / qn, z = qv[3] / qn;
  T R[3][3] = {
      {1.0 - 2.0 * (y * y + z * z), 2.0 * (x * y - w * z), 2.0 * (x * z + w * y)},
      {2.0 * (x * y + w * z), 1.0 - 2.0 * (x * x + z * z), 2.0 * (y * z - w * x)},
      {2.0 * (x * z - w * y), 2.0 * (y * z + w * x), 1.0 - 2.0 * (x * x + y * y)}};
  // Sigma = (R S)(R S)^T   (Eq. 2)
  T M[3][3], Sig[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) M[i][j] = R[i][j] * sc[j];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      T s(0.0);
      for (int k = 0; k < 3; ++k) s = s + M[i][k] * M[j][k];
      Sig[i][j] = s;
    }
  // V = W Sigma W^T (rotation part of the view matrix)
  T RS[3][3], V[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      T s(0.0);
      for (int k = 0; k < 3; ++k) s = s + cam.R[i][k] * Sig[k][j];
      RS[i][j] = s;
    }
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      T s(0.0);
      for (int k = 0; k < 3; ++k) s = s + RS[i][k] * cam.R[j][k];
      V[i][j] = s;
    }
  // local affine Jacobian of the perspective map, with t_x/t_z, t_y/t_z
  // clamped to 1.3x the half field of view (reading of Eq. 3).
  double W = cam.W, H = cam.H;
  double lxl = (cam.cx + 0.15 * W) / cam.fx, lxh = (W - cam.cx + 0.15 * W) / cam.fx;
  double lyl = (cam.cy + 0.15 * H) / cam.fy, lyh = (H - cam.cy + 0.15 * H) / cam.fy;
  T ux = clampv(t[0] / t[2], -lxl, lxh);
  T uy = clampv(t[1] / t[2], -lyl, lyh);
  T J[2][3] = {{cam.fx / t[2], T(0.0), -cam.fx * ux / t[2]},
               {T(0.0), cam.fy / t[2], -cam.fy * uy / t[2]}};
  // Sigma_2D = J V J^T  (Eq. 3-4)
  T JV[2][3], S2[2][2];
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 3; ++j) {
      T s(0.0);
      for (int k = 0; k < 3; ++k) s = s + J[i][k] * V[k][j];
      JV[i][j] = s;
    }
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 2; ++j) {
      T s(0.0);
      for (int k = 0; k < 3; ++k) s = s + JV[i][k] * J[j][k];
      S2[i][j] = s;
    }
  T sxx = S2[0][0] + P.eps2d, syy = S2[1][1] + P.eps2d, sxy = S2[0][1];
  T det = sxx * syy - sxy * sxy;
  if (!(val(det) > 0)) return false;
  T oe = o;
  if (P.antialias) {
    T det0 = S2[0][0] * S2[1][1] - S2[0][1] * S2[0][1];
    oe = o * dsqrt(relu(det0 / det));
  }
  if (!(val(oe) >= P.alpha_min)) return false;
  double xs = kern_support(P.kernel, val(oe), P.alpha_min);
  if (!(xs > 0)) return false;
  double rho = P.lambda * xs;
  // colour from SH at the viewing direction (mu - camera centre)
  double cc[3];
  for (int i = 0; i < 3; ++i)
    cc[i] = -(cam.R[0][i] * cam.t[0] + cam.R[1][i] * cam.t[1] + cam.R[2][i] * cam.t[2]);
  T dv[3] = {mu[0] - cc[0], mu[1] - cc[1], mu[2] - cc[2]};
  T dn = dsqrt(dv[0] * dv[0] + dv[1] * dv[1] + dv[2] * dv[2]);
  T Y[16];
  sh_basis(deg, dv[0] / dn, dv[1] / dn, dv[2] / dn, Y);
  int K = (deg + 1) * (deg + 1);
  for (int ch = 0; ch < 3; ++ch) {
    T s(0.0);
    for (int k = 0; k < K; ++k) s = s + sh[3 * k + ch] * Y[k];
    out[P_R + ch] = relu(s + 0.5);
  }
  out[P_MX] = cam.fx * t[0] / t[2] + cam.cx;
  out[P_MY] = cam.fy * t[1] / t[2] + cam.cy;
  out[P_A] = syy / det;
  out[P_B] = -sxy / det;
  out[P_C] = sxx / det;
  out[P_O] = oe;
  out[P_RHO2] = T(rho * rho);
  out[P_DEPTH] = t[2];
  out[P_EX] = rho * dsqrt(sxx);
  out[P_EY] = rho * dsqrt(syy);
  out[P_SXX] = sxx;
  out[P_SXY] = sxy;
  out[P_SYY] = syy;
  return true;
}

// ---------------------------------------------------------------- tile rule
struct Rect { int x0, x1, y0, y1; bool empty; };

// Pixel range of the exact bounding box of the support ellipse, pixel centre
// at +0.5; FP64 reading.
Rect rect_f64(double mx, double my, double ex, double ey, int W, int H) {
  Rect r;
  double xl = std::ceil(mx - ex - 0.5), xh = std::floor(mx + ex - 0.5);
  double yl = std::ceil(my - ey - 0.5), yh = std::floor(my + ey - 0.5);
  r.empty = !(xl <= xh && yl <= yh) || xh < 0 || yh < 0 || xl > W - 1 || yl > H - 1;
  if (r.empty) { r.x0 = r.x1 = r.y0 = r.y1 = 0; return r; }
  r.x0 = (int)std::max(xl, 0.0);
  r.x1 = (int)std::min(xh, (double)(W - 1));
  r.y0 = (int)std::max(yl, 0.0);
  r.y1 = (int)std::min(yh, (double)(H - 1));
  return r;
}

// The same rule in IEEE binary32, evaluated as written (this file is built
// with -ffp-contract=off, so no fused multiply-add is formed).
Rect rect_f32(float mx, float my, float ex, float ey, int W, int H) {
  Rect r;
  volatile float a = mx - ex, b = mx + ex, c = my - ey, d = my + ey;
  float xl = std::ceil((float)(a - 0.5f)), xh = std::floor((float)(b - 0.5f));
  float yl = std::ceil((float)(c - 0.5f)), yh = std::floor((float)(d - 0.5f));
  r.empty = !(xl <= xh && yl <= yh) || xh < 0.0f || yh < 0.0f || xl > (float)(W - 1) ||
            yl > (float)(H - 1);
  if (r.empty) { r.x0 = r.x1 = r.y0 = r.y1 = 0; return r; }
  r.x0 = (int)std::max(xl, 0.0f);
  r.x1 = (int)std::min(xh, (float)(W - 1));
  r.y0 = (int)std::max(yl, 0.0f);
  r.y1 = (int)std::min(yh, (float)(H - 1));
  return r;
}

uint32_t f32bits(double x) {
  float f = (float)x;
  uint32_t u;
  std::memcpy(&u, &f, 4);
  return u;
}

// Per-tile lists in front-to-back order: (depth as binary32 bits, id).
struct Lists {
  int tiles_x, tiles_y;
  std::vector<std::vector<int>> L;
};
Lists build_lists(int n, const double* proj, const unsigned char* vis, int W, int H, const Par& P,
                  int rule_f32, const uint32_t* dkey) {
  Lists out;
  out.tiles_x = (W + P.tile_w - 1) / P.tile_w;
  out.tiles_y = (H + P.tile_h - 1) / P.tile_h;
  out.L.assign((size_t)out.tiles_x * out.tiles_y, {});
  for (int i = 0; i < n; ++i) {
    if (!vis[i]) continue;
    const double* p = proj + (size_t)i * NP;
    Rect r = rule_f32 ? rect_f32((float)p[P_MX], (float)p[P_MY], (float)p[P_EX], (float)p[P_EY], W, H)
                      : rect_f64(p[P_MX], p[P_MY], p[P_EX], p[P_EY], W, H);
    if (r.empty) continue;
    for (int ty = r.y0 / P.tile_h; ty <= r.y1 / P.tile_h; ++ty)
      for (int tx = r.x0 / P.tile_w; tx <= r.x1 / P.tile_w; ++tx)
        out.L[(size_t)ty * out.tiles_x + tx].push_back(i);
  }
  auto key = [&](int i) -> uint32_t { return dkey ? dkey[i] : f32bits(proj[(size_t)i * NP + P_DEPTH]); };
  for (auto& l : out.L)
    std::stable_sort(l.begin(), l.end(), [&](int a, int b) { return key(a) < key(b); });
  return out;
}

// ---------------------------------------------------------------- blending
struct PixOut {
  double C[3], T;
  int n_last, last_id;
  bool flag;
  int stop_index;  // index at which the pixel finished, or list length
  long long n_contrib;
};

struct PairRec { int id; double alpha, T, dx, dy, D, fx; bool clamped; };

// One pixel, front to back over `list` (Eq. 6 with the kernel of Eq. 12).
PixOut blend_pixel(const std::vector<int>& list, const double* proj, double x, double y, const Par& P,
                   std::vector<PairRec>* rec) {
  PixOut o;
  o.C[0] = o.C[1] = o.C[2] = 0.0;
  o.T = 1.0;
  o.n_last = 0;
  o.last_id = -1;
  o.flag = false;
  o.stop_index = (int)list.size();
  o.n_contrib = 0;
  for (size_t k = 0; k < list.size(); ++k) {
    const double* p = proj + (size_t)list[k] * NP;
    double dx = x - p[P_MX], dy = y - p[P_MY];
    double q = p[P_A] * dx * dx + 2.0 * p[P_B] * dx * dy + p[P_C] * dy * dy;
    double D = std::sqrt(std::max(q, 0.0));
    double xk = D / P.lambda;
    double araw = p[P_O] * kern_f(P.kernel, xk);
    if (std::fabs(araw - P.alpha_min) < 1e-5) o.flag = true;
    if (q > p[P_RHO2]) continue;
    if (std::fabs(araw - P.alpha_max) < 1e-6) o.flag = true;
    double a = std::min(P.alpha_max, araw);
    if (a < P.alpha_min) continue;
    double Tn = o.T * (1.0 - a);
    if (std::fabs(Tn - P.t_min) < 1e-9) o.flag = true;
    if (Tn < P.t_min) { o.stop_index = (int)k; break; }
    for (int c = 0; c < 3; ++c) o.C[c] += p[P_R + c] * a * o.T;
    if (rec) rec->push_back({list[k], a, o.T, dx, dy, D, xk, araw > P.alpha_max});
    o.T = Tn;
    o.n_last = (int)k + 1;
    o.last_id = list[k];
    o.n_contrib++;
  }
  return o;
}

int g_threads = 1;

}  // namespace

extern "C" {

void lso_set_threads(int n) { g_threads = n > 0 ? n : 1; }

int lso_np() { return NP; }

// Projection of n primitives through one camera, FP64.  cam: [viewmat 16
// row-major, fx, fy, cx, cy, W, H]; par: see unpack_par.  out: [n][NP].
int lso_project(int n, const double* means, const double* scales, const double* quats,
                const double* opac, const double* sh, const double* camv, const double* parv,
                double* out, unsigned char* visible) {
  Cam cam = unpack_cam(camv);
  Par P = unpack_par(parv);
  int K = (P.sh_degree + 1) * (P.sh_degree + 1);
#pragma omp parallel for num_threads(g_threads) schedule(static)
  for (int i = 0; i < n; ++i) {
    double* o = out + (size_t)i * NP;
    for (int k = 0; k < NP; ++k) o[k] = 0.0;
    visible[i] = project_one<double>(means + 3 * (size_t)i, scales + 3 * (size_t)i, quats + 4 * (size_t)i,
                                     opac[i], sh + (size_t)i * K * 3, P.sh_degree, cam, P, o)
                     ? 1 : 0;
  }
  return 0;
}

// Real SH basis values for unit directions dirs [m][3] -> out [m][16].
void lso_sh_basis(int m, int deg, const double* dirs, double* out) {
  for (int i = 0; i < m; ++i) {
    for (int k = 0; k < 16; ++k) out[16 * i + k] = 0.0;
    sh_basis<double>(deg, dirs[3 * i], dirs[3 * i + 1], dirs[3 * i + 2], out + 16 * i);
  }
}

double lso_kernel_f(int k, double x) { return kern_f(k, x); }
double lso_kernel_support(int k, double o, double amin) { return kern_support(k, o, amin); }

// Tile rectangle of one footprint: out[4] = x0 x1 y0 y1 (pixels), returns
// 1 when non-empty.  f32 selects the binary32 rule.
int lso_rect(double mx, double my, double ex, double ey, int W, int H, int f32, int* out) {
  Rect r = f32 ? rect_f32((float)mx, (float)my, (float)ex, (float)ey, W, H) : rect_f64(mx, my, ex, ey, W, H);
  out[0] = r.x0; out[1] = r.x1; out[2] = r.y0; out[3] = r.y1;
  return r.empty ? 0 : 1;
}

// Tiles of support-box row ty that a record's support ellipse reaches, in
// binary32 with every operation rounded once (the rule the tile lists
// follow): the ellipse D^2 <= L, L = 1.02 rho^2 + 1e-3, D^2 = (l00 dx +
// l01 dy)^2 + (l11 dy)^2, cut by the row's band of pixel-centre heights
// (widened by 0.01 px), is convex; its x-extent follows from its left and
// right boundaries at the leftmost / rightmost point's dy clamped into the
// band (widened by 0.01 px), and a tile is reached when its pixel-centre
// columns meet that extent.  Boxes of at most 2 tiles are taken whole.
// Result [tx_a, tx_b] clamped to the box columns [x0, x1] (empty: tx_b < tx_a).
struct ReachRec {
  bool whole;
  float mx, my, a01, inv_l00, l11, L, dyl, ext;
};
static ReachRec reach_rec(float mx, float my, float l00, float l01, float l11, float rho2, int box_tiles) {
  ReachRec t{};
  t.whole = box_tiles <= 2;
  if (t.whole) return t;
  volatile float L = std::fma(rho2, 1.02f, 1e-3f);
  volatile float sL = std::sqrt((float)L);
  volatile float inv_l00 = 1.f / l00;
  volatile float a01 = l01 * inv_l00;
  volatile float nn = std::fma(l11, l11, l01 * l01);
  volatile float nrm = std::sqrt((float)nn);
  volatile float num = sL * l01, den = l11 * nrm;
  t.mx = mx;
  t.my = my;
  t.a01 = a01;
  t.inv_l00 = inv_l00;
  t.l11 = l11;
  t.L = L;
  t.dyl = num / den;
  t.ext = sL / l11;
  return t;
}
static void reach_row(const ReachRec& t, int ty, int TW, int TH, int x0, int x1, int& tx_a, int& tx_b) {
  if (t.whole) {
    tx_a = x0;
    tx_b = x1;
    return;
  }
  const float eps = 0.01f;
  volatile float Y0 = (float)(ty * TH) + 0.5f;
  volatile float Y1 = Y0 + (float)(TH - 1);
  volatile float a = Y0 - t.my, b = Y1 - t.my;
  volatile float lo0 = a - eps, hi0 = b + eps;
  const float lo = std::fmax((float)lo0, -t.ext), hi = std::fmin((float)hi0, t.ext);
  tx_a = x0;
  tx_b = x0 - 1;
  if (!(lo <= hi)) return;
  const float d1 = std::fmin(std::fmax(t.dyl, lo), hi), d2 = std::fmin(std::fmax(-t.dyl, lo), hi);
  volatile float e1 = t.l11 * d1, e2 = t.l11 * d2;
  volatile float s1 = std::sqrt(std::fmax(std::fma(-(float)e1, (float)e1, t.L), 0.f));
  volatile float s2 = std::sqrt(std::fmax(std::fma(-(float)e2, (float)e2, t.L), 0.f));
  volatile float p1 = t.a01 * d1, p2 = t.a01 * d2;
  volatile float f1 = std::fma((float)s1, t.inv_l00, (float)p1), f2 = std::fma((float)s2, t.inv_l00, -(float)p2);
  volatile float xl0 = t.mx - f1, xh0 = t.mx + f2;
  volatile float xlo = xl0 - eps, xhi = xh0 + eps;
  const float inv_tw = 1.f / (float)TW;
  volatile float xa = xlo + 0.5f, xb = xhi - 0.5f;
  volatile float ga = std::fma((float)xa, inv_tw, -1.f), gb = xb * inv_tw;
  const float fa = std::ceil((float)ga), fb = std::floor((float)gb);
  tx_a = fa <= (float)x0 ? x0 : (fa > (float)x1 ? x1 + 1 : (int)fa);
  tx_b = fb >= (float)x1 ? x1 : (fb < (float)x0 ? x0 - 1 : (int)fb);
}

// Duplication + stable sort of binary32 footprints (the integer part of the
// pipeline).  foot [R][4] = mx my ex ey (float), dkey [R] = depth bits or
// 0xFFFFFFFF when invisible.  Without ellipses (chol == NULL) every tile of
// the support box gets a key; with chol [R][3] = l00 l01 l11 and rho2 [R]
// (binary32, mx my from foot) only the tiles reach_row gives.  Keys are tile
// ids (ty*tiles_x + tx), values record ids, ordered by (tile, dkey, id).
// ranges [2*tiles] = start/end per tile.  Returns K, or -1 when K exceeds cap.
long long lso_dupsort_f32(long long R, const float* foot, const uint32_t* dkey, const float* chol,
                          const float* rho2, int W, int H, int TW, int TH, long long cap, uint32_t* keys,
                          uint32_t* vals, int32_t* ranges) {
  int tx_n = (W + TW - 1) / TW, ty_n = (H + TH - 1) / TH;
  std::vector<std::pair<uint64_t, uint32_t>> kv;  // (tile << 32 | dkey, id), emitted in id order
  for (long long r = 0; r < R; ++r) {
    if (dkey[r] == 0xFFFFFFFFu) continue;
    Rect rc = rect_f32(foot[4 * r], foot[4 * r + 1], foot[4 * r + 2], foot[4 * r + 3], W, H);
    if (rc.empty) continue;
    const int x0 = rc.x0 / TW, x1 = rc.x1 / TW, y0 = rc.y0 / TH, y1 = rc.y1 / TH;
    ReachRec t{};
    t.whole = true;
    if (chol)
      t = reach_rec(foot[4 * r], foot[4 * r + 1], chol[3 * r], chol[3 * r + 1], chol[3 * r + 2], rho2[r],
                    (x1 - x0 + 1) * (y1 - y0 + 1));
    for (int ty = y0; ty <= y1; ++ty) {
      int a, b;
      reach_row(t, ty, TW, TH, x0, x1, a, b);
      for (int tx = a; tx <= b; ++tx) kv.push_back({((uint64_t)(ty * tx_n + tx) << 32) | dkey[r], (uint32_t)r});
    }
  }
  std::stable_sort(kv.begin(), kv.end(), [](const std::pair<uint64_t, uint32_t>& a,
                                            const std::pair<uint64_t, uint32_t>& b) { return a.first < b.first; });
  long long K = (long long)kv.size();
  for (int t = 0; t < 2 * tx_n * ty_n; ++t) ranges[t] = 0;
  if (K > cap) return -1;
  for (long long k = 0; k < K; ++k) {
    keys[k] = (uint32_t)(kv[k].first >> 32);
    vals[k] = kv[k].second;
  }
  for (long long k = 0; k < K; ++k) {
    uint32_t t = keys[k];
    if (k == 0 || keys[k - 1] != t) ranges[2 * t] = (int32_t)k;
    if (k == K - 1 || keys[k + 1] != t) ranges[2 * t + 1] = (int32_t)(k + 1);
  }
  return K;
}

// (tile, record) pairs that every tile list must hold: tiles of a record's
// binary32 support box (the rule above) with at least one pixel centre
// (px + 1/2, py + 1/2) inside the shrunken support ellipse
// q = a dx^2 + 2 b dx dy + c dy^2 <= shrink * rho^2 (FP64, brute force over
// the tile's pixels).  conic [R][3] = a b c, rho2 [R].  A tile list that
// holds these pairs lets the blend composite every pair whose alpha reaches
// alpha_min (compact support of the kernel, Sec. 3.2 Eq. 11-12); pairs on
// the boundary (shrink < 1) are left to binary32 rounding.  Returns the count
// (pairs written while it is below cap).
long long lso_touch_pairs(long long R, const float* foot, const uint32_t* dkey, const double* conic,
                          const double* rho2, int W, int H, int TW, int TH, double shrink, long long cap,
                          uint32_t* tile_out, uint32_t* rec_out) {
  int tx_n = (W + TW - 1) / TW;
  long long n = 0;
  for (long long r = 0; r < R; ++r) {
    if (dkey[r] == 0xFFFFFFFFu) continue;
    Rect rc = rect_f32(foot[4 * r], foot[4 * r + 1], foot[4 * r + 2], foot[4 * r + 3], W, H);
    if (rc.empty) continue;
    const double a = conic[3 * r], b = conic[3 * r + 1], c = conic[3 * r + 2], lim = shrink * rho2[r];
    for (int ty = rc.y0 / TH; ty <= rc.y1 / TH; ++ty)
      for (int tx = rc.x0 / TW; tx <= rc.x1 / TW; ++tx) {
        bool hit = false;
        for (int py = std::max(ty * TH, rc.y0); py <= std::min(ty * TH + TH - 1, rc.y1) && !hit; ++py)
          for (int px = std::max(tx * TW, rc.x0); px <= std::min(tx * TW + TW - 1, rc.x1) && !hit; ++px) {
            const double dx = px + 0.5 - foot[4 * r], dy = py + 0.5 - foot[4 * r + 1];
            hit = a * dx * dx + 2.0 * b * dx * dy + c * dy * dy <= lim;
          }
        if (!hit) continue;
        if (n < cap) {
          tile_out[n] = (uint32_t)(ty * tx_n + tx);
          rec_out[n] = (uint32_t)r;
        }
        ++n;
      }
  }
  return n;
}

// Per-tile inputs of the termination network from binary32 footprints foot
// [R][4] and depth bits dkey, with each record's opacity, squared support
// radius and conic taken from proj [R][NP]: counts [tiles] = records whose
// support box covers the tile; coverage [tiles][32] = for bin b, the summed
// expected coverage o/3 * min(1, support-ellipse area / box area) of those
// records in bins 0..b.  Bin i holds depths in [e_i, e_{i+1}), e_i =
// binary32(0.5 * 64^(i/32)), i = 1..31 (bin 0 below e_1, bin 31 from e_31).
void lso_tile_depth_hist(long long R, const float* foot, const uint32_t* dkey, const double* proj, int W, int H,
                         int TW, int TH, int32_t* counts, double* coverage) {
  int tx_n = (W + TW - 1) / TW, ty_n = (H + TH - 1) / TH;
  float edge[31];
  for (int i = 0; i < 31; ++i) edge[i] = (float)(0.5 * std::pow(64.0, (i + 1) / 32.0));
  for (int t = 0; t < tx_n * ty_n; ++t) {
    counts[t] = 0;
    for (int b = 0; b < 32; ++b) coverage[32 * t + b] = 0.0;
  }
  for (long long r = 0; r < R; ++r) {
    if (dkey[r] == 0xFFFFFFFFu) continue;
    Rect rc = rect_f32(foot[4 * r], foot[4 * r + 1], foot[4 * r + 2], foot[4 * r + 3], W, H);
    if (rc.empty) continue;
    float d;
    std::memcpy(&d, &dkey[r], 4);
    int b = 0;
    while (b < 31 && d >= edge[b]) ++b;
    const double* p = proj + (size_t)r * NP;
    const double detA = p[P_A] * p[P_C] - p[P_B] * p[P_B];
    const double ellipse = PI * p[P_RHO2] / std::sqrt(detA);
    const int tx0 = rc.x0 / TW, tx1 = rc.x1 / TW, ty0 = rc.y0 / TH, ty1 = rc.y1 / TH;
    const double box = (double)(tx1 - tx0 + 1) * (ty1 - ty0 + 1) * TW * TH;
    const double w = p[P_O] / 3.0 * std::min(1.0, ellipse / box);
    for (int ty = ty0; ty <= ty1; ++ty)
      for (int tx = tx0; tx <= tx1; ++tx) {
        counts[ty * tx_n + tx]++;
        for (int bb = b; bb < 32; ++bb) coverage[(ty * tx_n + tx) * 32 + bb] += w;
      }
  }
}

// Forward render of projected records proj [n][NP] (Eq. 6).  brute = 1 skips
// the tiles: every pixel runs over all visible records in (depth, id) order.
// rule_f32 / dkey select the binary32 tile rule and sort bits (dkey may be
// NULL: binary32 rounding of the FP64 depth).  Outputs: image [H][W][3] (with
// background), T [H][W], n_last (tile-list count), last_id, flags, stats[0] =
// evaluated pairs, stats[1] = composited pairs.  window (NULL = whole image):
// {x0, x1, y0, y1}, only pixels in [x0, x1) x [y0, y1) are composited.
// tile_mask (NULL = every tile): only tiles with a non-zero entry are
// composited (a sample of the frame, for timing).
int lso_render(int n, const double* proj, const unsigned char* vis, int W, int H, const double* parv,
               int rule_f32, const uint32_t* dkey, int brute, double* image, double* T, int32_t* n_last,
               int32_t* last_id, unsigned char* flags, long long* stats, const int32_t* window, double* labels,
               const unsigned char* tile_mask) {
  Par P = unpack_par(parv);
  // pixel window [x0, x1) x [y0, y1); pixels outside it are left untouched
  int wx0 = window ? window[0] : 0, wx1 = window ? window[1] : W;
  int wy0 = window ? window[2] : 0, wy1 = window ? window[3] : H;
  long long n_eval = 0, n_contrib = 0;
  if (brute) {
    std::vector<int> all;
    for (int i = 0; i < n; ++i)
      if (vis[i]) all.push_back(i);
    auto key = [&](int i) -> uint32_t { return dkey ? dkey[i] : f32bits(proj[(size_t)i * NP + P_DEPTH]); };
    std::stable_sort(all.begin(), all.end(), [&](int a, int b) { return key(a) < key(b); });
#pragma omp parallel for num_threads(g_threads) schedule(dynamic, 4) reduction(+ : n_contrib)
    for (int py = wy0; py < wy1; ++py)
      for (int px = wx0; px < wx1; ++px) {
        PixOut o = blend_pixel(all, proj, px + 0.5, py + 0.5, P, nullptr);
        size_t pi = (size_t)py * W + px;
        for (int c = 0; c < 3; ++c) image[3 * pi + c] = o.C[c] + o.T * P.bg[c];
        T[pi] = o.T;
        n_last[pi] = o.n_last;
        last_id[pi] = o.last_id;
        flags[pi] = o.flag;
        n_contrib += o.n_contrib;
      }
    stats[0] = -1;
    stats[1] = n_contrib;
    return 0;
  }
  Lists Ls = build_lists(n, proj, vis, W, H, P, rule_f32, dkey);
  int ntiles = Ls.tiles_x * Ls.tiles_y;
#pragma omp parallel for num_threads(g_threads) schedule(dynamic, 1) reduction(+ : n_eval, n_contrib)
  for (int t = 0; t < ntiles; ++t) {
    if (tile_mask && !tile_mask[t]) continue;
    int tx = t % Ls.tiles_x, ty = t / Ls.tiles_x;
    int emax = 0, npix = 0, smax = -1;
    bool never = false;
    for (int py = std::max(ty * P.tile_h, wy0); py < std::min(std::min(H, (ty + 1) * P.tile_h), wy1); ++py)
      for (int px = std::max(tx * P.tile_w, wx0); px < std::min(std::min(W, (tx + 1) * P.tile_w), wx1); ++px) {
        PixOut o = blend_pixel(Ls.L[t], proj, px + 0.5, py + 0.5, P, nullptr);
        if (o.stop_index >= (int)Ls.L[t].size()) never = true;
        else smax = std::max(smax, o.stop_index);
        size_t pi = (size_t)py * W + px;
        for (int c = 0; c < 3; ++c) image[3 * pi + c] = o.C[c] + o.T * P.bg[c];
        T[pi] = o.T;
        n_last[pi] = o.n_last;
        last_id[pi] = o.last_id;
        flags[pi] = o.flag;
        n_contrib += o.n_contrib;
        int e = o.stop_index < (int)Ls.L[t].size() ? o.stop_index + 1 : (int)Ls.L[t].size();
        emax = std::max(emax, e);
        ++npix;
      }
    n_eval += (long long)emax * npix;
    // termination depth of the tile: depth of the entry at which its last
    // pixel stopped; +inf if a pixel never stops; 0 for an empty list
    if (labels) {
      if (Ls.L[t].empty() || npix == 0) labels[t] = 0.0;
      else if (never) labels[t] = INFINITY;
      else labels[t] = proj[(size_t)Ls.L[t][smax] * NP + P_DEPTH];
    }
  }
  stats[0] = n_eval;
  stats[1] = n_contrib;
  return 0;
}

// Adjoint of lso_render (tiled lists) with respect to the projected record:
// g2d [n][9] = d/d(mx, my, a, b, c, o_eff, r, g, b).  gC [H][W][3], gT [H][W].
// Forward transmittances are kept per pixel, not recomputed.  With ags != 0
// the kernel-derivative path is scaled by w(D) (Eq. 13-14), so the result is
// no longer an exact gradient.  window and tile_mask as for lso_render.
int lso_render_bwd(int n, const double* proj, const unsigned char* vis, int W, int H, const double* parv,
                   int rule_f32, const uint32_t* dkey, const double* gC, const double* gT, double* g2d,
                   const int32_t* window, const unsigned char* tile_mask) {
  Par P = unpack_par(parv);
  int wx0 = window ? window[0] : 0, wx1 = window ? window[1] : W;
  int wy0 = window ? window[2] : 0, wy1 = window ? window[3] : H;
  for (size_t i = 0; i < (size_t)n * 9; ++i) g2d[i] = 0.0;
  Lists Ls = build_lists(n, proj, vis, W, H, P, rule_f32, dkey);
  int ntiles = Ls.tiles_x * Ls.tiles_y;
#pragma omp parallel for num_threads(g_threads) schedule(dynamic, 1)
  for (int t = 0; t < ntiles; ++t) {
    if (tile_mask && !tile_mask[t]) continue;
    int tx = t % Ls.tiles_x, ty = t / Ls.tiles_x;
    std::vector<PairRec> rec;
    for (int py = std::max(ty * P.tile_h, wy0); py < std::min(std::min(H, (ty + 1) * P.tile_h), wy1); ++py)
      for (int px = std::max(tx * P.tile_w, wx0); px < std::min(std::min(W, (tx + 1) * P.tile_w), wx1); ++px) {
        rec.clear();
        PixOut o = blend_pixel(Ls.L[t], proj, px + 0.5, py + 0.5, P, &rec);
        size_t pi = (size_t)py * W + px;
        const double* g = gC + 3 * pi;
        double Tf = o.T;
        // S_k = sum_{l>k} c_l a_l T_l + bg T_final, built back to front.
        double S[3] = {P.bg[0] * Tf, P.bg[1] * Tf, P.bg[2] * Tf};
        for (int k = (int)rec.size() - 1; k >= 0; --k) {
          const PairRec& r = rec[k];
          const double* p = proj + (size_t)r.id * NP;
          double ga = 0.0;
          for (int c = 0; c < 3; ++c) ga += g[c] * (p[P_R + c] * r.T - S[c] / (1.0 - r.alpha));
          ga -= gT[pi] * Tf / (1.0 - r.alpha);
          double loc[9] = {0};
          for (int c = 0; c < 3; ++c) {
            loc[6 + c] = r.alpha * r.T * g[c];
            S[c] += p[P_R + c] * r.alpha * r.T;
          }
          if (!r.clamped) {
            double f = kern_f(P.kernel, r.fx);
            loc[5] = f * ga;
            double gD = p[P_O] * ga * kern_df(P.kernel, r.fx) / P.lambda;
            if (P.ags == 1) gD *= std::exp(-r.D * r.D);
            if (P.ags == 2) gD *= std::exp(-(r.D / P.lambda) * (r.D / P.lambda));
            double gq = r.D > 0 ? gD / (2.0 * r.D) : 0.0;
            loc[0] = -gq * 2.0 * (p[P_A] * r.dx + p[P_B] * r.dy);
            loc[1] = -gq * 2.0 * (p[P_B] * r.dx + p[P_C] * r.dy);
            loc[2] = gq * r.dx * r.dx;
            loc[3] = gq * 2.0 * r.dx * r.dy;
            loc[4] = gq * r.dy * r.dy;
          }
          double* dst = g2d + (size_t)r.id * 9;
          for (int j = 0; j < 9; ++j) {
#pragma omp atomic
            dst[j] += loc[j];
          }
        }
      }
  }
  return 0;
}

// Chain rule from g2d [n][9] to the 3D parameters, by forward-mode dual
// numbers through project_one (one pass per parameter).  Outputs are
// overwritten: g_means [n][3], g_scales [n][3], g_quats [n][4], g_opac [n],
// g_sh [n][K][3].
int lso_project_bwd(int n, const double* means, const double* scales, const double* quats, const double* opac,
                    const double* sh, const double* camv, const double* parv, const double* g2d,
                    double* g_means, double* g_scales, double* g_quats, double* g_opac, double* g_sh) {
  Cam cam = unpack_cam(camv);
  Par P = unpack_par(parv);
  int K = (P.sh_degree + 1) * (P.sh_degree + 1);
  int npar = 3 + 3 + 4 + 1 + 3 * K;
  const int outs[9] = {P_MX, P_MY, P_A, P_B, P_C, P_O, P_R, P_G, P_BL};
#pragma omp parallel for num_threads(g_threads) schedule(static)
  for (int i = 0; i < n; ++i) {
    std::vector<double> gp(npar, 0.0);
    const double* gi = g2d + (size_t)i * 9;
    bool any = false;
    for (int j = 0; j < 9; ++j) any = any || gi[j] != 0.0;
    if (any) {
      std::vector<Dual> x(npar);
      for (int j = 0; j < 3; ++j) x[j] = Dual(means[3 * (size_t)i + j]);
      for (int j = 0; j < 3; ++j) x[3 + j] = Dual(scales[3 * (size_t)i + j]);
      for (int j = 0; j < 4; ++j) x[6 + j] = Dual(quats[4 * (size_t)i + j]);
      x[10] = Dual(opac[i]);
      for (int j = 0; j < 3 * K; ++j) x[11 + j] = Dual(sh[(size_t)i * 3 * K + j]);
      Dual out[NP];
      for (int d = 0; d < npar; ++d) {
        x[d].d = 1.0;
        bool v = project_one<Dual>(&x[0], &x[3], &x[6], x[10], &x[11], P.sh_degree, cam, P, out);
        x[d].d = 0.0;
        if (!v) break;
        double s = 0.0;
        for (int j = 0; j < 9; ++j) s += gi[j] * out[outs[j]].d;
        gp[d] = s;
      }
    }
    for (int j = 0; j < 3; ++j) g_means[3 * (size_t)i + j] = gp[j];
    for (int j = 0; j < 3; ++j) g_scales[3 * (size_t)i + j] = gp[3 + j];
    for (int j = 0; j < 4; ++j) g_quats[4 * (size_t)i + j] = gp[6 + j];
    g_opac[i] = gp[10];
    for (int j = 0; j < 3 * K; ++j) g_sh[(size_t)i * 3 * K + j] = gp[11 + j];
  }
  return 0;
}

}  // extern "C"
