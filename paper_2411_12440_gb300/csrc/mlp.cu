// a8: the per-tile termination-depth MLP, 48 (35 used) -> 64 -> 64 -> 1 with
// ReLU, FP16 inputs/weights and FP32 accumulation on the tensor cores
// (mma.sync.m16n8k16 f16 x f16 -> f32; the layers are 16-row x 64 GEMMs, far
// too small for tcgen05's 128-row tiles to pay off).
//
// Forward: one warp per 16 rows.  Layer-1 and layer-2 accumulators are laid
// out exactly like the next layer's A fragments, so after bias + ReLU they
// are converted to f16x2 in registers without touching shared memory.  The
// 64 -> 1 output layer is an FP32 dot product reduced over the four lanes of
// a row group.
//
// Backward (training): 128 rows per CTA (8 warps).  Each warp recomputes its
// rows' forward, forms dy from an asymmetric squared loss, dh2 = dy w3 * relu',
// and dh1 = (dh2 W2^T) * relu' on the tensor cores, and stores x, h1, dh1, dh2
// (f16) for its rows in shared memory.  The CTA then forms the weight
// gradients dW2 = h1^T dh2 and dW1 = x^T dh1 (K = 128 rows) on the tensor
// cores from transposed ldmatrix loads, accumulates them in registers over
// its chunks, and adds them to global memory once at the end.
#include <cuda_fp16.h>

#include "kernels.h"

namespace ls {

namespace {

constexpr int IN = LS_MLP_IN;     // 48
constexpr int HID = LS_MLP_HID;   // 64
constexpr int LDX = IN + 8;       // padded shared-memory row strides (halves)
constexpr int LDH = HID + 8;
constexpr int OFF_W1 = 0;
constexpr int OFF_B1 = OFF_W1 + HID * IN;
constexpr int OFF_W2 = OFF_B1 + HID;
constexpr int OFF_B2 = OFF_W2 + HID * HID;
constexpr int OFF_W3 = OFF_B2 + HID;
constexpr int OFF_B3 = OFF_W3 + HID;
static_assert(OFF_B3 + 1 == LS_MLP_NPARAM, "packed parameter layout");

__device__ __forceinline__ void mma16816(float* d, const uint32_t* a, const uint32_t* b) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void ldsm_x4_trans(uint32_t* r, const void* row) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(smem_u32(row)));
}

__device__ __forceinline__ uint32_t pack_h2(float lo, float hi) {
  __half2 h = __floats2half2_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&h);
}

// B fragment (16 x 8, k x n) of a matrix stored [n][k] (k contiguous).
__device__ __forceinline__ void load_b_nk(uint32_t* b, const __half* S, int ld, int n0, int k0, int g, int t) {
  b[0] = *reinterpret_cast<const uint32_t*>(S + (n0 + g) * ld + k0 + 2 * t);
  b[1] = *reinterpret_cast<const uint32_t*>(S + (n0 + g) * ld + k0 + 8 + 2 * t);
}

// A fragment (16 x 16) of a row-major matrix in shared memory.
__device__ __forceinline__ void load_a_rm(uint32_t* a, const __half* S, int ld, int r0, int c0, int g, int t) {
  a[0] = *reinterpret_cast<const uint32_t*>(S + (r0 + g) * ld + c0 + 2 * t);
  a[1] = *reinterpret_cast<const uint32_t*>(S + (r0 + g + 8) * ld + c0 + 2 * t);
  a[2] = *reinterpret_cast<const uint32_t*>(S + (r0 + g) * ld + c0 + 8 + 2 * t);
  a[3] = *reinterpret_cast<const uint32_t*>(S + (r0 + g + 8) * ld + c0 + 8 + 2 * t);
}

struct MlpSmem {
  __align__(16) __half w1t[HID * LDX];  // [out][in]
  __align__(16) __half w2t[HID * LDH];  // [out][in]
  __align__(16) __half w2[HID * LDH];   // [in][out] (backward)
  float b1[HID], b2[HID], w3[HID], b3;
};

__device__ __forceinline__ void load_weights(MlpSmem& S, const __half* w1t, const float* b1, const __half* w2t,
                                             const float* b2, const __half* w3, const float* b3, bool with_w2) {
  for (int i = threadIdx.x; i < HID * IN; i += blockDim.x) S.w1t[(i / IN) * LDX + i % IN] = w1t[i];
  for (int i = threadIdx.x; i < HID * HID; i += blockDim.x) {
    const __half v = w2t[i];
    S.w2t[(i / HID) * LDH + i % HID] = v;
    if (with_w2) S.w2[(i % HID) * LDH + i / HID] = v;
  }
  for (int i = threadIdx.x; i < HID; i += blockDim.x) {
    S.b1[i] = b1[i];
    S.b2[i] = b2[i];
    S.w3[i] = __half2float(w3[i]);
  }
  if (threadIdx.x == 0) S.b3 = b3[0];
  __syncthreads();
}

// Forward of one warp's 16 rows from A fragments of x (3 k-chunks).  Leaves
// the pre-activations z1, z2 (FP32, accumulator layout) and returns y for
// rows g and g + 8 (valid in every lane).
__device__ __forceinline__ void warp_forward(const MlpSmem& S, const uint32_t (&ax)[3][4], float (&z1)[8][4],
                                             float (&z2)[8][4], float& y0, float& y1, int g, int t) {
#pragma unroll
  for (int nt = 0; nt < 8; ++nt)
#pragma unroll
    for (int q = 0; q < 4; ++q) z1[nt][q] = 0.f;
#pragma unroll
  for (int kc = 0; kc < 3; ++kc)
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
      uint32_t b[2];
      load_b_nk(b, S.w1t, LDX, nt * 8, kc * 16, g, t);
      mma16816(z1[nt], ax[kc], b);
    }
  uint32_t ah[4][4];  // relu(z1 + b1) as f16 A fragments of layer 2
#pragma unroll
  for (int nt = 0; nt < 8; ++nt) {
    const int c = nt * 8 + 2 * t;
    z1[nt][0] += S.b1[c];
    z1[nt][1] += S.b1[c + 1];
    z1[nt][2] += S.b1[c];
    z1[nt][3] += S.b1[c + 1];
    const uint32_t lo = pack_h2(fmaxf(z1[nt][0], 0.f), fmaxf(z1[nt][1], 0.f));
    const uint32_t hi = pack_h2(fmaxf(z1[nt][2], 0.f), fmaxf(z1[nt][3], 0.f));
    ah[nt >> 1][(nt & 1) * 2] = lo;
    ah[nt >> 1][(nt & 1) * 2 + 1] = hi;
  }
#pragma unroll
  for (int nt = 0; nt < 8; ++nt)
#pragma unroll
    for (int q = 0; q < 4; ++q) z2[nt][q] = 0.f;
#pragma unroll
  for (int kc = 0; kc < 4; ++kc)
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
      uint32_t b[2];
      load_b_nk(b, S.w2t, LDH, nt * 8, kc * 16, g, t);
      mma16816(z2[nt], ah[kc], b);
    }
  float s0 = 0.f, s1 = 0.f;
#pragma unroll
  for (int nt = 0; nt < 8; ++nt) {
    const int c = nt * 8 + 2 * t;
    z2[nt][0] += S.b2[c];
    z2[nt][1] += S.b2[c + 1];
    z2[nt][2] += S.b2[c];
    z2[nt][3] += S.b2[c + 1];
    // layer 3 reads h2 rounded to f16, like every other layer input
    s0 += __half2float(__float2half_rn(fmaxf(z2[nt][0], 0.f))) * S.w3[c] +
          __half2float(__float2half_rn(fmaxf(z2[nt][1], 0.f))) * S.w3[c + 1];
    s1 += __half2float(__float2half_rn(fmaxf(z2[nt][2], 0.f))) * S.w3[c] +
          __half2float(__float2half_rn(fmaxf(z2[nt][3], 0.f))) * S.w3[c + 1];
  }
  s0 += __shfl_xor_sync(0xffffffffu, s0, 1);
  s0 += __shfl_xor_sync(0xffffffffu, s0, 2);
  s1 += __shfl_xor_sync(0xffffffffu, s1, 1);
  s1 += __shfl_xor_sync(0xffffffffu, s1, 2);
  y0 = s0 + S.b3;
  y1 = s1 + S.b3;
}

// A fragments of x rows r0..r0+15 straight from global memory (zero past m).
__device__ __forceinline__ void load_x_frags(uint32_t (&ax)[3][4], const __half* x, int64_t m, int64_t r0, int g,
                                             int t) {
  const int64_t ra = r0 + g, rb = r0 + g + 8;
#pragma unroll
  for (int kc = 0; kc < 3; ++kc) {
    const int c = kc * 16 + 2 * t;
    ax[kc][0] = ra < m ? *reinterpret_cast<const uint32_t*>(x + ra * IN + c) : 0u;
    ax[kc][1] = rb < m ? *reinterpret_cast<const uint32_t*>(x + rb * IN + c) : 0u;
    ax[kc][2] = ra < m ? *reinterpret_cast<const uint32_t*>(x + ra * IN + c + 8) : 0u;
    ax[kc][3] = rb < m ? *reinterpret_cast<const uint32_t*>(x + rb * IN + c + 8) : 0u;
  }
}

__global__ void __launch_bounds__(128) mlp_forward_kernel(int64_t m, const __half* __restrict__ x,
                                                          const __half* w1t, const float* b1, const __half* w2t,
                                                          const float* b2, const __half* w3, const float* b3,
                                                          float* __restrict__ y) {
  __shared__ MlpSmem S;
  load_weights(S, w1t, b1, w2t, b2, w3, b3, false);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, g = lane >> 2, t = lane & 3;
  const int64_t tiles = (m + 15) / 16;
  for (int64_t tile = (int64_t)blockIdx.x * 4 + warp; tile < tiles; tile += (int64_t)gridDim.x * 4) {
    const int64_t r0 = tile * 16;
    uint32_t ax[3][4];
    load_x_frags(ax, x, m, r0, g, t);
    float z1[8][4], z2[8][4], y0, y1;
    warp_forward(S, ax, z1, z2, y0, y1, g, t);
    if (t == 0) {
      if (r0 + g < m) y[r0 + g] = y0;
      if (r0 + g + 8 < m) y[r0 + g + 8] = y1;
    }
  }
}

struct MlpBwdSmem {
  MlpSmem W;
  __align__(16) __half xs[128 * LDX];
  __align__(16) __half h1[128 * LDH];
  __align__(16) __half dh1[128 * LDH];
  __align__(16) __half dh2[128 * LDH];
};

__global__ void __launch_bounds__(256) mlp_backward_kernel(int64_t m, const __half* __restrict__ x,
                                                           const __half* w1t, const float* b1, const __half* w2t,
                                                           const float* b2, const __half* w3, const float* b3,
                                                           const float* __restrict__ target, float under_weight,
                                                           float inv_m, float* __restrict__ grad, float* loss) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  MlpBwdSmem& S = *reinterpret_cast<MlpBwdSmem*>(smem_raw);
  load_weights(S.W, w1t, b1, w2t, b2, w3, b3, true);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, g = lane >> 2, t = lane & 3;
  // register accumulators of this warp's share of the weight gradients
  float dw2[4][4], dw1[3][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int q = 0; q < 4; ++q) dw2[i][q] = 0.f;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int q = 0; q < 4; ++q) dw1[i][q] = 0.f;
  float db1[8][2], db2[8][2], dw3[8][2], db3 = 0.f, lsum = 0.f;
#pragma unroll
  for (int nt = 0; nt < 8; ++nt) db1[nt][0] = db1[nt][1] = db2[nt][0] = db2[nt][1] = dw3[nt][0] = dw3[nt][1] = 0.f;

  const int64_t chunks = (m + 127) / 128;
  for (int64_t ch = blockIdx.x; ch < chunks; ch += gridDim.x) {
    const int64_t rbase = ch * 128;
    // stage x rows of the chunk (zero past m)
    for (int i = threadIdx.x; i < 128 * (IN / 8); i += blockDim.x) {
      const int r = i / (IN / 8), c8 = (i % (IN / 8)) * 8;
      uint4 v = make_uint4(0u, 0u, 0u, 0u);
      if (rbase + r < m) v = *reinterpret_cast<const uint4*>(x + (rbase + r) * IN + c8);
      *reinterpret_cast<uint4*>(S.xs + r * LDX + c8) = v;
    }
    __syncthreads();
    const int lr0 = warp * 16;
    const int64_t r0 = rbase + lr0;
    uint32_t ax[3][4];
#pragma unroll
    for (int kc = 0; kc < 3; ++kc) load_a_rm(ax[kc], S.xs, LDX, lr0, kc * 16, g, t);
    float z1[8][4], z2[8][4], y0, y1;
    warp_forward(S.W, ax, z1, z2, y0, y1, g, t);
    // asymmetric squared loss on the predicted log-depth
    float d0 = 0.f, d1 = 0.f;
    if (r0 + g < m) {
      const float e = y0 - target[r0 + g];
      const float w = e < 0.f ? under_weight : 1.f;
      d0 = 2.f * w * e * inv_m;
      if (t == 0) lsum += w * e * e * inv_m;
    }
    if (r0 + g + 8 < m) {
      const float e = y1 - target[r0 + g + 8];
      const float w = e < 0.f ? under_weight : 1.f;
      d1 = 2.f * w * e * inv_m;
      if (t == 0) lsum += w * e * e * inv_m;
    }
    if (t == 0) db3 += d0 + d1;
    // dh2 = dy w3 relu'(z2); dw3 += h2 dy; h1 and dh2 to shared memory
    uint32_t adh2[4][4];
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
      const int c = nt * 8 + 2 * t;
      const float h20 = __half2float(__float2half_rn(fmaxf(z2[nt][0], 0.f)));
      const float h21 = __half2float(__float2half_rn(fmaxf(z2[nt][1], 0.f)));
      const float h22 = __half2float(__float2half_rn(fmaxf(z2[nt][2], 0.f)));
      const float h23 = __half2float(__float2half_rn(fmaxf(z2[nt][3], 0.f)));
      dw3[nt][0] += h20 * d0 + h22 * d1;
      dw3[nt][1] += h21 * d0 + h23 * d1;
      const float e0 = z2[nt][0] > 0.f ? d0 * S.W.w3[c] : 0.f;
      const float e1 = z2[nt][1] > 0.f ? d0 * S.W.w3[c + 1] : 0.f;
      const float e2 = z2[nt][2] > 0.f ? d1 * S.W.w3[c] : 0.f;
      const float e3 = z2[nt][3] > 0.f ? d1 * S.W.w3[c + 1] : 0.f;
      db2[nt][0] += e0 + e2;
      db2[nt][1] += e1 + e3;
      const uint32_t lo = pack_h2(e0, e1), hi = pack_h2(e2, e3);
      adh2[nt >> 1][(nt & 1) * 2] = lo;
      adh2[nt >> 1][(nt & 1) * 2 + 1] = hi;
      *reinterpret_cast<uint32_t*>(S.dh2 + (lr0 + g) * LDH + c) = lo;
      *reinterpret_cast<uint32_t*>(S.dh2 + (lr0 + g + 8) * LDH + c) = hi;
      *reinterpret_cast<uint32_t*>(S.h1 + (lr0 + g) * LDH + c) =
          pack_h2(fmaxf(z1[nt][0], 0.f), fmaxf(z1[nt][1], 0.f));
      *reinterpret_cast<uint32_t*>(S.h1 + (lr0 + g + 8) * LDH + c) =
          pack_h2(fmaxf(z1[nt][2], 0.f), fmaxf(z1[nt][3], 0.f));
    }
    // dh1 = (dh2 W2^T) relu'(z1): B[k = out][n = in] = W2[in][out]
    float a1[8][4];
#pragma unroll
    for (int nt = 0; nt < 8; ++nt)
#pragma unroll
      for (int q = 0; q < 4; ++q) a1[nt][q] = 0.f;
#pragma unroll
    for (int kc = 0; kc < 4; ++kc)
#pragma unroll
      for (int nt = 0; nt < 8; ++nt) {
        uint32_t b[2];
        load_b_nk(b, S.W.w2, LDH, nt * 8, kc * 16, g, t);
        mma16816(a1[nt], adh2[kc], b);
      }
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
      const int c = nt * 8 + 2 * t;
      const float e0 = z1[nt][0] > 0.f ? a1[nt][0] : 0.f;
      const float e1 = z1[nt][1] > 0.f ? a1[nt][1] : 0.f;
      const float e2 = z1[nt][2] > 0.f ? a1[nt][2] : 0.f;
      const float e3 = z1[nt][3] > 0.f ? a1[nt][3] : 0.f;
      db1[nt][0] += e0 + e2;
      db1[nt][1] += e1 + e3;
      *reinterpret_cast<uint32_t*>(S.dh1 + (lr0 + g) * LDH + c) = pack_h2(e0, e1);
      *reinterpret_cast<uint32_t*>(S.dh1 + (lr0 + g + 8) * LDH + c) = pack_h2(e2, e3);
    }
    __syncthreads();
    // weight gradients over the chunk's 128 rows (K), transposed loads:
    // dW2[in i][out j] = sum_r h1[r][i] dh2[r][j]; warp: i-tile (warp >> 1),
    // j-tiles (warp & 1) * 4 .. +4
    {
      const int mt = warp >> 1, nb = (warp & 1) * 4;
      const int q = lane >> 3, rr = lane & 7;
#pragma unroll
      for (int ks = 0; ks < 8; ++ks) {
        uint32_t a[4];
        ldsm_x4_trans(a, S.h1 + (ks * 16 + (q >> 1) * 8 + rr) * LDH + mt * 16 + (q & 1) * 8);
#pragma unroll
        for (int np = 0; np < 2; ++np) {
          uint32_t bb[4];  // two n-tiles: (b0, b1) of nb + 2np and nb + 2np + 1
          ldsm_x4_trans(bb, S.dh2 + (ks * 16 + (q & 1) * 8 + rr) * LDH + (nb + 2 * np + (q >> 1)) * 8);
          mma16816(dw2[2 * np], a, bb);
          mma16816(dw2[2 * np + 1], a, bb + 2);
        }
      }
      // dW1[in k][out i] = sum_r x[r][k] dh1[r][i]; warp: (m, n) tiles 3w..3w+2
#pragma unroll
      for (int s = 0; s < 3; ++s) {
        const int idx = warp * 3 + s, m1 = idx >> 3, n1 = idx & 7;
#pragma unroll
        for (int ks = 0; ks < 8; ++ks) {
          uint32_t a[4], bb[4];
          ldsm_x4_trans(a, S.xs + (ks * 16 + (q >> 1) * 8 + rr) * LDX + m1 * 16 + (q & 1) * 8);
          ldsm_x4_trans(bb, S.dh1 + (ks * 16 + (q & 1) * 8 + rr) * LDH + n1 * 8);
          mma16816(dw1[s], a, bb);
        }
      }
    }
    __syncthreads();
  }
  // ---- commit: weight gradients in the packed [out][in] layout
  {
    const int mt = warp >> 1, nb = (warp & 1) * 4;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int i0 = mt * 16 + g, o0 = (nb + j) * 8 + 2 * t;  // in index, out index
      atomicAdd(&grad[OFF_W2 + o0 * HID + i0], dw2[j][0]);
      atomicAdd(&grad[OFF_W2 + (o0 + 1) * HID + i0], dw2[j][1]);
      atomicAdd(&grad[OFF_W2 + o0 * HID + i0 + 8], dw2[j][2]);
      atomicAdd(&grad[OFF_W2 + (o0 + 1) * HID + i0 + 8], dw2[j][3]);
    }
#pragma unroll
    for (int s = 0; s < 3; ++s) {
      const int idx = warp * 3 + s, m1 = idx >> 3, n1 = idx & 7;
      const int k0 = m1 * 16 + g, o0 = n1 * 8 + 2 * t;
      atomicAdd(&grad[OFF_W1 + o0 * IN + k0], dw1[s][0]);
      atomicAdd(&grad[OFF_W1 + (o0 + 1) * IN + k0], dw1[s][1]);
      atomicAdd(&grad[OFF_W1 + o0 * IN + k0 + 8], dw1[s][2]);
      atomicAdd(&grad[OFF_W1 + (o0 + 1) * IN + k0 + 8], dw1[s][3]);
    }
  }
  // biases and w3: reduce over the 8 row groups (lanes with equal t)
#pragma unroll
  for (int nt = 0; nt < 8; ++nt)
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      float v1 = db1[nt][e], v2 = db2[nt][e], v3 = dw3[nt][e];
#pragma unroll
      for (int o = 4; o < 32; o <<= 1) {
        v1 += __shfl_xor_sync(0xffffffffu, v1, o);
        v2 += __shfl_xor_sync(0xffffffffu, v2, o);
        v3 += __shfl_xor_sync(0xffffffffu, v3, o);
      }
      if (g == 0) {
        const int c = nt * 8 + 2 * t + e;
        atomicAdd(&grad[OFF_B1 + c], v1);
        atomicAdd(&grad[OFF_B2 + c], v2);
        atomicAdd(&grad[OFF_W3 + c], v3);
      }
    }
#pragma unroll
  for (int o = 4; o < 32; o <<= 1) {
    db3 += __shfl_xor_sync(0xffffffffu, db3, o);
    lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
  }
  if (lane == 0) {
    atomicAdd(&grad[OFF_B3], db3);
    if (loss) atomicAdd(loss, lsum);
  }
}

// Adam on the packed FP32 master parameters, then refresh the FP16 weights
// and FP32 biases the forward reads.
__global__ void __launch_bounds__(256) mlp_adam_kernel(int step, float lr, float beta1, float beta2, float eps,
                                                       float* __restrict__ master, const float* __restrict__ grad,
                                                       float* __restrict__ m1, float* __restrict__ m2,
                                                       __half* w1t, float* b1, __half* w2t, float* b2, __half* w3,
                                                       float* b3) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= LS_MLP_NPARAM) return;
  const float gi = grad[i];
  const float a = beta1 * m1[i] + (1.f - beta1) * gi;
  const float b = beta2 * m2[i] + (1.f - beta2) * gi * gi;
  m1[i] = a;
  m2[i] = b;
  const float c1 = 1.f - powf(beta1, (float)step), c2 = 1.f - powf(beta2, (float)step);
  const float p = master[i] - lr * (a / c1) / (sqrtf(b / c2) + eps);
  master[i] = p;
  if (i < OFF_B1) w1t[i - OFF_W1] = __float2half_rn(p);
  else if (i < OFF_W2) b1[i - OFF_B1] = p;
  else if (i < OFF_B2) w2t[i - OFF_W2] = __float2half_rn(p);
  else if (i < OFF_W3) b2[i - OFF_B2] = p;
  else if (i < OFF_B3) w3[i - OFF_W3] = __float2half_rn(p);
  else b3[0] = p;
}

}  // namespace

cudaError_t launch_mlp_forward(int64_t m, const void* x, const MlpDev& net, float* y, cudaStream_t st) {
  if (m <= 0) return cudaSuccess;
  const int64_t tiles = (m + 15) / 16;
  int sms = 0;
  cudaError_t e = current_sm_count(&sms);
  if (e != cudaSuccess) return e;
  int grid = (int)((tiles + 3) / 4);
  if (grid > sms * 8) grid = sms * 8;
  mlp_forward_kernel<<<grid, 128, 0, st>>>(m, static_cast<const __half*>(x), static_cast<const __half*>(net.w1t),
                                           net.b1, static_cast<const __half*>(net.w2t), net.b2,
                                           static_cast<const __half*>(net.w3), net.b3, y);
  return cudaGetLastError();
}

cudaError_t launch_mlp_backward(int64_t m, const void* x, const MlpDev& net, const float* target, float under_weight,
                                float* grad, float* loss, cudaStream_t st) {
  if (m <= 0) return cudaSuccess;
  static bool attr_set[64] = {false};
  const size_t sm = sizeof(MlpBwdSmem);
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64 || !attr_set[dev]) {
    e = cudaFuncSetAttribute(mlp_backward_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev < 64) attr_set[dev] = true;
  }
  const int64_t chunks = (m + 127) / 128;
  int sms = 0;
  e = current_sm_count(&sms);
  if (e != cudaSuccess) return e;
  int grid = (int)(chunks < 2 * sms ? chunks : 2 * sms);
  mlp_backward_kernel<<<grid, 256, sm, st>>>(m, static_cast<const __half*>(x), static_cast<const __half*>(net.w1t),
                                            net.b1, static_cast<const __half*>(net.w2t), net.b2,
                                            static_cast<const __half*>(net.w3), net.b3, target, under_weight,
                                            1.f / (float)m, grad, loss);
  return cudaGetLastError();
}

cudaError_t launch_mlp_adam(int step, float lr, float beta1, float beta2, float eps, float* master, const float* grad,
                            float* m1, float* m2, const MlpMut& net, cudaStream_t st) {
  mlp_adam_kernel<<<ceil_div(LS_MLP_NPARAM, 256), 256, 0, st>>>(
      step, lr, beta1, beta2, eps, master, grad, m1, m2, static_cast<__half*>(net.w1t), net.b1,
      static_cast<__half*>(net.w2t), net.b2, static_cast<__half*>(net.w3), net.b3);
  return cudaGetLastError();
}

}  // namespace ls
