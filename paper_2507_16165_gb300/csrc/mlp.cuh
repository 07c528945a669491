// Small MLP of the surrogate: inputs (b/M, r_obs/M, plane angle) -> three
// hidden layers of 64 with SiLU -> (deflection, u b at the first two disk
// nodes) on the tensor cores (mma.sync m16n8k16) with FP32 accumulation.
// Training runs in BF16 (weights; inputs and activations as BF16 high + low
// pairs); inference holds the trained BF16 weights exactly in FP16, with
// inputs and activations as FP16 high + low pairs.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include <cmath>

namespace bhs {

constexpr int K0 = 16;    // input width: NFEAT features, zero padded to one k16 block
constexpr int NFEAT = 12; // features derived from (b, r_obs, psi0)
constexpr int HID = 64;   // hidden width
constexpr int NO = 16;    // output width in storage (3 used, zero padded)
constexpr int NOUT = 3;

// FP32 parameter vector layout (row-major W[in][out]).
constexpr int OW1 = 0;
constexpr int OB1 = OW1 + K0 * HID;
constexpr int OW2 = OB1 + HID;
constexpr int OB2 = OW2 + HID * HID;
constexpr int OW3 = OB2 + HID;
constexpr int OB3 = OW3 + HID * HID;
constexpr int OW4 = OB3 + HID;
constexpr int OB4 = OW4 + HID * NO;
constexpr int NPARAM = OB4 + NO;

// Target normalisation (b, r in units of M):
//   y0 = (delta b / 4 - D_C) / D_S               delta = phi_inf - alpha
//   y1 = u(psi0) b,  y2 = u(psi0 + pi) b
// Features: see surrogate_features.
constexpr float LB_C = -1.155f, LB_S = 8.06f;
constexpr float R_C = 57.5f, R_S = 42.5f;
constexpr float P_C = 1.5707963f, P_S = 1.5707963f;
constexpr float D_C = 3.0f, D_S = 3.0f;

// Fragment-ordered FP16 weights for inference (the trained BF16 values, those
// of the hidden layers halved): for each layer, k16 block kb and n8 tile j,
// lane l holds uint2{b0, b1} of the mma B operand.
constexpr int FR1 = 0;                      // 1 x 8 x 32
constexpr int FR2 = FR1 + 1 * 8 * 32;       // 4 x 8 x 32
constexpr int FR3 = FR2 + 4 * 8 * 32;       // 4 x 8 x 32
constexpr int FR4 = FR3 + 4 * 8 * 32;       // 4 x 1 x 32
constexpr int NFRAG = FR4 + 4 * 1 * 32;
constexpr int NBIAS = 3 * HID + 8;          // b1 / 2, b2 / 2, b3 / 2, first 8 of b4

// The network's features: the three inputs (b/M, r_obs/M, psi0) and
// transforms of them that carry the known structure of the orbit --
// ln(b - 3 sqrt 3) for the logarithmic divergence at the photon sphere,
// b_c / b and M / r for the weak-field terms, sin and cos of the flat-space
// exit angle alpha, and sin / cos of psi0 and of (alpha - psi0), the phase
// of the straight line the orbit reduces to far from the hole.  Used
// identically by training (double) and inference (float).
template <typename T>
__host__ __device__ inline void surrogate_features(T b, T r, T psi, T* f) {
  using std::log;
  using std::sqrt;
  using std::sin;
  using std::cos;
  const T bc = T(5.19615242270663188);
  const T s = b * sqrt(T(1) - T(2) / r) / r;                 // sin alpha
  const T c = sqrt(T(1) - (s < T(1) ? s * s : T(1)));        // |cos alpha|
  const T cp = cos(psi), sp = sin(psi);
  f[0] = (log(b - bc) - T(LB_C)) / T(LB_S);
  f[1] = (r - T(R_C)) / T(R_S);
  f[2] = (psi - T(P_C)) / T(P_S);
  f[3] = bc / b;
  f[4] = s;
  f[5] = c;
  f[6] = cp;
  f[7] = sp;
  f[8] = s * cp + c * sp;     // sin(alpha - psi0) with alpha = pi - asin(s)
  f[9] = s * sp - c * cp;     // cos(alpha - psi0)
  f[10] = T(10) / r;
  f[11] = (bc / b) * (bc / b);
  for (int k = NFEAT; k < K0; ++k) f[k] = T(0);
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&v);
}

// D = A (16x16, row) * B (16x8, col) + C, BF16 inputs, FP32 accumulate.
__device__ __forceinline__ void mma_bf16(float* d, const uint32_t* a, uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
      "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// SiLU z sigma(z) with sigma(z) = (1 + tanh(z/2)) / 2, so that each
// activation takes one special-function instruction (the hardware tanh
// approximation, relative error about 2^-11) instead of an exponential and a
// reciprocal: the inference pass is bound by that unit.  Training and
// inference use the same formula; silu_grad is its derivative
// sigma (1 + z (1 - sigma)).
__device__ __forceinline__ float tanh_approx(float x) {
  float t;
  asm("tanh.approx.f32 %0, %1;" : "=f"(t) : "f"(x));
  return t;
}
__device__ __forceinline__ float silu(float z) {
  const float h = 0.5f * z;
  return fmaf(h, tanh_approx(h), h);
}
__device__ __forceinline__ float silu_grad(float z) {
  const float s = fmaf(0.5f, tanh_approx(0.5f * z), 0.5f);
  return s * (1.0f + z * (1.0f - s));
}

// Split of an FP32 pair into BF16 high and low parts (x = hi + lo to about
// 2^-17 relative): the activations enter the tensor cores as two BF16
// operands, so only the weights are BF16-limited.
__device__ __forceinline__ void split_pack(float x0, float x1, uint32_t* hi, uint32_t* lo) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(x0, x1);
  const float2 hf = __bfloat1622float2(h);
  const __nv_bfloat162 l = __floats2bfloat162_rn(x0 - hf.x, x1 - hf.y);
  *hi = *reinterpret_cast<const uint32_t*>(&h);
  *lo = *reinterpret_cast<const uint32_t*>(&l);
}

// ---------------------------------------------------------------------------
// Inference (the render's warp MLP).  The weights are the trained network's
// BF16 values, held exactly in FP16 fragments; those of the three hidden
// layers, and their biases, are halved (exact), so a hidden accumulator
// started at b/2 ends at h = z/2 and SiLU(z) = h + h tanh(h).  Inputs and
// activations enter as FP16 high + low pairs (x = hi + lo to about 2^-22
// relative), one mma per part; every layer needs both parts: with single
// FP16 activations in any one hidden layer the calibrated share of samples
// within 1e-3 rad fell from 80% to between 37% and 58%.
__device__ __forceinline__ void mma_f16(float* d, const uint32_t* a, uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 "
      "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// Split of an FP32 pair into FP16 high and low parts.
__device__ __forceinline__ void split_pack_h(float x0, float x1, uint32_t* hi, uint32_t* lo) {
  const __half2 h = __floats2half2_rn(x0, x1);
  const float2 hf = __half22float2(h);
  const __half2 l = __floats2half2_rn(x0 - hf.x, x1 - hf.y);
  *hi = *reinterpret_cast<const uint32_t*>(&h);
  *lo = *reinterpret_cast<const uint32_t*>(&l);
}

// One hidden layer for one m16 tile: split A fragments in (KB k16 blocks;
// hi and lo parts) -> SiLU -> split A fragments of the next layer.  The
// accumulator of n8 tiles 2kb and 2kb+1 is exactly the A operand of k16
// block kb of the next layer, so activations stay in registers.  bias: the
// halved biases.
template <int KB>
__device__ __forceinline__ void mlp_hidden(const uint2* frag, const float* bias, const uint32_t (*ahi)[4],
                                           const uint32_t (*alo)[4], uint32_t (*ohi)[4],
                                           uint32_t (*olo)[4], int lane) {
  const int t = lane & 3;
#pragma unroll
  for (int kbo = 0; kbo < 4; ++kbo) {
    float acc[2][4];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int j = 2 * kbo + h;
      const float b0 = bias[8 * j + 2 * t], b1 = bias[8 * j + 2 * t + 1];
      acc[h][0] = b0;
      acc[h][1] = b1;
      acc[h][2] = b0;
      acc[h][3] = b1;
#pragma unroll
      for (int kb = 0; kb < KB; ++kb) {
        const uint2 b = frag[(kb * 8 + j) * 32 + lane];
        mma_f16(acc[h], alo[kb], b.x, b.y);
        mma_f16(acc[h], ahi[kb], b.x, b.y);
      }
#pragma unroll
      for (int e = 0; e < 4; ++e) acc[h][e] = fmaf(acc[h][e], tanh_approx(acc[h][e]), acc[h][e]);
    }
    split_pack_h(acc[0][0], acc[0][1], &ohi[kbo][0], &olo[kbo][0]);
    split_pack_h(acc[0][2], acc[0][3], &ohi[kbo][1], &olo[kbo][1]);
    split_pack_h(acc[1][0], acc[1][1], &ohi[kbo][2], &olo[kbo][2]);
    split_pack_h(acc[1][2], acc[1][3], &ohi[kbo][3], &olo[kbo][3]);
  }
}

// The MLP for the 32 rays of a warp.  X: the warp's 32 x K0 feature rows
// (row l = ray of lane l; shared or global memory).  Lane l receives the
// three normalised outputs of ray l.  All 32 lanes must call it together.
// frag / bias: the inference fragments and biases (in shared memory).  The
// two m16 tiles (rays 0-15, 16-31) run one after the other to keep the live
// registers down.
__device__ __forceinline__ void mlp_warp(const uint2* frag, const float* bias, const float* X,
                                         float o[3]) {
  const int lane = threadIdx.x & 31;
  const int g = lane >> 2, t = lane & 3;
  const int src = 4 * (lane & 7);       // lane holding outputs 0, 1 of my row
  const bool hi = (lane & 15) >= 8;     // my row is in the upper half of the tile
#pragma unroll 1
  for (int mt = 0; mt < 2; ++mt) {
    // layer-1 A fragment from feature rows 16 mt + g and 16 mt + g + 8
    const float* x0 = X + (16 * mt + g) * K0 + 2 * t;
    const float* x1 = x0 + 8 * K0;
    uint32_t x_hi[1][4], x_lo[1][4];
    split_pack_h(x0[0], x0[1], &x_hi[0][0], &x_lo[0][0]);
    split_pack_h(x1[0], x1[1], &x_hi[0][1], &x_lo[0][1]);
    split_pack_h(x0[8], x0[9], &x_hi[0][2], &x_lo[0][2]);
    split_pack_h(x1[8], x1[9], &x_hi[0][3], &x_lo[0][3]);
    uint32_t a_hi[4][4], a_lo[4][4], b_hi[4][4], b_lo[4][4];
    mlp_hidden<1>(frag + FR1, bias, x_hi, x_lo, a_hi, a_lo, lane);
    mlp_hidden<4>(frag + FR2, bias + HID, a_hi, a_lo, b_hi, b_lo, lane);
    mlp_hidden<4>(frag + FR3, bias + 2 * HID, b_hi, b_lo, a_hi, a_lo, lane);
    const float c0 = bias[3 * HID + 2 * t], c1 = bias[3 * HID + 2 * t + 1];
    float acc[4] = {c0, c1, c0, c1};
#pragma unroll
    for (int kb = 0; kb < 4; ++kb) {
      const uint2 b = frag[FR4 + kb * 32 + lane];
      mma_f16(acc, a_lo[kb], b.x, b.y);
      mma_f16(acc, a_hi[kb], b.x, b.y);
    }
    // output j of tile row (l % 16) sits in lane 4 (l % 8) + j / 2: acc[0]/[1]
    // for the upper 8 rows, acc[2]/[3] for the lower 8
    const float v00 = __shfl_sync(0xFFFFFFFFu, acc[0], src);
    const float v01 = __shfl_sync(0xFFFFFFFFu, acc[1], src);
    const float v02 = __shfl_sync(0xFFFFFFFFu, acc[0], src + 1);
    const float v10 = __shfl_sync(0xFFFFFFFFu, acc[2], src);
    const float v11 = __shfl_sync(0xFFFFFFFFu, acc[3], src);
    const float v12 = __shfl_sync(0xFFFFFFFFu, acc[2], src + 1);
    if ((lane >> 4) == mt) {
      o[0] = hi ? v10 : v00;
      o[1] = hi ? v11 : v01;
      o[2] = hi ? v12 : v02;
    }
  }
}

}  // namespace bhs
