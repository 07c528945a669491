// Small MLP of the surrogate: inputs (b/M, r_obs/M, plane angle) -> three
// hidden layers of 64 with SiLU -> (deflection, u b at the first two disk
// nodes) on the tensor cores with FP32 accumulation.  Training runs in BF16
// on warp-level mma.sync m16n8k16 (weights; inputs and activations as BF16
// high + low pairs; this file); inference runs on tcgen05 with the trained
// BF16 weights held exactly in FP16 and inputs and activations as FP16 high
// + low pairs (mlp_tc.cuh).
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

}  // namespace bhs
