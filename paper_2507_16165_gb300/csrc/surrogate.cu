// MLP surrogate: labels from the FP64 integrator, BF16 tensor-core training
// (forward, backward, Adam with FP32 master weights), calibration of the
// served domain, persistence, and the surrogate render.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "mlp.cuh"
#include "mlp_tc.cuh"
#include "runtime.h"
#include "tracer.cuh"

using namespace bhk;
using bf16 = __nv_bfloat16;

static_assert(bhs::NPARAM == BH_MLP_NPARAM, "parameter count of the C-ABI");

// Trained surrogate of a scene.
struct SurrogateState {
  std::vector<float> params;        // bhs::NPARAM, FP32 master weights
  int nb_lb = 0, nb_r = 0;          // calibration table dims
  std::vector<unsigned char> table; // served (1) / fallback (0)
  uint16_t* d_w = nullptr;
  float* d_bias = nullptr;
  unsigned char* d_table = nullptr;
  int* d_list = nullptr;            // fallback list
  size_t list_cap = 0;
  std::vector<float> cal_pd, cal_pr;  // per-bin p99.9 deflection / radius error
  std::vector<int> cal_n;             // per-bin calibration sample count
};

namespace {

constexpr double kBc = 5.19615242270663188;  // 3 sqrt 3

// ---------------------------------------------------------------------------
// Labels: bare FP64 orbits from (b, r_obs) with the static-observer initial
// state, integrated until escape and past psi0 + pi.
// ---------------------------------------------------------------------------
__global__ void k_labels(int n, double M, const double* __restrict__ bs, const double* __restrict__ rs,
                         const double* __restrict__ psis, double rtol, double* phi_inf,
                         double* u_a, double* u_b, int* status) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double b = bs[i], r = rs[i], psi = psis[i];
  const double u0 = 1.0 / r;
  const double v2 = 1.0 / (b * b) - u0 * u0 + 2.0 * M * u0 * u0 * u0;
  phi_inf[i] = NAN;
  u_a[i] = NAN;
  u_b[i] = NAN;
  if (!(v2 >= 0.0) || !(b > 0.0)) {
    status[i] = 1;  // no ray from this observer has this impact parameter
    return;
  }
  const double M3 = 3.0 * M;
  double u = u0, v = sqrt(v2), f = accel(M3, u), phi = 0.0;
  double h = initial_step<double>(M3, u, v, rtol, rtol, 0.01);
  const double ta = psi, tb = psi + 3.14159265358979323846;
  const double u_capt = M > 0.0 ? 1.0 / (2.0 * M) : INFINITY;
  bool esc = false, got_a = false, got_b = false;
  int st = 3;
  for (int steps = 0; steps < 100000 && phi < 64.0; ++steps) {
    double un, vn, fn;
    float err2;
    dp5_attempt<double>(M3, u, v, f, h, rtol, rtol, un, vn, fn, err2);
    const double hs = h;
    h = hs * step_factor<double>(err2);
    if (!(err2 <= 1.0f)) continue;
    const double pb = phi + hs;
    Hermite<double> H;
    H.make(phi, hs, u, v, f, un, vn, fn);
    if (!esc && un >= u_capt) {
      st = 2;
      break;
    }
    if (!esc && un <= 0.0) {
      phi_inf[i] = phi + hs * hermite_root<double>(H, 0.0, 0.0, 1.0);
      esc = true;
    }
    if (!got_a && ta <= pb) {
      u_a[i] = H.u_at(ta);
      got_a = true;
    }
    if (!got_b && tb <= pb) {
      u_b[i] = H.u_at(tb);
      got_b = true;
    }
    u = un;
    v = vn;
    f = fn;
    phi = pb;
    if (esc && got_a && got_b) {
      st = 0;
      break;
    }
  }
  status[i] = st;
}

// ---------------------------------------------------------------------------
// Training kernels.  Row-major BF16 activations [B][width], weights W[in][out]
// (BF16 copies of the FP32 masters), FP32 accumulation on mma.sync.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t ld_pair(const bf16* p) {
  return *reinterpret_cast<const uint32_t*>(p);
}
__device__ __forceinline__ uint32_t pack_raw(bf16 lo, bf16 hi) {
  return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

// Z = X W + b, H = act(Z); one warp per 32 rows.  X enters the tensor cores
// as BF16 high + low parts (two mma per block), W as BF16.
template <int KP, int NP, bool ACT>
__global__ void k_fwd(int B, const float* __restrict__ X, const bf16* __restrict__ W,
                      const float* __restrict__ bias, float* __restrict__ Z, float* __restrict__ Hout) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  if (warp * 32 >= B) return;
  for (int mt = 0; mt < 2; ++mt) {
    const int row0 = warp * 32 + mt * 16;
    for (int j = 0; j < NP / 8; ++j) {
      float acc[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
      for (int kb = 0; kb < KP / 16; ++kb) {
        uint32_t ah[4], al[4];
        const float* x0 = X + (row0 + g) * KP + 16 * kb + 2 * t;
        const float* x1 = X + (row0 + g + 8) * KP + 16 * kb + 2 * t;
        bhs::split_pack(x0[0], x0[1], &ah[0], &al[0]);
        bhs::split_pack(x1[0], x1[1], &ah[1], &al[1]);
        bhs::split_pack(x0[8], x0[9], &ah[2], &al[2]);
        bhs::split_pack(x1[8], x1[9], &ah[3], &al[3]);
        const int n = 8 * j + g;
        const uint32_t b0 = pack_raw(W[(16 * kb + 2 * t) * NP + n], W[(16 * kb + 2 * t + 1) * NP + n]);
        const uint32_t b1 = pack_raw(W[(16 * kb + 8 + 2 * t) * NP + n], W[(16 * kb + 9 + 2 * t) * NP + n]);
        bhs::mma_bf16(acc, al, b0, b1);
        bhs::mma_bf16(acc, ah, b0, b1);
      }
      const int c = 8 * j + 2 * t;
      const float zz[4] = {acc[0] + bias[c], acc[1] + bias[c + 1], acc[2] + bias[c], acc[3] + bias[c + 1]};
      const int rows[2] = {row0 + g, row0 + g + 8};
      for (int q = 0; q < 4; ++q) {
        const int rr = rows[q >> 1], cc = c + (q & 1);
        Z[rr * NP + cc] = zz[q];
        Hout[rr * NP + cc] = ACT ? bhs::silu(zz[q]) : zz[q];
      }
    }
  }
}

// Output gradient of the weighted mean squared error over the 3 used
// outputs (target row: 3 targets, then their 3 weights):
// dZ = 2 w (Z - T) / (B * 3), loss += sum w (Z - T)^2 / (B * 3).
__global__ void k_outgrad(int B, const float* __restrict__ Z, const float* __restrict__ T,
                          bf16* __restrict__ dZ, float* loss) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  float l = 0.0f;
  if (i < B * bhs::NO) {
    const int c = i % bhs::NO;
    float d = 0.0f;
    if (c < bhs::NOUT) {
      const float e = Z[i] - T[i], wt = T[i + bhs::NOUT];
      d = 2.0f * wt * e / (B * bhs::NOUT);
      l = wt * e * e / (B * bhs::NOUT);
    }
    dZ[i] = __float2bfloat16_rn(d);
  }
  for (int off = 16; off > 0; off >>= 1) l += __shfl_down_sync(0xFFFFFFFFu, l, off);
  if ((threadIdx.x & 31) == 0 && l != 0.0f) atomicAdd(loss, l);
}

// dZprev = (dZ W^T) * silu'(Zprev); one warp per 32 rows.
template <int KP, int NP>
__global__ void k_bwd_dx(int B, const bf16* __restrict__ dZ, const bf16* __restrict__ W,
                         const float* __restrict__ Zprev, bf16* __restrict__ dZprev) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  if (warp * 32 >= B) return;
  for (int mt = 0; mt < 2; ++mt) {
    const int row0 = warp * 32 + mt * 16;
    for (int j = 0; j < KP / 8; ++j) {
      float acc[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
      for (int nb = 0; nb < NP / 16; ++nb) {
        uint32_t a[4];
        a[0] = ld_pair(dZ + (row0 + g) * NP + 16 * nb + 2 * t);
        a[1] = ld_pair(dZ + (row0 + g + 8) * NP + 16 * nb + 2 * t);
        a[2] = ld_pair(dZ + (row0 + g) * NP + 16 * nb + 8 + 2 * t);
        a[3] = ld_pair(dZ + (row0 + g + 8) * NP + 16 * nb + 8 + 2 * t);
        // B = W^T: (k = n of W, n = k of W) -> W[8j + g][16 nb + 2t ...]
        const bf16* wr = W + (8 * j + g) * NP + 16 * nb;
        bhs::mma_bf16(acc, a, ld_pair(wr + 2 * t), ld_pair(wr + 8 + 2 * t));
      }
      const int c = 8 * j + 2 * t;
      const int rows[2] = {row0 + g, row0 + g + 8};
      for (int q = 0; q < 4; ++q) {
        const int rr = rows[q >> 1], cc = c + (q & 1);
        dZprev[rr * KP + cc] = __float2bfloat16_rn(acc[q] * bhs::silu_grad(Zprev[rr * KP + cc]));
      }
    }
  }
}

// dW += Hprev^T dZ over a batch slice (Hprev rounded to BF16); one warp per
// (m16 tile of KP, slice).
template <int KP, int NP>
__global__ void k_bwd_dw(int B, int slice, const float* __restrict__ Hp, const bf16* __restrict__ dZ,
                         float* __restrict__ dW) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const int nmt = KP / 16;
  const int mt = warp % nmt, sl = warp / nmt;
  const int k0 = sl * slice;
  if (k0 >= B) return;
  float acc[NP / 8][4];
#pragma unroll
  for (int j = 0; j < NP / 8; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.0f;
  for (int kb = 0; kb < slice / 16; ++kb) {
    const int k = k0 + 16 * kb;
    if (k >= B) break;
    const int m = 16 * mt + g;
    uint32_t a[4];
    a[0] = bhs::pack_bf16(Hp[(k + 2 * t) * KP + m], Hp[(k + 2 * t + 1) * KP + m]);
    a[1] = bhs::pack_bf16(Hp[(k + 2 * t) * KP + m + 8], Hp[(k + 2 * t + 1) * KP + m + 8]);
    a[2] = bhs::pack_bf16(Hp[(k + 8 + 2 * t) * KP + m], Hp[(k + 9 + 2 * t) * KP + m]);
    a[3] = bhs::pack_bf16(Hp[(k + 8 + 2 * t) * KP + m + 8], Hp[(k + 9 + 2 * t) * KP + m + 8]);
#pragma unroll
    for (int j = 0; j < NP / 8; ++j) {
      const int n = 8 * j + g;
      const uint32_t b0 = pack_raw(dZ[(k + 2 * t) * NP + n], dZ[(k + 2 * t + 1) * NP + n]);
      const uint32_t b1 = pack_raw(dZ[(k + 8 + 2 * t) * NP + n], dZ[(k + 9 + 2 * t) * NP + n]);
      bhs::mma_bf16(acc[j], a, b0, b1);
    }
  }
#pragma unroll
  for (int j = 0; j < NP / 8; ++j) {
    const int r0 = 16 * mt + g, c = 8 * j + 2 * t;
    atomicAdd(&dW[r0 * NP + c], acc[j][0]);
    atomicAdd(&dW[r0 * NP + c + 1], acc[j][1]);
    atomicAdd(&dW[(r0 + 8) * NP + c], acc[j][2]);
    atomicAdd(&dW[(r0 + 8) * NP + c + 1], acc[j][3]);
  }
}

// db += column sums of dZ; one block of NP threads per 256-row slice.
template <int NP>
__global__ void k_bias_grad(int B, const bf16* __restrict__ dZ, float* __restrict__ db) {
  const int c = threadIdx.x, r0 = blockIdx.x * 256;
  float s = 0.0f;
  for (int r = r0; r < min(B, r0 + 256); ++r) s += __bfloat162float(dZ[r * NP + c]);
  atomicAdd(&db[c], s);
}

// Adam on the FP32 masters (trainable entries only), refresh the BF16
// copies, clear the gradient.
__global__ void k_adam(int n, float* __restrict__ w, float* __restrict__ m, float* __restrict__ v,
                       float* __restrict__ grad, bf16* __restrict__ wb,
                       const unsigned char* __restrict__ trainable, float lr, float b1, float b2,
                       float eps, float bc1, float bc2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (trainable[i]) {
    const float g = grad[i];
    const float mi = b1 * m[i] + (1.0f - b1) * g;
    const float vi = b2 * v[i] + (1.0f - b2) * g * g;
    m[i] = mi;
    v[i] = vi;
    w[i] -= lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
  }
  wb[i] = __float2bfloat16_rn(w[i]);
  grad[i] = 0.0f;
}

// Gather a batch by index.
__global__ void k_gather(int B, const int* __restrict__ idx, const float* __restrict__ X,
                         const float* __restrict__ T, float* __restrict__ Xb, float* __restrict__ Tb) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= B) return;
  const int s = idx[i];
  for (int k = 0; k < bhs::K0; ++k) Xb[i * bhs::K0 + k] = X[s * bhs::K0 + k];
  for (int k = 0; k < bhs::NO; ++k) Tb[i * bhs::NO + k] = T[s * bhs::NO + k];
}

// Inference on feature rows x[n][K0] on the tensor cores (tcgen05): one CTA
// of 128 threads per 128 rows, persistent over the row groups.  A layer that
// does not complete in time sets *status and ends the CTA's loop.
__global__ void __launch_bounds__(128) k_mlp_infer_tc(int n, const float* __restrict__ x,
                                                      const uint16_t* __restrict__ wtc,
                                                      const float* __restrict__ bias_g,
                                                      float* __restrict__ y, unsigned* status) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  bhs::TcSmem& s = *reinterpret_cast<bhs::TcSmem*>(smem_raw);
  const int tid = threadIdx.x;
  for (int i = tid; i < bhs::TC_NW / 8; i += 128)
    reinterpret_cast<uint4*>(s.w)[i] = reinterpret_cast<const uint4*>(wtc)[i];
  for (int i = tid; i < bhs::NBIAS; i += 128) s.bias[i] = bias_g[i];
  if (tid < 32) bhs::tmem_alloc(bhs::smem_u32(&s.tmem), bhs::TC_COLS);
  if (tid == 0) bhs::mbar_init(bhs::smem_u32(&s.mbar), 1);
  bhs::tc_fence_before();
  __syncthreads();
  bhs::tc_fence_after();
  const uint32_t tmem = s.tmem;
  uint32_t phase = 0;
  for (long long g = blockIdx.x; g * 128 < n; g += gridDim.x) {
    const long long i = g * 128 + tid;
    float f[bhs::K0];
#pragma unroll
    for (int k = 0; k < bhs::K0; ++k) f[k] = i < n ? x[i * bhs::K0 + k] : 0.0f;
    float o[3];
    const bool ok = bhs::mlp_cta_tc(s, tmem, phase, f, o);
    if (i < n) {
      y[3 * i] = o[0];
      y[3 * i + 1] = o[1];
      y[3 * i + 2] = o[2];
    }
    if (__syncthreads_or(!ok)) {
      if (tid == 0) atomicOr(status, 1u);
      break;
    }
  }
  bhs::tc_fence_before();
  __syncthreads();
  if (tid < 32) {
    bhs::tc_fence_after();
    bhs::tmem_dealloc(tmem, bhs::TC_COLS);
  }
}

// The wait of the tensor-core kernels run out on purpose: tensor memory
// allocated, an mbarrier that nothing arrives on, the same bounded wait,
// then the same release of the tensor memory.  out[0] = 1 when the wait
// gave up, out[1] = the clock64 cycles it took.
__global__ void __launch_bounds__(32) k_tc_wait_probe(int tries, unsigned wait_ns,
                                                      unsigned long long* out) {
  __shared__ unsigned long long mbar;
  __shared__ uint32_t taddr;
  bhs::tmem_alloc(bhs::smem_u32(&taddr), bhs::TC_COLS);
  if (threadIdx.x == 0) bhs::mbar_init(bhs::smem_u32(&mbar), 1);
  bhs::tc_fence_before();
  __syncwarp();
  bhs::tc_fence_after();
  if (threadIdx.x == 0) {
    const long long t0 = clock64();
    bool done = false;
    for (int i = 0; i < tries && !done; ++i) done = bhs::mbar_wait(bhs::smem_u32(&mbar), 0u, wait_ns);
    out[0] = done ? 0ull : 1ull;
    out[1] = (unsigned long long)(clock64() - t0);
  }
  bhs::tc_fence_before();
  __syncwarp();
  bhs::tc_fence_after();
  bhs::tmem_dealloc(taddr, bhs::TC_COLS);
}

// FP16 W^T tiles of the tensor-core path (the trained BF16 values, the
// hidden layers' halved) from FP32 masters.
void pack_tc_weights(const std::vector<float>& p, std::vector<uint16_t>* w) {
  w->assign(bhs::TC_NW, 0);
  auto h = [](float x, float sc) {
    return (uint16_t)__half_as_ushort(__float2half_rn(sc * __bfloat162float(__float2bfloat16_rn(x))));
  };
  for (int n = 0; n < bhs::HID; ++n) {
    for (int k = 0; k < bhs::K0; ++k)
      (*w)[bhs::TC_W1 + bhs::tc_off(n, k, 16)] = h(p[bhs::OW1 + k * bhs::HID + n], 0.5f);
    for (int k = 0; k < bhs::HID; ++k) {
      (*w)[bhs::TC_W2 + bhs::tc_off(n, k, 64)] = h(p[bhs::OW2 + k * bhs::HID + n], 0.5f);
      (*w)[bhs::TC_W3 + bhs::tc_off(n, k, 64)] = h(p[bhs::OW3 + k * bhs::HID + n], 0.5f);
    }
  }
  for (int n = 0; n < bhs::NO; ++n)
    for (int k = 0; k < bhs::HID; ++k)
      (*w)[bhs::TC_W4 + bhs::tc_off(n, k, 64)] = h(p[bhs::OW4 + k * bhs::NO + n], 1.0f);
}

// ---------------------------------------------------------------------------
// Host helpers
// ---------------------------------------------------------------------------
uint64_t splitmix(uint64_t& s) {
  uint64_t z = (s += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
double uniform01(uint64_t& s) { return (splitmix(s) >> 11) * (1.0 / 9007199254740992.0); }

bf16 to_bf16(float x) { return __float2bfloat16_rn(x); }

// Which parameters train: the padded input rows of W1 and padded output
// columns of W4, b4 stay zero.
std::vector<unsigned char> trainable_mask() {
  std::vector<unsigned char> m(bhs::NPARAM, 1);
  for (int k = bhs::NFEAT; k < bhs::K0; ++k)
    for (int n = 0; n < bhs::HID; ++n) m[bhs::OW1 + k * bhs::HID + n] = 0;
  for (int k = 0; k < bhs::HID; ++k)
    for (int n = bhs::NOUT; n < bhs::NO; ++n) m[bhs::OW4 + k * bhs::NO + n] = 0;
  for (int n = bhs::NOUT; n < bhs::NO; ++n) m[bhs::OB4 + n] = 0;
  return m;
}

// Xavier-uniform weights from splitmix64, zero biases and padding.
std::vector<float> init_params(uint64_t seed) {
  std::vector<float> p(bhs::NPARAM, 0.0f);
  uint64_t s = seed * 0x2545F4914F6CDD1Dull + 1;
  auto fill = [&](int off, int fan_in, int fan_out, int rows, int cols, int ld) {
    const double a = std::sqrt(6.0 / (fan_in + fan_out));
    for (int k = 0; k < rows; ++k)
      for (int n = 0; n < cols; ++n) p[off + k * ld + n] = (float)((2.0 * uniform01(s) - 1.0) * a);
  };
  fill(bhs::OW1, bhs::NFEAT, bhs::HID, bhs::NFEAT, bhs::HID, bhs::HID);
  fill(bhs::OW2, bhs::HID, bhs::HID, bhs::HID, bhs::HID, bhs::HID);
  fill(bhs::OW3, bhs::HID, bhs::HID, bhs::HID, bhs::HID, bhs::HID);
  fill(bhs::OW4, bhs::HID, 3, bhs::HID, 3, bhs::NO);
  return p;
}

// Biases of the inference path: those of the hidden layers halved (the
// tensor-core tiles hold the hidden layers' weights halved, so the
// pre-activations come out as z / 2).
void pack_bias(const std::vector<float>& p, std::vector<float>* bias) {
  bias->assign(bhs::NBIAS, 0.0f);
  for (int n = 0; n < bhs::HID; ++n) {
    (*bias)[n] = 0.5f * p[bhs::OB1 + n];
    (*bias)[bhs::HID + n] = 0.5f * p[bhs::OB2 + n];
    (*bias)[2 * bhs::HID + n] = 0.5f * p[bhs::OB3 + n];
  }
  for (int n = 0; n < 8; ++n) (*bias)[3 * bhs::HID + n] = p[bhs::OB4 + n];
}

// Flat-space exit angle alpha of the ray with impact parameter b at r.
double alpha_of(double b, double r) { return M_PI - std::asin(std::min(1.0, b * std::sqrt(1.0 - 2.0 / r) / r)); }

// Training-state device buffers.
struct DevBuf {
  std::vector<void*> ptrs;
  ~DevBuf() {
    for (void* p : ptrs) cudaFree(p);
  }
  template <typename T>
  cudaError_t alloc(T** p, size_t n) {
    cudaError_t e = cudaMalloc((void**)p, std::max<size_t>(1, n) * sizeof(T));
    if (e == cudaSuccess) ptrs.push_back(*p);
    return e;
  }
};

// Forward + backward of one batch on the device (gradients accumulate into
// d_grad).  All buffers sized for B rows; B a multiple of 32.
struct Net {
  int B = 0;
  float *X = nullptr, *H1 = nullptr, *H2 = nullptr, *H3 = nullptr, *H4 = nullptr;
  float *Z1 = nullptr, *Z2 = nullptr, *Z3 = nullptr, *Z4 = nullptr, *T = nullptr;
  bf16 *dZ1 = nullptr, *dZ2 = nullptr, *dZ3 = nullptr, *dZ4 = nullptr;
  float *w = nullptr, *grad = nullptr, *loss = nullptr;
  bf16* wb = nullptr;
  cudaError_t alloc(DevBuf& db, int b) {
    B = b;
    cudaError_t e = cudaSuccess;
    auto A = [&](auto** p, size_t n) {
      if (e == cudaSuccess) e = db.alloc(p, n);
    };
    A(&X, (size_t)B * bhs::K0);
    A(&H1, (size_t)B * bhs::HID);
    A(&H2, (size_t)B * bhs::HID);
    A(&H3, (size_t)B * bhs::HID);
    A(&H4, (size_t)B * bhs::NO);
    A(&Z1, (size_t)B * bhs::HID);
    A(&Z2, (size_t)B * bhs::HID);
    A(&Z3, (size_t)B * bhs::HID);
    A(&Z4, (size_t)B * bhs::NO);
    A(&T, (size_t)B * bhs::NO);
    A(&dZ1, (size_t)B * bhs::HID);
    A(&dZ2, (size_t)B * bhs::HID);
    A(&dZ3, (size_t)B * bhs::HID);
    A(&dZ4, (size_t)B * bhs::NO);
    A(&w, bhs::NPARAM);
    A(&grad, bhs::NPARAM);
    A(&wb, bhs::NPARAM);
    A(&loss, 1);
    return e;
  }
  void step(cudaStream_t s) {
    const int wb_blocks = (B / 32 * 32 + 255) / 256;
    k_fwd<bhs::K0, bhs::HID, true><<<wb_blocks, 256, 0, s>>>(B, X, wb + bhs::OW1, w + bhs::OB1, Z1, H1);
    k_fwd<bhs::HID, bhs::HID, true><<<wb_blocks, 256, 0, s>>>(B, H1, wb + bhs::OW2, w + bhs::OB2, Z2, H2);
    k_fwd<bhs::HID, bhs::HID, true><<<wb_blocks, 256, 0, s>>>(B, H2, wb + bhs::OW3, w + bhs::OB3, Z3, H3);
    k_fwd<bhs::HID, bhs::NO, false><<<wb_blocks, 256, 0, s>>>(B, H3, wb + bhs::OW4, w + bhs::OB4, Z4, H4);
    k_outgrad<<<(B * bhs::NO + 255) / 256, 256, 0, s>>>(B, Z4, T, dZ4, loss);
    const int slice = 512;
    const int nsl = (B + slice - 1) / slice;
    k_bwd_dw<bhs::HID, bhs::NO><<<(4 * nsl * 32 + 255) / 256, 256, 0, s>>>(B, slice, H3, dZ4, grad + bhs::OW4);
    k_bias_grad<bhs::NO><<<(B + 255) / 256, bhs::NO, 0, s>>>(B, dZ4, grad + bhs::OB4);
    k_bwd_dx<bhs::HID, bhs::NO><<<wb_blocks, 256, 0, s>>>(B, dZ4, wb + bhs::OW4, Z3, dZ3);
    k_bwd_dw<bhs::HID, bhs::HID><<<(4 * nsl * 32 + 255) / 256, 256, 0, s>>>(B, slice, H2, dZ3, grad + bhs::OW3);
    k_bias_grad<bhs::HID><<<(B + 255) / 256, bhs::HID, 0, s>>>(B, dZ3, grad + bhs::OB3);
    k_bwd_dx<bhs::HID, bhs::HID><<<wb_blocks, 256, 0, s>>>(B, dZ3, wb + bhs::OW3, Z2, dZ2);
    k_bwd_dw<bhs::HID, bhs::HID><<<(4 * nsl * 32 + 255) / 256, 256, 0, s>>>(B, slice, H1, dZ2, grad + bhs::OW2);
    k_bias_grad<bhs::HID><<<(B + 255) / 256, bhs::HID, 0, s>>>(B, dZ2, grad + bhs::OB2);
    k_bwd_dx<bhs::HID, bhs::HID><<<wb_blocks, 256, 0, s>>>(B, dZ2, wb + bhs::OW2, Z1, dZ1);
    k_bwd_dw<bhs::K0, bhs::HID><<<(1 * nsl * 32 + 255) / 256, 256, 0, s>>>(B, slice, X, dZ1, grad + bhs::OW1);
    k_bias_grad<bhs::HID><<<(B + 255) / 256, bhs::HID, 0, s>>>(B, dZ1, grad + bhs::OB1);
  }
};

int upload_surrogate(bh_scene* sc, SurrogateState* s) {
  std::vector<float> bias;
  pack_bias(s->params, &bias);
  std::vector<uint16_t> wtc;
  pack_tc_weights(s->params, &wtc);
  cudaError_t e = cudaSuccess;
  if (!s->d_w) e = cudaMalloc((void**)&s->d_w, bhs::TC_NW * sizeof(uint16_t));
  if (e == cudaSuccess && !s->d_bias) e = cudaMalloc((void**)&s->d_bias, bhs::NBIAS * sizeof(float));
  if (e == cudaSuccess) {
    if (s->d_table) cudaFree(s->d_table);
    s->d_table = nullptr;
    e = cudaMalloc((void**)&s->d_table, std::max<size_t>(1, s->table.size()));
  }
  if (e == cudaSuccess) e = cudaMemcpy(s->d_w, wtc.data(), bhs::TC_NW * sizeof(uint16_t), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(s->d_bias, bias.data(), bhs::NBIAS * sizeof(float), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(s->d_table, s->table.data(), s->table.size(), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return bh_cuda_fail(e, "surrogate upload");
  (void)sc;
  return BH_OK;
}

uint64_t fnv1a(const void* data, size_t n, uint64_t h = 0xcbf29ce484222325ull) {
  const unsigned char* p = (const unsigned char*)data;
  for (size_t i = 0; i < n; ++i) h = (h ^ p[i]) * 0x100000001b3ull;
  return h;
}

// Run the inference kernel on host features (normalised), host outputs.
int infer_host(const std::vector<float>& params, int n, const float* x, float* y, cudaStream_t st) {
  std::vector<float> bias;
  pack_bias(params, &bias);
  std::vector<uint16_t> wtc;
  pack_tc_weights(params, &wtc);
  DevBuf db;
  uint16_t* d_w;
  float *d_bias, *d_x, *d_y;
  unsigned* d_status;
  cudaError_t e = db.alloc(&d_w, bhs::TC_NW);
  if (e == cudaSuccess) e = db.alloc(&d_bias, bhs::NBIAS);
  if (e == cudaSuccess) e = db.alloc(&d_x, (size_t)bhs::K0 * n);
  if (e == cudaSuccess) e = db.alloc(&d_y, (size_t)3 * n);
  if (e == cudaSuccess) e = db.alloc(&d_status, 1);
  if (e == cudaSuccess) e = cudaMemsetAsync(d_status, 0, sizeof(unsigned), st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_w, wtc.data(), bhs::TC_NW * sizeof(uint16_t), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_bias, bias.data(), bhs::NBIAS * sizeof(float), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_x, x, (size_t)bhs::K0 * n * sizeof(float), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_mlp_infer_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(bhs::TcSmem));
  if (e != cudaSuccess) return bh_cuda_fail(e, "mlp inference setup");
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int groups = (n + 127) / 128;
  const int blocks = std::max(1, std::min(groups, 2 * sms));
  k_mlp_infer_tc<<<blocks, 128, sizeof(bhs::TcSmem), st>>>(n, d_x, d_w, d_bias, d_y, d_status);
  e = cudaGetLastError();
  unsigned status = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(y, d_y, (size_t)3 * n * sizeof(float), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&status, d_status, sizeof(unsigned), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return bh_cuda_fail(e, "mlp inference");
  if (status) return bh_fail(BH_E_DEVICE, "mlp inference: a tensor-core layer did not complete");
  return BH_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
// C-ABI
// ---------------------------------------------------------------------------
extern "C" int bh_surrogate_labels(double mass, int n, const double* b, const double* r_obs,
                                   const double* psi0, double* phi_inf, double* u_a, double* u_b,
                                   int* status, void* stream) {
  if (n < 0 || !(mass >= 0.0)) return bh_fail(BH_E_INVALID, "bh_surrogate_labels: bad size or mass");
  if (n == 0) return BH_OK;
  if (!b || !r_obs || !psi0 || !phi_inf || !u_a || !u_b || !status)
    return bh_fail(BH_E_INVALID, "bh_surrogate_labels: null pointer");
  k_labels<<<(n + 127) / 128, 128, 0, (cudaStream_t)stream>>>(n, mass, b, r_obs, psi0, 1e-10, phi_inf,
                                                              u_a, u_b, status);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return bh_cuda_fail(e, "bh_surrogate_labels");
  return BH_OK;
}

extern "C" int bh_mlp_grad(const float* params, int n, const float* x, const float* t, float* y,
                           float* grad, float* loss, void* stream) {
  if (!params || !x || !t || n < 32 || n % 32)
    return bh_fail(BH_E_INVALID, "bh_mlp_grad: need params, x, t and n a positive multiple of 32");
  cudaStream_t st = (cudaStream_t)stream;
  DevBuf db;
  Net net;
  cudaError_t e = net.alloc(db, n);
  if (e != cudaSuccess) return bh_cuda_fail(e, "bh_mlp_grad: allocation");
  std::vector<float> xb(x, x + (size_t)n * bhs::K0);
  std::vector<float> tb((size_t)n * bhs::NO, 0.0f);
  for (int i = 0; i < n; ++i)
    for (int k = 0; k < bhs::NOUT; ++k) {
      tb[(size_t)i * bhs::NO + k] = t[3 * i + k];
      tb[(size_t)i * bhs::NO + bhs::NOUT + k] = 1.0f;  // unweighted
    }
  std::vector<bf16> wbh(bhs::NPARAM);
  for (int i = 0; i < bhs::NPARAM; ++i) wbh[i] = to_bf16(params[i]);
  e = cudaMemcpyAsync(net.X, xb.data(), xb.size() * sizeof(float), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(net.T, tb.data(), tb.size() * sizeof(float), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(net.w, params, bhs::NPARAM * sizeof(float), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(net.wb, wbh.data(), bhs::NPARAM * sizeof(bf16), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(net.grad, 0, bhs::NPARAM * sizeof(float), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(net.loss, 0, sizeof(float), st);
  if (e != cudaSuccess) return bh_cuda_fail(e, "bh_mlp_grad: upload");
  net.step(st);
  e = cudaGetLastError();
  std::vector<float> z4((size_t)n * bhs::NO);
  if (e == cudaSuccess) e = cudaMemcpyAsync(z4.data(), net.Z4, z4.size() * sizeof(float), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && grad) e = cudaMemcpyAsync(grad, net.grad, bhs::NPARAM * sizeof(float), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && loss) e = cudaMemcpyAsync(loss, net.loss, sizeof(float), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return bh_cuda_fail(e, "bh_mlp_grad: run");
  if (y)
    for (int i = 0; i < n; ++i)
      for (int k = 0; k < bhs::NOUT; ++k) y[3 * i + k] = z4[(size_t)i * bhs::NO + k];
  return BH_OK;
}

extern "C" int bh_selftest_wait_timeout(int tries, int wait_ns, int* timed_out, double* waited_ms) {
  if (!timed_out || !waited_ms) return bh_fail(BH_E_INVALID, "bh_selftest_wait_timeout: null output");
  tries = std::min(10000, std::max(1, tries));
  wait_ns = std::min(1000000, std::max(1, wait_ns));
  DevBuf db;
  unsigned long long* d_out;
  cudaError_t e = db.alloc(&d_out, 2);
  if (e == cudaSuccess) e = cudaMemset(d_out, 0, 2 * sizeof(unsigned long long));
  if (e != cudaSuccess) return bh_cuda_fail(e, "bh_selftest_wait_timeout: setup");
  k_tc_wait_probe<<<1, 32>>>(tries, (unsigned)wait_ns, d_out);
  e = cudaGetLastError();
  unsigned long long h[2] = {0, 0};
  if (e == cudaSuccess) e = cudaMemcpy(h, d_out, sizeof(h), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return bh_cuda_fail(e, "bh_selftest_wait_timeout");
  int dev = 0, khz = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, dev);
  *timed_out = (int)h[0];
  *waited_ms = khz > 0 ? (double)h[1] / (double)khz : 0.0;
  return BH_OK;
}

extern "C" int bh_mlp_infer(const float* params, int n, const float* x, float* y, void* stream) {
  if (!params || !x || !y || n < 0) return bh_fail(BH_E_INVALID, "bh_mlp_infer: null argument");
  if (n == 0) return BH_OK;
  std::vector<float> p(params, params + bhs::NPARAM);
  return infer_host(p, n, x, y, (cudaStream_t)stream);
}

namespace {

// Labelled samples: FP64 integrator labels of host samples (units of M),
// feature rows X[nv][K0], normalised targets Y[nv][3], and b, r of each.
struct Labelled {
  std::vector<float> X, Y;
  std::vector<double> b, r;
  int n = 0;
};

int label_samples(cudaStream_t st, int n, const double* hb, const double* hr, const double* hpsi,
                  Labelled* L) {
  DevBuf db;
  double *d_b, *d_r, *d_p, *d_phi, *d_ua, *d_ub;
  int* d_st;
  cudaError_t e = db.alloc(&d_b, n);
  if (e == cudaSuccess) e = db.alloc(&d_r, n);
  if (e == cudaSuccess) e = db.alloc(&d_p, n);
  if (e == cudaSuccess) e = db.alloc(&d_phi, n);
  if (e == cudaSuccess) e = db.alloc(&d_ua, n);
  if (e == cudaSuccess) e = db.alloc(&d_ub, n);
  if (e == cudaSuccess) e = db.alloc(&d_st, n);
  if (e != cudaSuccess) return bh_cuda_fail(e, "surrogate labels: buffers");
  e = cudaMemcpyAsync(d_b, hb, n * sizeof(double), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_r, hr, n * sizeof(double), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_p, hpsi, n * sizeof(double), cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return bh_cuda_fail(e, "surrogate labels: upload");
  int rc = bh_surrogate_labels(1.0, n, d_b, d_r, d_p, d_phi, d_ua, d_ub, d_st, st);
  if (rc) return rc;
  std::vector<double> phi(n), ua(n), ub(n);
  std::vector<int> status(n);
  e = cudaMemcpyAsync(phi.data(), d_phi, n * sizeof(double), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(ua.data(), d_ua, n * sizeof(double), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(ub.data(), d_ub, n * sizeof(double), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(status.data(), d_st, n * sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return bh_cuda_fail(e, "surrogate labels");
  L->X.clear();
  L->Y.clear();
  L->b.clear();
  L->r.clear();
  for (int i = 0; i < n; ++i) {
    if (!(status[i] == 0 && hb[i] > kBc + 1e-5 && std::isfinite(ua[i]) && std::isfinite(ub[i]))) continue;
    double xd[bhs::K0];
    bhs::surrogate_features<double>(hb[i], hr[i], hpsi[i], xd);
    for (int k = 0; k < bhs::K0; ++k) L->X.push_back((float)xd[k]);
    const double delta = phi[i] - alpha_of(hb[i], hr[i]);
    L->Y.push_back((float)((delta * hb[i] / 4.0 - bhs::D_C) / bhs::D_S));
    L->Y.push_back((float)(ua[i] * hb[i]));
    L->Y.push_back((float)(ub[i] * hb[i]));
    L->b.push_back(hb[i]);
    L->r.push_back(hr[i]);
  }
  L->n = (int)L->b.size();
  return BH_OK;
}

// Calibrate the served domain: run the inference kernel on labelled
// samples [first, first + count) and, per bin of (feature x0 =
// normalised ln(b - 3 sqrt 3), r_obs), take the 99.9th percentile of the
// deflection error (rad) and of the relative disk-crossing radius error
// |dr| / r (for true crossings at 2.5 M < r < 60 M; the disk colour is a
// function of ln r, so a relative bound is a bound on the shading error).  A bin is served when it holds at least
// 50 samples and both percentiles are within the thresholds.
int calibrate(SurrogateState* s, cudaStream_t st, const Labelled& L, int first, int count, int nb_lb,
              int nb_r, double thr_d, double thr_r, std::vector<float>* pd_out,
              std::vector<float>* pr_out, std::vector<int>* n_out, double se[3], double* served) {
  std::vector<float> yv((size_t)count * 3);
  int rc = infer_host(s->params, count, L.X.data() + (size_t)first * bhs::K0, yv.data(), st);
  if (rc) return rc;
  const int nbin = nb_lb * nb_r;
  std::vector<std::vector<float>> ed(nbin), er(nbin);
  for (int k = 0; k < 3; ++k) se[k] = 0.0;
  for (int j = 0; j < count; ++j) {
    const int i = first + j;
    const float x0 = L.X[(size_t)i * bhs::K0];
    const int ib = std::min(nb_lb - 1, std::max(0, (int)((x0 + 1.0f) * 0.5f * nb_lb)));
    const int ir = std::min(nb_r - 1, std::max(0, (int)((L.r[i] - 15.0) / 85.0 * nb_r)));
    const int bin = ib * nb_r + ir;
    const float* y = yv.data() + (size_t)j * 3;
    const float* t = L.Y.data() + (size_t)i * 3;
    for (int k = 0; k < 3; ++k) se[k] += (double)(y[k] - t[k]) * (y[k] - t[k]);
    ed[bin].push_back((float)std::fabs((double)(y[0] - t[0]) * bhs::D_S * 4.0 / L.b[i]));
    for (int k = 1; k < 3; ++k) {
      const double ut = t[k] / L.b[i], up = y[k] / L.b[i];
      if (ut > 1.0 / 60.0 && ut < 1.0 / 2.5)
        er[bin].push_back((float)(up > 0 ? std::min(std::fabs(ut / up - 1.0), 1e9) : 1e9));
    }
  }
  auto q999 = [](std::vector<float>& v) -> double {
    if (v.empty()) return 0.0;
    std::sort(v.begin(), v.end());
    return v[std::min(v.size() - 1, (size_t)std::ceil(0.999 * (v.size() - 1)))];
  };
  s->nb_lb = nb_lb;
  s->nb_r = nb_r;
  s->table.assign(nbin, 0);
  pd_out->assign(nbin, 0.0f);
  pr_out->assign(nbin, 0.0f);
  n_out->assign(nbin, 0);
  size_t served_n = 0;
  for (int bin = 0; bin < nbin; ++bin) {
    const double pd = q999(ed[bin]), pr = q999(er[bin]);
    (*pd_out)[bin] = (float)pd;
    (*pr_out)[bin] = (float)pr;
    (*n_out)[bin] = (int)ed[bin].size();
    s->table[bin] = (ed[bin].size() >= 50 && pd <= thr_d && pr <= thr_r) ? 1 : 0;
    if (s->table[bin]) served_n += ed[bin].size();
  }
  *served = (double)served_n / std::max(1, count);
  return BH_OK;
}

}  // namespace

extern "C" int bh_surrogate_train(bh_scene* sc, int n, const double* hb, const double* hr,
                                  const double* hpsi, const bh_train_opts* opts,
                                  bh_train_report* rep) {
  if (!sc || !hb || !hr || !hpsi || !opts || n < 1024)
    return bh_fail(BH_E_INVALID, "bh_surrogate_train: need a scene, samples (n >= 1024) and options");
  if (!(sc->sk.M > 0.0)) return bh_fail(BH_E_INVALID, "bh_surrogate_train: needs M > 0");
  DeviceGuard dg(sc->device);
  cudaStream_t st = (cudaStream_t)opts->stream;
  const auto t0 = std::chrono::steady_clock::now();
  Labelled L;
  int rc = label_samples(st, n, hb, hr, hpsi, &L);
  if (rc) return rc;
  const auto t1 = std::chrono::steady_clock::now();
  const int nv = L.n;
  const int n_val = std::max(32, (int)(opts->val_fraction > 0 ? opts->val_fraction * nv : 0.05 * nv)) / 32 * 32;
  const int n_tr = nv - n_val;
  const int B = opts->batch > 0 ? opts->batch / 32 * 32 : 16384;
  if (n_tr < B) return bh_fail(BH_E_INVALID, "bh_surrogate_train: %d valid training samples < batch %d", n_tr, B);
  // targets with the weights of the loss: the deflection error in radians
  // is 12 |dy0| / b, so its term is weighted by min(25, (10/b)^2)
  std::vector<float> T((size_t)nv * bhs::NO, 0.0f);
  for (int j = 0; j < nv; ++j) {
    const float wts[3] = {(float)std::min(25.0, (10.0 / L.b[j]) * (10.0 / L.b[j])), 1.0f, 1.0f};
    for (int k = 0; k < 3; ++k) {
      T[(size_t)j * bhs::NO + k] = L.Y[(size_t)j * 3 + k];
      T[(size_t)j * bhs::NO + bhs::NOUT + k] = wts[k];
    }
  }
  DevBuf db;
  float* d_X;
  float* d_T;
  int* d_idx;
  float *d_m, *d_v;
  unsigned char* d_mask;
  Net net;
  cudaError_t e = db.alloc(&d_X, L.X.size());
  if (e == cudaSuccess) e = db.alloc(&d_T, T.size());
  if (e == cudaSuccess) e = db.alloc(&d_idx, (size_t)n_tr);
  if (e == cudaSuccess) e = db.alloc(&d_m, bhs::NPARAM);
  if (e == cudaSuccess) e = db.alloc(&d_v, bhs::NPARAM);
  if (e == cudaSuccess) e = db.alloc(&d_mask, bhs::NPARAM);
  if (e == cudaSuccess) e = net.alloc(db, B);
  if (e != cudaSuccess) return bh_cuda_fail(e, "bh_surrogate_train: buffers");
  std::vector<float> params = init_params(opts->seed);
  std::vector<bf16> wbh(bhs::NPARAM);
  for (int i = 0; i < bhs::NPARAM; ++i) wbh[i] = to_bf16(params[i]);
  const std::vector<unsigned char> mask = trainable_mask();
  e = cudaMemcpyAsync(d_X, L.X.data(), L.X.size() * sizeof(float), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_T, T.data(), T.size() * sizeof(float), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(net.w, params.data(), bhs::NPARAM * sizeof(float), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(net.wb, wbh.data(), bhs::NPARAM * sizeof(bf16), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_mask, mask.data(), bhs::NPARAM, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(d_m, 0, bhs::NPARAM * sizeof(float), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(d_v, 0, bhs::NPARAM * sizeof(float), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(net.grad, 0, bhs::NPARAM * sizeof(float), st);
  if (e != cudaSuccess) return bh_cuda_fail(e, "bh_surrogate_train: init");

  // Adam over shuffled mini-batches, cosine learning-rate decay
  const int epochs = opts->epochs > 0 ? opts->epochs : 20;
  const double lr0 = opts->lr > 0 ? opts->lr : 2e-3;
  const int steps_per_epoch = n_tr / B;
  const int total = epochs * steps_per_epoch;
  std::vector<int> perm(n_tr);
  for (int i = 0; i < n_tr; ++i) perm[i] = i;
  uint64_t rs = opts->seed ^ 0x5DEECE66Dull;
  const float b1 = 0.9f, b2 = 0.999f;
  double bc1 = 1.0, bc2 = 1.0;
  int step = 0;
  float last_loss = 0.0f;
  for (int ep = 0; ep < epochs; ++ep) {
    for (int i = n_tr - 1; i > 0; --i) std::swap(perm[i], perm[splitmix(rs) % (uint64_t)(i + 1)]);
    e = cudaMemcpyAsync(d_idx, perm.data(), n_tr * sizeof(int), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return bh_cuda_fail(e, "bh_surrogate_train: shuffle");
    cudaMemsetAsync(net.loss, 0, sizeof(float), st);
    for (int s = 0; s < steps_per_epoch; ++s, ++step) {
      k_gather<<<(B + 255) / 256, 256, 0, st>>>(B, d_idx + (size_t)s * B, d_X, d_T, net.X, net.T);
      net.step(st);
      bc1 *= b1;
      bc2 *= b2;
      const double lr = 1e-2 * lr0 + 0.5 * (lr0 - 1e-2 * lr0) * (1.0 + std::cos(M_PI * step / total));
      k_adam<<<(bhs::NPARAM + 255) / 256, 256, 0, st>>>(bhs::NPARAM, net.w, d_m, d_v, net.grad, net.wb, d_mask,
                                                       (float)lr, b1, b2, 1e-8f, (float)(1.0 - bc1),
                                                       (float)(1.0 - bc2));
    }
    // the read-back throttles the host so queued launches stay bounded
    e = cudaMemcpyAsync(&last_loss, net.loss, sizeof(float), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return bh_cuda_fail(e, "bh_surrogate_train: epoch");
    last_loss /= std::max(1, steps_per_epoch);
  }
  e = cudaMemcpyAsync(params.data(), net.w, bhs::NPARAM * sizeof(float), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return bh_cuda_fail(e, "bh_surrogate_train: download");
  const auto t2 = std::chrono::steady_clock::now();

  SurrogateState* s = sc->surr ? sc->surr : new SurrogateState();
  s->params = params;
  sc->surr = s;
  double se[3], served = 0.0;
  rc = calibrate(s, st, L, n_tr, n_val, 24, 4,
                 opts->err_threshold > 0 ? opts->err_threshold : 1e-3,
                 opts->r_err_threshold > 0 ? opts->r_err_threshold : 2e-3, &s->cal_pd, &s->cal_pr,
                 &s->cal_n, se, &served);
  if (rc) return rc;
  rc = upload_surrogate(sc, s);
  if (rc) return rc;
  const auto t3 = std::chrono::steady_clock::now();
  if (rep) {
    memset(rep, 0, sizeof *rep);
    rep->n_samples = n;
    rep->n_valid = nv;
    rep->n_train = n_tr;
    rep->n_val = n_val;
    rep->steps = total;
    rep->final_loss = last_loss;
    for (int k = 0; k < 3; ++k) rep->val_rmse[k] = (float)std::sqrt(se[k] / std::max(1, n_val));
    rep->served_fraction = (float)served;
    rep->label_ms = std::chrono::duration<float, std::milli>(t1 - t0).count();
    rep->train_ms = std::chrono::duration<float, std::milli>(t2 - t1).count();
    rep->calib_ms = std::chrono::duration<float, std::milli>(t3 - t2).count();
  }
  return BH_OK;
}

extern "C" int bh_surrogate_calibrate(bh_scene* sc, int n, const double* hb, const double* hr,
                                      const double* hpsi, const bh_calib_opts* opts,
                                      float* p999_delta, float* p999_r, int* counts,
                                      float* served_fraction) {
  if (!sc || !hb || !hr || !hpsi || !opts || n < 32)
    return bh_fail(BH_E_INVALID, "bh_surrogate_calibrate: need a scene, samples (n >= 32) and options");
  if (!sc->surr) return bh_fail(BH_E_NO_SURROGATE, "bh_surrogate_calibrate: no trained surrogate");
  const int nb_lb = opts->nb_lb > 0 ? opts->nb_lb : 32, nb_r = opts->nb_r > 0 ? opts->nb_r : 8;
  if (nb_lb > 1024 || nb_r > 1024) return bh_fail(BH_E_INVALID, "bh_surrogate_calibrate: too many bins");
  DeviceGuard dg(sc->device);
  cudaStream_t st = (cudaStream_t)opts->stream;
  Labelled L;
  int rc = label_samples(st, n, hb, hr, hpsi, &L);
  if (rc) return rc;
  if (L.n < 32) return bh_fail(BH_E_INVALID, "bh_surrogate_calibrate: fewer than 32 valid samples");
  SurrogateState* s = sc->surr;
  double se[3], served = 0.0;
  rc = calibrate(s, st, L, 0, L.n, nb_lb, nb_r, opts->err_threshold > 0 ? opts->err_threshold : 1e-3,
                 opts->r_err_threshold > 0 ? opts->r_err_threshold : 2e-3, &s->cal_pd, &s->cal_pr,
                 &s->cal_n, se, &served);
  if (rc) return rc;
  rc = upload_surrogate(sc, s);
  if (rc) return rc;
  const size_t nbin = (size_t)nb_lb * nb_r;
  if (p999_delta) memcpy(p999_delta, s->cal_pd.data(), nbin * sizeof(float));
  if (p999_r) memcpy(p999_r, s->cal_pr.data(), nbin * sizeof(float));
  if (counts) memcpy(counts, s->cal_n.data(), nbin * sizeof(int));
  if (served_fraction) *served_fraction = (float)served;
  return BH_OK;
}

extern "C" int bh_surrogate_get(const bh_scene* sc, float* params, unsigned char* table, int* nb_lb,
                                int* nb_r) {
  if (!sc) return bh_fail(BH_E_INVALID, "bh_surrogate_get: null scene");
  if (!sc->surr) return bh_fail(BH_E_NO_SURROGATE, "bh_surrogate_get: no trained surrogate");
  if (params) memcpy(params, sc->surr->params.data(), bhs::NPARAM * sizeof(float));
  if (table) memcpy(table, sc->surr->table.data(), sc->surr->table.size());
  if (nb_lb) *nb_lb = sc->surr->nb_lb;
  if (nb_r) *nb_r = sc->surr->nb_r;
  return BH_OK;
}

// File: "BHSURR01", u32 version, u32 nparam, u32 nb_lb, u32 nb_r,
// f32 params[nparam], u8 table[nb_lb * nb_r], u64 FNV-1a of everything before.
extern "C" int bh_surrogate_save(const bh_scene* sc, const char* path) {
  if (!sc || !path) return bh_fail(BH_E_INVALID, "bh_surrogate_save: null argument");
  if (!sc->surr) return bh_fail(BH_E_NO_SURROGATE, "bh_surrogate_save: no trained surrogate");
  const SurrogateState* s = sc->surr;
  std::vector<unsigned char> buf;
  auto put = [&](const void* p, size_t n) {
    const unsigned char* c = (const unsigned char*)p;
    buf.insert(buf.end(), c, c + n);
  };
  const uint32_t hdr[4] = {1u, (uint32_t)bhs::NPARAM, (uint32_t)s->nb_lb, (uint32_t)s->nb_r};
  put("BHSURR01", 8);
  put(hdr, sizeof hdr);
  put(s->params.data(), s->params.size() * sizeof(float));
  put(s->table.data(), s->table.size());
  const uint64_t h = fnv1a(buf.data(), buf.size());
  put(&h, sizeof h);
  FILE* f = fopen(path, "wb");
  if (!f) return bh_fail(BH_E_IO, "bh_surrogate_save: cannot open %s", path);
  const size_t w = fwrite(buf.data(), 1, buf.size(), f);
  fclose(f);
  if (w != buf.size()) return bh_fail(BH_E_IO, "bh_surrogate_save: short write to %s", path);
  return BH_OK;
}

extern "C" int bh_surrogate_load(bh_scene* sc, const char* path) {
  if (!sc || !path) return bh_fail(BH_E_INVALID, "bh_surrogate_load: null argument");
  FILE* f = fopen(path, "rb");
  if (!f) return bh_fail(BH_E_IO, "bh_surrogate_load: cannot open %s", path);
  std::vector<unsigned char> buf;
  unsigned char tmp[4096];
  size_t r;
  while ((r = fread(tmp, 1, sizeof tmp, f)) > 0) buf.insert(buf.end(), tmp, tmp + r);
  fclose(f);
  const size_t head = 8 + 16;
  if (buf.size() < head + 8 || memcmp(buf.data(), "BHSURR01", 8) != 0)
    return bh_fail(BH_E_IO, "bh_surrogate_load: %s is not a surrogate file", path);
  uint32_t hdr[4];
  memcpy(hdr, buf.data() + 8, sizeof hdr);
  const size_t body = (size_t)hdr[1] * sizeof(float) + (size_t)hdr[2] * hdr[3];
  if (hdr[0] != 1u || hdr[1] != (uint32_t)bhs::NPARAM || hdr[2] == 0 || hdr[3] == 0 || hdr[2] > 1024 ||
      hdr[3] > 1024 || buf.size() != head + body + 8)
    return bh_fail(BH_E_IO, "bh_surrogate_load: %s has an unexpected layout", path);
  uint64_t h;
  memcpy(&h, buf.data() + head + body, sizeof h);
  if (h != fnv1a(buf.data(), head + body)) return bh_fail(BH_E_IO, "bh_surrogate_load: checksum mismatch in %s", path);
  DeviceGuard dg(sc->device);
  SurrogateState* s = sc->surr ? sc->surr : new SurrogateState();
  s->params.assign(bhs::NPARAM, 0.0f);
  memcpy(s->params.data(), buf.data() + head, bhs::NPARAM * sizeof(float));
  s->nb_lb = (int)hdr[2];
  s->nb_r = (int)hdr[3];
  s->table.assign(buf.begin() + head + bhs::NPARAM * sizeof(float), buf.begin() + head + body);
  sc->surr = s;
  return upload_surrogate(sc, s);
}

// ---------------------------------------------------------------------------
// Surrogate render
// ---------------------------------------------------------------------------
// Host-side preparation of a surrogate render: the integrator passes run in
// MIXED arithmetic with the launch shape tuned for the surrogate mode; the
// fallback list is sized; the FP64 band pass is set to run on the scene's
// side stream.  cams_dev as for prepare_render.
int surrogate_prepare(bh_scene* sc, const bh_camera* cams, int n_cams, const int* w, const int* h,
                      void* dirs, uint16_t* flags, uint32_t* rgba, const bh_render_opts* opts,
                      cudaStream_t upload_stream, CamK* cams_dev, PreparedRender* pr) {
  if (!sc->surr || !sc->surr->d_w)
    return bh_fail(BH_E_NO_SURROGATE, "surrogate mode: no trained weights on this scene");
  if (sc->sk.ic != BH_IC_STATIC && sc->sk.ic != BH_IC_EUCLIDEAN)
    return bh_fail(BH_E_INVALID, "surrogate mode: unknown initial-condition convention");
  {
    const cudaError_t e = surrogate_kernel_setup();
    if (e != cudaSuccess) return bh_cuda_fail(e, "surrogate mode: kernel set-up");
  }
  const TunedShape t = tuned_shape(sc, BH_MODE_SURROGATE);
  bh_render_opts o = *opts;
  o.mode = BH_MODE_MIXED;
  if (!o.tile_w && !o.tile_h) {
    o.tile_w = t.tile_w;
    o.tile_h = t.tile_h;
  }
  if (!o.queue_chunk) o.queue_chunk = t.chunk;
  if (!o.budget) o.budget = t.budget;
  int rc = prepare_render(sc, cams, n_cams, w, h, dirs, flags, rgba, &o, upload_stream, cams_dev, pr);
  if (rc) return rc;
  SurrogateState* s = sc->surr;
  const size_t need = (size_t)pr->p.n_queue;
  if (s->list_cap < need) {
    if (s->d_list) cudaFree(s->d_list);
    s->d_list = nullptr;
    s->list_cap = 0;
    cudaError_t e = cudaMalloc((void**)&s->d_list, need * sizeof(int));
    if (e != cudaSuccess) return bh_cuda_fail(e, "surrogate: fallback list");
    s->list_cap = need;
  }
  // the FP64 band pass runs on the side stream beside the surrogate pass
  pr->ls.side = sc->side;
  pr->ls.fork = sc->fork;
  pr->ls.join = sc->join;
  pr->ls.band_ev = sc->band_ev;
  pr->ls.band_warps = t.band_warps;
  pr->p.band_trim = 0;  // the band pass keeps its warps beside the surrogate pass
  pr->p.mlp_w = s->d_w;
  pr->p.mlp_bias = s->d_bias;
  pr->p.surr_table = s->d_table;
  pr->p.surr_nb_lb = s->nb_lb;
  pr->p.surr_nb_r = s->nb_r;
  pr->p.surr_list = s->d_list;
  pr->mode = BH_MODE_SURROGATE;
  return BH_OK;
}

// Device work of a prepared surrogate render (also what a graph captures).
int surrogate_enqueue(bh_scene* sc, const PreparedRender& pr, cudaStream_t stream) {
  cudaError_t e = cudaMemsetAsync(sc->d_ws, 0, sizeof(WorkK), stream);
  if (e == cudaSuccess) e = launch_surrogate(pr.p, pr.ls, stream, sc->ev);
  if (e != cudaSuccess) return bh_cuda_fail(e, "surrogate render: launch");
  return BH_OK;
}

int surrogate_render(bh_scene* sc, const bh_camera* cams, int n_cams, const int* w, const int* h,
                     void* dirs, uint16_t* flags, uint32_t* rgba, const bh_render_opts* opts) {
  cudaStream_t stream = (cudaStream_t)opts->stream;
  PreparedRender pr;
  int rc = surrogate_prepare(sc, cams, n_cams, w, h, dirs, flags, rgba, opts, stream, nullptr, &pr);
  if (rc) return rc;
  rc = surrogate_enqueue(sc, pr, stream);
  if (rc) return rc;
  sc->last_stream = stream;
  sc->timed = true;
  sc->band_used = true;
  return BH_OK;
}

void surrogate_release(bh_scene* sc) {
  if (!sc->surr) return;
  SurrogateState* s = sc->surr;
  cudaFree(s->d_w);
  cudaFree(s->d_bias);
  cudaFree(s->d_table);
  cudaFree(s->d_list);
  delete s;
  sc->surr = nullptr;
}
