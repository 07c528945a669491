// The surrogate MLP on the fifth-generation tensor cores: one CTA of 128
// threads evaluates the network for 128 rows at a time (row r = thread r).
// Each layer is D[128 x N] = A[128 x K] B[K x N] by tcgen05.mma (kind::f16,
// FP16 operands, FP32 accumulation in tensor memory), issued by one thread.
// A (the inputs, or the previous layer's activations as FP16 high parts and
// negated low parts: two MMAs per K block, the second with A negated) is
// read from tensor memory, row m in lane m; B (the layer's weights, W^T)
// from shared memory through matrix descriptors; D starts from the layer's
// bias.  Warp w reads rows 32w..32w+31 of D from tensor memory lanes
// 32w..32w+31 (tcgen05.ld), applies the SiLU and writes the next layer's A
// and bias into the same lanes (tcgen05.st): the activations never leave
// tensor memory and registers.
//
// The weight tiles in shared memory use the canonical K-major layout
// without swizzling: 8 x 8 core matrices of 8 rows of 16 bytes (8 FP16
// values along K), the core matrices adjacent along K 128 bytes apart (the
// leading-dimension byte offset) and the groups of 8 rows K/8 * 128 bytes
// apart (the stride byte offset).
#pragma once

#include <cuda_fp16.h>
#include <stdint.h>

#include "mlp.cuh"

namespace bhs {

// W^T tiles (N rows x K columns) of the four layers, FP16, in the layout above.
constexpr int TC_W1 = 0;                // 64 x 16
constexpr int TC_W2 = TC_W1 + 64 * 16;  // 64 x 64
constexpr int TC_W3 = TC_W2 + 64 * 64;  // 64 x 64
constexpr int TC_W4 = TC_W3 + 64 * 64;  // 16 x 64
constexpr int TC_NW = TC_W4 + 16 * 64;  // FP16 values
// Tensor-memory columns a CTA allocates: the accumulators (columns 0-63,
// FP32) and the layer inputs as packed FP16 pairs, high parts (64-95) and
// negated low parts (96-127).  Every kernel that allocates tensor memory
// (the surrogate pass, the inference kernel) holds about 54 KB of shared
// memory a CTA (TcSmem::reserve), so at most four such CTAs share an SM: its
// 512 columns, and an allocation never has to wait for another CTA's.
constexpr int TC_COLS = 128;
constexpr uint32_t TC_A_HI = 64, TC_A_LO = 96;

// FP16 element offset of (row, k) in a tile of K columns (K = 16 or 64).
__host__ __device__ constexpr int tc_off(int row, int k, int K) {
  return (row >> 3) * (8 * K) + (k >> 3) * 64 + (row & 7) * 8 + (k & 7);
}

struct TcSmem {
  uint16_t w[TC_NW];        // weights (the hidden layers' halved)
  unsigned char reserve[32768];  // unused: keeps four CTAs an SM (see TC_COLS)
  float bias[NBIAS];        // b1 / 2, b2 / 2, b3 / 2, first 8 of b4
  unsigned long long mbar;  // completion of the layer's MMAs
  uint32_t tmem;            // tensor-memory base address
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// Shared-memory matrix descriptor: start address, leading- and stride-
// dimension byte offsets (all >> 4), descriptor version 1, no swizzle.
__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)(lbo >> 4) << 16) |
         ((uint64_t)(sbo >> 4) << 32) | (1ull << 46);
}

// Instruction descriptor of kind::f16: FP32 D, FP16 A and B, both K-major,
// N >> 3 at bit 17, M >> 4 at bit 24.
__host__ __device__ constexpr uint32_t tc_idesc(int M, int N) {
  return (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
// Negate-A bit of the instruction descriptor (bit 13): D += -A B.
constexpr uint32_t TC_NEG_A = 1u << 13;

// D (+)= A B with A read from tensor memory (a_tmem: lane 0, first column of
// the K block; row m of A in lane m, two FP16 values a column) and B from a
// shared-memory descriptor.
__device__ __forceinline__ void tc_mma_ta(uint32_t d_tmem, uint32_t a_tmem, uint64_t b, uint32_t idesc,
                                          uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}\n" ::"r"(d_tmem),
      "r"(a_tmem), "l"(b), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void tc_commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
               : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// generic-proxy shared-memory writes -> visible to the tensor cores
__device__ __forceinline__ void fence_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_init(uint32_t mbar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mbar), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Wait of up to about suspend_ns for the barrier's phase with the given
// parity to complete (the thread sleeps meanwhile); true when it has.
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity, uint32_t suspend_ns) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(mbar), "r"(parity), "r"(suspend_ns)
      : "memory");
  return ok != 0;
}

// Tensor-memory allocation of ncols columns by one whole warp; the address
// is written to shared memory at dst.
__device__ __forceinline__ void tmem_alloc(uint32_t dst, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst), "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
               : "memory");
}

// 16 consecutive 32-bit columns of this thread's tensor-memory lane, waited.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
      "[%16];\n\ttcgen05.wait::ld.sync.aligned;\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
        "=r"(r[15])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// An FP32 pair as FP16 high parts hi = fp16(x) and negated low parts
// nlo = fp16(hi - x): hi - x is exact in FP32, and with the hi operand
// added and the nlo operand subtracted (the MMA's negate-A bit) the two
// MMAs of a K block sum to x to about 2^-22 relative.  The difference is
// one mixed-precision subtract per value (FP16 minuend, FP32 subtrahend).
__device__ __forceinline__ void split_pair(float x0, float x1, uint32_t* hi, uint32_t* nlo) {
  const __half2 h = __floats2half2_rn(x0, x1);
  const uint32_t hb = *reinterpret_cast<const uint32_t*>(&h);
  float d0, d1;
  asm("{\n\t.reg .b16 a, b;\n\tmov.b32 {a, b}, %2;\n\t"
      "sub.rn.f32.f16 %0, a, %3;\n\tsub.rn.f32.f16 %1, b, %4;\n\t}\n"
      : "=f"(d0), "=f"(d1)
      : "r"(hb), "f"(x0), "f"(x1));
  const __half2 l = __floats2half2_rn(d0, d1);
  *hi = hb;
  *nlo = *reinterpret_cast<const uint32_t*>(&l);
}

// 16 consecutive 32-bit columns of this thread's tensor-memory lane set to
// v (completion is waited for with tmem_st_wait).
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const float* v) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16};\n" ::"r"(taddr),
      "f"(v[0]), "f"(v[1]), "f"(v[2]), "f"(v[3]), "f"(v[4]), "f"(v[5]), "f"(v[6]), "f"(v[7]), "f"(v[8]),
      "f"(v[9]), "f"(v[10]), "f"(v[11]), "f"(v[12]), "f"(v[13]), "f"(v[14]), "f"(v[15])
      : "memory");
}
__device__ __forceinline__ void tmem_st_wait() {
  asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

// Eight consecutive 32-bit columns of this thread's tensor-memory lane set
// to u (completion is waited for with tmem_st_wait).
__device__ __forceinline__ void tmem_st8u(uint32_t taddr, const uint32_t* u) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};\n" ::"r"(taddr),
               "r"(u[0]), "r"(u[1]), "r"(u[2]), "r"(u[3]), "r"(u[4]), "r"(u[5]), "r"(u[6]), "r"(u[7])
               : "memory");
}

// Sixteen FP32 values as the high and negated low FP16 parts of eight
// packed columns of A, written to this thread's lane at column col.
__device__ __forceinline__ void a_to_tmem(uint32_t lane_addr, uint32_t col, const float* x) {
  uint32_t h[8], l[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) split_pair(x[2 * q], x[2 * q + 1], &h[q], &l[q]);
  tmem_st8u(lane_addr + TC_A_HI + col, h);
  tmem_st8u(lane_addr + TC_A_LO + col, l);
}

// A layer's bias, columns 16c..16c+15, into this thread's accumulator lane
// (the layer's MMAs then accumulate onto it).  The output layer has 8
// stored bias values; its columns 8..15 are not read.
__device__ __forceinline__ void bias_to_tmem(const TcSmem& s, uint32_t lane_addr, int layer, int c) {
  float b[16];
  if (layer < 3) {
    const float4* src = reinterpret_cast<const float4*>(s.bias + HID * layer + 16 * c);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float4 t = src[q];
      b[4 * q] = t.x;
      b[4 * q + 1] = t.y;
      b[4 * q + 2] = t.z;
      b[4 * q + 3] = t.w;
    }
  } else {
    const float4* src = reinterpret_cast<const float4*>(s.bias + 3 * HID);
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const float4 t = src[q];
      b[4 * q] = t.x;
      b[4 * q + 1] = t.y;
      b[4 * q + 2] = t.z;
      b[4 * q + 3] = t.w;
    }
#pragma unroll
    for (int j = 8; j < 16; ++j) b[j] = 0.0f;
  }
  tmem_st16(lane_addr + 16u * c, b);
}

// Waits of up to kTcWaitNs each allowed on a layer's completion before the
// pass gives up (20 ms in all; a layer's MMAs take a few microseconds).
constexpr int kTcSpin = 200;
constexpr uint32_t kTcWaitNs = 100000;

// The network for the CTA's 128 rows: all 128 threads call it together with
// their row's features f (K0 values); thread r receives row r's three
// outputs.  tmem: the CTA's tensor-memory columns; phase: the completion
// barrier's parity, advanced per layer.  Returns false when a layer's MMAs
// did not complete within kTcSpin polls (the outputs are then garbage).
__device__ __forceinline__ bool mlp_cta_tc(TcSmem& s, uint32_t tmem, uint32_t& phase, const float* f,
                                           float o[3]) {
  const int r = threadIdx.x;
  const int w = r >> 5;
  const uint32_t mbar = smem_u32(&s.mbar);
  const uint32_t lane_addr = tmem + ((uint32_t)(32 * w) << 16);
  a_to_tmem(lane_addr, 0, f);
#pragma unroll
  for (int c = 0; c < 4; ++c) bias_to_tmem(s, lane_addr, 0, c);
  tmem_st_wait();
  // the weights staged in shared memory by these threads, for the MMAs
  fence_async_smem();
  tc_fence_before();
  __syncthreads();
  bool ok = true;
#pragma unroll 1
  for (int L = 0; L < 4; ++L) {
    if (r == 0) {
      tc_fence_after();
      // A from tensor memory (8 columns a K block), accumulating onto the
      // bias; the low parts subtracted
      if (L == 0) {
        const uint64_t b = tc_desc(smem_u32(s.w + TC_W1), 128, 256);
        tc_mma_ta(tmem, tmem + TC_A_LO, b, tc_idesc(128, 64) | TC_NEG_A, 1u);
        tc_mma_ta(tmem, tmem + TC_A_HI, b, tc_idesc(128, 64), 1u);
      } else {
        const int wo = L == 1 ? TC_W2 : (L == 2 ? TC_W3 : TC_W4);
        const uint32_t id = tc_idesc(128, L == 3 ? 16 : 64);
        const uint32_t wb = smem_u32(s.w + wo);
#pragma unroll
        for (int kb = 0; kb < 4; ++kb) {
          const uint64_t b = tc_desc(wb + 256u * kb, 128, 1024);
          tc_mma_ta(tmem, tmem + TC_A_LO + 8u * kb, b, id | TC_NEG_A, 1u);
          tc_mma_ta(tmem, tmem + TC_A_HI + 8u * kb, b, id, 1u);
        }
      }
      tc_commit(mbar);
    }
    // thread 0 sleeps on the barrier; the others wait at the CTA barrier
    bool done = true;
    if (r == 0) {
      done = false;
      for (int i = 0; i < kTcSpin && !done; ++i) done = mbar_wait(mbar, phase, kTcWaitNs);
    }
    phase ^= 1u;
    if (__syncthreads_or(!done)) ok = false;
    tc_fence_after();
    if (L < 3) {
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        float v[16];
        tmem_ld16(lane_addr + 16u * c, v);
        // the next layer's bias into the columns just read
        if (L < 2 || c == 0) bias_to_tmem(s, lane_addr, L + 1, c);
#pragma unroll
        for (int j = 0; j < 16; ++j) v[j] = fmaf(v[j], tanh_approx(v[j]), v[j]);
        a_to_tmem(lane_addr, 8u * c, v);
      }
      tmem_st_wait();
      tc_fence_before();
      __syncthreads();
    } else {
      float v[16];
      tmem_ld16(lane_addr, v);
      o[0] = v[0];
      o[1] = v[1];
      o[2] = v[2];
      tc_fence_before();
    }
  }
  return ok;
}

}  // namespace bhs
