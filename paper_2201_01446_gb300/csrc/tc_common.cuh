// tcgen05 / mbarrier / bulk-copy helpers shared by the tensor-core kernels
// (inline PTX for sm_103a).  Every wait is bounded by kSpinLimit polls.
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

namespace dp_tc {

constexpr long long kSpinLimit = 20000000;  // bounded mbarrier waits

// element offset of (row r, column k) inside one piece of a tiled block:
// 8-row groups 128 elements apart, K groups 64 apart, rows 8 apart
__host__ __device__ __forceinline__ int tile_off(int r, int k) {
  return (r >> 3) * 128 + ((k >> 3) & 1) * 64 + (r & 7) * 8 + (k & 7);
}


__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// 64-bit shared-memory matrix descriptor, no swizzle, K-major:
// start address, leading byte offset (K direction), stride byte offset
// (8-row groups), version 1 (bits 46-47), layout type 0 (bits 61-63).
__device__ __forceinline__ uint64_t make_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// instruction descriptor for kind::f16: D f32, A/B bf16, both K-major
__host__ __device__ constexpr uint32_t make_idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

// instruction descriptor for kind::f16: D f32, A/B f16, both K-major
__host__ __device__ constexpr uint32_t make_idesc_f16(int M, int N) {
  return (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(done)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return done != 0;
}

// bounded wait of at most `limit` polls; false on timeout (which raises the
// CTA's abort flag) or when another role has already raised it (abort ==
// nullptr: only the time limit)
__device__ __forceinline__ bool mbar_wait_lim(uint64_t* bar, uint32_t parity,
                                              volatile int* abort, long long limit) {
  for (long long it = 0; it < limit; ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if (abort && *abort) return false;
  }
  if (abort) *abort = 1;
  return false;
}
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, volatile int* abort) {
  return mbar_wait_lim(bar, parity, abort, kSpinLimit);
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

// bulk global -> shared copy (16-byte aligned, size a multiple of 16) whose
// completion is counted in bytes on the mbarrier
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes,
                                         uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::
          "r"(dst),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,"
      "%15}, [%16];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
  for (int k = 0; k < 16; ++k) v[k] = __uint_as_float(r[k]);
}

// x = h + m + l with h, m, l BF16 (the FP32 value to ~2^-25 relative)
template <int PC>
__device__ __forceinline__ void split8(const float* x, __nv_bfloat16 (&pv)[3][8]) {
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    pv[0][j] = __float2bfloat16_rn(x[j]);
    if (PC > 1) {
      const float r1 = x[j] - __bfloat162float(pv[0][j]);
      pv[1][j] = __float2bfloat16_rn(r1);
      pv[2][j] = __float2bfloat16_rn(r1 - __bfloat162float(pv[1][j]));
    }
  }
}

// pieces (a, b) multiplied for PC = 3: every product down to 2^-16 relative
__device__ __forceinline__ void prod_pieces(int q, int& pa, int& pb) {
  // (h,h) (h,m) (m,h) (h,l) (l,h) (m,m)
  const int a[6] = {0, 0, 1, 0, 2, 1};
  const int b[6] = {0, 1, 0, 2, 0, 1};
  pa = a[q];
  pb = b[q];
}

}  // namespace dp_tc
