// Fitting net (Sec. 2.1) and descriptor (Eq. 2) on the 5th-generation tensor
// cores: tcgen05.mma with BF16 operands in shared memory and the FP32
// accumulator in tensor memory (TMEM), read back with tcgen05.ld for fused
// epilogues (bias, tanh, shortcut, per-atom energy, gradient of tanh).
//
// One CTA (4 warps) computes a 128-row x NT-column tile of C = A B^T with A
// [rows x K] and B [N x K] both K-contiguous BF16 in global memory.  K is
// walked in chunks of 64 through two shared-memory stages filled with
// cp.async (16-byte pieces written straight into the no-swizzle K-major core
// matrix layout: 8 rows x 16 bytes per core matrix, consecutive K groups 128
// bytes apart, consecutive 8-row groups 1024 bytes apart).  Thread 0 issues
// four K=16 MMAs per chunk and commits them to the stage's mbarrier; a stage
// is refilled only after that barrier's phase completes.  Every wait is
// bounded: on timeout the kernel records an error word, stops issuing work,
// waits (bounded) for its MMAs, frees its TMEM and returns.
#include <cuda_bf16.h>
#include <math.h>

#include "dp_internal.h"

namespace {

constexpr int kBM = 128;        // rows per tile (one TMEM lane per row)
// TMEM columns: one accumulator of NT <= 256 columns, or (split operands) the
// exact hi*hi products in columns 0..255 and the five small piece products
// in columns 256..511, so the dominant sum sees 6x fewer FP32 accumulations
template <int PC>
struct TmemCols {
  static constexpr int value = PC == 1 ? 256 : 512;
};
constexpr long long kSpinLimit = 20000000;  // bounded mbarrier waits

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

// bounded wait; false on timeout
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  for (long long it = 0; it < kSpinLimit; ++it)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src, bool valid) {
  const int sz = valid ? 16 : 0;  // size 0: fill the 16 bytes with zeros
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst), "l"(src), "r"(sz)
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

// TC_L0: layer 0, its A operand (the descriptor D of Eq. 2) formed from T in
// the producer; TC_DT: the input gradient dE/dD contracted with T into dE/dT
// in the epilogue (D and dE/dD never reach global memory)
enum { TC_PLAIN = 0, TC_L0 = 1, TC_MID = 2, TC_LAST = 3, TC_BWD = 4, TC_DT = 5 };

struct TcEpi {
  const float* bias;       // [N]
  const float* R;          // residual rows (ldr), ldr = 0: broadcast row
  int ldr;
  const float* Tt;         // tanh values of the layer below (TC_BWD), ld = ldt
  int ldt;
  const float* wout;       // output weights (TC_LAST)
  float bout;
  float* out_a;            // FP32 [rows][ldo]: t (L0, MID) or C (PLAIN)
  float* out_b;            // FP32 [rows][ldo]: z (MID) or gz (BWD)
  __nv_bfloat16* out_h;    // BF16 pieces [PC][rows][ldo] of the next A operand
  int64_t h_ps;            // element stride between pieces of out_h
  int ldo;
  double* e_atom;          // TC_LAST: E_i written at idx[row] (or row)
  const int32_t* idx;
  int32_t* err;            // error word (timeouts)
  const float* T;          // TC_L0 / TC_DT: T rows [4][Mw] at tidx[row] (or row)
  float* dT;               // TC_DT: dE/dT rows, same indexing as T
  const int32_t* tidx;
  int Mw;                  // embedding width M
  float* part;             // TC_DT: per (N tile, half) partial sums [slot][rows][64]
  int64_t part_ps;         // elements between slots
};

// x = h + m + l with h, m, l BF16 (the FP32 value to ~2^-25 relative)
template <int PC>
__device__ __forceinline__ void split_store(__nv_bfloat16* out, int64_t ps, size_t o, const float (&x)[8]) {
  __align__(16) __nv_bfloat16 hv[8], mv[8], lv[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    hv[k] = __float2bfloat16_rn(x[k]);
    if (PC > 1) {
      const float r1 = x[k] - __bfloat162float(hv[k]);
      mv[k] = __float2bfloat16_rn(r1);
      lv[k] = __float2bfloat16_rn(r1 - __bfloat162float(mv[k]));
    }
  }
  *reinterpret_cast<uint4*>(out + o) = *reinterpret_cast<const uint4*>(hv);
  if (PC > 1) {
    *reinterpret_cast<uint4*>(out + ps + o) = *reinterpret_cast<const uint4*>(mv);
    *reinterpret_cast<uint4*>(out + 2 * ps + o) = *reinterpret_cast<const uint4*>(lv);
  }
}

template <int PC>
struct TcCfg {
  static constexpr int BK = PC == 1 ? 64 : 32;                 // K per stage
  static constexpr int SBO = BK * 16;                          // bytes between 8-row groups
  static constexpr int A_BYTES = kBM * BK * 2;                 // one piece of A
  static constexpr int B_BYTES = 256 * BK * 2;                 // one piece of B
  static constexpr int STAGE = PC * (A_BYTES + B_BYTES);
  static constexpr int NPROD = PC == 1 ? 1 : 6;                // piece products
  static constexpr size_t SMEM = 1024 + 2 * (size_t)STAGE + 64;
};

// pieces (a, b) multiplied for PC = 3: every product down to 2^-16 relative
__device__ __forceinline__ void prod_pieces(int q, int& pa, int& pb) {
  // (h,h) (h,m) (m,h) (h,l) (l,h) (m,m)
  const int a[6] = {0, 0, 1, 0, 2, 1};
  const int b[6] = {0, 1, 0, 2, 0, 1};
  pa = a[q];
  pb = b[q];
}

constexpr int kTcThreads = 256;

template <int EPI, int PC>
__global__ void __launch_bounds__(kTcThreads, 1) k_tc_gemm(int M, int N, int K, int NT,
                                                           const __nv_bfloat16* __restrict__ A,
                                                           int lda, int64_t a_ps,
                                                           const __nv_bfloat16* __restrict__ B,
                                                           int ldb, int64_t b_ps, TcEpi ep) {
  using C = TcCfg<PC>;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* base = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* bars = (uint64_t*)(base + 2 * C::STAGE);  // [2] stage barriers
  uint32_t* tmem_slot = (uint32_t*)(bars + 2);
  __shared__ int s_abort;
  __shared__ float s_e[2][kBM];

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.x * kBM, n0 = blockIdx.y * NT;
  const int ntile = min(NT, N - n0);  // columns of this tile (multiple of 16)

  if (tid == 0) {
    mbar_init(&bars[0], 1);
    mbar_init(&bars[1], 1);
    s_abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(TmemCols<PC>::value));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n");
  const uint32_t tmem = *tmem_slot;

  const int nk = (K + C::BK - 1) / C::BK;
  const uint32_t idesc = make_idesc_bf16(kBM, ntile);
  constexpr int KG = C::BK / 8;  // 16-byte K groups per row in a stage

  auto stage_ptr = [&](int s) { return base + s * C::STAGE; };
  // TC_L0: this thread's T[row][c][hal*8 .. hal*8+7], kept for every K chunk
  float ta[4][8];
  const float* trow_ptr = nullptr;
  if (EPI == TC_L0) {
    const int r = tid >> 1, hal = tid & 1;
    const int gm = m0 + r;
    if (gm < M) trow_ptr = ep.T + (size_t)(ep.tidx ? ep.tidx[gm] : gm) * 4 * ep.Mw;
#pragma unroll
    for (int c = 0; c < 4; ++c)
#pragma unroll
      for (int j = 0; j < 8; ++j) ta[c][j] = trow_ptr ? __ldg(trow_ptr + c * ep.Mw + hal * 8 + j) : 0.0f;
  }
  // fill stage s with chunk kc: every piece of A rows m0.. and B rows n0..
  auto load_stage = [&](int s, int kc) {
    const int k0 = kc * C::BK;
    const uint32_t st0 = smem_u32(stage_ptr(s));
    if (EPI == TC_L0) {
      // D[r][k] = sum_c T[c][k/16] T[c][k%16]: two threads per row, thread
      // (row, hal) forms the 8-wide groups whose a-range is hal*8..hal*8+7
      const int r = tid >> 1, hal = tid & 1;
      const int gm = m0 + r;
      unsigned char* sa = stage_ptr(s);
      for (int kg = hal; kg < KG; kg += 2) {
        const int k = k0 + kg * 8;
        float x[8];
        if (gm < M && k < K) {
          const int b = k >> 4;
          float tb[4];
#pragma unroll
          for (int c = 0; c < 4; ++c) tb[c] = __ldg(trow_ptr + c * ep.Mw + b);
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            float acc = 0.0f;
#pragma unroll
            for (int c = 0; c < 4; ++c) acc = fmaf(tb[c], ta[c][j], acc);
            x[j] = acc;
          }
        } else {
#pragma unroll
          for (int j = 0; j < 8; ++j) x[j] = 0.0f;
        }
        __align__(16) __nv_bfloat16 pv[3][8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          pv[0][j] = __float2bfloat16_rn(x[j]);
          if (PC > 1) {
            const float r1 = x[j] - __bfloat162float(pv[0][j]);
            pv[1][j] = __float2bfloat16_rn(r1);
            pv[2][j] = __float2bfloat16_rn(r1 - __bfloat162float(pv[1][j]));
          }
        }
        const int off = (r >> 3) * C::SBO + kg * 128 + (r & 7) * 16;
#pragma unroll
        for (int p = 0; p < PC; ++p)
          *reinterpret_cast<uint4*>(sa + p * C::A_BYTES + off) = *reinterpret_cast<const uint4*>(pv[p]);
      }
    }
#pragma unroll
    for (int p = 0; p < PC; ++p) {
      const uint32_t a0 = st0 + p * C::A_BYTES;
      const __nv_bfloat16* Ap = A + p * a_ps;
      for (int q = tid; q < (EPI == TC_L0 ? 0 : kBM * KG); q += kTcThreads) {
        const int r = q / KG, kg = q % KG;
        const int gm = m0 + r, gk = k0 + kg * 8;
        const bool ok = gm < M && gk < K;
        cp_async16(a0 + (r >> 3) * C::SBO + kg * 128 + (r & 7) * 16,
                   ok ? Ap + (size_t)gm * lda + gk : Ap, ok);
      }
      const uint32_t b0 = st0 + PC * C::A_BYTES + p * C::B_BYTES;
      const __nv_bfloat16* Bp = B + p * b_ps;
      for (int q = tid; q < ntile * KG; q += kTcThreads) {
        const int r = q / KG, kg = q % KG;
        const int gn = n0 + r, gk = k0 + kg * 8;
        const bool ok = gn < N && gk < K;
        cp_async16(b0 + (r >> 3) * C::SBO + kg * 128 + (r & 7) * 16,
                   ok ? Bp + (size_t)gn * ldb + gk : Bp, ok);
      }
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
  };

  load_stage(0, 0);
  int uses[2] = {0, 0};
  bool ok_run = true;
  for (int kc = 0; kc < nk; ++kc) {
    const int s = kc & 1;
    if (kc + 1 < nk) {
      const int s1 = (kc + 1) & 1;
      if (uses[s1] > 0 && !mbar_wait(&bars[s1], (uses[s1] - 1) & 1)) atomicExch(&s_abort, 1);
      __syncthreads();
      if (s_abort) {
        ok_run = false;
        break;
      }
      load_stage(s1, kc + 1);
      asm volatile("cp.async.wait_group 1;\n" ::: "memory");
    } else {
      asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    }
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;\n");
      const uint32_t st0 = smem_u32(stage_ptr(s));
#pragma unroll
      for (int j = 0; j < C::BK / 16; ++j) {
#pragma unroll
        for (int q = 0; q < C::NPROD; ++q) {
          int pa = 0, pb = 0;
          if (PC > 1) prod_pieces(q, pa, pb);
          // K = 16 covers two 8-element K groups (128 bytes apart)
          const uint64_t ad = make_desc(st0 + pa * C::A_BYTES + j * 256, 128, C::SBO);
          const uint64_t bd = make_desc(st0 + PC * C::A_BYTES + pb * C::B_BYTES + j * 256, 128,
                                        C::SBO);
          // accumulator 0: (h,h); accumulator 1 (PC = 3): the other products
          const uint32_t dst = tmem + (q > 0 ? 256u : 0u);
          const uint32_t acc = (kc > 0 || j > 0 || q > 1) ? 1u : 0u;
          asm volatile(
              "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
              " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dst),
              "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
        }
      }
      asm volatile(
          "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
              smem_u32(&bars[s])));
    }
    uses[s] += 1;
  }
  // wait for the MMAs (bounded); commits complete in order
  bool done = ok_run;
  for (int t = 0; t < 2; ++t)
    if (uses[t] > 0 && !mbar_wait(&bars[t], (uses[t] - 1) & 1)) done = false;
  if (!done) atomicExch(&s_abort, 1);
  asm volatile("tcgen05.fence::after_thread_sync;\n");
  __syncthreads();
  done = s_abort == 0;  // uniform over the CTA (the epilogue synchronises)
  if (!done) {
    if (tid == 0 && ep.err) atomicAdd(ep.err, 1);
  } else {
    // epilogue: warp w reads TMEM lanes 32*(w%4).. (its 32 rows) and one half
    // of the tile's 16-column chunks
    const int lg = warp & 3, half = warp >> 2;
    const int row_t = lg * 32 + lane;
    const int row = m0 + row_t;
    const bool rok = row < M;
    const uint32_t tbase = tmem + ((uint32_t)(lg * 32) << 16);
    const int nch = ntile / 16;
    const int c_beg = half ? (nch + 1) / 2 : 0, c_end = half ? nch : (nch + 1) / 2;
    float e_acc = 0.0f;
    // TC_DT: T[row][c][0..15] and the partial sums of the second factor
    float tl[4][16], part[4][16];
    const float* tr = nullptr;
    float* dtr = nullptr;
    if (EPI == TC_DT) {
      if (rok) {
        const size_t trow = (size_t)(ep.tidx ? ep.tidx[row] : row) * 4 * ep.Mw;
        tr = ep.T + trow;
        dtr = ep.dT + trow;
      }
#pragma unroll
      for (int c = 0; c < 4; ++c)
#pragma unroll
        for (int a = 0; a < 16; ++a) {
          tl[c][a] = tr ? __ldg(tr + c * ep.Mw + a) : 0.0f;
          part[c][a] = 0.0f;
        }
    }
    for (int ch = c_beg; ch < c_end; ++ch) {
      const int c0 = ch * 16;
      float v[16];
      tmem_ld16(tbase + (uint32_t)c0, v);
      if (PC > 1) {
        float v2[16];
        tmem_ld16(tbase + 256u + (uint32_t)c0, v2);
#pragma unroll
        for (int k = 0; k < 16; ++k) v[k] += v2[k];
      }
      if (!rok) continue;
      const int n = n0 + c0;
      if (EPI == TC_DT) {
        // v = dE/dD[b][0..15] with b = n/16 (Eq. 2: D[b][a] = sum_c T[c][b] T[c][a])
        const int b = n >> 4;
        float tb[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          tb[c] = __ldg(tr + c * ep.Mw + b);
          float acc = 0.0f;
#pragma unroll
          for (int a = 0; a < 16; ++a) acc = fmaf(v[a], tl[c][a], acc);
          dtr[c * ep.Mw + b] = acc;  // first factor: complete for this b
        }
#pragma unroll
        for (int c = 0; c < 4; ++c)
#pragma unroll
          for (int a = 0; a < 16; ++a) part[c][a] = fmaf(v[a], tb[c], part[c][a]);
        continue;
      }
      const size_t o = (size_t)row * ep.ldo + n;
      float r[16], b[16], tt[16], oa[16], ob[16], oh[16];
      if (EPI == TC_L0 || EPI == TC_MID || EPI == TC_LAST) {
#pragma unroll
        for (int k = 0; k < 16; k += 4) *reinterpret_cast<float4*>(b + k) = *reinterpret_cast<const float4*>(ep.bias + n + k);
      }
      if ((EPI == TC_MID || EPI == TC_LAST || EPI == TC_BWD)) {
        if (ep.R) {
#pragma unroll
          for (int k = 0; k < 16; k += 4)
            *reinterpret_cast<float4*>(r + k) =
                *reinterpret_cast<const float4*>(ep.R + (size_t)row * ep.ldr + n + k);
        } else {
#pragma unroll
          for (int k = 0; k < 16; ++k) r[k] = 0.0f;
        }
      }
      if (EPI == TC_BWD) {
#pragma unroll
        for (int k = 0; k < 16; k += 4)
          *reinterpret_cast<float4*>(tt + k) =
              *reinterpret_cast<const float4*>(ep.Tt + (size_t)row * ep.ldt + n + k);
      }
#pragma unroll
      for (int k = 0; k < 16; ++k) {
        if (EPI == TC_PLAIN) {
          oa[k] = v[k];
        } else if (EPI == TC_L0) {
          const float t = tanhf(v[k] + b[k]);
          oa[k] = t;
          oh[k] = t;
        } else if (EPI == TC_MID) {
          const float t = tanhf(v[k] + b[k]);
          oa[k] = t;
          ob[k] = r[k] + t;
          oh[k] = ob[k];
        } else if (EPI == TC_LAST) {
          const float t = tanhf(v[k] + b[k]);
          const float w = ep.wout[n + k];
          e_acc = fmaf(r[k] + t, w, e_acc);
          oh[k] = w * (1.0f - t * t);
        } else {  // TC_BWD
          const float gz = v[k] + r[k];
          ob[k] = gz;
          oh[k] = gz * (1.0f - tt[k] * tt[k]);
        }
      }
      if (EPI == TC_PLAIN || EPI == TC_L0 || EPI == TC_MID) {
#pragma unroll
        for (int k = 0; k < 16; k += 4)
          *reinterpret_cast<float4*>(ep.out_a + o + k) = *reinterpret_cast<const float4*>(oa + k);
      }
      if (EPI == TC_MID || EPI == TC_BWD) {
#pragma unroll
        for (int k = 0; k < 16; k += 4)
          *reinterpret_cast<float4*>(ep.out_b + o + k) = *reinterpret_cast<const float4*>(ob + k);
      }
      if (EPI != TC_PLAIN) {
        split_store<PC>(ep.out_h, ep.h_ps, o, *reinterpret_cast<const float(*)[8]>(oh));
        split_store<PC>(ep.out_h, ep.h_ps, o + 8, *reinterpret_cast<const float(*)[8]>(oh + 8));
      }
    }
    if (EPI == TC_LAST) {
      s_e[half][row_t] = e_acc;
    }
    if (EPI == TC_DT) {
      // second factor (a < 16): the two halves meet in the (now idle) stage
      // memory, row stride 65 floats (conflict-free); one partial per N tile
      float* sp = reinterpret_cast<float*>(base) + row_t * 65;
      if (half) {
#pragma unroll
        for (int c = 0; c < 4; ++c)
#pragma unroll
          for (int a = 0; a < 16; ++a) sp[c * 16 + a] = part[c][a];
      }
      __syncthreads();
      if (!half && rok) {
        float* pp = ep.part + (size_t)blockIdx.y * ep.part_ps + (size_t)row * 64;
#pragma unroll
        for (int c = 0; c < 4; ++c)
#pragma unroll
          for (int a = 0; a < 16; a += 4)
            *reinterpret_cast<float4*>(pp + c * 16 + a) =
                make_float4(part[c][a] + sp[c * 16 + a], part[c][a + 1] + sp[c * 16 + a + 1],
                            part[c][a + 2] + sp[c * 16 + a + 2], part[c][a + 3] + sp[c * 16 + a + 3]);
      }
    }
  }
  if (EPI == TC_LAST) {
    __syncthreads();
    if (done && tid < kBM && m0 + tid < M) {
      const int row = m0 + tid;
      ep.e_atom[ep.idx ? ep.idx[row] : row] = (double)(s_e[0][tid] + s_e[1][tid] + ep.bout);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem),
                 "r"(TmemCols<PC>::value));
}

template <int EPI, int PC>
int tc_gemm(cudaStream_t st, int M, int N, int K, const __nv_bfloat16* A, int lda, int64_t a_ps,
            const __nv_bfloat16* B, int ldb, int64_t b_ps, const TcEpi& ep) {
  if (M <= 0) return 0;
  if (K % 8 || lda % 8 || ldb % 8 || N % 16 || ep.ldo % 8) return -1;
  const int NT = N <= 256 ? N : 256;
  if (N > 256 && N % 256) return -1;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_tc_gemm<EPI, PC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)TcCfg<PC>::SMEM);
    attr = true;
  }
  dim3 grid((M + kBM - 1) / kBM, (N + NT - 1) / NT);
  DP_LAUNCHED(1);
  k_tc_gemm<EPI, PC><<<grid, kTcThreads, TcCfg<PC>::SMEM, st>>>(M, N, K, NT, A, lda, a_ps, B, ldb,
                                                               b_ps, ep);
  return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

// dE/dT[c][x] for x < 16 gets the second factor of Eq. 2's derivative,
// sum_b dE/dD[b][x] T[c][b], as the fixed-order sum of the per-N-tile partials
__global__ void k_dt_reduce(int64_t rows, const int32_t* __restrict__ idx, int M, int slots,
                            int64_t part_ps, const float* __restrict__ part, float* __restrict__ dT) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= rows * 64) return;
  const int64_t r = i >> 6;
  const int e = (int)(i & 63);  // c * 16 + x
  float acc = 0.0f;
  for (int sl = 0; sl < slots; ++sl) acc += part[(size_t)sl * part_ps + (size_t)r * 64 + e];
  const int64_t a = idx ? idx[r] : r;
  dT[(size_t)a * 4 * M + (e >> 4) * M + (e & 15)] += acc;
}

// FP32 -> PC BF16 pieces, piece p at out + p*n
__global__ void k_split_pieces(int64_t n, const float* __restrict__ in, __nv_bfloat16* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float x = in[i];
  const __nv_bfloat16 h = __float2bfloat16_rn(x);
  const float r1 = x - __bfloat162float(h);
  const __nv_bfloat16 m = __float2bfloat16_rn(r1);
  out[i] = h;
  out[n + i] = m;
  out[2 * n + i] = __float2bfloat16_rn(r1 - __bfloat162float(m));
}

}  // namespace

void launch_split_pieces(cudaStream_t st, int64_t n, const float* in, __nv_bfloat16* out) {
  if (n <= 0) return;
  DP_LAUNCHED(1);
  k_split_pieces<<<(int)((n + 255) / 256), 256, 0, st>>>(n, in, out);
}

template <int PC>
static int fit_tc_impl(cudaStream_t st, int64_t n, const int32_t* idx, const FitNetTC& net, int M,
                       int m_lt, const float* T, float* dT, double* e_atom, const FitScratchTC& s,
                       int32_t* err) {
  const int din = M * m_lt;
  const int nl = net.nl;
  if (nl < 2 || nl > DP_MAXFIT) return -1;
  for (int k = 0; k < nl; ++k)
    if (net.wout[k] > 256 || net.wout[k] % 16) return -1;
  if (din % 16 || m_lt != 16 || M < 16) return -1;  // the fused descriptor wants M< = 16
  const int64_t R = s.rows;  // piece strides of the activation scratch: R * width
  for (int64_t r0 = 0; r0 < n; r0 += R) {
    const int rows = (int)((n - r0) < R ? (n - r0) : R);
    const int32_t* id = idx ? idx + r0 : nullptr;
    const float* Tc = idx ? T : T + (size_t)r0 * 4 * M;
    float* dTc = idx ? dT : dT + (size_t)r0 * 4 * M;
    // forward: layer 0 (its A operand D formed from T in the producer), hidden
    // layers, last layer with the energy
    const __nv_bfloat16* in = nullptr;
    int win = din;
    for (int k = 0; k < nl; ++k) {
      TcEpi ep{};
      ep.bias = net.b[k];
      ep.ldo = net.wout[k];
      ep.err = err;
      // z of the layer below (z_0 = t_0: the first layer has no shortcut)
      const float* zb = k == 0 ? nullptr : (k == 1 ? s.t[0] : s.z[k - 1]);
      int rc;
      if (k == 0) {
        ep.out_a = s.t[0];
        ep.out_h = s.zh[0];
        ep.h_ps = R * net.wout[0];
        ep.T = Tc;
        ep.tidx = id;
        ep.Mw = M;
        rc = tc_gemm<TC_L0, PC>(st, rows, net.wout[0], din, in, din, 0, net.WTh[0], din,
                                net.w_ps[0], ep);
      } else if (k == nl - 1) {
        ep.R = net.shortcut[k] ? zb : nullptr;
        ep.ldr = net.wout[k - 1];
        ep.wout = net.w_out;
        ep.bout = net.b_out;
        ep.out_h = s.gph[0];
        ep.h_ps = R * s.wmax;
        ep.ldo = net.wout[k];
        ep.e_atom = e_atom + (idx ? 0 : r0);
        ep.idx = id;
        rc = tc_gemm<TC_LAST, PC>(st, rows, net.wout[k], win, in, win, R * win, net.WTh[k], win,
                                  net.w_ps[k], ep);
      } else {
        ep.R = net.shortcut[k] ? zb : nullptr;
        ep.ldr = net.wout[k - 1];
        ep.out_a = s.t[k];
        ep.out_b = s.z[k];
        ep.out_h = s.zh[k];
        ep.h_ps = R * net.wout[k];
        rc = tc_gemm<TC_MID, PC>(st, rows, net.wout[k], win, in, win, R * win, net.WTh[k], win,
                                 net.w_ps[k], ep);
      }
      if (rc) return rc;
      in = s.zh[k];
      win = net.wout[k];
    }
    // backward: gz_last = w_out (row stride 0); gp of the last layer from the
    // TC_LAST epilogue; gz updated in place, gp ping-pongs
    const float* gz_prev = net.w_out;
    int ldgz = 0;
    int gi = 0;
    for (int k = nl - 1; k >= 1; --k) {
      TcEpi ep{};
      ep.R = net.shortcut[k] ? gz_prev : nullptr;
      ep.ldr = ldgz;
      ep.Tt = s.t[k - 1];
      ep.ldt = net.win[k];
      ep.out_b = s.gz;
      ep.out_h = s.gph[gi ^ 1];
      ep.h_ps = R * s.wmax;
      ep.ldo = net.win[k];
      ep.err = err;
      const int rc = tc_gemm<TC_BWD, PC>(st, rows, net.win[k], net.wout[k], s.gph[gi],
                                         net.wout[k], R * s.wmax, net.Wh[k], net.wout[k],
                                         net.w_ps[k], ep);
      if (rc) return rc;
      gz_prev = s.gz;
      ldgz = net.win[k];
      gi ^= 1;
    }
    {
      // dE/dD = gp_0 W_0^T never leaves the chip: the epilogue contracts it
      // with T into dE/dT and leaves per-N-tile partials of the x < 16 term
      TcEpi ep{};
      ep.ldo = din;
      ep.err = err;
      ep.T = Tc;
      ep.dT = dTc;
      ep.tidx = id;
      ep.Mw = M;
      ep.part = s.part;
      ep.part_ps = R * 64;
      const int rc = tc_gemm<TC_DT, PC>(st, rows, din, net.wout[0], s.gph[gi], net.wout[0],
                                        R * s.wmax, net.Wh[0], net.wout[0], net.w_ps[0], ep);
      if (rc) return rc;
    }
    const int slots = din <= 256 ? 1 : din / 256;
    DP_LAUNCHED(1);
    k_dt_reduce<<<(int)((rows * 64 + 255) / 256), 256, 0, st>>>(rows, id, M, slots, R * 64, s.part,
                                                                dTc);
  }
  return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

int fit_tc(cudaStream_t st, int64_t n, const int32_t* idx, const FitNetTC& net, int M, int m_lt,
           const float* T, float* dT, double* e_atom, const FitScratchTC& s, int pieces,
           int32_t* err) {
  if (n <= 0) return 0;
  if (pieces == 1) return fit_tc_impl<1>(st, n, idx, net, M, m_lt, T, dT, e_atom, s, err);
  if (pieces == 3) return fit_tc_impl<3>(st, n, idx, net, M, m_lt, T, dT, e_atom, s, err);
  return -1;
}
