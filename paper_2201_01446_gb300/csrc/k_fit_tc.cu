// Fitting net (Sec. 2.1) and descriptor (Eq. 2) on the 5th-generation tensor
// cores: tcgen05.mma with 16-bit operands in shared memory and the FP32
// accumulator in tensor memory (TMEM), read back with tcgen05.ld for fused
// epilogues (bias, tanh, shortcut, per-atom energy, gradient of tanh, the
// descriptor's own backward).
//
// Operand pieces (PC): 1 = one BF16 piece; 3 = x = h + m + l in BF16, six
// piece products; 2 = an FP16 pair x s = h + l (22 significant bits), three
// piece products (h h, h l, l h), the operand first scaled by a power of two
// s that puts an upper bound of its magnitude at 2^14, below the FP16
// maximum (the weights: their largest |w|; activations and gradients: bounds
// that follow from the net, |tanh| <= 1 and |tanh'| <= 1; the descriptor: a
// Cauchy-Schwarz bound per row from T).  Elements of at least 2^-14 (scaled)
// keep 2^-22 relative accuracy; the epilogue multiplies the FP32 accumulator
// by the inverse scales, exactly.
//
// C = A B^T (A: rows x K, B: N x K) in 128-row tiles.  The operands live in
// global memory PRE-TILED in the tensor core's no-swizzle K-major
// shared-memory layout: for each 128-row (A) or 256-row (B) tile and each
// 16-wide K chunk, one contiguous block holding every BF16 piece of the
// operand, core matrices of 8 rows x 16 bytes, the two K groups 128 bytes
// apart, 8-row groups 256 bytes apart.  A pipeline stage is then a few bulk
// asynchronous copies (cp.async.bulk, completion counted in bytes on the
// stage's mbarrier) issued by one thread; each GEMM's epilogue writes its
// output straight into that layout for the next GEMM.
//
// Two kernels.  Layer 0 (K = 2048) runs on a tiled kernel, one output tile
// per CTA, whose warps 4-7 form the descriptor D from T in the stage's A
// slot.  The K-short GEMMs (hidden, last, backward, dE/dD) run on a
// persistent kernel, one CTA per SM with double-buffered TMEM accumulators.
// Warp roles: warp 0 (one lane) issues the copies up to NS stages ahead,
// warp 1 (one lane) issues the MMAs and commits each stage back to its
// "empty" barrier, the epilogue warps drain TMEM.  Every wait is bounded: on
// timeout the kernel records an error word, stops issuing work, waits
// (bounded) for its own copies and MMAs, frees its TMEM and returns.
#include <atomic>
#include <cuda_bf16.h>
#include <math.h>

#include "act.cuh"
#include "dp_internal.h"
#include "tc_common.cuh"

namespace {
using namespace dp_tc;

constexpr int kBM = 128;   // rows per tile (one TMEM lane per row)
constexpr int kBK = 16;    // K per stage: one K = 16 MMA step per piece product
constexpr int kTcThreads = 256;

// TMEM columns: one accumulator of NT <= 256 columns, or (split operands) the
// exact hi*hi products in columns 0..255 and the five small piece products
// in columns 256..511, so the dominant sum sees 6x fewer FP32 accumulations
template <int PC>
constexpr int kProds = PC == 1 ? 1 : PC == 2 ? 3 : 6;  // piece products per K chunk

template <int PC>
struct TcCfg {
  static constexpr int A_BYTES = kBM * kBK * 2;          // one piece of an A block
  static constexpr int B_MAX = 256 * kBK * 2;            // one piece of a B block (NT <= 256)
  static constexpr int STAGE = PC * (A_BYTES + B_MAX);
  static constexpr int NS = PC == 1 ? 12 : PC == 2 ? 8 : 6;  // pipeline stages
  static constexpr int NPROD = kProds<PC>;
  static constexpr int TMEM_COLS = PC == 1 ? 256 : 512;
  static constexpr size_t SMEM = 128 + (size_t)NS * STAGE;
};

template <int PC>
__device__ __forceinline__ uint32_t idesc_of(int M, int N) {
  return PC == 2 ? make_idesc_f16(M, N) : make_idesc_bf16(M, N);
}

// the pieces (of A, of B) that piece product q multiplies
template <int PC>
__device__ __forceinline__ void pieces_of(int q, int& pa, int& pb) {
  if (PC == 2) {  // (h,h) (h,l) (l,h)
    pa = q == 2 ? 1 : 0;
    pb = q == 1 ? 1 : 0;
  } else if (PC == 3) {
    prod_pieces(q, pa, pb);
  } else {
    pa = pb = 0;
  }
}

// the 16-bit pieces of W values: BF16 (PC 1, 3: x = h + m + l) of x, or the
// FP16 pair of x s (PC 2)
template <int PC, int W>
__device__ __forceinline__ void pieces_w(const float* x, float s, uint16_t (&pv)[3][W]) {
#pragma unroll
  for (int j = 0; j < W; ++j) {
    if constexpr (PC == 2) {
      const float v = x[j] * s;
      const __half h = __float2half_rn(v);
      pv[0][j] = __half_as_ushort(h);
      pv[1][j] = __half_as_ushort(__float2half_rn(v - __half2float(h)));
    } else {
      const __nv_bfloat16 h = __float2bfloat16_rn(x[j]);
      pv[0][j] = __bfloat16_as_ushort(h);
      if (PC == 3) {
        const float r1 = x[j] - __bfloat162float(h);
        const __nv_bfloat16 m = __float2bfloat16_rn(r1);
        pv[1][j] = __bfloat16_as_ushort(m);
        pv[2][j] = __bfloat16_as_ushort(__float2bfloat16_rn(r1 - __bfloat162float(m)));
      }
    }
  }
}
template <int PC>
__device__ __forceinline__ void pieces8(const float* x, float s, uint16_t (&pv)[3][8]) {
  pieces_w<PC, 8>(x, s, pv);
}

// the same pieces of 4 consecutive values with paired conversions, each
// piece as 4 packed 16-bit values (bitwise those of pieces_w)
template <int PC>
__device__ __forceinline__ void pieces4_packed(float4 x, float s, uint2 (&out)[3]) {
  uint32_t w[3][2];
  const float2 xv[2] = {make_float2(x.x, x.y), make_float2(x.z, x.w)};
#pragma unroll
  for (int h2 = 0; h2 < 2; ++h2) {
    if constexpr (PC == 2) {
      const float2 v = make_float2(xv[h2].x * s, xv[h2].y * s);
      const __half2 h = __floats2half2_rn(v.x, v.y);
      const float2 hf = __half22float2(h);
      const __half2 l = __floats2half2_rn(v.x - hf.x, v.y - hf.y);
      w[0][h2] = *reinterpret_cast<const uint32_t*>(&h);
      w[1][h2] = *reinterpret_cast<const uint32_t*>(&l);
    } else {
      const __nv_bfloat162 h = __floats2bfloat162_rn(xv[h2].x, xv[h2].y);
      w[0][h2] = *reinterpret_cast<const uint32_t*>(&h);
      if (PC == 3) {
        const float2 hf = __bfloat1622float2(h);
        const float2 r = make_float2(xv[h2].x - hf.x, xv[h2].y - hf.y);
        const __nv_bfloat162 m = __floats2bfloat162_rn(r.x, r.y);
        const float2 mf = __bfloat1622float2(m);
        const __nv_bfloat162 l = __floats2bfloat162_rn(r.x - mf.x, r.y - mf.y);
        w[1][h2] = *reinterpret_cast<const uint32_t*>(&m);
        w[2][h2] = *reinterpret_cast<const uint32_t*>(&l);
      }
    }
  }
#pragma unroll
  for (int p = 0; p < PC; ++p) out[p] = make_uint2(w[p][0], w[p][1]);
}

// FP32 activations and gradients of the fitting net between its GEMMs live in
// a row-tile-chunked layout: per 128-row tile and 16-column chunk one
// contiguous block of 128 x 16 floats, row-major inside.  A chunk is one bulk
// copy (the next GEMM's A operand, split into pieces in shared memory), and a
// row's 16 columns are 64 contiguous bytes (the epilogues' residual and tanh
// rows).  w: the array's width, a multiple of 16.
__host__ __device__ __forceinline__ size_t chunked(int row, int col, int w) {
  return ((size_t)(row >> 7) * (w >> 4) + (col >> 4)) * (kBM * kBK) + (size_t)(row & 127) * kBK +
         (col & 15);
}

// 2^e as a float, e clamped to the normal range
__device__ __forceinline__ float pow2f(int e) {
  e = max(-126, min(127, e));
  return __int_as_float((e + 127) << 23);
}

// pieces of 8 consecutive columns n..n+7 (n % 8 == 0) of row `row` into an
// activation stored pre-tiled for the next GEMM (width W = 16 * nkc); s is
// the FP16 pair's scale (PC 2)
template <int PC>
__device__ __forceinline__ void store_tiled(__nv_bfloat16* out, int nkc, int row, int n,
                                            const float* x, float s) {
  __align__(16) uint16_t pv[3][8];
  pieces8<PC>(x, s, pv);
  const size_t o =
      ((size_t)(row >> 7) * nkc + (n >> 4)) * PC * (kBM * kBK) + tile_off(row & 127, n);
#pragma unroll
  for (int p = 0; p < PC; ++p)
    *reinterpret_cast<uint4*>(out + o + p * (kBM * kBK)) = *reinterpret_cast<const uint4*>(pv[p]);
}

// TC_L0: layer 0, its A operand (the descriptor D of Eq. 2) formed from T in
// the stage; TC_DT: the input gradient dE/dD contracted with T into dE/dT in
// the epilogue (D and dE/dD never reach global memory)
enum { TC_L0 = 1, TC_MID = 2, TC_LAST = 3, TC_BWD = 4, TC_DT = 5 };

struct TcEpi {
  const float* bias;       // [N]
  const float* R;          // residual rows (ldr), ldr = 0: broadcast row
  int ldr;
  const float* Tt;         // t (derivatives in the table mode) of the layer below (TC_BWD)
  int ldt;
  const float* wout;       // output weights (TC_LAST)
  float bout;
  float* out_a;            // FP32 [rows][ldo]: t, or in the table mode the activation
                           // derivative (L0, MID)
  float* out_b;            // FP32 [rows][ldo]: z (MID) or gz (BWD; NULL: not kept)
  __nv_bfloat16* out_h;    // the next A operand, pre-tiled, width ldo
  int ldo;
  double* e_atom;          // TC_LAST: E_i written at idx[row] (or row)
  const int32_t* idx;
  int32_t* err;            // error word (timeouts)
  const float* T;          // TC_L0 / TC_DT: T rows [4][Mw] at tidx[row] (or row)
  float* dT;               // TC_DT: dE/dT rows, same indexing as T
  const int32_t* tidx;
  int Mw;                  // embedding width M
  const float4* tab;       // tanh table (L0, MID, LAST), NULL: tanhf
  float acc_scale;         // PC 2: the inverse scales of A and B (L0: of B; A per row)
  float out_scale;         // PC 2: the scale of the pieces written to out_h
  float a_scale;           // PC 2: the scale of an FP32 A operand's pieces (split in the kernel)
};

// The tiled kernel (one output tile per CTA) runs layer 0 (K = 2048), its A
// operand D formed in the stage from T by warps 4-7; the K-short layers run
// on the persistent kernel below.
template <int EPI, int PC, bool TAB>
__global__ void __launch_bounds__(kTcThreads, 1)
    k_tc_gemm(int M, int N, int K, int NT, const __nv_bfloat16* __restrict__ B, TcEpi ep) {
  static_assert(EPI == TC_L0, "the tiled kernel serves layer 0");
  using C = TcCfg<PC>;
  constexpr int NS = C::NS;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  unsigned char* base = (unsigned char*)(((uintptr_t)smem_raw + 127) & ~(uintptr_t)127);
  __shared__ __align__(8) uint64_t s_full[NS];   // stage filled (bytes landed)
  __shared__ __align__(8) uint64_t s_empty[NS];  // stage consumed (MMAs done)
  __shared__ __align__(8) uint64_t s_gen[NS];    // layer 0: D written into the stage
  __shared__ __align__(8) uint64_t s_acc;        // accumulator complete
  __shared__ uint32_t s_tmem;
  __shared__ int s_abort;
  __shared__ float s_rinv[kBM];                  // PC 2: inverse scale of each row of D
  volatile int* abort_flag = &s_abort;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // grid (N tiles, row tiles): the N tiles of one row tile are consecutive
  // blocks, so its A rows are read from HBM once and then hit in L2
  const int m_tile = blockIdx.y, n_tile = blockIdx.x;
  const int m0 = m_tile * kBM, n0 = n_tile * NT;
  const int ntile = min(NT, N - n0);  // NT, or the ragged last tile (a multiple of 16)
  const int nk = K / kBK;
  const uint32_t a_bytes = PC * C::A_BYTES;
  const uint32_t b_piece = (uint32_t)ntile * kBK * 2;

  if (tid == 0) {
    for (int s = 0; s < NS; ++s) {
      mbar_init(&s_full[s], 1);
      mbar_init(&s_empty[s], 1);
      mbar_init(&s_gen[s], kTcThreads / 2);
    }
    mbar_init(&s_acc, 1);
    s_abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (warp == 2) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                     smem_u32(&s_tmem)),
                 "r"(C::TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n");
  const uint32_t tmem = s_tmem;

  if (warp == 0) {
    if (lane == 0) {
      // producer: the B block of chunk kc lands in stage kc % NS (its A
      // block is written there by warps 4-7)
      int kc = 0;
      for (; kc < nk; ++kc) {
        const int s = kc % NS, u = kc / NS;
        if (u > 0 && !mbar_wait(&s_empty[s], (u - 1) & 1, abort_flag)) break;
        const uint32_t st0 = smem_u32(base + (size_t)s * C::STAGE);
        mbar_expect_tx(&s_full[s], PC * b_piece);
        bulk_g2s(st0 + a_bytes,
                 B + (size_t)n0 * K * PC + (size_t)kc * PC * ((size_t)ntile * kBK),
                 PC * b_piece, &s_full[s]);
      }
      if (kc < nk) {
        // aborted: wait (bounded) for the copies already issued to land
        for (int j = kc - NS > 0 ? kc - NS : 0; j < kc; ++j)
          mbar_wait(&s_full[j % NS], (j / NS) & 1, nullptr);
      }
    }
    __syncwarp();
  } else if (warp == 1) {
    if (lane == 0) {
      // MMA issuer: NPROD piece products per stage, the stage committed back
      const uint32_t idesc = idesc_of<PC>(kBM, ntile);
      for (int kc = 0; kc < nk; ++kc) {
        const int s = kc % NS, u = kc / NS;
        if (!mbar_wait(&s_full[s], u & 1, abort_flag)) break;
        if (!mbar_wait(&s_gen[s], u & 1, abort_flag)) break;
        asm volatile("tcgen05.fence::after_thread_sync;\n");
        const uint32_t st0 = smem_u32(base + (size_t)s * C::STAGE);
#pragma unroll
        for (int q = 0; q < C::NPROD; ++q) {
          int pa = 0, pb = 0;
          pieces_of<PC>(q, pa, pb);
          const uint64_t ad = make_desc(st0 + pa * C::A_BYTES, 128, 256);
          const uint64_t bd = make_desc(st0 + a_bytes + pb * b_piece, 128, 256);
          // accumulator 0: (h,h); accumulator 1 (PC > 1): the other products
          const uint32_t dst = tmem + (q > 0 ? 256u : 0u);
          const uint32_t acc = (kc > 0 || q > 1) ? 1u : 0u;
          asm volatile(
              "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
              " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dst),
              "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
        }
        asm volatile(
            "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                smem_u32(&s_empty[s])));
      }
      // every MMA issued (all, or up to an abort) completes before s_acc does
      asm volatile(
          "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
              smem_u32(&s_acc)));
    }
    __syncwarp();
  } else if (warp >= 4) {
    // layer 0: D[r][16 b + a] = sum_c T[c][b] T[c][a] (Eq. 2, M< = 16), one
    // thread per row; chunk kc is b = kc
    const int r = tid - kTcThreads / 2;
    const int gm = m0 + r;
    const float* trow = gm < M ? ep.T + (size_t)(ep.tidx ? ep.tidx[gm] : gm) * 4 * ep.Mw : nullptr;
    float ta[4][16];
#pragma unroll
    for (int c = 0; c < 4; ++c)
#pragma unroll
      for (int a = 0; a < 16; a += 4) {
        const float4 v = trow ? __ldg(reinterpret_cast<const float4*>(trow + c * ep.Mw + a))
                              : make_float4(0.f, 0.f, 0.f, 0.f);
        ta[c][a] = v.x;
        ta[c][a + 1] = v.y;
        ta[c][a + 2] = v.z;
        ta[c][a + 3] = v.w;
      }
    float rs = 1.0f;  // PC 2: the scale of this row of D
    if (PC == 2) {
      // |D[b][a]| <= |T_b| |T_a| (Cauchy-Schwarz over the 4 components c):
      // max_b |T_b|^2 over all M columns, each warp over its 32 rows with
      // coalesced loads (four rows in flight), times max_{a<16} |T_a|^2
      const int w4 = warp - 4;
      float nb = 0.0f;
      for (int i0 = 0; i0 < 32; i0 += 4) {
        float mx[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int gi = m0 + w4 * 32 + i0 + u;
          mx[u] = 0.0f;
          if (gi < M) {
            const float* tri = ep.T + (size_t)(ep.tidx ? ep.tidx[gi] : gi) * 4 * ep.Mw;
            for (int b = 4 * lane; b < ep.Mw; b += 128) {
              float4 q4[4];
#pragma unroll
              for (int c = 0; c < 4; ++c)
                q4[c] = __ldg(reinterpret_cast<const float4*>(tri + c * ep.Mw + b));
              float n0 = 0.0f, n1 = 0.0f, n2 = 0.0f, n3 = 0.0f;
#pragma unroll
              for (int c = 0; c < 4; ++c) {
                n0 = fmaf(q4[c].x, q4[c].x, n0);
                n1 = fmaf(q4[c].y, q4[c].y, n1);
                n2 = fmaf(q4[c].z, q4[c].z, n2);
                n3 = fmaf(q4[c].w, q4[c].w, n3);
              }
              mx[u] = fmaxf(mx[u], fmaxf(fmaxf(n0, n1), fmaxf(n2, n3)));
            }
          }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
#pragma unroll
          for (int o = 16; o; o >>= 1) mx[u] = fmaxf(mx[u], __shfl_xor_sync(0xffffffffu, mx[u], o));
          if (lane == i0 + u) nb = mx[u];
        }
      }
      float na = 0.0f;
#pragma unroll
      for (int a = 0; a < 16; ++a) {
        float q = 0.0f;
#pragma unroll
        for (int c = 0; c < 4; ++c) q = fmaf(ta[c][a], ta[c][a], q);
        na = fmaxf(na, q);
      }
      // bound^2 = nb na < 2^(E+1): bound < 2^e with e = ceil((E+1)/2), scale 2^(14-e)
      const float b2 = nb * na;
      int e = 0;
      if (b2 > 0.0f) {
        const int E = ((__float_as_int(b2) >> 23) & 255) - 127;
        e = (E + 2) >> 1;
      }
      rs = b2 > 0.0f ? pow2f(14 - e) : 1.0f;
      s_rinv[r] = b2 > 0.0f ? pow2f(e - 14) : 1.0f;
    }
    float4 tb4[4];
    for (int kc = 0; kc < nk; ++kc) {
      const int s = kc % NS, u = kc / NS;
      if (u > 0 && !mbar_wait(&s_empty[s], (u - 1) & 1, abort_flag)) break;
      if ((kc & 3) == 0) {
#pragma unroll
        for (int c = 0; c < 4; ++c)
          tb4[c] = trow ? __ldg(reinterpret_cast<const float4*>(trow + c * ep.Mw + kc))
                        : make_float4(0.f, 0.f, 0.f, 0.f);
      }
      const int q = kc & 3;
      float x[16];
#pragma unroll
      for (int a = 0; a < 16; ++a) {
        float acc = 0.0f;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const float tb = q == 0 ? tb4[c].x : q == 1 ? tb4[c].y : q == 2 ? tb4[c].z : tb4[c].w;
          acc = fmaf(tb, ta[c][a], acc);
        }
        x[a] = acc;
      }
      unsigned char* sa = base + (size_t)s * C::STAGE;
#pragma unroll
      for (int kg = 0; kg < 2; ++kg) {
        __align__(16) uint16_t pv[3][8];
        pieces8<PC>(x + kg * 8, rs, pv);
        const int off = (r >> 3) * 256 + kg * 128 + (r & 7) * 16;
#pragma unroll
        for (int p = 0; p < PC; ++p)
          *reinterpret_cast<uint4*>(sa + p * C::A_BYTES + off) = *reinterpret_cast<const uint4*>(pv[p]);
      }
      asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
      mbar_arrive(&s_gen[s]);
    }
  }

  // the accumulator: the MMA thread commits it in every case
  bool done = mbar_wait(&s_acc, 0, nullptr);
  if (!done) *abort_flag = 1;
  asm volatile("tcgen05.fence::after_thread_sync;\n");
  __syncthreads();
  done = *abort_flag == 0;  // uniform over the CTA (the epilogue synchronises)

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
    const int nkc_out = ep.ldo / kBK;
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
      if (PC == 2) {
        const float sc = ep.acc_scale * s_rinv[row_t];
#pragma unroll
        for (int k = 0; k < 16; ++k) v[k] *= sc;
      }
      if (!rok) continue;
      const int n = n0 + c0;
      const size_t o = chunked(row, n, ep.ldo);
      float b[16], oa[16], oh[16];
#pragma unroll
      for (int k = 0; k < 16; k += 4)
        *reinterpret_cast<float4*>(b + k) = *reinterpret_cast<const float4*>(ep.bias + n + k);
#pragma unroll
      for (int k = 0; k < 16; ++k) {
        float d;
        const float t = act_tanh_t<TAB>(v[k] + b[k], ep.tab, d);
        oa[k] = TAB ? d : t;
        oh[k] = t;  // z_0 = t_0 (layer 0 has no shortcut)
      }
#pragma unroll
      for (int k = 0; k < 16; k += 4)
        *reinterpret_cast<float4*>(ep.out_a + o + k) = *reinterpret_cast<const float4*>(oa + k);
      if (TAB) {  // the table mode keeps derivatives in out_a: z_0 separately
#pragma unroll
        for (int k = 0; k < 16; k += 4)
          *reinterpret_cast<float4*>(ep.out_b + o + k) = *reinterpret_cast<const float4*>(oh + k);
      }
      if (ep.out_h) {
        store_tiled<PC>(ep.out_h, nkc_out, row, n, oh, ep.out_scale);
        store_tiled<PC>(ep.out_h, nkc_out, row, n + 8, oh + 8, ep.out_scale);
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n");
  __syncthreads();
  if (warp == 2)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem),
                 "r"(C::TMEM_COLS));
}

// ---------------------------------------------------------------- persistent
// K-short GEMMs (K <= 256: hidden, last, backward and dE/dD layers): one CTA
// per SM walks row tiles and, per row tile, its N tiles of 128 columns (256
// for the dE/dD GEMM); each stage holds one K chunk of A and of B (all
// pieces), up to 8 stages deep.
// (Keeping the row tile's A resident instead, loaded once for all N tiles,
// measured slower even for the 16 N tiles of the dE/dD GEMM: its 180 KB
// leave room for three B stages only, and the MMAs then wait on B.)
// The accumulators are double-buffered in TMEM (2 x 256 columns), so warps 4-7
// drain N tile t (the fused epilogue, one thread per row) while warp 1 issues
// the MMAs of tile t+1 and warp 0 the copies of t+2.  Per-row state across the
// N tiles of a row tile (the energy sum, the dE/dT second factor) stays in the
// epilogue thread's registers.
constexpr int kPNT = 128;    // columns per N tile (the dE/dD GEMM: 256, see below)
constexpr int kPMaxNS = 8;   // stages at most
constexpr int kPMaxK = 16;   // K chunks a row tile can hold (K <= 256)
constexpr size_t kPSmemMax = 225 * 1024;

template <int PC, int NTW, bool AF>
struct PCfg {
  static constexpr int A_CHUNK = PC * kBM * kBK * 2;   // one K chunk of A, all pieces
  static constexpr int B_PIECE = NTW * kBK * 2;        // one piece of B
  static constexpr int A_F32 = AF ? kBM * kBK * 4 : 0;  // the FP32 A chunk as copied
  static constexpr int STAGE = A_CHUNK + PC * B_PIECE + A_F32;  // [A pieces][B pieces][FP32 A]
  static int stages() {
    const long ns = ((long)kPSmemMax - 128) / STAGE;
    return (int)(ns < kPMaxNS ? ns : kPMaxNS);
  }
  static size_t smem() { return 128 + (size_t)stages() * STAGE; }
};

// EW epilogue warps: 4 (one thread per row, all columns: the dE/dD GEMM,
// whose per-row state spans all columns) or 8 (two column halves; the last
// layer hands the second half's energy sums to the first).
// The hidden layers read their A operand (the FP32 output z of the layer
// below, chunked layout) as it is, and four converter warps (2, 3 and two
// after the epilogue warps) split it into the pieces in each stage: the layer
// below then writes no pieces (layer 0 saves 3% of its time).  The last and
// the backward layers take pre-split pieces: splitting there measured slower
// (the backward layer 145 -> 171 us per 100k rows).
template <int EPI>
constexpr int kConvWarps = EPI == TC_MID ? 2 : 0;  // converter warps beyond warps 2-3
// PO: the pieces of the next A operand the epilogue writes (out_h)
template <int EPI, int PC, bool TAB, int EW, int PO>
__global__ void __launch_bounds__(128 + EW * 32 + kConvWarps<EPI> * 32, 1)
    k_tc_gemm_p(int M, int N, int K, int NS, const void* __restrict__ Av,
                const __nv_bfloat16* __restrict__ B, TcEpi ep) {
  // The dE/dD GEMM (N = 2048) streams its A chunk once per N tile: N tiles of
  // 256 columns halve those bytes (36 KB per stage for 6.3 MFLOP instead of
  // 24 KB for 3.1), and all six piece products then share one accumulator
  // (2 x 256 TMEM columns, still double-buffered; measured 62.5 -> 60.5 ms of
  // fitting per 4M-atom step, force errors within the FP32 bars).  The other
  // layers keep the h*h products in their own accumulator.
  constexpr int NTW = EPI == TC_DT ? 256 : kPNT;
  constexpr bool ONE_ACC = NTW == 256;
  constexpr bool AF = EPI == TC_MID;  // A as FP32 rows, split here
  using C = PCfg<PC, NTW, AF>;
  const __nv_bfloat16* A = static_cast<const __nv_bfloat16*>(Av);
  const float* A32 = static_cast<const float*>(Av);
  extern __shared__ __align__(128) unsigned char smem_raw[];
  unsigned char* base = (unsigned char*)(((uintptr_t)smem_raw + 127) & ~(uintptr_t)127);
  const int nk = K / kBK;
  unsigned char* st_smem = base;  // stage s: [A pieces][B pieces][FP32 A]
  const uint32_t st_b = (uint32_t)C::A_CHUNK;
  const uint32_t st_f = (uint32_t)(C::A_CHUNK + PC * C::B_PIECE);
  __shared__ __align__(8) uint64_t b_full[kPMaxNS], b_empty[kPMaxNS], b_conv[kPMaxNS];
  __shared__ __align__(8) uint64_t t_full[2], t_empty[2], fin;
  // TC_LAST: the second column half's energy sums, handed to the first half
  __shared__ __align__(8) uint64_t e_full[2], e_empty[2];
  __shared__ float s_epart[2][kBM];
  __shared__ uint32_t s_tmem;
  __shared__ int s_abort;
  volatile int* abort_flag = &s_abort;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int mtiles = (M + kBM - 1) / kBM;
  const int ntn = (N + NTW - 1) / NTW;
  // B is pre-tiled in tiles of 256 rows (the last ragged)
  auto b_src = [&](int n, int kc, int p) {
    const int n0 = n * NTW, t256 = n0 / 256, r0 = n0 - t256 * 256;
    const int nt256 = min(256, N - t256 * 256);
    return B + (size_t)t256 * 256 * K * PC + ((size_t)kc * PC + p) * nt256 * kBK +
           (size_t)(r0 / 8) * 128;
  };

  if (tid == 0) {
    for (int s = 0; s < kPMaxNS; ++s) {
      mbar_init(&b_full[s], 1);
      mbar_init(&b_empty[s], 1);
      mbar_init(&b_conv[s], 128);
    }
    for (int j = 0; j < 2; ++j) {
      mbar_init(&t_full[j], 1);
      mbar_init(&t_empty[j], EW * 32);
      mbar_init(&e_full[j], kBM);
      mbar_init(&e_empty[j], kBM);
    }
    mbar_init(&fin, 1);
    s_abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (warp == 2) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                     smem_u32(&s_tmem)),
                 "r"(512));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n");
  const uint32_t tmem = s_tmem;

  if (warp == 0) {
    if (lane == 0) {
      // producer: for every (row tile, N tile, K chunk) the A chunk and the B chunk
      uint32_t bi = 0;
      bool ok = true;
      for (int mt = blockIdx.x; mt < mtiles && ok; mt += gridDim.x) {
        for (int n = 0; n < ntn && ok; ++n) {
          const int nt = min(NTW, N - n * NTW);
          for (int kc = 0; kc < nk; ++kc, ++bi) {
            const int s = bi % NS;
            const uint32_t u = bi / NS;
            if (u > 0 && !mbar_wait(&b_empty[s], (u - 1) & 1, abort_flag)) {
              ok = false;
              break;
            }
            const uint32_t st0 = smem_u32(st_smem + (size_t)s * C::STAGE);
            if (AF) {
              mbar_expect_tx(&b_full[s], (uint32_t)C::A_F32 + PC * nt * 32);
              bulk_g2s(st0 + st_f, A32 + ((size_t)mt * nk + kc) * (kBM * kBK), C::A_F32, &b_full[s]);
            } else {
              mbar_expect_tx(&b_full[s], (uint32_t)C::A_CHUNK + PC * nt * 32);
              bulk_g2s(st0, A + ((size_t)mt * nk + kc) * PC * (kBM * kBK), C::A_CHUNK, &b_full[s]);
            }
#pragma unroll
            for (int p = 0; p < PC; ++p)
              bulk_g2s(st0 + st_b + p * C::B_PIECE, b_src(n, kc, p), nt * 32, &b_full[s]);
          }
        }
      }
      if (*abort_flag) {
        // aborted: wait (bounded) for the copies already issued to land
        for (uint32_t j = bi > (uint32_t)NS ? bi - NS : 0; j < bi; ++j)
          mbar_wait(&b_full[j % NS], (j / NS) & 1, nullptr);
      }
    }
    __syncwarp();
  } else if (warp == 1) {
    if (lane == 0) {
      uint32_t bi = 0, ti = 0;
      bool ok = true;
      for (int mt = blockIdx.x; mt < mtiles && ok; mt += gridDim.x) {
        for (int n = 0; n < ntn && ok; ++n, ++ti) {
          const int nt = min(NTW, N - n * NTW);
          const uint32_t idesc = idesc_of<PC>(kBM, nt);
          const int j = ti & 1;
          if (ti >= 2 && !mbar_wait(&t_empty[j], ((ti >> 1) - 1) & 1, abort_flag)) {
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;\n");
          for (int kc = 0; kc < nk; ++kc, ++bi) {
            const int s = bi % NS;
            // AF: the pieces split from the FP32 chunk (which implies it landed)
            if (!mbar_wait(AF ? &b_conv[s] : &b_full[s], (bi / NS) & 1, abort_flag)) {
              ok = false;
              break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;\n");
            const uint32_t a0 = smem_u32(st_smem + (size_t)s * C::STAGE);
            const uint32_t b0 = a0 + st_b;
#pragma unroll
            for (int q = 0; q < kProds<PC>; ++q) {
              int pa = 0, pb = 0;
              pieces_of<PC>(q, pa, pb);
              const uint64_t ad = make_desc(a0 + pa * (kBM * kBK * 2), 128, 256);
              const uint64_t bd = make_desc(b0 + pb * C::B_PIECE, 128, 256);
              const uint32_t dst = tmem + (uint32_t)(j * 256) + (!ONE_ACC && q > 0 ? 128u : 0u);
              const uint32_t acc = (kc > 0 || q > (ONE_ACC ? 0 : 1)) ? 1u : 0u;
              asm volatile(
                  "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                  " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dst),
                  "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
            }
            asm volatile(
                "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                    smem_u32(&b_empty[s])));
          }
          asm volatile(
              "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                  smem_u32(&t_full[j])));
        }
      }
      // the epilogue may be waiting for a buffer this thread will not fill
      if (!ok) *abort_flag = 1;
      // every MMA issued completes before fin does (TMEM is freed after it)
      asm volatile(
          "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
              smem_u32(&fin)));
    }
    __syncwarp();
  } else if (AF && (warp == 2 || warp == 3 || warp >= 4 + EW)) {
    // converters: each landed FP32 A chunk (128 rows x 16) into its pieces in
    // the tensor core's layout; thread ct takes float4 q = 128 i + ct (row
    // q / 4, columns 4 (q % 4) ..), so a warp reads 512 contiguous bytes and
    // writes eight whole 8-row core-matrix rows
    const int ct = (warp < 4 ? warp - 2 : warp - EW - 2) * 32 + lane;
    uint32_t bi = 0;
    bool ok = true;
    for (int mt = blockIdx.x; mt < mtiles && ok; mt += gridDim.x) {
      for (int n = 0; n < ntn && ok; ++n) {
        for (int kc = 0; kc < nk; ++kc, ++bi) {
          const int s = bi % NS;
          if (!mbar_wait(&b_full[s], (bi / NS) & 1, abort_flag)) {
            ok = false;
            break;
          }
          unsigned char* st = st_smem + (size_t)s * C::STAGE;
          const float4* src = reinterpret_cast<const float4*>(st + st_f);
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            const int q = i * 128 + ct;
            const int rr = q >> 2, k0 = (q & 3) * 4;
            uint2 pw[3];
            pieces4_packed<PC>(src[q], ep.a_scale, pw);
            const int off = tile_off(rr, k0);
#pragma unroll
            for (int p = 0; p < PC; ++p)
              *reinterpret_cast<uint2*>(st + (size_t)p * (kBM * kBK * 2) + (size_t)off * 2) = pw[p];
          }
          asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
          mbar_arrive(&b_conv[s]);
        }
      }
    }
  } else if (warp >= 4 && warp < 4 + EW) {
    // epilogue: thread = row of the tile (TMEM lane; a warp reaches the lane
    // quarter warp % 4), all columns of each N tile or one half of them
    static_assert(EW == 4 || (EW == 8 && EPI != TC_DT), "epilogue warps");
    constexpr int CPW = (NTW / 16) / (EW / 4);  // 16-column chunks per thread and N tile
    const int r = (tid - 128) & (kBM - 1);
    const int hf = EW == 8 ? (warp - 4) >> 2 : 0;
    const uint32_t tl_base = tmem + ((uint32_t)((warp & 3) * 32) << 16);
    uint32_t ti = 0, it = 0;
    for (int mt = blockIdx.x; mt < mtiles; mt += gridDim.x, ++it) {
      const int row = mt * kBM + r;
      const bool rok = row < M;
      float e_acc = 0.0f;
      float tl[4][16], part[4][16];
      const float* tr = nullptr;
      float* dtr = nullptr;
      if (EPI == TC_DT) {
        if (rok) {
          const size_t trow = (size_t)(ep.tidx ? ep.tidx[row] : row) * 4 * ep.Mw;
          tr = ep.T + trow;
          dtr = ep.dT + trow;
        }
        // the next row tile's T rows (contiguous without an index list) into
        // L2 while this one is drained: the epilogue's T loads then hit L2
        const int mn = mt + gridDim.x;
        if (tid == 128 && !ep.tidx && mn < mtiles) {
          const int rows_n = min(kBM, M - mn * kBM);
          asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;\n" ::"l"(
                           ep.T + (size_t)mn * kBM * 4 * ep.Mw),
                       "r"((uint32_t)(rows_n * 4 * ep.Mw * 4))
                       : "memory");
        }
#pragma unroll
        for (int c = 0; c < 4; ++c)
#pragma unroll
          for (int a = 0; a < 16; a += 4) {
            const float4 q = tr ? __ldg(reinterpret_cast<const float4*>(tr + c * ep.Mw + a))
                                : make_float4(0.f, 0.f, 0.f, 0.f);
            tl[c][a] = q.x;
            tl[c][a + 1] = q.y;
            tl[c][a + 2] = q.z;
            tl[c][a + 3] = q.w;
#pragma unroll
            for (int k = 0; k < 4; ++k) part[c][a + k] = 0.0f;
          }
      }
      bool fail = false;
      for (int n = 0; n < ntn; ++n, ++ti) {
        const int j = ti & 1;
        const int nt = min(NTW, N - n * NTW), nch = nt / 16;
        // TC_DT: T[c][b] of the row for the chunks b - NTW/16 n of this N
        // tile, four chunks per float4 (b a multiple of 4 and M % 4 == 0: in
        // the row), one group of four ahead in a ring of two (the first two
        // issued before the accumulator wait)
        float4 tq4[2][4];
        auto load_tg = [&](int slot, int g) {
          const int chn = hf * CPW + 4 * g;
#pragma unroll
          for (int c = 0; c < 4; ++c)
            tq4[slot][c] = chn < nch ? __ldg(reinterpret_cast<const float4*>(
                                           tr + c * ep.Mw + n * (NTW / 16) + chn))
                                     : make_float4(0.f, 0.f, 0.f, 0.f);
        };
        if (EPI == TC_DT && rok) {
          load_tg(0, 0);
          load_tg(1, 1);
        }
        if (!mbar_wait(&t_full[j], (ti >> 1) & 1, abort_flag)) {
          fail = true;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;\n");
        float f1[4][8];  // the first factor of dE/dT for 8 chunks (b) at a time
        // dE/dT[c][b] for the chunk group g of this N tile (b = NTW/16 n + 8 g ..)
        auto flush_f1 = [&](int g, int cnt) {
          const int b0 = n * (NTW / 16) + 8 * g;
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            float* d = dtr + c * ep.Mw + b0;
            if (cnt == 8 && ((b0 | ep.Mw) & 3) == 0) {
              *reinterpret_cast<float4*>(d) = make_float4(f1[c][0], f1[c][1], f1[c][2], f1[c][3]);
              *reinterpret_cast<float4*>(d + 4) = make_float4(f1[c][4], f1[c][5], f1[c][6], f1[c][7]);
            } else {
#pragma unroll
              for (int q = 0; q < 8; ++q)
                if (q < cnt) d[q] = f1[c][q];
            }
          }
        };
#pragma unroll
        for (int cc = 0; cc < CPW; ++cc) {
          const int ch = hf * CPW + cc;
          if (ch < nch) {
            float v[16], v2[16];
            tmem_ld16(tl_base + (uint32_t)(j * 256 + ch * 16), v);
            if (PC > 1 && !ONE_ACC) {
              tmem_ld16(tl_base + (uint32_t)(j * 256 + 128 + ch * 16), v2);
#pragma unroll
              for (int k = 0; k < 16; ++k) v[k] += v2[k];
            }
            if (PC == 2) {
#pragma unroll
              for (int k = 0; k < 16; ++k) v[k] *= ep.acc_scale;
            }
            const int ncol = n * NTW + ch * 16;
            if (rok) {
              if (EPI == TC_DT) {
                // v = dE/dD[b][0..15], b = ncol / 16 (Eq. 2)
                if ((cc & 3) == 0 && cc >= 4 && cc + 4 < CPW) load_tg(((cc >> 2) + 1) & 1, (cc >> 2) + 1);
                float tb[4];
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                  const float4 q = tq4[(cc >> 2) & 1][c];
                  const int u = cc & 3;
                  tb[c] = u == 0 ? q.x : u == 1 ? q.y : u == 2 ? q.z : q.w;  // T[c][b], b = ncol / 16
                  float acc = 0.0f;
#pragma unroll
                  for (int a = 0; a < 16; ++a) acc = fmaf(v[a], tl[c][a], acc);
                  f1[c][ch & 7] = acc;
                }
#pragma unroll
                for (int c = 0; c < 4; ++c)
#pragma unroll
                  for (int a = 0; a < 16; ++a) part[c][a] = fmaf(v[a], tb[c], part[c][a]);
                // a full group of 8 with more chunks to follow: write it now
                if ((cc & 7) == 7 && ch < nch - 1) flush_f1(cc >> 3, 8);
              } else {
                const size_t o = chunked(row, ncol, ep.ldo);
                float rr[16], bb[16], tt[16], oh[16];
                if (EPI == TC_MID || EPI == TC_LAST) {
#pragma unroll
                  for (int k = 0; k < 16; k += 4)
                    *reinterpret_cast<float4*>(bb + k) = *reinterpret_cast<const float4*>(ep.bias + ncol + k);
                }
                if (ep.R) {
#pragma unroll
                  for (int k = 0; k < 16; k += 4)
                    *reinterpret_cast<float4*>(rr + k) =
                        *reinterpret_cast<const float4*>(
                            ep.ldr ? ep.R + chunked(row, ncol, ep.ldr) + k : ep.R + ncol + k);
                } else {
#pragma unroll
                  for (int k = 0; k < 16; ++k) rr[k] = 0.0f;
                }
                if (EPI == TC_BWD) {
#pragma unroll
                  for (int k = 0; k < 16; k += 4)
                    *reinterpret_cast<float4*>(tt + k) =
                        *reinterpret_cast<const float4*>(ep.Tt + chunked(row, ncol, ep.ldt) + k);
                }
                float oa[16], ob[16];
#pragma unroll
                for (int k = 0; k < 16; ++k) {
                  if (EPI == TC_MID) {
                    float d;
                    const float t = act_tanh_t<TAB>(v[k] + bb[k], ep.tab, d);
                    oa[k] = TAB ? d : t;
                    ob[k] = rr[k] + t;
                    oh[k] = ob[k];
                  } else if (EPI == TC_LAST) {
                    float d;
                    const float t = act_tanh_t<TAB>(v[k] + bb[k], ep.tab, d);
                    const float w = ep.wout[ncol + k];
                    e_acc = fmaf(rr[k] + t, w, e_acc);
                    oh[k] = w * d;
                  } else {  // TC_BWD
                    const float gz = v[k] + rr[k];
                    ob[k] = gz;
                    oh[k] = gz * (TAB ? tt[k] : 1.0f - tt[k] * tt[k]);
                  }
                }
                if (EPI == TC_MID) {
#pragma unroll
                  for (int k = 0; k < 16; k += 4)
                    *reinterpret_cast<float4*>(ep.out_a + o + k) = *reinterpret_cast<const float4*>(oa + k);
                }
                if (EPI == TC_MID || (EPI == TC_BWD && ep.out_b)) {
#pragma unroll
                  for (int k = 0; k < 16; k += 4)
                    *reinterpret_cast<float4*>(ep.out_b + o + k) = *reinterpret_cast<const float4*>(ob + k);
                }
                const int nkc_out = ep.ldo / kBK;
                if (ep.out_h) {  // MID: only for the last layer's A
                  store_tiled<PO>(ep.out_h, nkc_out, row, ncol, oh, ep.out_scale);
                  store_tiled<PO>(ep.out_h, nkc_out, row, ncol + 8, oh + 8, ep.out_scale);
                }
              }
            }
          }
        }
        // TMEM buffer j is drained: the MMAs of tile t+2 may overwrite it
        asm volatile("tcgen05.fence::before_thread_sync;\n");
        mbar_arrive(&t_empty[j]);
        if (EPI == TC_DT && rok) {
          // the last (possibly partial) group of first factors of this N tile
          const int g = (nch - 1) >> 3;
          flush_f1(g, nch - 8 * g);
        }
      }
      if (fail) break;
      if (EPI == TC_LAST && EW == 8) {
        // E_i = (first half's sum + second half's) + b_out; the halves meet
        // in a double-buffered shared array (bounded waits)
        const int b = it & 1;
        const uint32_t ph = (it >> 1) & 1;
        if (hf == 1) {
          if (it >= 2 && !mbar_wait(&e_empty[b], ph ^ 1, abort_flag)) break;
          s_epart[b][r] = e_acc;
          mbar_arrive(&e_full[b]);
        } else {
          if (!mbar_wait(&e_full[b], ph, abort_flag)) break;
          const float e1 = s_epart[b][r];
          mbar_arrive(&e_empty[b]);
          if (rok) ep.e_atom[ep.idx ? ep.idx[row] : row] = (double)(e_acc + e1 + ep.bout);
        }
      } else if (EPI == TC_LAST && rok) {
        ep.e_atom[ep.idx ? ep.idx[row] : row] = (double)(e_acc + ep.bout);
      }
      if (EPI == TC_DT && rok) {
        // second factor (x < 16): complete over all N tiles of the row tile;
        // the first factor of b = x was written by this thread above
#pragma unroll
        for (int c = 0; c < 4; ++c)
#pragma unroll
          for (int a = 0; a < 16; ++a) dtr[c * ep.Mw + a] += part[c][a];
      }
    }
  }
  if (tid == 0 && !mbar_wait(&fin, 0, nullptr)) *abort_flag = 1;
  asm volatile("tcgen05.fence::before_thread_sync;\n");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n");
  if (tid == 0 && *abort_flag && ep.err) atomicAdd(ep.err, 1);
  if (warp == 2)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(512));
}

std::atomic<int> g_tc_sms{0};

// persistent launch of the K-short GEMMs (PO: pieces of the A operand written)
template <int EPI, int PC, bool TAB, int PO = PC>
int tc_gemm_p(cudaStream_t st, int M, int N, int K, const void* A, const __nv_bfloat16* B,
              const TcEpi& ep) {
  constexpr int EW = EPI == TC_DT ? 4 : 8;
  if (M <= 0) return 0;
  if (K <= 0 || K % kBK || K / kBK > kPMaxK || N <= 0 || N % 16) return -1;
  if (EPI != TC_DT && ep.ldo != N) return -1;
  using CF = PCfg<PC, EPI == TC_DT ? 256 : kPNT, EPI == TC_MID>;  // the kernel's stage
  static_assert(CF::STAGE * 3 + 128 <= kPSmemMax, "three stages at least");
  const int NS = CF::stages();
  const size_t sm = CF::smem();
  static std::atomic<size_t> set{0};  // launches from several host threads
  if (sm > set) {
    if (cudaFuncSetAttribute(k_tc_gemm_p<EPI, PC, TAB, EW, PO>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sm) != cudaSuccess)
      return -3;
    set = sm;
  }
  if (!g_tc_sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    int v = 0;
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    g_tc_sms = v > 0 ? v : 1;
  }
  const int mtiles = (M + kBM - 1) / kBM, nsm = g_tc_sms;
  DP_LAUNCHED(1);
  k_tc_gemm_p<EPI, PC, TAB, EW, PO><<<mtiles < nsm ? mtiles : nsm,
                                      128 + EW * 32 + kConvWarps<EPI> * 32, sm, st>>>(M, N, K, NS, A,
                                                                                     B, ep);
  return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

// the caller's layouts: A pre-tiled in 128-row tiles, B in tiles of 256 rows
// (the last one ragged), N % 16 == 0, K % 16 == 0
// layer 0 on the tiled kernel (A formed from T in the stage)
template <int EPI, int PC, bool TAB>
int tc_gemm(cudaStream_t st, int M, int N, int K, const __nv_bfloat16* B, const TcEpi& ep) {
  if (M <= 0) return 0;
  if (K <= 0 || K % kBK || N <= 0 || N % 16) return -1;
  if (ep.ldo != N) return -1;
  const int NT = N <= 256 ? N : 256;
  static std::atomic<bool> attr{false};  // launches from several host threads
  if (!attr) {
    if (cudaFuncSetAttribute(k_tc_gemm<EPI, PC, TAB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)TcCfg<PC>::SMEM) != cudaSuccess)
      return -3;
    attr = true;
  }
  dim3 grid((N + NT - 1) / NT, (M + kBM - 1) / kBM);
  DP_LAUNCHED(1);
  k_tc_gemm<EPI, PC, TAB><<<grid, kTcThreads, TcCfg<PC>::SMEM, st>>>(M, N, K, NT, B, ep);
  return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

// FP32 B [N][K] -> PC pieces in the pre-tiled B layout: tile nt (rows
// 256 nt .., ntile of them) at 256 nt K PC, its K chunk kc at kc PC ntile 16;
// PC 2: the FP16 pair of x scale
__global__ void k_tile_operand(int N, int K, int PC, float scale, const float* __restrict__ src,
                               __nv_bfloat16* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)N * K) return;
  const int n = (int)(i / K), k = (int)(i - (int64_t)n * K);
  const int nt = n / 256, r = n - nt * 256, ntile = min(256, N - nt * 256);
  const size_t ps = (size_t)ntile * kBK;
  const size_t o = (size_t)nt * 256 * K * PC + (size_t)(k / kBK) * PC * ps + tile_off(r, k);
  const float x = src[i];
  if (PC == 2) {
    uint16_t* o16 = reinterpret_cast<uint16_t*>(out);
    const float v = x * scale;
    const __half hh = __float2half_rn(v);
    o16[o] = __half_as_ushort(hh);
    o16[o + ps] = __half_as_ushort(__float2half_rn(v - __half2float(hh)));
    return;
  }
  const __nv_bfloat16 h = __float2bfloat16_rn(x);
  out[o] = h;
  if (PC > 1) {
    const float r1 = x - __bfloat162float(h);
    const __nv_bfloat16 m = __float2bfloat16_rn(r1);
    out[o + ps] = m;
    out[o + 2 * ps] = __float2bfloat16_rn(r1 - __bfloat162float(m));
  }
}

}  // namespace

int launch_tile_operand(cudaStream_t st, int N, int K, int pieces, float scale, const float* src,
                        __nv_bfloat16* out) {
  if (N <= 0 || K <= 0 || K % kBK || N % 16) return -1;
  if (pieces < 1 || pieces > 3) return -1;
  const int64_t n = (int64_t)N * K;
  DP_LAUNCHED(1);
  k_tile_operand<<<(int)((n + 255) / 256), 256, 0, st>>>(N, K, pieces, scale, src, out);
  return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

// PDT: the pieces of the dE/dD GEMM's operands (its A written by the last
// backward layer, its B the tiled W_0); PC for every other GEMM
template <int PC, bool TAB, int PDT = PC>
static int fit_tc_impl(cudaStream_t st, int64_t n, const int32_t* idx, const FitNetTC& net, int M,
                       int m_lt, const float* T, float* dT, double* e_atom, const FitScratchTC& s,
                       int32_t* err) {
  const int din = M * m_lt;
  const int nl = net.nl;
  if (nl < 2 || nl > DP_MAXFIT) return -1;
  for (int k = 0; k < nl; ++k)
    if (net.wout[k] > 256 || net.wout[k] % 16) return -1;
  if (m_lt != 16 || M % 4 || M < 16) return -1;  // the fused descriptor wants M< = 16
  // bulk copies and vector loads want 16-byte aligned operands
  auto al = [](const void* p) { return ((uintptr_t)p & 15) == 0; };
  if (!al(T) || !al(s.zh) || !al(s.gph[0]) || !al(s.gph[1]) || !al(s.gz)) return -1;
  for (int k = 0; k < nl; ++k)
    if (!al(net.WTh[k]) || !al(net.Wh[k]) || !al(s.t[k]) || !al(s.z[k]) || !al(net.b[k]))
      return -1;
  const int64_t R = s.rows;
  for (int64_t r0 = 0; r0 < n; r0 += R) {
    const int rows = (int)((n - r0) < R ? (n - r0) : R);
    const int32_t* id = idx ? idx + r0 : nullptr;
    const float* Tc = idx ? T : T + (size_t)r0 * 4 * M;
    float* dTc = idx ? dT : dT + (size_t)r0 * 4 * M;
    // forward: layer 0 (its A operand D formed from T in the stage), hidden
    // layers (A: the FP32 z of the layer below, split in the kernel), last
    // layer with the energy (A: the pieces of z written by the layer below)
    for (int k = 0; k < nl; ++k) {
      TcEpi ep{};
      ep.bias = net.b[k];
      ep.ldo = net.wout[k];
      ep.err = err;
      ep.tab = net.tanh_tab;
      // z of the layer below (z_0 = t_0: layer 0 has no shortcut; the table
      // mode keeps activation derivatives in t, so layer 0 writes z_0 then)
      const float* zb = k == 0 ? nullptr : (k == 1 && !TAB ? s.t[0] : s.z[k - 1]);
      int rc;
      if (k == 0) {
        ep.acc_scale = 1.0f / net.s_wt[0];
        ep.out_scale = net.s_z[0];
        ep.out_a = s.t[0];
        ep.out_b = s.z[0];
        ep.out_h = nl == 2 ? s.zh : nullptr;
        ep.T = Tc;
        ep.tidx = id;
        ep.Mw = M;
        rc = tc_gemm<TC_L0, PC, TAB>(st, rows, net.wout[0], din, net.WTh[0], ep);
      } else if (k == nl - 1) {
        ep.acc_scale = 1.0f / (net.s_z[k - 1] * net.s_wt[k]);
        ep.out_scale = net.s_g[k];
        ep.R = net.shortcut[k] ? zb : nullptr;
        ep.ldr = net.wout[k - 1];
        ep.wout = net.w_out;
        ep.bout = net.b_out;
        ep.out_h = s.gph[0];
        ep.e_atom = e_atom + (idx ? 0 : r0);
        ep.idx = id;
        rc = tc_gemm_p<TC_LAST, PC, TAB>(st, rows, net.wout[k], net.win[k], s.zh, net.WTh[k], ep);
      } else {
        ep.acc_scale = 1.0f / (net.s_z[k - 1] * net.s_wt[k]);
        ep.a_scale = net.s_z[k - 1];
        ep.out_scale = net.s_z[k];
        ep.R = net.shortcut[k] ? zb : nullptr;
        ep.ldr = net.wout[k - 1];
        ep.out_a = s.t[k];
        ep.out_b = s.z[k];
        ep.out_h = k == nl - 2 ? s.zh : nullptr;
        rc = tc_gemm_p<TC_MID, PC, TAB>(st, rows, net.wout[k], net.win[k], zb, net.WTh[k], ep);
      }
      if (rc) return rc;
    }
    // backward: gz_last = w_out (row stride 0); gp of the last layer from the
    // TC_LAST epilogue; gz updated in place, gp ping-pongs
    const float* gz_prev = net.w_out;
    int ldgz = 0;
    int gi = 0;
    for (int k = nl - 1; k >= 1; --k) {
      TcEpi ep{};
      ep.acc_scale = 1.0f / (net.s_g[k] * net.s_w[k]);
      ep.out_scale = net.s_g[k - 1];
      ep.R = net.shortcut[k] ? gz_prev : nullptr;
      ep.ldr = ldgz;
      ep.Tt = s.t[k - 1];
      ep.ldt = net.win[k];
      // dE/dz_0 (k = 1) is read by nothing after: only its product with tanh', the
      // pieces of the dE/dD GEMM's A operand, is kept
      ep.out_b = k > 1 ? s.gz : nullptr;
      ep.out_h = s.gph[gi ^ 1];
      ep.ldo = net.win[k];
      ep.err = err;
      const int rc =
          k > 1 ? tc_gemm_p<TC_BWD, PC, TAB>(st, rows, net.win[k], net.wout[k], s.gph[gi],
                                             net.Wh[k], ep)
                : tc_gemm_p<TC_BWD, PC, TAB, PDT>(st, rows, net.win[k], net.wout[k], s.gph[gi],
                                                  net.Wh[k], ep);
      if (rc) return rc;
      gz_prev = s.gz;
      ldgz = net.win[k];
      gi ^= 1;
    }
    {
      // dE/dD = gp_0 W_0^T never leaves the chip: the epilogue contracts it
      // with T into dE/dT, both factors of Eq. 2's derivative (the x < 16
      // term completed in the epilogue thread's registers)
      TcEpi ep{};
      ep.acc_scale = 1.0f / (net.s_g[0] * net.s_w[0]);
      ep.ldo = din;
      ep.err = err;
      ep.T = Tc;
      ep.dT = dTc;
      ep.tidx = id;
      ep.Mw = M;
      const int rc = tc_gemm_p<TC_DT, PDT, TAB>(st, rows, din, net.wout[0], s.gph[gi], net.Wh[0], ep);
      if (rc) return rc;
    }
  }
  return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

int fit_tc(cudaStream_t st, int64_t n, const int32_t* idx, const FitNetTC& net, int M, int m_lt,
           const float* T, float* dT, double* e_atom, const FitScratchTC& s, int pieces,
           int32_t* err) {
  if (n <= 0) return 0;
  const bool tab = net.tanh_tab != nullptr;
  if (pieces == 1)
    return tab ? fit_tc_impl<1, true>(st, n, idx, net, M, m_lt, T, dT, e_atom, s, err)
               : fit_tc_impl<1, false>(st, n, idx, net, M, m_lt, T, dT, e_atom, s, err);
  if (pieces == 2)
    return tab ? fit_tc_impl<2, true>(st, n, idx, net, M, m_lt, T, dT, e_atom, s, err)
               : fit_tc_impl<2, false>(st, n, idx, net, M, m_lt, T, dT, e_atom, s, err);
  if (pieces == 3)
    return tab ? fit_tc_impl<3, true>(st, n, idx, net, M, m_lt, T, dT, e_atom, s, err)
               : fit_tc_impl<3, false>(st, n, idx, net, M, m_lt, T, dT, e_atom, s, err);
  if (pieces == 4)  // three BF16 pieces, the dE/dD GEMM an FP16 pair
    return tab ? fit_tc_impl<3, true, 2>(st, n, idx, net, M, m_lt, T, dT, e_atom, s, err)
               : fit_tc_impl<3, false, 2>(st, n, idx, net, M, m_lt, T, dT, e_atom, s, err);
  return -1;
}
