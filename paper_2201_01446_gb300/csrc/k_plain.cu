// Plain (untabulated) embedding path in FP32: the comparator of the paper's
// tabulation.  Every pair within rc evaluates the embedding net of Eq. 3-5
//   h0 = tanh(s W0 + b0),  h1 = (h0,h0) + tanh(h0 W1 + b1),
//   G  = (h1,h1) + tanh(h1 W2 + b2)
// and contracts T_i = (1/N_m) sum_j R_ij^T G_ij (Eq. 2's R^T G).  The
// backward recomputes the net per pair and propagates dE/dT back to s and R.
// This is the computation the paper's baseline ran as GEMMs (Fig. 1e); here
// it is fused per atom and G is never stored either, so the comparison with
// the tabulated kernels isolates the tabulation itself.
//
// One warp per atom; pairs are processed in blocks of kP = 8 so that every
// weight load feeds 8 multiply-adds.  Lanes own layer outputs: h0[k] for
// k = lane, h1[m] for m = lane, lane + 32, and embedding columns 4*lane.. .
// Requires the doubling widths of Eq. 5 with d1 <= 32 (M <= 128).
#include <atomic>
#include <math.h>

#include "dp_internal.h"

namespace {

constexpr int kP = 8;       // pairs per block
constexpr int kWpb = 4;     // warps per CTA

struct PlainNet {           // FP32 weights of one (centre, neighbor) type pair
  const float* W0;          // [d1]
  const float* b0;          // [d1]
  const float* W1;          // [d1][d2]
  const float* b1;          // [d2]
  const float* W2;          // [d2][M]
  const float* b2;          // [M]
  const float* W1T;         // [d2][d1]
  const float* W2T;         // [M][d2]
};

struct PlainSmem {          // per warp
  float h0[32][kP];         // layer-0 outputs  [k][p]
  float h1[64][kP];         // layer-1 outputs  [m][p]
  float t1[64][kP];         // layer-1 tanh part
  float dg[128][kP];        // dE/dG            [col][p]
  float dp2[128][kP];       // dE/d(pre-activation of layer 2)
  float dp1[64][kP];        // dE/d(pre-activation of layer 1)
  float R[32][4];           // staged pair data (one chunk of the list)
  float s[32];
  float geo[32][8];         // ds/dr, 1/r, dx, dy, dz
  int jj[32];               // neighbor atom index
};

__device__ __forceinline__ void plain_pair(const EnvParams& ep, float dx, float dy, float dz,
                                           float r2, float& s, float& dsdr, float& ir) {
  const float r = sqrtf(r2);
  ir = 1.0f / r;
  float sw, dsw;
  if (r < ep.rcs) {
    sw = 1.0f;
    dsw = 0.0f;
  } else {
    const float x = (r - ep.rcs) * ep.inv_w;
    const float om = 1.0f - x;
    sw = om * om * om * fmaf(fmaf(6.0f, x, 3.0f), x, 1.0f);
    dsw = -30.0f * x * x * om * om * ep.inv_w;
  }
  s = sw * ir;
  dsdr = (dsw - s) * ir;
}

__device__ __forceinline__ void load_pair_p(const float4& oi, const float4* __restrict__ off,
                                            const CellGeom& g, uint32_t e, float& dx, float& dy,
                                            float& dz, int& tj) {
  const int j = (int)(e >> 5), code = (int)(e & 31u);
  const float4 oj = off[j];
  dx = (oj.x - oi.x) + (float)(code / 9 - 1) * g.edgef[0];
  dy = (oj.y - oi.y) + (float)((code / 3) % 3 - 1) * g.edgef[1];
  dz = (oj.z - oi.z) + (float)(code % 3 - 1) * g.edgef[2];
  tj = __float_as_int(oj.w);
}

// layers 0 and 1 for the block's kP pairs (s from smem); writes h0, h1, t1
__device__ __forceinline__ void plain_layers01(const PlainNet& w, int d1, PlainSmem& S,
                                               const float (&sv)[kP], int lane) {
  const int d2 = 2 * d1;
  if (lane < d1) {
    const float W = w.W0[lane], b = w.b0[lane];
#pragma unroll
    for (int p = 0; p < kP; ++p) S.h0[lane][p] = tanhf(fmaf(sv[p], W, b));
  }
  __syncwarp();
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int m = lane + 32 * h;
    if (m < d2) {
      float acc[kP];
      const float b = w.b1[m];
#pragma unroll
      for (int p = 0; p < kP; ++p) acc[p] = b;
      for (int k = 0; k < d1; ++k) {
        const float W = __ldg(w.W1 + k * d2 + m);
        const float4 a0 = *reinterpret_cast<const float4*>(&S.h0[k][0]);
        const float4 a1 = *reinterpret_cast<const float4*>(&S.h0[k][4]);
        acc[0] = fmaf(a0.x, W, acc[0]);
        acc[1] = fmaf(a0.y, W, acc[1]);
        acc[2] = fmaf(a0.z, W, acc[2]);
        acc[3] = fmaf(a0.w, W, acc[3]);
        acc[4] = fmaf(a1.x, W, acc[4]);
        acc[5] = fmaf(a1.y, W, acc[5]);
        acc[6] = fmaf(a1.z, W, acc[6]);
        acc[7] = fmaf(a1.w, W, acc[7]);
      }
      const int src = m < d1 ? m : m - d1;  // (x, x): column m repeats m mod d1
#pragma unroll
      for (int p = 0; p < kP; ++p) {
        const float t = tanhf(acc[p]);
        S.t1[m][p] = t;
        S.h1[m][p] = S.h0[src][p] + t;
      }
    }
  }
  __syncwarp();
}

// layer 2 for the lane's 4 columns: G[p][q] (and the tanh part t2)
__device__ __forceinline__ void plain_layer2(const PlainNet& w, int d1, int M, PlainSmem& S,
                                             int lane, float (&G)[kP][4], float (&t2)[kP][4]) {
  const int d2 = 2 * d1;
  const int cl = lane * 4;
  if (cl >= M) {
#pragma unroll
    for (int p = 0; p < kP; ++p)
#pragma unroll
      for (int q = 0; q < 4; ++q) G[p][q] = t2[p][q] = 0.0f;
    return;
  }
  const float4 b = __ldg(reinterpret_cast<const float4*>(w.b2 + cl));
  float acc[kP][4];
#pragma unroll
  for (int p = 0; p < kP; ++p) {
    acc[p][0] = b.x;
    acc[p][1] = b.y;
    acc[p][2] = b.z;
    acc[p][3] = b.w;
  }
  for (int l = 0; l < d2; ++l) {
    const float4 W = __ldg(reinterpret_cast<const float4*>(w.W2 + l * M + cl));
    const float4 a0 = *reinterpret_cast<const float4*>(&S.h1[l][0]);
    const float4 a1 = *reinterpret_cast<const float4*>(&S.h1[l][4]);
    const float hv[kP] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
#pragma unroll
    for (int p = 0; p < kP; ++p) {
      acc[p][0] = fmaf(hv[p], W.x, acc[p][0]);
      acc[p][1] = fmaf(hv[p], W.y, acc[p][1]);
      acc[p][2] = fmaf(hv[p], W.z, acc[p][2]);
      acc[p][3] = fmaf(hv[p], W.w, acc[p][3]);
    }
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int col = cl + q;
    const int src = col - (col / d2) * d2;  // (x, x): column repeats col mod d2
#pragma unroll
    for (int p = 0; p < kP; ++p) {
      const float t = tanhf(acc[p][q]);
      t2[p][q] = t;
      G[p][q] = S.h1[src][p] + t;
    }
  }
}

// ------------------------------------------------------------------ forward
// One warp per atom.  The pairs within rc of one neighbor type are staged in
// list order (s and the R row) until a block of kPF = 16 is full; each block
// then runs the net as register-tiled products: layer 1 with lane (m group of
// 4 columns, pair group of 8) owning a 4 x 8 tile, layer 2 with lane owning 4
// embedding columns of all 16 pairs (4 x 16 accumulators: one float4 weight
// load and four broadcast loads of h1 feed 64 multiply-adds).  G goes
// straight into the lane's 4 x 4 block of T.  The last block of an atom and
// type is padded with s = 0, R = 0 (contributes nothing).  Four CTAs (16
// warps) per SM at 128 registers, a few spilled, measured 4% faster than three
// at 167: the kernel is issue-bound and needs the warps to hide the shared-
// memory broadcasts and tanh.
constexpr int kPF = 16;      // pairs per block (forward)
constexpr int kStage = 48;   // staged pairs: < 16 waiting + one list round of 32

struct PlainFwdSmem {        // per warp
  float h0[32][kPF];         // layer-0 outputs [k][p]
  float h1[64][kPF];         // layer-1 outputs [m][p]
  float4 R[kStage];          // staged R rows
  float s[kStage];           // staged s
};

// one block of kPF staged pairs (from the stage front) through the net into
// the lane's T accumulators
template <bool VEC1>
__device__ __forceinline__ void plain_fwd_block(const PlainNet* __restrict__ wp, int d1, int M,
                                                PlainFwdSmem& S, int lane, float (&tacc)[4][4]) {
  // the weight pointers are read from the (L1-resident) record where used:
  // none of them stays live in registers across the atom loop
  const PlainNet& w = *wp;
  const int d2 = 2 * d1;
  // layer 0: lane k < d1, all pairs
  if (lane < d1) {
    const float W = w.W0[lane], b = w.b0[lane];
#pragma unroll
    for (int p = 0; p < kPF; p += 4) {
      float4 h;
      h.x = tanhf(fmaf(S.s[p], W, b));
      h.y = tanhf(fmaf(S.s[p + 1], W, b));
      h.z = tanhf(fmaf(S.s[p + 2], W, b));
      h.w = tanhf(fmaf(S.s[p + 3], W, b));
      *reinterpret_cast<float4*>(&S.h0[lane][p]) = h;
    }
  }
  __syncwarp();
  // layer 1: columns m0..m0+3, pairs p0..p0+7
  {
    const int m0 = (lane & 15) * 4, p0 = (lane >> 4) * 8;
    if (m0 < d2) {
      float acc[8][4];
      float bv[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) bv[q] = m0 + q < d2 ? w.b1[m0 + q] : 0.0f;
#pragma unroll
      for (int p = 0; p < 8; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[p][q] = bv[q];
#pragma unroll 2
      for (int k = 0; k < d1; ++k) {
        float W[4];
        if (VEC1) {
          const float4 w4 = __ldg(reinterpret_cast<const float4*>(w.W1 + k * d2 + m0));
          W[0] = w4.x;
          W[1] = w4.y;
          W[2] = w4.z;
          W[3] = w4.w;
        } else {
#pragma unroll
          for (int q = 0; q < 4; ++q) W[q] = m0 + q < d2 ? __ldg(w.W1 + k * d2 + m0 + q) : 0.0f;
        }
        const float4 a0 = *reinterpret_cast<const float4*>(&S.h0[k][p0]);
        const float4 a1 = *reinterpret_cast<const float4*>(&S.h0[k][p0 + 4]);
        const float hv[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
#pragma unroll
        for (int p = 0; p < 8; ++p)
#pragma unroll
          for (int q = 0; q < 4; ++q) acc[p][q] = fmaf(hv[p], W[q], acc[p][q]);
      }
      // h1 = (h0, h0) + tanh: column m repeats h0 column m mod d1
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int m = m0 + q;
        if (m < d2) {
          const int src = m < d1 ? m : m - d1;
          const float4 a0 = *reinterpret_cast<const float4*>(&S.h0[src][p0]);
          const float4 a1 = *reinterpret_cast<const float4*>(&S.h0[src][p0 + 4]);
          *reinterpret_cast<float4*>(&S.h1[m][p0]) =
              make_float4(a0.x + tanhf(acc[0][q]), a0.y + tanhf(acc[1][q]),
                          a0.z + tanhf(acc[2][q]), a0.w + tanhf(acc[3][q]));
          *reinterpret_cast<float4*>(&S.h1[m][p0 + 4]) =
              make_float4(a1.x + tanhf(acc[4][q]), a1.y + tanhf(acc[5][q]),
                          a1.z + tanhf(acc[6][q]), a1.w + tanhf(acc[7][q]));
        }
      }
    }
  }
  __syncwarp();
  // layer 2: columns c0..c0+3 of all pairs, then G into T
  const int c0 = lane * 4;
  if (c0 < M) {
    float acc[kPF][4];
    const float4 b = __ldg(reinterpret_cast<const float4*>(w.b2 + c0));
#pragma unroll
    for (int p = 0; p < kPF; ++p) {
      acc[p][0] = b.x;
      acc[p][1] = b.y;
      acc[p][2] = b.z;
      acc[p][3] = b.w;
    }
#pragma unroll 2
    for (int l = 0; l < d2; ++l) {
      const float4 W = __ldg(reinterpret_cast<const float4*>(w.W2 + l * M + c0));
      const float4* hr = reinterpret_cast<const float4*>(&S.h1[l][0]);
#pragma unroll
      for (int g4 = 0; g4 < kPF / 4; ++g4) {
        const float4 a = hr[g4];
        const float hv[4] = {a.x, a.y, a.z, a.w};
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int p = g4 * 4 + j;
          acc[p][0] = fmaf(hv[j], W.x, acc[p][0]);
          acc[p][1] = fmaf(hv[j], W.y, acc[p][1]);
          acc[p][2] = fmaf(hv[j], W.z, acc[p][2]);
          acc[p][3] = fmaf(hv[j], W.w, acc[p][3]);
        }
      }
    }
    // G = (h1, h1) + tanh: column c repeats h1 column c mod d2
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int c = c0 + q;
      const int src = c - (c / d2) * d2;
      const float4* hr = reinterpret_cast<const float4*>(&S.h1[src][0]);
#pragma unroll
      for (int g4 = 0; g4 < kPF / 4; ++g4) {
        const float4 a = hr[g4];
        const float hv[4] = {a.x, a.y, a.z, a.w};
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int p = g4 * 4 + j;
          const float G = hv[j] + tanhf(acc[p][q]);
          const float4 R = S.R[p];
          tacc[0][q] = fmaf(R.x, G, tacc[0][q]);
          tacc[1][q] = fmaf(R.y, G, tacc[1][q]);
          tacc[2][q] = fmaf(R.z, G, tacc[2][q]);
          tacc[3][q] = fmaf(R.w, G, tacc[3][q]);
        }
      }
    }
  }
  __syncwarp();
}

template <bool VEC1>
__global__ void __launch_bounds__(kWpb * 32, 4) k_plain_fwd(int64_t n, const float4* __restrict__ off,
                                                         const uint32_t* __restrict__ nlist,
                                                         const int32_t* __restrict__ nn, int cap,
                                                         CellGeom g, EnvParams ep,
                                                         const PlainNet* __restrict__ nets, int d1,
                                                         float* __restrict__ T,
                                                         unsigned long long* __restrict__ pair_count) {
  extern __shared__ float4 smem4[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  PlainFwdSmem& S = reinterpret_cast<PlainFwdSmem*>(smem4)[wib];
  const int M = ep.M, nt = ep.ntypes;
  const int cl = lane * 4;
  const unsigned below = (1u << lane) - 1u;
  unsigned long long npairs = 0;
  for (int64_t i = (int64_t)blockIdx.x * kWpb + wib; i < n; i += (int64_t)gridDim.x * kWpb) {
    const float4 oi = off[i];
    const int ti = __float_as_int(oi.w);
    const int cnt = min(nn[i], cap);
    const uint32_t* L = nlist + (size_t)i * cap;
    float tacc[4][4];
#pragma unroll
    for (int c = 0; c < 4; ++c)
#pragma unroll
      for (int q = 0; q < 4; ++q) tacc[c][q] = 0.0f;
    for (int tj = 0; tj < nt; ++tj) {
      const PlainNet* w = nets + ti * nt + tj;
      int nst = 0;  // staged pairs
      uint32_t e_next = lane < cnt ? L[lane] : 0u;
      for (int b0 = 0; b0 < cnt; b0 += 32) {
        const int k = b0 + lane;
        const uint32_t e = e_next;
        if (k + 32 < cnt) e_next = L[k + 32];
        bool in = false;
        float s = 0.f, dsdr, ir, dx = 0.f, dy = 0.f, dz = 0.f;
        if (k < cnt) {
          int t;
          load_pair_p(oi, off, g, e, dx, dy, dz, t);
          const float r2 = dx * dx + dy * dy + dz * dz;
          if (r2 < ep.rc2 && t == tj) {
            in = true;
            plain_pair(ep, dx, dy, dz, r2, s, dsdr, ir);
          }
        }
        const unsigned m = __ballot_sync(0xffffffffu, in);
        // the stage holds < kPF pairs here, so nst + 32 <= kStage
        const int slot = nst + __popc(m & below);
        if (in && slot < kStage) {
          S.s[slot] = s;
          S.R[slot] = make_float4(s, s * dx * ir, s * dy * ir, s * dz * ir);
        }
        nst += __popc(m);
        npairs += __popc(m);
        __syncwarp();
        while (nst >= kPF) {
          plain_fwd_block<VEC1>(w, d1, M, S, lane, tacc);
          // the rest of the stage (< 32 pairs) to its front
          const int rest = nst - kPF;
          float sv = 0.f;
          float4 rv = make_float4(0.f, 0.f, 0.f, 0.f);
          if (lane < rest) {
            sv = S.s[kPF + lane];
            rv = S.R[kPF + lane];
          }
          __syncwarp();
          if (lane < rest) {
            S.s[lane] = sv;
            S.R[lane] = rv;
          }
          __syncwarp();
          nst = rest;
        }
      }
      if (nst > 0) {
        // the last partial block, padded with zero rows
        if (lane < kPF && lane >= nst) {
          S.s[lane] = 0.0f;
          S.R[lane] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
        __syncwarp();
        plain_fwd_block<VEC1>(w, d1, M, S, lane, tacc);
      }
    }
    if (cl < M) {
      float* Ti = T + (size_t)i * 4 * M + cl;
#pragma unroll
      for (int cc = 0; cc < 4; ++cc)
        *reinterpret_cast<float4*>(Ti + cc * M) =
            make_float4(tacc[cc][0] * ep.inv_nm, tacc[cc][1] * ep.inv_nm, tacc[cc][2] * ep.inv_nm,
                        tacc[cc][3] * ep.inv_nm);
    }
  }
  if (lane == 0 && pair_count) atomicAdd(pair_count, npairs);
}

// sum of 32 per-lane values across the warp; lane l receives the total of
// value l (a transposing butterfly: 31 shuffles)
__device__ __forceinline__ float transpose_sum32(float (&v)[32], int lane) {
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) {
    const bool hi = (lane & o) != 0;
#pragma unroll
    for (int k = 0; k < o; ++k) {
      const float send = hi ? v[k] : v[k + o];
      const float keep = hi ? v[k + o] : v[k];
      v[k] = keep + __shfl_xor_sync(0xffffffffu, send, o);
    }
  }
  return v[0];
}

// sum of 16 per-lane values across the warp; lanes l and l + 16 receive the
// total of value l % 16 (a fold of the two half-warps, then a transposing
// butterfly: 31 shuffles)
__device__ __forceinline__ float transpose_sum16(float (&v)[16], int lane) {
#pragma unroll
  for (int k = 0; k < 16; ++k) v[k] += __shfl_xor_sync(0xffffffffu, v[k], 16);
#pragma unroll
  for (int o = 8; o >= 1; o >>= 1) {
    const bool hi = (lane & o) != 0;
#pragma unroll
    for (int k = 0; k < o; ++k) {
      const float send = hi ? v[k] : v[k + o];
      const float keep = hi ? v[k + o] : v[k];
      v[k] = keep + __shfl_xor_sync(0xffffffffu, send, o);
    }
  }
  return v[0];
}

// ------------------------------------------------------------------ backward
// One warp per atom, pairs staged in blocks of kPF = 16 as in the forward.
// Per block: the forward recomputed (h0, t1, h1 in shared memory, layer 2 in
// the lane's 4 x 16 registers), then
//   dE/dG[c][p] = (1/N_m) sum_cc dT[cc][c] R[p][cc],  dp2 = dE/dG (1 - t2^2),
//   dE/dR[p][cc] = (1/N_m) sum_c dT[cc][c] G[p][c]   (a transposing warp sum),
//   dh1 = dE/dG[l] + dE/dG[l + d2] + W2 dp2           (lane tile 4 l x 8 p),
//   dp1 = dh1 (1 - t1^2),
//   dh0 = dh1[k] + dh1[k + d1] + W1 dp1               (lane tile 4 k x 4 p),
//   dE/ds = sum_k W0[k] dh0[k] (1 - h0[k]^2),
// and the chain rule through Eq. 1 per pair (lanes 0..15) to the forces and
// the virial.
struct PlainBwdSmem {        // per warp
  float h0[32][kPF];         // layer-0 outputs
  float t1[64][kPF];         // layer-1 tanh part
  float h1[64][kPF];         // layer-1 outputs, then dE/dh1
  float dp[128][kPF];        // dE/d(pre-activation): layer 2, then layer 1
  float4 R[kStage];          // staged pairs: R row
  float4 geo[kStage];        // ds/dr, 1/r, dx, dy
  float dz[kStage];
  float s[kStage];
  int jj[kStage];            // neighbor atom index
  float4 gR[kPF];            // dE/dR of the block's pairs
  float gs[kPF];             // dE/ds (through the net) of the block's pairs
  double vacc[9];            // the warp's virial (lane 0)
};

template <bool VEC>
__device__ __forceinline__ void plain_bwd_block(const PlainNet& w, int d1, int M, float inv_nm,
                                                PlainBwdSmem& S, int lane,
                                                const float (&dTv)[4][4],
                                                const float* __restrict__ dTi, int c, int& nbad,
                                                float& fx, float& fy, float& fz, float (&vl)[9],
                                                unsigned long long* __restrict__ ffix) {
  const int d2 = 2 * d1;
  // ---- forward: layer 0
  if (lane < d1) {
    const float W = w.W0[lane], b = w.b0[lane];
#pragma unroll
    for (int p = 0; p < kPF; p += 4) {
      float4 h;
      h.x = tanhf(fmaf(S.s[p], W, b));
      h.y = tanhf(fmaf(S.s[p + 1], W, b));
      h.z = tanhf(fmaf(S.s[p + 2], W, b));
      h.w = tanhf(fmaf(S.s[p + 3], W, b));
      *reinterpret_cast<float4*>(&S.h0[lane][p]) = h;
    }
  }
  __syncwarp();
  // ---- forward: layer 1 (tile 4 m x 8 p)
  {
    const int m0 = (lane & 15) * 4, p0 = (lane >> 4) * 8;
    if (m0 < d2) {
      float acc[8][4];
      float bv[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) bv[q] = m0 + q < d2 ? w.b1[m0 + q] : 0.0f;
#pragma unroll
      for (int p = 0; p < 8; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[p][q] = bv[q];
            for (int k = 0; k < d1; ++k) {
        float W[4];
        if (VEC) {
          const float4 w4 = __ldg(reinterpret_cast<const float4*>(w.W1 + k * d2 + m0));
          W[0] = w4.x;
          W[1] = w4.y;
          W[2] = w4.z;
          W[3] = w4.w;
        } else {
#pragma unroll
          for (int q = 0; q < 4; ++q) W[q] = m0 + q < d2 ? __ldg(w.W1 + k * d2 + m0 + q) : 0.0f;
        }
        const float4 a0 = *reinterpret_cast<const float4*>(&S.h0[k][p0]);
        const float4 a1 = *reinterpret_cast<const float4*>(&S.h0[k][p0 + 4]);
        const float hv[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
#pragma unroll
        for (int p = 0; p < 8; ++p)
#pragma unroll
          for (int q = 0; q < 4; ++q) acc[p][q] = fmaf(hv[p], W[q], acc[p][q]);
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int m = m0 + q;
        if (m < d2) {
          const int src = m < d1 ? m : m - d1;
          float t[8];
#pragma unroll
          for (int p = 0; p < 8; ++p) t[p] = tanhf(acc[p][q]);
          const float4 a0 = *reinterpret_cast<const float4*>(&S.h0[src][p0]);
          const float4 a1 = *reinterpret_cast<const float4*>(&S.h0[src][p0 + 4]);
          *reinterpret_cast<float4*>(&S.t1[m][p0]) = make_float4(t[0], t[1], t[2], t[3]);
          *reinterpret_cast<float4*>(&S.t1[m][p0 + 4]) = make_float4(t[4], t[5], t[6], t[7]);
          *reinterpret_cast<float4*>(&S.h1[m][p0]) =
              make_float4(a0.x + t[0], a0.y + t[1], a0.z + t[2], a0.w + t[3]);
          *reinterpret_cast<float4*>(&S.h1[m][p0 + 4]) =
              make_float4(a1.x + t[4], a1.y + t[5], a1.z + t[6], a1.w + t[7]);
        }
      }
    }
  }
  __syncwarp();
  // ---- forward layer 2 and its backward epilogue, per half of the pairs
  // (lane's 4 columns x 8 pairs in registers): G, dE/dG and dp2 of the
  // lane's columns, and the lane's partial dE/dR summed across the warp (lane
  // l receives pair 8 h + l / 4, component l % 4)
  const int c0 = lane * 4;
#pragma unroll 1
  for (int hf = 0; hf < 2; ++hf) {
    const int pb = hf * 8;
    float acc[8][4];
    if (c0 < M) {
      const float4 b = __ldg(reinterpret_cast<const float4*>(w.b2 + c0));
#pragma unroll
      for (int p = 0; p < 8; ++p) {
        acc[p][0] = b.x;
        acc[p][1] = b.y;
        acc[p][2] = b.z;
        acc[p][3] = b.w;
      }
            for (int l = 0; l < d2; ++l) {
        const float4 W = __ldg(reinterpret_cast<const float4*>(w.W2 + l * M + c0));
        const float4 a0 = *reinterpret_cast<const float4*>(&S.h1[l][pb]);
        const float4 a1 = *reinterpret_cast<const float4*>(&S.h1[l][pb + 4]);
        const float hv[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
#pragma unroll
        for (int p = 0; p < 8; ++p) {
          acc[p][0] = fmaf(hv[p], W.x, acc[p][0]);
          acc[p][1] = fmaf(hv[p], W.y, acc[p][1]);
          acc[p][2] = fmaf(hv[p], W.z, acc[p][2]);
          acc[p][3] = fmaf(hv[p], W.w, acc[p][3]);
        }
      }
    } else {
#pragma unroll
      for (int p = 0; p < 8; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[p][q] = 0.0f;
    }
#pragma unroll
    for (int qt = 0; qt < 2; ++qt) {  // quarters of 4 pairs: 16 partial sums each
      float part[16];
#pragma unroll
      for (int j = 0; j < 16; ++j) part[j] = 0.0f;
#pragma unroll
      for (int pq = 0; pq < 4; ++pq) {
        const int pp = qt * 4 + pq, p = pb + pp;
        const float4 R = S.R[p];
        const float rv[4] = {R.x, R.y, R.z, R.w};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int col = c0 + q;
          float G = 0.0f, t = 0.0f, dg = 0.0f;
          if (col < M) {
            const int src = col - (col / d2) * d2;
            t = tanhf(acc[pp][q]);
            G = S.h1[src][p] + t;
#pragma unroll
            for (int cc = 0; cc < 4; ++cc) dg = fmaf(dTv[cc][q], rv[cc], dg);
            dg *= inv_nm;
          }
#pragma unroll
          for (int cc = 0; cc < 4; ++cc)
            part[pq * 4 + cc] = fmaf(dTv[cc][q], G, part[pq * 4 + cc]);
          if (col < M) S.dp[col][p] = dg * (1.0f - t * t);
        }
      }
      // lane l (< 16) receives pair pb + 4 qt + l / 4, component l % 4
      const float dR = transpose_sum16(part, lane) * inv_nm;
      if (lane < 16) reinterpret_cast<float*>(S.gR)[4 * (pb + 4 * qt) + lane] = dR;
    }
  }
  __syncwarp();
  // ---- layer 2 backward (tile 4 l x 8 p): dE/dh1 = the (x, x) shortcut's
  // dE/dG[l] + dE/dG[l + d2] = (1/N_m) R . (dT[.][l] + dT[.][l + d2]), plus
  // W2 dp2; then dp1
  {
    const int l0 = (lane & 15) * 4, p0 = (lane >> 4) * 8;
    float acc[8][4];
    if (l0 < d2) {
      float dsum[4][4];  // [cc][q]: dT[cc][l] + dT[cc][l + d2]
#pragma unroll
      for (int cc = 0; cc < 4; ++cc)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int l = l0 + q;
          dsum[cc][q] = l < d2 ? (__ldg(dTi + cc * M + l) + __ldg(dTi + cc * M + l + d2)) * inv_nm
                               : 0.0f;
        }
#pragma unroll
      for (int p = 0; p < 8; ++p) {
        const float4 R = S.R[p0 + p];
#pragma unroll
        for (int q = 0; q < 4; ++q)
          acc[p][q] = fmaf(R.x, dsum[0][q],
                           fmaf(R.y, dsum[1][q], fmaf(R.z, dsum[2][q], R.w * dsum[3][q])));
      }
            for (int cc = 0; cc < M; ++cc) {
        float W[4];
        if (VEC) {
          const float4 w4 = __ldg(reinterpret_cast<const float4*>(w.W2T + cc * d2 + l0));
          W[0] = w4.x;
          W[1] = w4.y;
          W[2] = w4.z;
          W[3] = w4.w;
        } else {
#pragma unroll
          for (int q = 0; q < 4; ++q) W[q] = l0 + q < d2 ? __ldg(w.W2T + cc * d2 + l0 + q) : 0.0f;
        }
        const float4 a0 = *reinterpret_cast<const float4*>(&S.dp[cc][p0]);
        const float4 a1 = *reinterpret_cast<const float4*>(&S.dp[cc][p0 + 4]);
        const float dv[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
#pragma unroll
        for (int p = 0; p < 8; ++p)
#pragma unroll
          for (int q = 0; q < 4; ++q) acc[p][q] = fmaf(dv[p], W[q], acc[p][q]);
      }
    }
    __syncwarp();  // every lane is done with dp2 and the shortcut part of dE/dh1
    if (l0 < d2) {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int l = l0 + q;
        if (l < d2) {
          float dpv[8];
#pragma unroll
          for (int p = 0; p < 8; ++p) {
            const float t = S.t1[l][p0 + p];
            dpv[p] = acc[p][q] * (1.0f - t * t);
          }
          *reinterpret_cast<float4*>(&S.dp[l][p0]) = make_float4(dpv[0], dpv[1], dpv[2], dpv[3]);
          *reinterpret_cast<float4*>(&S.dp[l][p0 + 4]) =
              make_float4(dpv[4], dpv[5], dpv[6], dpv[7]);
          *reinterpret_cast<float4*>(&S.h1[l][p0]) =
              make_float4(acc[0][q], acc[1][q], acc[2][q], acc[3][q]);
          *reinterpret_cast<float4*>(&S.h1[l][p0 + 4]) =
              make_float4(acc[4][q], acc[5][q], acc[6][q], acc[7][q]);
        }
      }
    }
  }
  __syncwarp();
  // ---- layer 1 and layer 0 backward: dh0 (tile 4 k x 4 p), dE/ds
  {
    const int k0 = (lane & 7) * 4, p0 = (lane >> 3) * 4;
    float acc[4][4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int k = k0 + q;
#pragma unroll
      for (int p = 0; p < 4; ++p)
        acc[p][q] = k < d1 ? S.h1[k][p0 + p] + S.h1[k + d1][p0 + p] : 0.0f;
    }
    if (k0 < d1) {
            for (int m = 0; m < d2; ++m) {
        float W[4];
        if (VEC && (d1 % 4) == 0) {
          const float4 w4 = __ldg(reinterpret_cast<const float4*>(w.W1T + m * d1 + k0));
          W[0] = w4.x;
          W[1] = w4.y;
          W[2] = w4.z;
          W[3] = w4.w;
        } else {
#pragma unroll
          for (int q = 0; q < 4; ++q) W[q] = k0 + q < d1 ? __ldg(w.W1T + m * d1 + k0 + q) : 0.0f;
        }
        const float4 a = *reinterpret_cast<const float4*>(&S.dp[m][p0]);
        const float dv[4] = {a.x, a.y, a.z, a.w};
#pragma unroll
        for (int p = 0; p < 4; ++p)
#pragma unroll
          for (int q = 0; q < 4; ++q) acc[p][q] = fmaf(dv[p], W[q], acc[p][q]);
      }
    }
    float dsp[4];
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      float v = 0.0f;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int k = k0 + q;
        if (k < d1) {
          const float h0 = S.h0[k][p0 + p];
          v = fmaf(w.W0[k] * acc[p][q], 1.0f - h0 * h0, v);
        }
      }
      dsp[p] = v;
    }
    // sum over the 8 lanes of a pair group (lane bits 0..2)
#pragma unroll
    for (int o = 1; o < 8; o <<= 1)
#pragma unroll
      for (int p = 0; p < 4; ++p) dsp[p] += __shfl_xor_sync(0xffffffffu, dsp[p], o);
    if ((lane & 7) == 0) {
#pragma unroll
      for (int p = 0; p < 4; ++p) S.gs[p0 + p] = dsp[p];
    }
  }
  __syncwarp();
  // ---- per pair: chain rule through Eq. 1 (lanes 0..c-1 of the block)
  if (lane < c) {
    const float4 gR = S.gR[lane];
    const float gsv = S.gs[lane];
    const float4 ge = S.geo[lane];
    const float sgeo = S.s[lane];
    const float dsr = ge.x, irr = ge.y, ddx = ge.z, ddy = ge.w, ddz = S.dz[lane];
    const float ux = ddx * irr, uy = ddy * irr, uz = ddz * irr;
    const float a0 = gR.x + gsv;
    const float dot = gR.y * ux + gR.z * uy + gR.w * uz;
    const float sor = sgeo * irr;
    const float coef = dsr * (a0 + dot) - sor * dot;
    float gx = coef * ux + sor * gR.y;
    float gy = coef * uy + sor * gR.z;
    float gz = coef * uz + sor * gR.w;
    if (!(isfinite(gx) && isfinite(gy) && isfinite(gz)) || fabsf(gx) > 4.0e6f ||
        fabsf(gy) > 4.0e6f || fabsf(gz) > 4.0e6f) {
      ++nbad;
      gx = gy = gz = 0.0f;
    }
    fx += gx;
    fy += gy;
    fz += gz;
    vl[0] -= ddx * gx;
    vl[1] -= ddx * gy;
    vl[2] -= ddx * gz;
    vl[3] -= ddy * gx;
    vl[4] -= ddy * gy;
    vl[5] -= ddy * gz;
    vl[6] -= ddz * gx;
    vl[7] -= ddz * gy;
    vl[8] -= ddz * gz;
    unsigned long long* fj = ffix + (size_t)S.jj[lane] * 3;
    atomicAdd(fj + 0, (unsigned long long)(-__float2ll_rn(gx * DP_FSCALE_F)));
    atomicAdd(fj + 1, (unsigned long long)(-__float2ll_rn(gy * DP_FSCALE_F)));
    atomicAdd(fj + 2, (unsigned long long)(-__float2ll_rn(gz * DP_FSCALE_F)));
  }
  __syncwarp();
}

template <bool VEC>
__global__ void __launch_bounds__(kWpb * 32) k_plain_bwd(int64_t n, const float4* __restrict__ off,
                                                         const uint32_t* __restrict__ nlist,
                                                         const int32_t* __restrict__ nn, int cap,
                                                         CellGeom g, EnvParams ep,
                                                         const PlainNet* __restrict__ nets, int d1,
                                                         const float* __restrict__ dT,
                                                         unsigned long long* __restrict__ ffix,
                                                         double* __restrict__ vir_part,
                                                         int32_t* __restrict__ status) {
  extern __shared__ float4 smem4[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  PlainBwdSmem& S = reinterpret_cast<PlainBwdSmem*>(smem4)[wib];
  const int M = ep.M, nt = ep.ntypes;
  const int cl = lane * 4;
  const unsigned below = (1u << lane) - 1u;
  if (lane < 9) S.vacc[lane] = 0.0;
  int nbad = 0;
  for (int64_t i = (int64_t)blockIdx.x * kWpb + wib; i < n; i += (int64_t)gridDim.x * kWpb) {
    const float4 oi = off[i];
    const int ti = __float_as_int(oi.w);
    const int cnt = min(nn[i], cap);
    const uint32_t* L = nlist + (size_t)i * cap;
    float dTv[4][4];  // dT[c][cl + q]
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const float4 t4 = cl < M ? *reinterpret_cast<const float4*>(dT + (size_t)i * 4 * M + c * M + cl)
                               : make_float4(0.f, 0.f, 0.f, 0.f);
      dTv[c][0] = t4.x;
      dTv[c][1] = t4.y;
      dTv[c][2] = t4.z;
      dTv[c][3] = t4.w;
    }
    float fx = 0.f, fy = 0.f, fz = 0.f;
    float vl[9];
#pragma unroll
    for (int a = 0; a < 9; ++a) vl[a] = 0.f;
    for (int tj = 0; tj < nt; ++tj) {
      const PlainNet w = nets[ti * nt + tj];
      int nst = 0;
      uint32_t e_next = lane < cnt ? L[lane] : 0u;
      for (int b0 = 0; b0 < cnt; b0 += 32) {
        const int k = b0 + lane;
        const uint32_t e = e_next;
        if (k + 32 < cnt) e_next = L[k + 32];
        bool in = false;
        float s = 0.f, dsdr = 0.f, ir = 0.f, dx = 0.f, dy = 0.f, dz = 0.f;
        if (k < cnt) {
          int t;
          load_pair_p(oi, off, g, e, dx, dy, dz, t);
          const float r2 = dx * dx + dy * dy + dz * dz;
          if (r2 < ep.rc2 && t == tj) {
            in = true;
            plain_pair(ep, dx, dy, dz, r2, s, dsdr, ir);
          }
        }
        const unsigned m = __ballot_sync(0xffffffffu, in);
        // the stage holds < kPF pairs here, so nst + 32 <= kStage
        const int slot = nst + __popc(m & below);
        if (in && slot < kStage) {
          S.s[slot] = s;
          S.R[slot] = make_float4(s, s * dx * ir, s * dy * ir, s * dz * ir);
          S.geo[slot] = make_float4(dsdr, ir, dx, dy);
          S.dz[slot] = dz;
          S.jj[slot] = (int)(e >> 5);
        }
        nst += __popc(m);
        __syncwarp();
        while (nst >= kPF) {
          plain_bwd_block<VEC>(w, d1, M, ep.inv_nm, S, lane, dTv, dT + (size_t)i * 4 * M, kPF,
                               nbad, fx, fy, fz, vl, ffix);
          const int rest = nst - kPF;
          float sv = 0.f, dzv = 0.f;
          float4 rv = make_float4(0.f, 0.f, 0.f, 0.f), gv = rv;
          int jv = 0;
          if (lane < rest) {
            sv = S.s[kPF + lane];
            rv = S.R[kPF + lane];
            gv = S.geo[kPF + lane];
            dzv = S.dz[kPF + lane];
            jv = S.jj[kPF + lane];
          }
          __syncwarp();
          if (lane < rest) {
            S.s[lane] = sv;
            S.R[lane] = rv;
            S.geo[lane] = gv;
            S.dz[lane] = dzv;
            S.jj[lane] = jv;
          }
          __syncwarp();
          nst = rest;
        }
      }
      if (nst > 0) {
        if (lane < kPF && lane >= nst) {
          S.s[lane] = 0.0f;
          S.R[lane] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
        __syncwarp();
        plain_bwd_block<VEC>(w, d1, M, ep.inv_nm, S, lane, dTv, dT + (size_t)i * 4 * M, nst,
                             nbad, fx, fy, fz, vl, ffix);
      }
    }
    double red[12] = {fx, fy, fz, vl[0], vl[1], vl[2], vl[3], vl[4], vl[5], vl[6], vl[7], vl[8]};
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1)
#pragma unroll
      for (int a = 0; a < 12; ++a) red[a] += __shfl_xor_sync(0xffffffffu, red[a], o);
    if (lane == 0) {
      unsigned long long* fi = ffix + (size_t)i * 3;
      atomicAdd(fi + 0, (unsigned long long)__double2ll_rn(red[0] * DP_FSCALE));
      atomicAdd(fi + 1, (unsigned long long)__double2ll_rn(red[1] * DP_FSCALE));
      atomicAdd(fi + 2, (unsigned long long)__double2ll_rn(red[2] * DP_FSCALE));
#pragma unroll
      for (int a = 0; a < 9; ++a) S.vacc[a] += red[3 + a];
    }
    __syncwarp();
  }
  if (lane == 0) {
    double* vp = vir_part + ((size_t)blockIdx.x * kWpb + wib) * 9;
#pragma unroll
    for (int a = 0; a < 9; ++a) vp[a] = S.vacc[a];
  }
  nbad = __reduce_add_sync(0xffffffffu, nbad);
  if (lane == 0 && nbad) atomicAdd(&status[ST_NONFINITE], nbad);
}

int plain_blocks(int64_t n) {
  int dev = 0, sms = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t want = (n + kWpb - 1) / kWpb;
  const int64_t capb = (int64_t)sms * 12;
  return (int)(want < capb ? (want > 0 ? want : 1) : capb);
}

bool plain_shape_ok(const EnvParams& ep, int d1) {
  return d1 >= 1 && d1 <= 32 && ep.M == 4 * d1 && ep.M % 4 == 0;
}


// ------------------------------------------------------------------ parameter gradients
// dE/d(embedding-net weights and biases) of one (centre, neighbor) type pair,
// reverse mode through Eq. 4-5 per pair: with dE/dG = (1/N_m) R^T dE/dT,
//   layer 2: dp2 = dE/dG (1 - t2^2), dW2[l][q] += h1[l] dp2[q], db2 += dp2,
//   layer 1: dp1 = dE/dh1 (1 - t1^2), dW1[k][m] += h0[k] dp1[m], db1 += dp1,
//   layer 0: dp0 = dE/dh0 (1 - h0^2), dW0[k] += s dp0[k], db0 += dp0,
// where dE/dh1 and dE/dh0 carry the (x,x) shortcuts.  One warp per CTA; the
// CTA's sums (one layout block per layer: W rows, then b) stay in its
// shared memory, every element owned by one lane (no atomics), and go to the
// CTA's row of part at the end; a second kernel adds the rows in order.
__global__ void __launch_bounds__(32) k_plain_wgrad(int64_t n, const float4* __restrict__ off,
                                                    const uint32_t* __restrict__ nlist,
                                                    const int32_t* __restrict__ nn, int cap,
                                                    CellGeom g, EnvParams ep,
                                                    const PlainNet* __restrict__ nets, int d1,
                                                    const float* __restrict__ dT, int ti, int tj,
                                                    int npar, float* __restrict__ part) {
  extern __shared__ float4 smem4[];
  PlainSmem& S = *reinterpret_cast<PlainSmem*>(smem4);
  float* acc = reinterpret_cast<float*>(reinterpret_cast<unsigned char*>(smem4) +
                                        (sizeof(PlainSmem) + 15) / 16 * 16);
  const int lane = threadIdx.x;
  const int M = ep.M, nt = ep.ntypes, d2 = 2 * d1;
  const int cl = lane * 4;
  const unsigned below = (1u << lane) - 1u;
  // the layer blocks: W0 [1][d1], b0; W1 [d1][d2], b1; W2 [d2][M], b2
  float* gW0 = acc;
  float* gb0 = gW0 + d1;
  float* gW1 = gb0 + d1;
  float* gb1 = gW1 + d1 * d2;
  float* gW2 = gb1 + d2;
  float* gb2 = gW2 + d2 * M;
  for (int e = lane; e < npar; e += 32) acc[e] = 0.0f;
  __syncwarp();
  const PlainNet w = nets[ti * nt + tj];
  for (int64_t i = blockIdx.x; i < n; i += gridDim.x) {
    const float4 oi = off[i];
    if (__float_as_int(oi.w) != ti) continue;
    const int cnt = min(nn[i], cap);
    const uint32_t* L = nlist + (size_t)i * cap;
    float dTv[4][4];  // dT[c][cl + q]
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const float4 t4 = cl < M ? *reinterpret_cast<const float4*>(dT + (size_t)i * 4 * M + c * M + cl)
                               : make_float4(0.f, 0.f, 0.f, 0.f);
      dTv[c][0] = t4.x;
      dTv[c][1] = t4.y;
      dTv[c][2] = t4.z;
      dTv[c][3] = t4.w;
    }
    for (int b0 = 0; b0 < cnt; b0 += 32) {
      const int k = b0 + lane;
      bool in = false;
      float s = 0.f, dsdr = 0.f, ir = 0.f, dx = 0.f, dy = 0.f, dz = 0.f;
      if (k < cnt) {
        int t;
        load_pair_p(oi, off, g, L[k], dx, dy, dz, t);
        const float r2 = dx * dx + dy * dy + dz * dz;
        if (r2 < ep.rc2 && t == tj) {
          in = true;
          plain_pair(ep, dx, dy, dz, r2, s, dsdr, ir);
        }
      }
      const unsigned m = __ballot_sync(0xffffffffu, in);
      if (in) {
        const int slot = __popc(m & below);
        S.s[slot] = s;
        S.R[slot][0] = s;
        S.R[slot][1] = s * dx * ir;
        S.R[slot][2] = s * dy * ir;
        S.R[slot][3] = s * dz * ir;
      }
      __syncwarp();
      const int c = __popc(m);
      for (int p0 = 0; p0 < c; p0 += kP) {
        float sv[kP];
#pragma unroll
        for (int p = 0; p < kP; ++p) sv[p] = p0 + p < c ? S.s[p0 + p] : 0.0f;
        plain_layers01(w, d1, S, sv, lane);
        float G[kP][4], t2[kP][4];
        plain_layer2(w, d1, M, S, lane, G, t2);
        // dE/dG and dp2 for the lane's columns (zero for padding pairs)
        float dp2[kP][4];
#pragma unroll
        for (int p = 0; p < kP; ++p) {
          float4 R = *reinterpret_cast<const float4*>(S.R[p0 + p < c ? p0 + p : p0]);
          if (p0 + p >= c) R = make_float4(0.f, 0.f, 0.f, 0.f);
          const float rv[4] = {R.x, R.y, R.z, R.w};
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            float dg = 0.0f;
#pragma unroll
            for (int cc = 0; cc < 4; ++cc) dg = fmaf(dTv[cc][q], rv[cc], dg);
            dg *= ep.inv_nm;
            dp2[p][q] = dg * (1.0f - t2[p][q] * t2[p][q]);
            if (cl < M) {
              S.dg[cl + q][p] = dg;
              S.dp2[cl + q][p] = dp2[p][q];
            }
          }
        }
        // layer 2: the lane's four columns of W2 and b2
        if (cl < M) {
          for (int l = 0; l < d2; ++l) {
            const float4 a0 = *reinterpret_cast<const float4*>(&S.h1[l][0]);
            const float4 a1 = *reinterpret_cast<const float4*>(&S.h1[l][4]);
            const float hv[kP] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
            // scalar accesses: the block's offset need not be a multiple of 4
            float* gr = gW2 + l * M + cl;
            float gw[4] = {gr[0], gr[1], gr[2], gr[3]};
#pragma unroll
            for (int p = 0; p < kP; ++p)
#pragma unroll
              for (int q = 0; q < 4; ++q) gw[q] = fmaf(hv[p], dp2[p][q], gw[q]);
#pragma unroll
            for (int q = 0; q < 4; ++q) gr[q] = gw[q];
          }
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            float sb = gb2[cl + q];
#pragma unroll
            for (int p = 0; p < kP; ++p) sb += dp2[p][q];
            gb2[cl + q] = sb;
          }
        }
        __syncwarp();
        // back to h1 (lanes own l = lane, lane + 32), then dp1
        float dh1[2][kP], dp1[2][kP];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int l = lane + 32 * h;
#pragma unroll
          for (int p = 0; p < kP; ++p) dh1[h][p] = dp1[h][p] = 0.0f;
          if (l < d2) {
#pragma unroll
            for (int p = 0; p < kP; ++p) dh1[h][p] = S.dg[l][p] + S.dg[l + d2][p];
            for (int q = 0; q < M; ++q) {
              const float W = __ldg(w.W2T + q * d2 + l);
              const float4 a0 = *reinterpret_cast<const float4*>(&S.dp2[q][0]);
              const float4 a1 = *reinterpret_cast<const float4*>(&S.dp2[q][4]);
              dh1[h][0] = fmaf(a0.x, W, dh1[h][0]);
              dh1[h][1] = fmaf(a0.y, W, dh1[h][1]);
              dh1[h][2] = fmaf(a0.z, W, dh1[h][2]);
              dh1[h][3] = fmaf(a0.w, W, dh1[h][3]);
              dh1[h][4] = fmaf(a1.x, W, dh1[h][4]);
              dh1[h][5] = fmaf(a1.y, W, dh1[h][5]);
              dh1[h][6] = fmaf(a1.z, W, dh1[h][6]);
              dh1[h][7] = fmaf(a1.w, W, dh1[h][7]);
            }
#pragma unroll
            for (int p = 0; p < kP; ++p) {
              const float t = S.t1[l][p];
              dp1[h][p] = dh1[h][p] * (1.0f - t * t);
            }
          }
        }
        __syncwarp();
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int l = lane + 32 * h;
          if (l < d2) {
#pragma unroll
            for (int p = 0; p < kP; ++p) {
              S.dp1[l][p] = dp1[h][p];
              S.h1[l][p] = dh1[h][p];  // h1 is no longer needed: keep dE/dh1 there
            }
            // layer 1: column l of W1 and b1
            float sb = gb1[l];
#pragma unroll
            for (int p = 0; p < kP; ++p) sb += dp1[h][p];
            gb1[l] = sb;
            for (int kk = 0; kk < d1; ++kk) {
              const float4 a0 = *reinterpret_cast<const float4*>(&S.h0[kk][0]);
              const float4 a1 = *reinterpret_cast<const float4*>(&S.h0[kk][4]);
              float gw = gW1[kk * d2 + l];
              gw = fmaf(a0.x, dp1[h][0], gw);
              gw = fmaf(a0.y, dp1[h][1], gw);
              gw = fmaf(a0.z, dp1[h][2], gw);
              gw = fmaf(a0.w, dp1[h][3], gw);
              gw = fmaf(a1.x, dp1[h][4], gw);
              gw = fmaf(a1.y, dp1[h][5], gw);
              gw = fmaf(a1.z, dp1[h][6], gw);
              gw = fmaf(a1.w, dp1[h][7], gw);
              gW1[kk * d2 + l] = gw;
            }
          }
        }
        __syncwarp();
        // back to h0 (lane = k), then layer 0
        if (lane < d1) {
          float dh0[kP];
#pragma unroll
          for (int p = 0; p < kP; ++p) dh0[p] = S.h1[lane][p] + S.h1[lane + d1][p];
          for (int mm = 0; mm < d2; ++mm) {
            const float W = __ldg(w.W1T + mm * d1 + lane);
            const float4 a0 = *reinterpret_cast<const float4*>(&S.dp1[mm][0]);
            const float4 a1 = *reinterpret_cast<const float4*>(&S.dp1[mm][4]);
            dh0[0] = fmaf(a0.x, W, dh0[0]);
            dh0[1] = fmaf(a0.y, W, dh0[1]);
            dh0[2] = fmaf(a0.z, W, dh0[2]);
            dh0[3] = fmaf(a0.w, W, dh0[3]);
            dh0[4] = fmaf(a1.x, W, dh0[4]);
            dh0[5] = fmaf(a1.y, W, dh0[5]);
            dh0[6] = fmaf(a1.z, W, dh0[6]);
            dh0[7] = fmaf(a1.w, W, dh0[7]);
          }
          float sw = gW0[lane], sb = gb0[lane];
#pragma unroll
          for (int p = 0; p < kP; ++p) {
            const float h0 = S.h0[lane][p];
            const float dp0 = dh0[p] * (1.0f - h0 * h0);
            sw = fmaf(sv[p], dp0, sw);
            sb += dp0;
          }
          gW0[lane] = sw;
          gb0[lane] = sb;
        }
        __syncwarp();
      }
    }
  }
  __syncwarp();
  float* dst = part + (size_t)blockIdx.x * npar;
  for (int e = lane; e < npar; e += 32) dst[e] = acc[e];
}

// g[e] += sum over the CTAs (in order) of part[cta][e], in FP64
__global__ void k_plain_wgrad_add(int nct, int npar, const float* __restrict__ part,
                                  double* __restrict__ g) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= npar) return;
  double s = 0.0;
  for (int k = 0; k < nct; ++k) s += (double)part[(size_t)k * npar + e];
  g[e] += s;
}

}  // namespace

int plain_kernel_slots(int64_t n) { return plain_blocks(n) * kWpb; }

int launch_plain_fwd(cudaStream_t st, int64_t n, const float4* off, const uint32_t* nlist,
                     const int32_t* nn, int cap, const CellGeom& g, const EnvParams& ep,
                     const void* nets, int d1, float* T, unsigned long long* pair_count) {
  if (n <= 0) return 0;
  if (!plain_shape_ok(ep, d1)) return -1;
  const size_t sm = sizeof(PlainFwdSmem) * kWpb;
  // float4 rows of W1 when its width 2 d1 is a multiple of 4
  const bool vec = (2 * d1) % 4 == 0;
  DP_LAUNCHED(1);
  if (vec)
    k_plain_fwd<true><<<plain_blocks(n), kWpb * 32, sm, st>>>(n, off, nlist, nn, cap, g, ep,
                                                            (const PlainNet*)nets, d1, T,
                                                            pair_count);
  else
    k_plain_fwd<false><<<plain_blocks(n), kWpb * 32, sm, st>>>(n, off, nlist, nn, cap, g, ep,
                                                             (const PlainNet*)nets, d1, T,
                                                             pair_count);
  return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

int launch_plain_bwd(cudaStream_t st, int64_t n, const float4* off, const uint32_t* nlist,
                     const int32_t* nn, int cap, const CellGeom& g, const EnvParams& ep,
                     const void* nets, int d1, const float* dT, unsigned long long* ffix,
                     double* vir_part, int vir_slots, int32_t* status) {
  if (n <= 0) return 0;
  if (!plain_shape_ok(ep, d1)) return -1;
  if (vir_slots < plain_kernel_slots(n)) return -1;
  const size_t sm = sizeof(PlainBwdSmem) * kWpb;
  // float4 rows of the transposed weights when the widths are multiples of 4
  const bool vec = (2 * d1) % 4 == 0;
  static std::atomic<bool> attr[2] = {{false}, {false}};  // launches from several host threads
  if (!attr[vec]) {
    if (cudaFuncSetAttribute(vec ? k_plain_bwd<true> : k_plain_bwd<false>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) != cudaSuccess)
      return -3;
    attr[vec] = true;
  }
  DP_LAUNCHED(1);
  if (vec)
    k_plain_bwd<true><<<plain_blocks(n), kWpb * 32, sm, st>>>(n, off, nlist, nn, cap, g, ep,
                                                            (const PlainNet*)nets, d1, dT, ffix,
                                                            vir_part, status);
  else
    k_plain_bwd<false><<<plain_blocks(n), kWpb * 32, sm, st>>>(n, off, nlist, nn, cap, g, ep,
                                                             (const PlainNet*)nets, d1, dT, ffix,
                                                             vir_part, status);
  return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

int plain_wgrad_params(int d1, int M) { return 2 * d1 + (d1 + 1) * 2 * d1 + (2 * d1 + 1) * M; }
int plain_wgrad_ctas() {
  int dev = 0, sms = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return 4 * (sms > 0 ? sms : 1);
}

int launch_plain_wgrad(cudaStream_t st, int64_t n, const float4* off, const uint32_t* nlist,
                       const int32_t* nn, int cap, const CellGeom& g, const EnvParams& ep,
                       const void* nets, int d1, const float* dT, int ti, int tj, float* part,
                       double* grad) {
  if (n <= 0) return 0;
  if (!plain_shape_ok(ep, d1)) return -1;
  const int npar = plain_wgrad_params(d1, ep.M);
  const size_t sm = (sizeof(PlainSmem) + 15) / 16 * 16 + sizeof(float) * (size_t)npar;
  static std::atomic<size_t> set{0};  // launches from several host threads
  if (sm > set) {
    if (cudaFuncSetAttribute(k_plain_wgrad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) !=
        cudaSuccess)
      return -3;
    set = sm;
  }
  const int grid = plain_wgrad_ctas();
  DP_LAUNCHED(2);
  k_plain_wgrad<<<grid, 32, sm, st>>>(n, off, nlist, nn, cap, g, ep, (const PlainNet*)nets, d1, dT,
                                      ti, tj, npar, part);
  k_plain_wgrad_add<<<(npar + 255) / 256, 256, 0, st>>>(grid, npar, part, grad);
  return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

size_t plain_net_bytes() { return sizeof(PlainNet); }

// pointers of a PlainNet record, in field order
// returns false unless W2 and b2 (read as float4) start on 16-byte boundaries
bool plain_net_fill(void* rec, const float* W0, const float* b0, const float* W1, const float* b1,
                    const float* W2, const float* b2, const float* W1T, const float* W2T) {
  PlainNet* r = (PlainNet*)rec;
  r->W0 = W0;
  r->b0 = b0;
  r->W1 = W1;
  r->b1 = b1;
  r->W2 = W2;
  r->b2 = b2;
  r->W1T = W1T;
  r->W2T = W2T;
  return ((uintptr_t)W2 % 16 == 0) && ((uintptr_t)b2 % 16 == 0);
}
