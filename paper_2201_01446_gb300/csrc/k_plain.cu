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
__global__ void __launch_bounds__(kWpb * 32) k_plain_fwd(int64_t n, const float4* __restrict__ off,
                                                         const uint32_t* __restrict__ nlist,
                                                         const int32_t* __restrict__ nn, int cap,
                                                         CellGeom g, EnvParams ep,
                                                         const PlainNet* __restrict__ nets, int d1,
                                                         float* __restrict__ T,
                                                         unsigned long long* __restrict__ pair_count) {
  extern __shared__ float4 smem4[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  PlainSmem& S = reinterpret_cast<PlainSmem*>(smem4)[wib];
  const int M = ep.M, nt = ep.ntypes;
  const int cl = lane * 4;
  const unsigned below = (1u << lane) - 1u;
  unsigned long long npairs = 0;
  for (int64_t i = (int64_t)blockIdx.x * kWpb + wib; i < n; i += (int64_t)gridDim.x * kWpb) {
    const float4 oi = off[i];
    const int ti = __float_as_int(oi.w);
    const int cnt = min(nn[i], cap);
    const uint32_t* L = nlist + (size_t)i * cap;
    float acc[4][4];
#pragma unroll
    for (int c = 0; c < 4; ++c)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[c][q] = 0.0f;
    for (int tj = 0; tj < nt; ++tj) {
      const PlainNet w = nets[ti * nt + tj];
      for (int b0 = 0; b0 < cnt; b0 += 32) {
        const int k = b0 + lane;
        bool in = false;
        float s = 0.f, dsdr, ir, dx = 0.f, dy = 0.f, dz = 0.f;
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
        npairs += c;
        for (int p0 = 0; p0 < c; p0 += kP) {
          float sv[kP];
#pragma unroll
          for (int p = 0; p < kP; ++p) sv[p] = p0 + p < c ? S.s[p0 + p] : 0.0f;
          plain_layers01(w, d1, S, sv, lane);
          float G[kP][4], t2[kP][4];
          plain_layer2(w, d1, M, S, lane, G, t2);
#pragma unroll
          for (int p = 0; p < kP; ++p) {
            if (p0 + p >= c) break;
            const float4 R = *reinterpret_cast<const float4*>(S.R[p0 + p]);
            const float rv[4] = {R.x, R.y, R.z, R.w};
#pragma unroll
            for (int cc = 0; cc < 4; ++cc)
#pragma unroll
              for (int q = 0; q < 4; ++q) acc[cc][q] = fmaf(rv[cc], G[p][q], acc[cc][q]);
          }
          __syncwarp();
        }
      }
    }
    if (cl < M) {
      float* Ti = T + (size_t)i * 4 * M + cl;
#pragma unroll
      for (int cc = 0; cc < 4; ++cc)
        *reinterpret_cast<float4*>(Ti + cc * M) =
            make_float4(acc[cc][0] * ep.inv_nm, acc[cc][1] * ep.inv_nm, acc[cc][2] * ep.inv_nm,
                        acc[cc][3] * ep.inv_nm);
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

// ------------------------------------------------------------------ backward
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
  PlainSmem& S = reinterpret_cast<PlainSmem*>(smem4)[wib];
  const int M = ep.M, nt = ep.ntypes, d2 = 2 * d1;
  const int cl = lane * 4;
  const unsigned below = (1u << lane) - 1u;
  double vacc[9];
#pragma unroll
  for (int a = 0; a < 9; ++a) vacc[a] = 0.0;
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
      for (int b0 = 0; b0 < cnt; b0 += 32) {
        const int k = b0 + lane;
        bool in = false;
        float s = 0.f, dsdr = 0.f, ir = 0.f, dx = 0.f, dy = 0.f, dz = 0.f;
        uint32_t e = 0;
        if (k < cnt) {
          int t;
          e = L[k];
          load_pair_p(oi, off, g, e, dx, dy, dz, t);
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
          S.geo[slot][0] = dsdr;
          S.geo[slot][1] = ir;
          S.geo[slot][2] = dx;
          S.geo[slot][3] = dy;
          S.geo[slot][4] = dz;
          S.jj[slot] = (int)(e >> 5);
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
          // dE/dG (lane's columns), dE/d(pre2), partial dE/dR over the columns
          float part[32];
#pragma unroll
          for (int p = 0; p < kP; ++p) {
            float4 R = *reinterpret_cast<const float4*>(S.R[p0 + p < c ? p0 + p : p0]);
            if (p0 + p >= c) R = make_float4(0.f, 0.f, 0.f, 0.f);
            const float rv[4] = {R.x, R.y, R.z, R.w};
#pragma unroll
            for (int cc = 0; cc < 4; ++cc) {
              float acc = 0.0f;
#pragma unroll
              for (int q = 0; q < 4; ++q) acc = fmaf(dTv[cc][q], G[p][q], acc);
              part[p * 4 + cc] = acc;
            }
            if (cl < M) {
#pragma unroll
              for (int q = 0; q < 4; ++q) {
                float dg = 0.0f;
#pragma unroll
                for (int cc = 0; cc < 4; ++cc) dg = fmaf(dTv[cc][q], rv[cc], dg);
                dg *= ep.inv_nm;
                S.dg[cl + q][p] = dg;
                S.dp2[cl + q][p] = dg * (1.0f - t2[p][q] * t2[p][q]);
              }
            }
          }
          const float dRtot = transpose_sum32(part, lane) * ep.inv_nm;  // (p, c) = (lane/4, lane%4)
          __syncwarp();
          // layer 2 backward: lanes own l = lane, lane + 32
          float dh1[2][kP];
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int l = lane + 32 * h;
#pragma unroll
            for (int p = 0; p < kP; ++p) dh1[h][p] = 0.0f;
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
            }
          }
          __syncwarp();
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int l = lane + 32 * h;
            if (l < d2) {
#pragma unroll
              for (int p = 0; p < kP; ++p) {
                const float t = S.t1[l][p];
                S.dp1[l][p] = dh1[h][p] * (1.0f - t * t);
                S.h1[l][p] = dh1[h][p];  // h1 is no longer needed: keep dE/dh1 there
              }
            }
          }
          __syncwarp();
          // layer 1 backward and layer 0: lanes own k = lane
          float dsp[kP];
#pragma unroll
          for (int p = 0; p < kP; ++p) dsp[p] = 0.0f;
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
            const float W0 = w.W0[lane];
#pragma unroll
            for (int p = 0; p < kP; ++p) {
              const float h0 = S.h0[lane][p];
              dsp[p] = W0 * dh0[p] * (1.0f - h0 * h0);
            }
          }
#pragma unroll
          for (int o = 16; o >= 1; o >>= 1)
#pragma unroll
            for (int p = 0; p < kP; ++p) dsp[p] += __shfl_xor_sync(0xffffffffu, dsp[p], o);
          // per pair: chain rule through Eq. 1, one pair per lane (lanes 0..kP-1)
          float gR[4];
#pragma unroll
          for (int cc = 0; cc < 4; ++cc) gR[cc] = __shfl_sync(0xffffffffu, dRtot, (4 * lane + cc) & 31);
          float gsv = dsp[0];
#pragma unroll
          for (int p = 1; p < kP; ++p) gsv = lane == p ? dsp[p] : gsv;
          const int pp = p0 + lane;
          if (lane < kP && pp < c) {
            const float sgeo = S.s[pp];
            const float dsr = S.geo[pp][0], irr = S.geo[pp][1];
            const float ddx = S.geo[pp][2], ddy = S.geo[pp][3], ddz = S.geo[pp][4];
            const float ux = ddx * irr, uy = ddy * irr, uz = ddz * irr;
            const float a0 = gR[0] + gsv;
            const float dot = gR[1] * ux + gR[2] * uy + gR[3] * uz;
            const float sor = sgeo * irr;
            const float coef = dsr * (a0 + dot) - sor * dot;
            float gx = coef * ux + sor * gR[1];
            float gy = coef * uy + sor * gR[2];
            float gz = coef * uz + sor * gR[3];
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
            unsigned long long* fj = ffix + (size_t)S.jj[pp] * 3;
            atomicAdd(fj + 0, (unsigned long long)(-__float2ll_rn(gx * DP_FSCALE_F)));
            atomicAdd(fj + 1, (unsigned long long)(-__float2ll_rn(gy * DP_FSCALE_F)));
            atomicAdd(fj + 2, (unsigned long long)(-__float2ll_rn(gz * DP_FSCALE_F)));
          }
          __syncwarp();
        }
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
      for (int a = 0; a < 9; ++a) vacc[a] += red[3 + a];
    }
  }
  if (lane == 0) {
    double* vp = vir_part + ((size_t)blockIdx.x * kWpb + wib) * 9;
#pragma unroll
    for (int a = 0; a < 9; ++a) vp[a] = vacc[a];
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
  const size_t sm = sizeof(PlainSmem) * kWpb;
  static std::atomic<bool> attr{false};  // launches from several host threads
  if (!attr) {
    cudaFuncSetAttribute(k_plain_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    attr = true;
  }
  DP_LAUNCHED(1);
  k_plain_fwd<<<plain_blocks(n), kWpb * 32, sm, st>>>(n, off, nlist, nn, cap, g, ep,
                                                      (const PlainNet*)nets, d1, T, pair_count);
  return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

int launch_plain_bwd(cudaStream_t st, int64_t n, const float4* off, const uint32_t* nlist,
                     const int32_t* nn, int cap, const CellGeom& g, const EnvParams& ep,
                     const void* nets, int d1, const float* dT, unsigned long long* ffix,
                     double* vir_part, int vir_slots, int32_t* status) {
  if (n <= 0) return 0;
  if (!plain_shape_ok(ep, d1)) return -1;
  if (vir_slots < plain_kernel_slots(n)) return -1;
  const size_t sm = sizeof(PlainSmem) * kWpb;
  static std::atomic<bool> attr{false};  // launches from several host threads
  if (!attr) {
    cudaFuncSetAttribute(k_plain_bwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    attr = true;
  }
  DP_LAUNCHED(1);
  k_plain_bwd<<<plain_blocks(n), kWpb * 32, sm, st>>>(n, off, nlist, nn, cap, g, ep,
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
