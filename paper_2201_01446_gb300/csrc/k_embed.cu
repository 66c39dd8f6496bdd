// Tabulated embedding net fused with the environment-matrix contraction
// (paper Sec. 3.2 tabulation, Sec. 3.3/3.4.1 kernel fusion, Sec. 3.4.2
// redundancy removal) and its backward pass down to the forces and virial.
//
// Forward, per atom i (Eq. 1, Eq. 2):
//   T_i[c][:] = (1/N_m) sum_{j: r_ij < rc} R_ij[c] g(s_ij),
//   R_ij = s (1, x/r, y/r, z/r), s = sw(r)/r,
// with g(s) on interval k given by the quintic sum_q c[k][q][:] u^q,
// u = s/h - k.  Regrouping the sum by interval (exact in real arithmetic),
//   T_i[c][:] = sum_k sum_q C_k[c][q] c[k][q][:],  C_k[c][q] = (1/N_m) sum_{j in k} R_ij[c] u_j^q,
// so the table row of an interval is read once per atom however many
// neighbors fall in it.  G is never formed, pairs beyond rc (the padding of
// the paper's N_m rows) cost nothing.
//
// Backward, given dT = dE_i/dT_i:
//   B_k[c][q] = (1/N_m) sum_eta c[k][q][eta] dT[c][eta]          (per occupied interval)
//   dE/dR_ij[c] = sum_q B_k[c][q] u^q,
//   dE/ds_ij (through g) = (1/h) sum_c R_ij[c] sum_q q B_k[c][q] u^(q-1),
//   g_ij = dE_i/dr_ij by the chain rule through Eq. 1,
//   F_i += g_ij, F_j -= g_ij, virial -= r_ij (x) g_ij.
// Forces go to int64 fixed-point accumulators (associative, deterministic);
// the virial to per-warp FP64 partials summed later in a fixed order.
#include <atomic>
#include <math.h>

#include "dp_internal.h"
#include "embed_common.cuh"

namespace {
using namespace dp_embed;

// ------------------------------------------------------------------ table
// One CTA per (type pair, node): the embedding net (Eq. 3-5) and its first
// and second derivative in s, by forward-mode propagation in FP64.
__global__ void k_table_nodes(const double* __restrict__ emb, const int64_t* __restrict__ emb_off,
                              int n_emb, int w0, int w1, int w2, int w3, int w4, int w5, double h,
                              int n_fine, double H, int n_nodes, double* __restrict__ node) {
  extern __shared__ double sm[];
  const int p = blockIdx.x / n_nodes, k = blockIdx.x % n_nodes;
  const int widths[6] = {w0, w1, w2, w3, w4, w5};
  int wmax = 0;
  for (int l = 0; l < n_emb; ++l) wmax = max(wmax, widths[l]);
  double* cur = sm;                 // [3][wmax]
  double* nxt = sm + 3 * wmax;      // [3][wmax]
  // node k: k h up to n_fine, then steps of H (the extrapolation region)
  const double s = k <= n_fine ? k * h : n_fine * h + (k - n_fine) * H;
  const int c = threadIdx.x;
  {
    const double* W = emb + emb_off[p * n_emb + 0];
    const double* b = W + widths[0];
    if (c < widths[0]) {
      double z = fma(s, W[c], b[c]), zp = W[c];
      double t = tanh(z), q = 1.0 - t * t;
      cur[c] = t;
      cur[wmax + c] = q * zp;
      cur[2 * wmax + c] = -2.0 * t * q * zp * zp;
    }
  }
  __syncthreads();
  int w = widths[0];
  for (int l = 1; l < n_emb; ++l) {
    const int wo = widths[l];
    const double* W = emb + emb_off[p * n_emb + l];
    const double* b = W + (size_t)w * wo;
    if (c < wo) {
      double z = b[c], zp = 0.0, zpp = 0.0;
      for (int r = 0; r < w; ++r) {
        double wk = W[(size_t)r * wo + c];
        z = fma(cur[r], wk, z);
        zp = fma(cur[wmax + r], wk, zp);
        zpp = fma(cur[2 * wmax + r], wk, zpp);
      }
      double t = tanh(z), q = 1.0 - t * t;
      int src = c - (c / w) * w;  // (x, x): output c repeats input c mod w
      nxt[c] = cur[src] + t;
      nxt[wmax + c] = cur[wmax + src] + q * zp;
      nxt[2 * wmax + c] = cur[2 * wmax + src] + q * zpp - 2.0 * t * q * zp * zp;
    }
    __syncthreads();
    double* tmp = cur;
    cur = nxt;
    nxt = tmp;
    w = wo;
  }
  if (c < w) {
    double* out = node + ((size_t)p * n_nodes + k) * 3 * w;
    out[c] = cur[c];
    out[w + c] = cur[wmax + c];
    out[2 * w + c] = cur[2 * wmax + c];
  }
}

// Quintic on u in [0,1] with f, f', f'' given at both ends (derivatives in u,
// i.e. the s-derivatives times the interval width w and w^2; w = h, or H
// in the extrapolation region).  With A, B, C the residuals of the value,
// slope and curvature left at u = 1 by the first three coefficients, the
// last three solve  p+q+w = A, 3p+4q+5w = B, 6p+12q+20w = C.
__global__ void k_table_coef(const double* __restrict__ node, int npair, int n_int, int M,
                             double h_fine, int n_fine, double H, float* __restrict__ table) {
  int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)npair * n_int * M) return;
  const int c = idx % M;
  const int k = (idx / M) % n_int;
  const int p = idx / ((int64_t)M * n_int);
  const double h = k < n_fine ? h_fine : H;
  const double* n0 = node + ((size_t)p * (n_int + 1) + k) * 3 * M;
  const double* n1 = n0 + 3 * M;
  const double f0 = n0[c], d0 = n0[M + c] * h, e0 = n0[2 * M + c] * h * h;
  const double f1 = n1[c], d1 = n1[M + c] * h, e1 = n1[2 * M + c] * h * h;
  const double A = f1 - f0 - d0 - 0.5 * e0;
  const double B = d1 - d0 - e0;
  const double C = e1 - e0;
  double q[6];
  q[0] = f0;
  q[1] = d0;
  q[2] = 0.5 * e0;
  q[3] = 10.0 * A - 4.0 * B + 0.5 * C;
  q[4] = -15.0 * A + 7.0 * B - C;
  q[5] = 6.0 * A - 3.0 * B + 0.5 * C;
  float* out = table + ((size_t)p * n_int + k) * 6 * M;
  for (int r = 0; r < 6; ++r) out[r * M + c] = (float)q[r];
}

__host__ __device__ inline int fwd_warp_words(int nbins, int scap) {
  return round4(nbins) + 4 * scap + round4(scap) + 32;
}
__host__ __device__ inline int bwd_warp_words(int nbins, int scap) {
  return round4(nbins) + round4(scap) + 32 * 24 + 2 * 10;
}

// ------------------------------------------------------------------ forward
__global__ void __launch_bounds__(256, 3) k_tab_fwd(int64_t n, const float4* __restrict__ off,
                                                 const uint32_t* __restrict__ nlist,
                                                 const int32_t* __restrict__ nn, int cap, CellGeom g,
                                                 EnvParams ep, const float* __restrict__ table,
                                                 int scap, float* __restrict__ T,
                                                 int32_t* __restrict__ status,
                                                 unsigned long long* __restrict__ pair_count) {
  extern __shared__ float4 smem4[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, wpb = blockDim.x >> 5;
  const int nt = ep.ntypes, n_int = ep.n_int, M = ep.M;
  const int nbins = nt * n_int;
  float* base = (float*)smem4 + (size_t)wib * fwd_warp_words(nbins, scap);
  int* hist = (int*)base;
  float4* sR = (float4*)(base + round4(nbins));
  float* sU = base + round4(nbins) + 4 * scap;
  float* Cb = sU + round4(scap);
  const int cl = lane * 4;
  const bool colok = cl < M;
  int nrange = 0, nover = 0;
  unsigned long long npairs = 0;
  for (int64_t i = (int64_t)blockIdx.x * wpb + wib; i < n; i += (int64_t)gridDim.x * wpb) {
    const float4 oi = off[i];
    const int ti = __float_as_int(oi.w);
    const int cnt = min(nn[i], cap);
    const uint32_t* L = nlist + (size_t)i * cap;
    for (int b = lane; b < nbins; b += 32) hist[b] = 0;
    __syncwarp();
    // pass 1: histogram of bins
    int np = 0;
    for (int b0 = 0; b0 < cnt; b0 += 32) {
      const int k = b0 + lane;
      bool in = false;
      if (k < cnt) {
        float dx, dy, dz;
        int tj;
        load_pair(oi, off, g, L[k], dx, dy, dz, tj);
        const float r2 = dx * dx + dy * dy + dz * dz;
        if (r2 < ep.rc2) {
          Pair P;
          pair_geom(ep, dx, dy, dz, r2, tj, P);
          atomicAdd(&hist[tj * n_int + P.th], 1);
          nrange += P.out_of_range;
          in = true;
        }
      }
      np += __popc(__ballot_sync(0xffffffffu, in));
    }
    __syncwarp();
    npairs += np;
    float acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[a][q] = 0.0f;
    if (np <= scap) {
      warp_exclusive_scan(hist, nbins, lane);
      // pass 2: stable scatter of (R, u) into bin order
      for (int b0 = 0; b0 < cnt; b0 += 32) {
        const int k = b0 + lane;
        bool in = false;
        Pair P;
        int bin = 0;
        if (k < cnt) {
          float dx, dy, dz;
          int tj;
          load_pair(oi, off, g, L[k], dx, dy, dz, tj);
          const float r2 = dx * dx + dy * dy + dz * dz;
          if (r2 < ep.rc2) {
            pair_geom(ep, dx, dy, dz, r2, tj, P);
            bin = tj * n_int + P.th;
            in = true;
          }
        }
        const int pos = sorted_slot(hist, in, bin, lane);
        if (in) {
          sR[pos] = make_float4(P.s, P.s * P.dx * P.ir, P.s * P.dy * P.ir, P.s * P.dz * P.ir);
          sU[pos] = P.u;
        }
      }
      __syncwarp();
      // per occupied bin: C[c][q] = sum over members R[c] u^q, then T += C . table row
      const int cc = lane / 6, qq = lane - (lane / 6) * 6;
      for (int b0 = 0; b0 < nbins; b0 += 32) {
        const int bl = b0 + lane;
        const bool occ = bl < nbins && hist[bl] > bin_begin(hist, bl);
        unsigned bits = __ballot_sync(0xffffffffu, occ);
        while (bits) {
          const int bin = b0 + __ffs(bits) - 1;
          bits &= bits - 1u;
          const int s0 = bin_begin(hist, bin), s1 = hist[bin];
          if (lane < 24) {
            float cacc = 0.0f;
            for (int k = s0; k < s1; ++k) {
              const float4 R = sR[k];
              const float u = sU[k];
              const float u2 = u * u;
              const float pw = qq == 0 ? 1.0f
                             : qq == 1 ? u
                             : qq == 2 ? u2
                             : qq == 3 ? u2 * u
                             : qq == 4 ? u2 * u2 : u2 * u2 * u;
              const float rv = cc == 0 ? R.x : (cc == 1 ? R.y : (cc == 2 ? R.z : R.w));
              cacc = fmaf(rv, pw, cacc);
            }
            Cb[lane] = cacc;
          }
          __syncwarp();
          if (colok) {
            float Cv[24];
#pragma unroll
            for (int v = 0; v < 6; ++v) {
              const float4 t4 = reinterpret_cast<const float4*>(Cb)[v];
              Cv[4 * v] = t4.x;
              Cv[4 * v + 1] = t4.y;
              Cv[4 * v + 2] = t4.z;
              Cv[4 * v + 3] = t4.w;
            }
            const float* tp = table + ((size_t)ti * nbins + bin) * 6 * M + cl;
#pragma unroll
            for (int q = 0; q < 6; ++q) {
              const float4 a = __ldg(reinterpret_cast<const float4*>(tp + q * M));
#pragma unroll
              for (int c = 0; c < 4; ++c) {
                const float cv = Cv[c * 6 + q];
                acc[c][0] = fmaf(cv, a.x, acc[c][0]);
                acc[c][1] = fmaf(cv, a.y, acc[c][1]);
                acc[c][2] = fmaf(cv, a.z, acc[c][2]);
                acc[c][3] = fmaf(cv, a.w, acc[c][3]);
              }
            }
          }
          __syncwarp();
        }
      }
    } else {
      ++nover;  // more pairs within rc than N_m + 32: an overflow of sel
    }
    if (colok) {
      float* Ti = T + (size_t)i * 4 * M + cl;
#pragma unroll
      for (int c = 0; c < 4; ++c)
        *reinterpret_cast<float4*>(Ti + c * M) =
            make_float4(acc[c][0] * ep.inv_nm, acc[c][1] * ep.inv_nm, acc[c][2] * ep.inv_nm,
                        acc[c][3] * ep.inv_nm);
    }
    __syncwarp();
  }
  nrange = __reduce_add_sync(0xffffffffu, nrange);
  if (lane == 0 && nrange) atomicAdd(&status[ST_RANGE], nrange);
  if (lane == 0 && nover) atomicAdd(&status[ST_SEL], nover);
  if (lane == 0 && pair_count) atomicAdd(pair_count, npairs);
}

// ------------------------------------------------------------------ backward
__global__ void __launch_bounds__(256, 3) k_tab_bwd(int64_t n, const float4* __restrict__ off,
                                                 const uint32_t* __restrict__ nlist,
                                                 const int32_t* __restrict__ nn, int cap, CellGeom g,
                                                 EnvParams ep, const float* __restrict__ table,
                                                 int scap, const float* __restrict__ dT,
                                                 unsigned long long* __restrict__ ffix,
                                                 double* __restrict__ vir_part,
                                                 int32_t* __restrict__ status) {
  extern __shared__ float4 smem4[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, wpb = blockDim.x >> 5;
  const int nt = ep.ntypes, n_int = ep.n_int, M = ep.M;
  const int nbins = nt * n_int;
  float* base = (float*)smem4 + (size_t)wib * bwd_warp_words(nbins, scap);
  int* hist = (int*)base;
  int* sK = (int*)(base + round4(nbins));
  float* Bb = base + round4(nbins) + round4(scap);  // [32 bins][24]
  double* vacc = reinterpret_cast<double*>(Bb + 32 * 24);  // [9] per warp
  // lane (c, grp): c = lane / 8 picks the row of dT, grp the 16 columns it sums
  const int lc = lane >> 3, lg = lane & 7;
  const int col0 = lg * 16;
  if (lane < 9) vacc[lane] = 0.0;
  __syncwarp();
  int nbad = 0;
  for (int64_t i = (int64_t)blockIdx.x * wpb + wib; i < n; i += (int64_t)gridDim.x * wpb) {
    const float4 oi = off[i];
    const int ti = __float_as_int(oi.w);
    const int cnt = min(nn[i], cap);
    const uint32_t* L = nlist + (size_t)i * cap;
    for (int b = lane; b < nbins; b += 32) hist[b] = 0;
    __syncwarp();
    int np = 0;
    for (int b0 = 0; b0 < cnt; b0 += 32) {
      const int k = b0 + lane;
      bool in = false;
      if (k < cnt) {
        float dx, dy, dz;
        int tj;
        load_pair(oi, off, g, L[k], dx, dy, dz, tj);
        const float r2 = dx * dx + dy * dy + dz * dz;
        if (r2 < ep.rc2) {
          Pair P;
          pair_geom(ep, dx, dy, dz, r2, tj, P);
          atomicAdd(&hist[tj * n_int + P.th], 1);
          in = true;
        }
      }
      np += __popc(__ballot_sync(0xffffffffu, in));
    }
    __syncwarp();
    float fx = 0.f, fy = 0.f, fz = 0.f;
    float vl[9];
#pragma unroll
    for (int a = 0; a < 9; ++a) vl[a] = 0.f;
    if (np <= scap) {
      warp_exclusive_scan(hist, nbins, lane);
      for (int b0 = 0; b0 < cnt; b0 += 32) {
        const int k = b0 + lane;
        bool in = false;
        int bin = 0;
        if (k < cnt) {
          float dx, dy, dz;
          int tj;
          load_pair(oi, off, g, L[k], dx, dy, dz, tj);
          const float r2 = dx * dx + dy * dy + dz * dz;
          if (r2 < ep.rc2) {
            Pair P;
            pair_geom(ep, dx, dy, dz, r2, tj, P);
            bin = tj * n_int + P.th;
            in = true;
          }
        }
        const int pos = sorted_slot(hist, in, bin, lane);
        if (in) sK[pos] = k | (bin << 16);
      }
      __syncwarp();
      // this lane's slice of dT: row lc, columns col0 .. col0+15
      float4 dTv[4];
#pragma unroll
      for (int v = 0; v < 4; ++v)
        dTv[v] = (col0 + 4 * v < M)
                     ? *reinterpret_cast<const float4*>(dT + (size_t)i * 4 * M + lc * M + col0 + 4 * v)
                     : make_float4(0.f, 0.f, 0.f, 0.f);
      for (int r0 = 0; r0 < nbins; r0 += 32) {
        const int sb = bin_begin(hist, r0), eb = hist[min(r0 + 32, nbins) - 1];
        if (eb == sb) continue;
        const int bl = r0 + lane;
        const bool occ = bl < nbins && hist[bl] > bin_begin(hist, bl);
        unsigned bits = __ballot_sync(0xffffffffu, occ);
        // B_k[c][q] = (1/N_m) sum_eta c[k][q][eta] dT[c][eta] for every occupied bin
        while (bits) {
          const int bo = __ffs(bits) - 1;
          bits &= bits - 1u;
          const float* tp = table + ((size_t)ti * nbins + r0 + bo) * 6 * M + col0;
          float v[8];
#pragma unroll
          for (int q = 0; q < 6; ++q) {
            float sacc = 0.0f;
#pragma unroll
            for (int w = 0; w < 4; ++w) {
              if (col0 + 4 * w < M) {
                const float4 a = __ldg(reinterpret_cast<const float4*>(tp + q * M + 4 * w));
                sacc = fmaf(a.x, dTv[w].x, sacc);
                sacc = fmaf(a.y, dTv[w].y, sacc);
                sacc = fmaf(a.z, dTv[w].z, sacc);
                sacc = fmaf(a.w, dTv[w].w, sacc);
              }
            }
            v[q] = sacc;
          }
          v[6] = 0.0f;
          v[7] = 0.0f;
          // sum over the 8 column groups; lane (c, grp) keeps q = grp
#pragma unroll
          for (int o = 4; o >= 1; o >>= 1) {
            const bool hi = (lane & o) != 0;
#pragma unroll
            for (int k = 0; k < o; ++k) {
              const float send = hi ? v[k] : v[k + o];
              const float keep = hi ? v[k + o] : v[k];
              v[k] = keep + __shfl_xor_sync(0xffffffffu, send, o);
            }
          }
          if (lg < 6) Bb[bo * 24 + lc * 6 + lg] = v[0] * ep.inv_nm;
        }
        __syncwarp();
        // members of this round's bins, one pair per lane
        for (int k0 = sb; k0 < eb; k0 += 32) {
          const int k = k0 + lane;
          if (k < eb) {
            const int key = sK[k];
            const uint32_t e = L[key & 0xffff];
            const int bo = (key >> 16) - r0;
            float dx, dy, dz;
            int tj;
            load_pair(oi, off, g, e, dx, dy, dz, tj);
            const float r2 = dx * dx + dy * dy + dz * dz;
            Pair P;
            pair_geom(ep, dx, dy, dz, r2, tj, P);
            const float* Bk = Bb + bo * 24;
            float Bv[24];
#pragma unroll
            for (int q = 0; q < 6; ++q) {
              const float4 t4 = reinterpret_cast<const float4*>(Bk)[q];
              Bv[4 * q] = t4.x;
              Bv[4 * q + 1] = t4.y;
              Bv[4 * q + 2] = t4.z;
              Bv[4 * q + 3] = t4.w;
            }
            const float u = P.u;
            float gR[4], dgu[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) {
              const float* b = Bv + c * 6;
              gR[c] = fmaf(fmaf(fmaf(fmaf(fmaf(b[5], u, b[4]), u, b[3]), u, b[2]), u, b[1]), u, b[0]);
              dgu[c] = fmaf(fmaf(fmaf(fmaf(5.0f * b[5], u, 4.0f * b[4]), u, 3.0f * b[3]), u,
                                  2.0f * b[2]),
                             u, b[1]);
            }
            const float ux = P.dx * P.ir, uy = P.dy * P.ir, uz = P.dz * P.ir;
            const float s = P.s;
            const float gs =
                interval_du_ds(ep, P.th) * s * (dgu[0] + ux * dgu[1] + uy * dgu[2] + uz * dgu[3]);
            const float a0 = gR[0] + gs;
            const float dot = gR[1] * ux + gR[2] * uy + gR[3] * uz;
            const float sor = s * P.ir;
            const float coef = P.dsdr * (a0 + dot) - sor * dot;
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
            vl[0] -= P.dx * gx;
            vl[1] -= P.dx * gy;
            vl[2] -= P.dx * gz;
            vl[3] -= P.dy * gx;
            vl[4] -= P.dy * gy;
            vl[5] -= P.dy * gz;
            vl[6] -= P.dz * gx;
            vl[7] -= P.dz * gy;
            vl[8] -= P.dz * gz;
            unsigned long long* fj = ffix + (size_t)(e >> 5) * 3;
            atomicAdd(fj + 0, (unsigned long long)(-__float2ll_rn(gx * DP_FSCALE_F)));
            atomicAdd(fj + 1, (unsigned long long)(-__float2ll_rn(gy * DP_FSCALE_F)));
            atomicAdd(fj + 2, (unsigned long long)(-__float2ll_rn(gz * DP_FSCALE_F)));
          }
        }
        __syncwarp();
      }
    } else {
      ++nbad;
    }
    // the centre's own force: lane partials (a few pairs each, FP32) summed
    // across the warp in FP64, where the pair terms largely cancel
    double red[3] = {fx, fy, fz};
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1)
#pragma unroll
      for (int a = 0; a < 3; ++a) red[a] += __shfl_xor_sync(0xffffffffu, red[a], o);
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1)
#pragma unroll
      for (int a = 0; a < 9; ++a) vl[a] += __shfl_xor_sync(0xffffffffu, vl[a], o);
    if (lane == 0) {
      unsigned long long* fi = ffix + (size_t)i * 3;
      atomicAdd(fi + 0, (unsigned long long)__double2ll_rn(red[0] * DP_FSCALE));
      atomicAdd(fi + 1, (unsigned long long)__double2ll_rn(red[1] * DP_FSCALE));
      atomicAdd(fi + 2, (unsigned long long)__double2ll_rn(red[2] * DP_FSCALE));
    }
    if (lane < 9) {
      float vv = vl[0];
#pragma unroll
      for (int a = 1; a < 9; ++a) vv = lane == a ? vl[a] : vv;
      vacc[lane] += (double)vv;
    }
    __syncwarp();
  }
  __syncwarp();
  if (lane < 9) vir_part[((size_t)blockIdx.x * wpb + wib) * 9 + lane] = vacc[lane];
  nbad = __reduce_add_sync(0xffffffffu, nbad);
  if (lane == 0 && nbad) atomicAdd(&status[ST_NONFINITE], nbad);
}

int g_num_sms = 0;
int num_sms() {
  if (!g_num_sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (g_num_sms <= 0) g_num_sms = 1;
  }
  return g_num_sms;
}

constexpr int kWarpsPerBlock = 8;

int tab_blocks(int64_t n) {
  int64_t want = (n + kWarpsPerBlock - 1) / kWarpsPerBlock;
  int64_t cap = (int64_t)num_sms() * 8;
  return (int)(want < cap ? (want > 0 ? want : 1) : cap);
}

int stage_cap(const EnvParams& ep) { return ((int)(1.0f / ep.inv_nm + 0.5f) + 32 + 31) / 32 * 32; }

size_t fwd_smem(const EnvParams& ep) {
  return (size_t)kWarpsPerBlock * fwd_warp_words(ep.ntypes * ep.n_int, stage_cap(ep)) * sizeof(float);
}
size_t bwd_smem(const EnvParams& ep) {
  return (size_t)kWarpsPerBlock * bwd_warp_words(ep.ntypes * ep.n_int, stage_cap(ep)) * sizeof(float);
}

}  // namespace

int tab_kernel_slots(int64_t n) { return tab_blocks(n) * kWarpsPerBlock; }

int table_build(cudaStream_t st, const double* emb64, const int64_t* emb_off, int n_emb,
                const int* emb_w, int npair, double h, int n_int, int n_fine, double H,
                float* table_out) {
  if (n_emb < 1 || n_emb > 6) return -1;
  int w[6] = {0, 0, 0, 0, 0, 0};
  int wmax = 0;
  for (int l = 0; l < n_emb; ++l) {
    w[l] = emb_w[l];
    wmax = wmax > w[l] ? wmax : w[l];
  }
  if (wmax > 1024) return -1;
  const int M = w[n_emb - 1];
  const int n_nodes = n_int + 1;
  double* node = nullptr;
  if (cudaMallocAsync(&node, sizeof(double) * (size_t)npair * n_nodes * 3 * M, st) != cudaSuccess)
    return -2;
  int threads = ((wmax + 31) / 32) * 32;
  DP_LAUNCHED(2);
  k_table_nodes<<<npair * n_nodes, threads, sizeof(double) * 6 * wmax, st>>>(
      emb64, emb_off, n_emb, w[0], w[1], w[2], w[3], w[4], w[5], h, n_fine, H, n_nodes, node);
  int64_t tot = (int64_t)npair * n_int * M;
  k_table_coef<<<(int)((tot + 255) / 256), 256, 0, st>>>(node, npair, n_int, M, h, n_fine, H,
                                                         table_out);
  cudaFreeAsync(node, st);
  return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

int launch_tab_fwd(cudaStream_t st, int64_t n, const float4* off, const uint32_t* nlist,
                   const int32_t* nn, int cap, const CellGeom& g, const EnvParams& ep,
                   const float* table, float* T, int32_t* status,
                   unsigned long long* pair_count) {
  if (n <= 0) return 0;
  if (ep.M > 128 || ep.M % 4 || ep.ntypes * ep.n_int > 32768) return -1;
  size_t sm = fwd_smem(ep);
  if (sm > 200 * 1024) return -1;
  static std::atomic<size_t> set_fwd{0};  // launches from several host threads
  if (sm > 48 * 1024 && sm > set_fwd) {
    cudaFuncSetAttribute(k_tab_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    set_fwd = sm;
  }
  DP_LAUNCHED(1);
  k_tab_fwd<<<tab_blocks(n), kWarpsPerBlock * 32, sm, st>>>(n, off, nlist, nn, cap, g, ep, table,
                                                          stage_cap(ep), T, status, pair_count);
  return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

int launch_tab_bwd(cudaStream_t st, int64_t n, const float4* off, const uint32_t* nlist,
                   const int32_t* nn, int cap, const CellGeom& g, const EnvParams& ep,
                   const float* table, const float* dT, unsigned long long* ffix,
                   double* vir_part, int vir_slots, int32_t* status) {
  if (n <= 0) return 0;
  if (ep.M > 128 || ep.M % 4 || ep.ntypes * ep.n_int > 32768) return -1;
  if (vir_slots < tab_kernel_slots(n)) return -1;
  size_t sm = bwd_smem(ep);
  if (sm > 200 * 1024) return -1;
  static std::atomic<size_t> set_bwd{0};
  if (sm > 48 * 1024 && sm > set_bwd) {
    cudaFuncSetAttribute(k_tab_bwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    set_bwd = sm;
  }
  DP_LAUNCHED(1);
  k_tab_bwd<<<tab_blocks(n), kWarpsPerBlock * 32, sm, st>>>(n, off, nlist, nn, cap, g, ep, table,
                                                          stage_cap(ep), dT, ffix, vir_part, status);
  return cudaGetLastError() == cudaSuccess ? 0 : -3;
}
