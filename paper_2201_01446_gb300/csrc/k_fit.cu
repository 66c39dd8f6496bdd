// Descriptor (Eq. 2) and fitting net (Sec. 2.1) on FP32 CUDA cores, forward
// and input-gradient backward.  This is the FP32 reference mode of the
// fitting stage; the tensor-core mode lives in k_fit_tc.cu.
//
//   D[b*m_lt + a] = sum_c T[c][b] T[c][a]       (a < M^<; the flattening
//                                                order is a reading)
//   z_0 = tanh(D W_0 + b_0)
//   z_k = z_{k-1} + tanh(z_{k-1} W_k + b_k)     (shortcut when widths match)
//   E_i = z_last . w_out + b_out
// Backward: gz_last = w_out; gp_k = gz_k (1 - t_k^2);
//   gz_{k-1} = [shortcut] gz_k + gp_k W_k^T;  dD = gp_0 W_0^T;
//   dT[c][x] = sum_a dD[x][a] T[c][a] + [x < M^<] sum_b dD[b][x] T[c][b].
#include <math.h>

#include "act.cuh"
#include "dp_internal.h"

namespace {

enum { EPI_PLAIN = 0, EPI_TANH = 1, EPI_BWD = 2 };

struct GemmEpi {
  const float* bias;  // [N]            (EPI_TANH)
  const float* R;     // residual, row stride ldr (0 = broadcast row)
  int ldr;
  float* out0;        // C / activation derivative / gz
  float* out1;        // z / gp
  int ldc;
  const float* Tt;    // activation derivatives of the previous layer (EPI_BWD)
  int ldt;
  const float4* tab;  // tanh table (EPI_TANH), NULL: tanhf
};

// C[M x N] = A[M x K] B[K x N], 128 x BN tiles, 8 x TN outputs per thread
template <int BN, int TN, int EPI>
__global__ void __launch_bounds__(256) k_gemm(int M, int N, int K, const float* __restrict__ A,
                                              int lda, const float* __restrict__ B, int ldb,
                                              GemmEpi ep) {
  constexpr int BM = 128, BK = 16, TM = 8;
  static_assert(BN / TN == 16, "16 x 16 threads");
  __shared__ float As[BK][BM + 4];
  __shared__ float Bs[BK][BN];
  const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
  const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
  float acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = 0.0f;
  const int ar = tid >> 1, ak = (tid & 1) * 8;
  for (int k0 = 0; k0 < K; k0 += BK) {
    {
      const int m = m0 + ar;
      float4 v0 = make_float4(0.f, 0.f, 0.f, 0.f), v1 = v0;
      if (m < M) {
        const float* ap = A + (size_t)m * lda + k0 + ak;
        v0 = *reinterpret_cast<const float4*>(ap);
        v1 = *reinterpret_cast<const float4*>(ap + 4);
      }
      As[ak + 0][ar] = v0.x;
      As[ak + 1][ar] = v0.y;
      As[ak + 2][ar] = v0.z;
      As[ak + 3][ar] = v0.w;
      As[ak + 4][ar] = v1.x;
      As[ak + 5][ar] = v1.y;
      As[ak + 6][ar] = v1.z;
      As[ak + 7][ar] = v1.w;
    }
    for (int idx = tid; idx < BK * BN; idx += 256) {
      const int kk = idx / BN, nn = idx % BN;
      Bs[kk][nn] = (n0 + nn < N) ? B[(size_t)(k0 + kk) * ldb + n0 + nn] : 0.0f;
    }
    __syncthreads();
    // two-level sum: each K tile is accumulated on its own and then added to
    // the running total, so rounding grows with K/16 + 16 instead of K
    float tacc[TM][TN];
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      float a[TM], b[TN];
#pragma unroll
      for (int i = 0; i < TM; ++i) a[i] = As[kk][ty * TM + i];
#pragma unroll
      for (int j = 0; j < TN; ++j) b[j] = Bs[kk][tx * TN + j];
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) tacc[i][j] = kk ? fmaf(a[i], b[j], tacc[i][j]) : a[i] * b[j];
    }
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
      for (int j = 0; j < TN; ++j) acc[i][j] += tacc[i][j];
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < TM; ++i) {
    const int m = m0 + ty * TM + i;
    if (m >= M) continue;
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      const int n = n0 + tx * TN + j;
      if (n >= N) continue;
      const float v = acc[i][j];
      const size_t o = (size_t)m * ep.ldc + n;
      if (EPI == EPI_PLAIN) {
        ep.out0[o] = v;
      } else if (EPI == EPI_TANH) {
        float d;
        const float t = act_tanh(v + ep.bias[n], ep.tab, d);
        ep.out0[o] = d;
        ep.out1[o] = (ep.R ? ep.R[(size_t)m * ep.ldr + n] : 0.0f) + t;
      } else {
        const float gz = v + (ep.R ? ep.R[(size_t)m * ep.ldr + n] : 0.0f);
        const float tt = ep.Tt[(size_t)m * ep.ldt + n];
        ep.out0[o] = gz;
        ep.out1[o] = gz * tt;
      }
    }
  }
}

template <int EPI>
void gemm(cudaStream_t st, int M, int N, int K, const float* A, int lda, const float* B, int ldb,
          const GemmEpi& ep) {
  DP_LAUNCHED(1);
  if (N <= 256 && N % 80 == 0) {
    dim3 grid((M + 127) / 128, (N + 79) / 80);
    k_gemm<80, 5, EPI><<<grid, 256, 0, st>>>(M, N, K, A, lda, B, ldb, ep);
  } else {
    dim3 grid((M + 127) / 128, (N + 127) / 128);
    k_gemm<128, 8, EPI><<<grid, 256, 0, st>>>(M, N, K, A, lda, B, ldb, ep);
  }
}

// one CTA per atom: D row from T (gathered through idx)
__global__ void k_descr(int64_t rows, const int32_t* __restrict__ idx, const float* __restrict__ T,
                        int M, int m_lt, float* __restrict__ D) {
  extern __shared__ float Ts[];  // [4][M]
  const int64_t r = blockIdx.x;
  const int64_t a = idx ? idx[r] : r;
  for (int k = threadIdx.x; k < 4 * M; k += blockDim.x) Ts[k] = T[(size_t)a * 4 * M + k];
  __syncthreads();
  for (int b = threadIdx.x; b < M; b += blockDim.x) {
    float* out = D + (size_t)r * M * m_lt + (size_t)b * m_lt;
    for (int q = 0; q < m_lt; ++q) {
      float s = 0.0f;
#pragma unroll
      for (int c = 0; c < 4; ++c) s = fmaf(Ts[c * M + b], Ts[c * M + q], s);
      out[q] = s;
    }
  }
}

__global__ void k_descr_bwd(int64_t rows, const int32_t* __restrict__ idx,
                            const float* __restrict__ T, const float* __restrict__ dD, int M,
                            int m_lt, float* __restrict__ dT) {
  extern __shared__ float sm[];
  float* Ts = sm;            // [4][M]
  float* dDs = sm + 4 * M;   // [M][m_lt]
  const int64_t r = blockIdx.x;
  const int64_t a = idx ? idx[r] : r;
  for (int k = threadIdx.x; k < 4 * M; k += blockDim.x) Ts[k] = T[(size_t)a * 4 * M + k];
  for (int k = threadIdx.x; k < M * m_lt; k += blockDim.x) dDs[k] = dD[(size_t)r * M * m_lt + k];
  __syncthreads();
  for (int x = threadIdx.x; x < M; x += blockDim.x) {
    float g[4] = {0.f, 0.f, 0.f, 0.f};
    for (int q = 0; q < m_lt; ++q) {
      const float d = dDs[x * m_lt + q];
#pragma unroll
      for (int c = 0; c < 4; ++c) g[c] = fmaf(d, Ts[c * M + q], g[c]);
    }
    if (x < m_lt) {
      for (int b = 0; b < M; ++b) {
        const float d = dDs[b * m_lt + x];
#pragma unroll
        for (int c = 0; c < 4; ++c) g[c] = fmaf(d, Ts[c * M + b], g[c]);
      }
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) dT[(size_t)a * 4 * M + c * M + x] = g[c];
  }
}

// one warp per atom: E_i = z . w + b
__global__ void k_energy(int64_t rows, const int32_t* __restrict__ idx, const float* __restrict__ z,
                         int W, const float* __restrict__ w, float b, double* __restrict__ e) {
  const int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (r >= rows) return;
  float s = 0.0f;
  for (int k = lane; k < W; k += 32) s = fmaf(z[(size_t)r * W + k], w[k], s);
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) e[idx ? idx[r] : r] = (double)(s + b);
}

// gp = w act'(a) for the last hidden layer (d: the stored derivatives)
__global__ void k_gp_last(int64_t rows, int W, const float* __restrict__ d,
                          const float* __restrict__ w, float* __restrict__ gp) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= rows * W) return;
  gp[k] = w[k % W] * d[k];
}

// Parameter gradients of one layer over a chunk of rows:
//   part[s][r][c] = sum over the rows i of split s of Xe[i][r] Ge[i][c]
// with Xe = [X | 1] (row r == win: the bias) and Ge = G, or a column of ones
// when G == NULL (the output layer: dE/dw_out = sum_i z_i, dE/db_out = rows).
// 64 x 64 output tiles, 4 x 4 per thread, rows staged 16 at a time.
__global__ void __launch_bounds__(256) k_wgrad_part(int rows, int per_split,
                                                    const float* __restrict__ X, int ldx, int win,
                                                    const float* __restrict__ G, int ldg, int wo,
                                                    float* __restrict__ part) {
  __shared__ float Xs[16][64], Gs[16][64];
  const int r0 = blockIdx.x * 64, c0 = blockIdx.y * 64, sp = blockIdx.z;
  const int i_beg = sp * per_split, i_end = min(rows, i_beg + per_split);
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  float acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = 0.0f;
  for (int i0 = i_beg; i0 < i_end; i0 += 16) {
    for (int q = threadIdx.x; q < 16 * 64; q += 256) {
      const int ii = q >> 6, cc = q & 63, i = i0 + ii;
      const int r = r0 + cc, c = c0 + cc;
      const bool in = i < i_end;
      Xs[ii][cc] = (in && r <= win) ? (r < win ? X[(size_t)i * ldx + r] : 1.0f) : 0.0f;
      Gs[ii][cc] = (in && c < wo) ? (G ? G[(size_t)i * ldg + c] : 1.0f) : 0.0f;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      float xa[4], gb[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) xa[a] = Xs[kk][ty * 4 + a];
#pragma unroll
      for (int b = 0; b < 4; ++b) gb[b] = Gs[kk][tx * 4 + b];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = fmaf(xa[a], gb[b], acc[a][b]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int r = r0 + ty * 4 + a;
    if (r > win) continue;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int c = c0 + tx * 4 + b;
      if (c < wo) part[((size_t)sp * (win + 1) + r) * wo + c] = acc[a][b];
    }
  }
}

// g[e] += sum over the splits (in order) of part[s][e], in FP64
__global__ void k_wgrad_add(int nsplit, int64_t n, const float* __restrict__ part,
                            double* __restrict__ g) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  double s = 0.0;
  for (int k = 0; k < nsplit; ++k) s += (double)part[(size_t)k * n + e];
  g[e] += s;
}

int wgrad_splits(int rows, int win, int wo) {
  const int tiles = ((win + 1 + 63) / 64) * ((wo + 63) / 64);
  int sp = (2 * 152 + tiles - 1) / tiles;
  const int maxsp = (rows + 255) / 256;
  return sp < 1 ? 1 : (sp > maxsp ? (maxsp < 1 ? 1 : maxsp) : sp);
}

// g_block [(win + 1)][wo] += [X | 1]^T G over rows
void wgrad(cudaStream_t st, int rows, const float* X, int ldx, int win, const float* G, int ldg,
           int wo, const FitGrad& fg, double* g_block) {
  int sp = wgrad_splits(rows, win, wo);
  const int64_t n = (int64_t)(win + 1) * wo;
  while (sp > 1 && (int64_t)sp * n > fg.part_floats) --sp;
  const int per = ((rows + sp - 1) / sp + 15) / 16 * 16;
  dim3 grid((win + 1 + 63) / 64, (wo + 63) / 64, sp);
  DP_LAUNCHED(2);
  k_wgrad_part<<<grid, 256, 0, st>>>(rows, per, X, ldx, win, G, ldg, wo, fg.part);
  k_wgrad_add<<<(int)((n + 255) / 256), 256, 0, st>>>(sp, n, fg.part, g_block);
}

}  // namespace

int64_t fit_grad_part_floats(const FitNet& net, int din, int64_t rows) {
  int64_t mx = 0;
  int win = din;
  for (int k = 0; k < net.nl; ++k) {
    const int64_t v = (int64_t)wgrad_splits((int)rows, win, net.wout[k]) * (win + 1) * net.wout[k];
    mx = v > mx ? v : mx;
    win = net.wout[k];
  }
  const int64_t v = (int64_t)wgrad_splits((int)rows, win, 1) * (win + 1);
  return v > mx ? v : mx;
}

int fit_simt(cudaStream_t st, int64_t n, const int32_t* idx, const FitNet& net, int M, int m_lt,
             const float* T, float* dT, double* e_atom, const FitScratch& s,
             const FitGrad* fg) {
  if (n <= 0) return 0;
  const int din = M * m_lt;
  const int nl = net.nl;
  // offsets of the layers' gradient blocks
  int64_t goff[DP_MAXFIT + 1];
  goff[0] = 0;
  for (int k = 0; k < nl; ++k) goff[k + 1] = goff[k] + (int64_t)(net.win[k] + 1) * net.wout[k];
  for (int64_t r0 = 0; r0 < n; r0 += s.rows) {
    const int rows = (int)((n - r0) < s.rows ? (n - r0) : s.rows);
    const int32_t* id = idx ? idx + r0 : nullptr;
    // T -> D  (rows gathered through idx; without idx the chunk starts at r0)
    const float* Tc = idx ? T : T + (size_t)r0 * 4 * M;
    float* dTc = idx ? dT : dT + (size_t)r0 * 4 * M;
    DP_LAUNCHED(4);  // descriptor, energy, last-layer gradient, descriptor backward
    k_descr<<<rows, 128, sizeof(float) * 4 * M, st>>>(rows, id, Tc, M, m_lt, s.D);
    // forward
    const float* in = s.D;
    int win = din;
    for (int k = 0; k < nl; ++k) {
      GemmEpi ep{};
      ep.bias = net.b[k];
      ep.R = net.shortcut[k] ? in : nullptr;
      ep.ldr = win;
      ep.out0 = s.t[k];
      ep.out1 = s.z[k];
      ep.ldc = net.wout[k];
      ep.tab = net.tanh_tab;
      gemm<EPI_TANH>(st, rows, net.wout[k], win, in, win, net.W[k], net.wout[k], ep);
      in = s.z[k];
      win = net.wout[k];
    }
    const int W = net.wout[nl - 1];
    k_energy<<<(rows * 32 + 255) / 256, 256, 0, st>>>(rows, id, s.z[nl - 1], W, net.w_out,
                                                      net.b_out, e_atom + (idx ? 0 : r0));
    // backward
    k_gp_last<<<(int)(((int64_t)rows * W + 255) / 256), 256, 0, st>>>(rows, W, s.t[nl - 1],
                                                                      net.w_out, s.gp);
    // gz of the last layer is w_out on every row (row stride 0); gz is
    // updated in place (each element is read and written by one thread),
    // gp ping-pongs because it is the A operand of the next GEMM
    const float* gz_prev = net.w_out;
    int ldgz = 0;
    float* gpin = s.gp;
    float* gpout = s.gz2;
    if (fg)  // dE/dw_out = sum_i z_i, dE/db_out = rows
      wgrad(st, rows, s.z[nl - 1], W, W, nullptr, 0, 1, *fg, fg->g + goff[nl]);
    for (int k = nl - 1; k >= 1; --k) {
      // gpin = gp_k: dE/dW_k = z_{k-1}^T gp_k, dE/db_k = sum_i gp_k
      if (fg)
        wgrad(st, rows, s.z[k - 1], net.win[k], net.win[k], gpin, net.wout[k], net.wout[k], *fg,
              fg->g + goff[k]);
      GemmEpi ep{};
      ep.R = net.shortcut[k] ? gz_prev : nullptr;
      ep.ldr = ldgz;
      ep.out0 = s.gz;
      ep.out1 = gpout;
      ep.ldc = net.win[k];
      ep.Tt = s.t[k - 1];
      ep.ldt = net.win[k];
      gemm<EPI_BWD>(st, rows, net.win[k], net.wout[k], gpin, net.wout[k], net.WT[k], net.win[k], ep);
      gz_prev = s.gz;
      ldgz = net.win[k];
      float* tmp = gpin;
      gpin = gpout;
      gpout = tmp;
    }
    if (fg)  // layer 0: dE/dW_0 = D^T gp_0
      wgrad(st, rows, s.D, din, din, gpin, net.wout[0], net.wout[0], *fg, fg->g);
    {
      GemmEpi ep{};
      ep.out0 = s.dD;
      ep.ldc = din;
      gemm<EPI_PLAIN>(st, rows, din, net.wout[0], gpin, net.wout[0], net.WT[0], din, ep);
    }
    k_descr_bwd<<<rows, 128, sizeof(float) * (4 * M + M * m_lt), st>>>(rows, id, Tc, s.dD, M,
                                                                      m_lt, dTc);
  }
  return cudaGetLastError() == cudaSuccess ? 0 : -3;
}
