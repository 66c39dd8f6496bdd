// Pair geometry and the per-atom counting sort by table interval, shared by
// the CUDA-core and tensor-core embedding kernels (one warp per atom).
#pragma once
#include <math.h>

#include "dp_internal.h"

namespace dp_embed {

// ------------------------------------------------------------------ pair geometry
struct Pair {
  float dx, dy, dz, r, ir, s, dsdr;
  int th, tj;
  float u;
  bool out_of_range;
};

// The table interval of s: floor(s/h) in the first region (intervals of
// width h up to s_fine), n_fine + floor((s - s_fine)/H) beyond it, clamped to
// the table (s beyond the last node is flagged by the caller).
__device__ __forceinline__ int interval_of(const EnvParams& ep, float s) {
  const float q = floorf(s * ep.inv_h);
  if (q < (float)ep.n_fine) return q < 0.0f ? 0 : (int)q;
  if (ep.n_int == ep.n_fine) return ep.n_fine - 1;
  // clamped in floating point first (fmaxf maps a NaN to 0)
  const float j = fminf(fmaxf(floorf((s - ep.s_fine) * ep.inv_H), 0.0f),
                        (float)(ep.n_int - ep.n_fine - 1));
  return ep.n_fine + (int)j;
}

// The normalised local variable of s on interval th, u = (s - x_th) / w_th,
// and the width's reciprocal du/ds.
__device__ __forceinline__ float interval_u(const EnvParams& ep, float s, int th) {
  return th < ep.n_fine ? s * ep.inv_h - (float)th
                        : (s - ep.s_fine) * ep.inv_H - (float)(th - ep.n_fine);
}
__device__ __forceinline__ float interval_du_ds(const EnvParams& ep, int th) {
  return th < ep.n_fine ? ep.inv_h : ep.inv_H;
}

__device__ __forceinline__ void pair_geom(const EnvParams& ep, float dx, float dy, float dz,
                                          float r2, int tj, Pair& P) {
  P.dx = dx;
  P.dy = dy;
  P.dz = dz;
  P.tj = tj;
  // 1/r from the hardware reciprocal square root (a few ulp), r = r2 / r
  const float ir = rsqrtf(r2);
  const float r = r2 * ir;
  float sw, dsw;
  if (r < ep.rcs) {
    sw = 1.0f;
    dsw = 0.0f;
  } else {
    // 1 - 10x^3 + 15x^4 - 6x^5 = (1-x)^3 (1 + 3x + 6x^2): the factored form
    // keeps its accuracy (and sign) next to rc where the expanded one cancels
    const float x = (r - ep.rcs) * ep.inv_w;
    const float om = 1.0f - x;
    sw = om * om * om * fmaf(fmaf(6.0f, x, 3.0f), x, 1.0f);
    dsw = -30.0f * x * x * om * om * ep.inv_w;
  }
  const float s = sw * ir;
  P.r = r;
  P.ir = ir;
  P.s = s;
  P.dsdr = (dsw - s) * ir;
  const int th = interval_of(ep, s);
  P.th = th;
  P.u = interval_u(ep, s, th);
  P.out_of_range = s > ep.smax;
}

__device__ __forceinline__ void load_pair(const float4& oi, const float4* __restrict__ off,
                                          const CellGeom& g, uint32_t e, float& dx, float& dy,
                                          float& dz, int& tj) {
  const int j = (int)(e >> 5), code = (int)(e & 31u);
  const float4 oj = off[j];
  dx = (oj.x - oi.x) + (float)(code / 9 - 1) * g.edgef[0];
  dy = (oj.y - oi.y) + (float)((code / 3) % 3 - 1) * g.edgef[1];
  dz = (oj.z - oi.z) + (float)(code % 3 - 1) * g.edgef[2];
  tj = __float_as_int(oj.w);
}

// the same with the neighbor's offset record oj already loaded
__device__ __forceinline__ void pair_from(const float4& oi, const float4& oj, const CellGeom& g,
                                          uint32_t e, float& dx, float& dy, float& dz, int& tj) {
  const int code = (int)(e & 31u);
  dx = (oj.x - oi.x) + (float)(code / 9 - 1) * g.edgef[0];
  dy = (oj.y - oi.y) + (float)((code / 3) % 3 - 1) * g.edgef[1];
  dz = (oj.z - oi.z) + (float)(code % 3 - 1) * g.edgef[2];
  tj = __float_as_int(oj.w);
}

// ------------------------------------------------------------------ per-atom interval sort
// The pairs of an atom within rc are counting-sorted by bin = (neighbor type,
// table interval): a histogram (integer atomics: order independent), an
// exclusive scan, then a stable scatter in list order (ranks within a chunk
// from __match_any_sync).  The result is deterministic.  After the scatter,
// hist[b] holds the end of bin b, so bin b spans [b ? hist[b-1] : 0, hist[b]).
__device__ __forceinline__ int bin_begin(const int* hist, int b) { return b ? hist[b - 1] : 0; }

// exclusive scan of hist[0..nb) in place; returns the total
__device__ __forceinline__ int warp_exclusive_scan(int* hist, int nb, int lane) {
  const int per = (nb + 31) / 32;
  const int b0 = min(lane * per, nb), b1 = min(b0 + per, nb);
  int sum = 0;
  for (int b = b0; b < b1; ++b) sum += hist[b];
  int incl = sum;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  int run = incl - sum;
  for (int b = b0; b < b1; ++b) {
    const int c = hist[b];
    hist[b] = run;
    run += c;
  }
  const int total = __shfl_sync(0xffffffffu, incl, 31);
  __syncwarp();
  return total;
}

// stable slot of this lane's pair in the bin-sorted order (all lanes call)
__device__ __forceinline__ int sorted_slot(int* hist, bool in, int bin, int lane) {
  const unsigned grp = __match_any_sync(0xffffffffu, in ? bin : (0x40000000 | lane));
  const int rank = __popc(grp & ((1u << lane) - 1u));
  const int pos = in ? hist[bin] + rank : -1;
  __syncwarp();
  if (in && rank == 0) hist[bin] += __popc(grp);
  __syncwarp();
  return pos;
}

__host__ __device__ inline int round4(int v) { return (v + 3) & ~3; }
}  // namespace dp_embed
