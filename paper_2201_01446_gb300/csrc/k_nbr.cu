// Cell-list neighbor build (paper Sec. 2.1: the neighbor set within the
// cutoff; Sec. 4: list with a buffer region, rebuilt periodically).
//
// The list of atom i holds every periodic image (j, n) with
// |x_j + n*L - x_i| < rlist, (j, n) != (i, 0), where x is wrapped into
// [0, L).  Entries are (j << 5) | code with code the 27-cell stencil offset
// o in {-1,0,1}^3 that found j; the image follows from the cells.  Entries
// are ordered by stencil slot, then by atom index within the cell (cells are
// sorted after binning), so the list is deterministic.
//
// Distances are tested in FP32 on cell offsets; a pair within a relative
// band of 1e-4 of rlist^2 is decided again in FP64 from the wrapped FP64
// positions, evaluated in the same operation order as the plain definition
// ((x_j - x_i) + n*L, squares summed in x, y, z order, no fused multiply-add),
// so the set equals the one an exact FP64 test gives.
#include "dp_internal.h"

namespace {

__device__ __forceinline__ double wrap1(double x, double L) {
  double w = __dsub_rn(x, __dmul_rn(floor(__ddiv_rn(x, L)), L));
  if (w >= L) w = __dsub_rn(w, L);
  if (w < 0.0) w = __dadd_rn(w, L);
  return w;
}

__device__ __forceinline__ int cell_of(double w, double L, int nc) {
  int c = (int)floor(__dmul_rn(__ddiv_rn(w, L), (double)nc));
  return c < 0 ? 0 : (c >= nc ? nc - 1 : c);
}

__global__ void k_wrap_bin(int64_t n, double* __restrict__ x, CellGeom g, int32_t* __restrict__ cellc,
                           int32_t* __restrict__ count) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int c[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    double w = wrap1(x[i * 3 + a], g.L[a]);
    x[i * 3 + a] = w;
    c[a] = cell_of(w, g.L[a], g.nc[a]);
  }
  int id = (c[0] * g.nc[1] + c[1]) * g.nc[2] + c[2];
  cellc[i] = id;
  atomicAdd(&count[id], 1);
}

// single-CTA exclusive scan of cell counts (ncell is at most a few million)
__global__ void __launch_bounds__(1024) k_scan(const int32_t* __restrict__ count,
                                               int32_t* __restrict__ start, long long ncell) {
  __shared__ int32_t warp_tot[32];
  __shared__ int32_t carry_s;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  if (tid == 0) carry_s = 0;
  __syncthreads();
  for (long long base = 0; base < ncell; base += 4096) {
    int32_t v[4];
    int32_t s = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      long long idx = base + tid * 4 + k;
      v[k] = idx < ncell ? count[idx] : 0;
      s += v[k];
    }
    int32_t incl = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int32_t y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    if (lane == 31) warp_tot[wid] = incl;
    __syncthreads();
    if (wid == 0) {
      int32_t t = warp_tot[lane];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        int32_t y = __shfl_up_sync(0xffffffffu, t, o);
        if (lane >= o) t += y;
      }
      warp_tot[lane] = t;  // inclusive over warps
    }
    __syncthreads();
    int32_t excl = carry_s + (wid ? warp_tot[wid - 1] : 0) + incl - s;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      long long idx = base + tid * 4 + k;
      if (idx < ncell) start[idx] = excl;
      excl += v[k];
    }
    __syncthreads();
    if (tid == 0) carry_s += warp_tot[31];
    __syncthreads();
  }
  if (tid == 0) start[ncell] = carry_s;
}

__global__ void k_scatter(int64_t n, const int32_t* __restrict__ cellc, const int32_t* __restrict__ start,
                          int32_t* __restrict__ fill, int32_t* __restrict__ out) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int c = cellc[i];
  int p = atomicAdd(&fill[c], 1);
  out[start[c] + p] = (int32_t)i;
}

// one warp per cell: rank sort of the cell's atom indices (all distinct)
__global__ void k_cell_sort(long long ncell, const int32_t* __restrict__ start,
                            const int32_t* __restrict__ in, int32_t* __restrict__ out) {
  long long c = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (c >= ncell) return;
  int s = start[c], e = start[c + 1];
  for (int k = s + lane; k < e; k += 32) {
    int v = in[k], r = 0;
    for (int q = s; q < e; ++q) r += (in[q] < v);
    out[s + r] = v;
  }
}

__global__ void k_mirror(int64_t n, const double* __restrict__ x, const int32_t* __restrict__ cellc,
                         const int32_t* __restrict__ types, CellGeom g, float4* __restrict__ off) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int id = cellc[i];
  int c2 = id % g.nc[2];
  int c1 = (id / g.nc[2]) % g.nc[1];
  int c0 = id / (g.nc[2] * g.nc[1]);
  float4 o;
  o.x = (float)(x[i * 3 + 0] - (c0 + 0.5) * g.edge[0]);
  o.y = (float)(x[i * 3 + 1] - (c1 + 0.5) * g.edge[1]);
  o.z = (float)(x[i * 3 + 2] - (c2 + 0.5) * g.edge[2]);
  o.w = __int_as_float(types[i]);
  off[i] = o;
}

// the same for several systems in one array: atom i uses the cell grid of
// its system sys_of[i] (cellc holds system-local cell indices)
__global__ void k_mirror_batch(int64_t n, const double* __restrict__ x,
                               const int32_t* __restrict__ cellc, const int32_t* __restrict__ types,
                               const int32_t* __restrict__ sys_of, const CellGeom* __restrict__ geoms,
                               float4* __restrict__ off) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const CellGeom& g = geoms[sys_of[i]];
  int id = cellc[i];
  int c2 = id % g.nc[2];
  int c1 = (id / g.nc[2]) % g.nc[1];
  int c0 = id / (g.nc[2] * g.nc[1]);
  float4 o;
  o.x = (float)(x[i * 3 + 0] - (c0 + 0.5) * g.edge[0]);
  o.y = (float)(x[i * 3 + 1] - (c1 + 0.5) * g.edge[1]);
  o.z = (float)(x[i * 3 + 2] - (c2 + 0.5) * g.edge[2]);
  o.w = __int_as_float(types[i]);
  off[i] = o;
}

// one warp per atom, atoms visited in cell order so that the warps of a CTA
// share their candidate cells in L1.  Lane l < 27 first looks up stencil
// slot l's cell (its atom range and image shift); the warp then walks the
// 27 ranges as one sequence of rounds of 32 candidates, with the next
// round's candidate indices and offsets loaded while the current round is
// tested (the slot order, hence the list order, is unchanged)
__global__ void __launch_bounds__(128) k_build_list(
    int64_t n, const double* __restrict__ x, const int32_t* __restrict__ cellc,
    const float4* __restrict__ off, const int32_t* __restrict__ cell_start,
    const int32_t* __restrict__ cell_atoms, CellGeom g, double rlist, float rc2, int ntypes,
    const int32_t* __restrict__ sel, int cap, uint32_t* __restrict__ nlist, int32_t* __restrict__ nn,
    int32_t* __restrict__ status) {
  const int lane = threadIdx.x & 31;
  int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (w >= n) return;
  const int i = cell_atoms[w];
  const int id = cellc[i];
  const int ci[3] = {id / (g.nc[2] * g.nc[1]), (id / g.nc[2]) % g.nc[1], id % g.nc[2]};
  const float4 oi = off[i];
  const double rl2 = rlist * rlist;
  const float rl2f = (float)rl2;
  const float lo = rl2f * (1.0f - 1e-4f), hi = rl2f * (1.0f + 1e-4f);
  uint32_t* L = nlist + (size_t)i * cap;
  // lane l < 27: stencil slot l's atom range [my_s, my_e) and image code
  int my_s = 0, my_e = 0, my_img = 0;
  if (lane < 27) {
    const int o[3] = {lane / 9 - 1, (lane / 3) % 3 - 1, lane % 3 - 1};
    int cc[3], im[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const int v = ci[a] + o[a];
      im[a] = v < 0 ? -1 : (v >= g.nc[a] ? 1 : 0);
      cc[a] = v - im[a] * g.nc[a];
    }
    const int cid = (cc[0] * g.nc[1] + cc[1]) * g.nc[2] + cc[2];
    my_s = cell_start[cid];
    my_e = cell_start[cid + 1];
    my_img = (im[0] + 1) * 9 + (im[1] + 1) * 3 + (im[2] + 1);
    // the slot's cell is skipped when its nearest point is farther from atom
    // i than r_list (oi: i's offset from its own cell's centre; along a
    // shifted axis the cell starts half an edge beyond the centre), with a
    // margin of 1e-4 on r^2 far above the FP32 error of the offsets: no atom
    // of a skipped cell could pass the test below, so the list is unchanged
    const float oia[3] = {oi.x, oi.y, oi.z};
    float d2 = 0.0f;
#pragma unroll
    for (int a = 0; a < 3; ++a)
      if (o[a] != 0) {
        const float d = 0.5f * g.edgef[a] - (float)o[a] * oia[a];
        if (d > 0.0f) d2 = fmaf(d, d, d2);
      }
    if (d2 > hi) my_e = my_s;
  }
  int cnt = 0;
  int cnt_t[DP_MAXT];
#pragma unroll
  for (int t = 0; t < DP_MAXT; ++t) cnt_t[t] = 0;
  const unsigned below = (1u << lane) - 1u;
  // the round sequence: (slot, base) with base stepping by 32 through the
  // slot's range; advance() moves to the next non-empty round
  int slot = 0, base = __shfl_sync(0xffffffffu, my_s, 0), e = __shfl_sync(0xffffffffu, my_e, 0);
  auto advance = [&](int& sl, int& b, int& en) {
    b += 32;
    while (b >= en && sl < 27) {
      ++sl;
      if (sl < 27) {
        b = __shfl_sync(0xffffffffu, my_s, sl);
        en = __shfl_sync(0xffffffffu, my_e, sl);
      }
    }
  };
  if (base >= e) {  // the first slot's cell is empty: find the first round
    base -= 32;
    advance(slot, base, e);
  }
  // the current slot's image shift (recomputed when the slot changes)
  auto shift_of = [&](int sl, float& x0, float& y0, float& z0) {
    x0 = (sl / 9 - 1) * g.edgef[0];
    y0 = ((sl / 3) % 3 - 1) * g.edgef[1];
    z0 = (sl % 3 - 1) * g.edgef[2];
  };
  float sx = 0.f, sy = 0.f, sz = 0.f;
  if (slot < 27) shift_of(slot, sx, sy, sz);
  // prefetched candidate of the current round
  int j_c = 0;
  float4 o_c = make_float4(0.f, 0.f, 0.f, 0.f);
  if (slot < 27 && base + lane < e) {
    j_c = cell_atoms[base + lane];
    o_c = off[j_c];
  }
  while (slot < 27) {
    // the next round and its candidate, loaded before this round is tested
    int nslot = slot, nbase = base, ne = e;
    advance(nslot, nbase, ne);
    int j_n = 0;
    float4 o_n = make_float4(0.f, 0.f, 0.f, 0.f);
    if (nslot < 27 && nbase + lane < ne) {
      j_n = cell_atoms[nbase + lane];
      o_n = off[j_n];
    }
    const int img_code = __shfl_sync(0xffffffffu, my_img, slot);
    const int k = base + lane;
    bool in = false, inrc = false;
    const int j = j_c;
    int tj = 0;
    if (k < e) {
      const float4 oj = o_c;
      tj = __float_as_int(oj.w);
      const float dx = (oj.x - oi.x) + sx, dy = (oj.y - oi.y) + sy, dz = (oj.z - oi.z) + sz;
      const float r2 = dx * dx + dy * dy + dz * dz;
      const bool self = (j == i) && slot == 13;
      if (!self) {
        if (r2 < lo) {
          in = true;
        } else if (r2 <= hi) {
          // boundary band: decide exactly as the FP64 definition does
          const int img[3] = {img_code / 9 - 1, (img_code / 3) % 3 - 1, img_code % 3 - 1};
          double r2d = 0.0;
#pragma unroll
          for (int a = 0; a < 3; ++a) {
            double d = __dadd_rn(__dsub_rn(x[(size_t)j * 3 + a], x[(size_t)i * 3 + a]),
                                 __dmul_rn((double)img[a], g.L[a]));
            r2d = __dadd_rn(r2d, __dmul_rn(d, d));
          }
          in = r2d < rl2;
        }
        inrc = r2 < rc2;
      }
    }
    const unsigned m = __ballot_sync(0xffffffffu, in);
    if (in) {
      const int p = cnt + __popc(m & below);
      if (p < cap) L[p] = ((uint32_t)j << 5) | (uint32_t)slot;
    }
    cnt += __popc(m);
    for (int t = 0; t < ntypes; ++t) cnt_t[t] += __popc(__ballot_sync(0xffffffffu, inrc && tj == t));
    if (nslot != slot && nslot < 27) shift_of(nslot, sx, sy, sz);
    slot = nslot;
    base = nbase;
    e = ne;
    j_c = j_n;
    o_c = o_n;
  }
  if (lane == 0) {
    nn[i] = cnt;
    atomicMax(&status[ST_MAXLIST], cnt);
    if (cnt > cap) atomicAdd(&status[ST_LISTOVF], 1);
    bool over = false;
    for (int t = 0; t < ntypes; ++t) over |= cnt_t[t] > sel[t];
    if (over) atomicAdd(&status[ST_SEL], 1);
  }
}

inline int nblk(int64_t n, int t) { return (int)((n + t - 1) / t); }

}  // namespace

void launch_wrap_bin(cudaStream_t st, int64_t n, double* x, const CellGeom& g, int32_t* cellc,
                     int32_t* cell_count) {
  if (n > 0) DP_LAUNCHED(1), k_wrap_bin<<<nblk(n, 256), 256, 0, st>>>(n, x, g, cellc, cell_count);
}

void launch_scan(cudaStream_t st, const int32_t* count, int32_t* start, long long ncell) {
  DP_LAUNCHED(1);
  k_scan<<<1, 1024, 0, st>>>(count, start, ncell);
}

void launch_scatter(cudaStream_t st, int64_t n, const int32_t* cellc, const int32_t* start,
                    int32_t* fill, int32_t* out) {
  if (n > 0) DP_LAUNCHED(1), k_scatter<<<nblk(n, 256), 256, 0, st>>>(n, cellc, start, fill, out);
}

void launch_cell_sort(cudaStream_t st, long long ncell, const int32_t* start, const int32_t* in,
                      int32_t* out) {
  DP_LAUNCHED(1);
  k_cell_sort<<<nblk(ncell * 32, 256), 256, 0, st>>>(ncell, start, in, out);
}

void launch_mirror(cudaStream_t st, int64_t n, const double* x, const int32_t* cellc,
                   const int32_t* types, const CellGeom& g, float4* off) {
  if (n > 0) DP_LAUNCHED(1), k_mirror<<<nblk(n, 256), 256, 0, st>>>(n, x, cellc, types, g, off);
}

void launch_mirror_batch(cudaStream_t st, int64_t n, const double* x, const int32_t* cellc,
                         const int32_t* types, const int32_t* sys_of, const CellGeom* geoms,
                         float4* off) {
  if (n > 0)
    DP_LAUNCHED(1), k_mirror_batch<<<nblk(n, 256), 256, 0, st>>>(n, x, cellc, types, sys_of, geoms,
                                                               off);
}

void launch_build_list(cudaStream_t st, int64_t n, const double* x, const int32_t* cellc,
                       const float4* off, const int32_t* cell_start, const int32_t* cell_atoms,
                       const CellGeom& g, double rlist, float rc2, int ntypes, const int32_t* sel,
                       int cap, uint32_t* nlist, int32_t* nn, int32_t* status) {
  if (n > 0)
    DP_LAUNCHED(1), k_build_list<<<nblk(n * 32, 128), 128, 0, st>>>(n, x, cellc, off, cell_start, cell_atoms, g,
                                                     rlist, rc2, ntypes, sel, cap, nlist, nn,
                                                     status);
}
