// dp_neighbor_pairs_static: the neighbor-pair build of dp_neighbor_pairs for
// callers that cannot allocate device memory -- for example an MD engine
// that hands every device allocation to its own memory pool, or a
// time-critical loop in which cudaMalloc/cudaFree (which can synchronise
// the whole device) must not run.  The caller passes device input and
// output buffers; every intermediate (wrapped positions, cell lists, pair
// counts and offsets) lives in one file-scope __device__ array of fixed
// size that each GPU loading this library keeps until the process exits.
//
// Limits: at most kStaticMaxAtoms atoms and kStaticMaxCells cells (cells
// have edge >= rlist); larger requests return DP_ERR_CAPACITY before any
// device work.  The array is shared by every call on a device and keeps
// the last call's contents: each call clears the parts that must start at
// zero, and calls whose device work overlaps (different streams or host
// threads without ordering) race on it.  The first call on a device looks
// up the array's device address (cudaGetSymbolAddress) with that device
// current; make that first call before any stream capture.
#include <cmath>
#include <mutex>

#include "dp_internal.h"

namespace {

constexpr int kStaticMaxAtoms = 65536;
constexpr int kStaticMaxCells = 65536;

constexpr size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }
// layout of the static scratch (byte offsets)
constexpr size_t kOffX = 0;                                               // double [N][3]
constexpr size_t kOffCellc = align256(kOffX + sizeof(double) * 3 * kStaticMaxAtoms);
constexpr size_t kOffTmp = align256(kOffCellc + sizeof(int) * kStaticMaxAtoms);
constexpr size_t kOffAtoms = align256(kOffTmp + sizeof(int) * kStaticMaxAtoms);
constexpr size_t kOffOff = align256(kOffAtoms + sizeof(int) * kStaticMaxAtoms);  // float4 [N]
constexpr size_t kOffTypes = align256(kOffOff + sizeof(float4) * kStaticMaxAtoms);
constexpr size_t kOffCnt = align256(kOffTypes + sizeof(int) * kStaticMaxAtoms);
constexpr size_t kOffRow = align256(kOffCnt + sizeof(int) * kStaticMaxAtoms);  // int64 [N+1]
constexpr size_t kOffCellCount = align256(kOffRow + sizeof(int64_t) * (kStaticMaxAtoms + 1));
constexpr size_t kOffCellFill = align256(kOffCellCount + sizeof(int) * (kStaticMaxCells + 1));
constexpr size_t kOffCellStart = align256(kOffCellFill + sizeof(int) * (kStaticMaxCells + 1));
constexpr size_t kStaticBytes = align256(kOffCellStart + sizeof(int) * (kStaticMaxCells + 1));

__device__ __align__(256) unsigned char g_static_scratch[kStaticBytes];

// device address of g_static_scratch per device, looked up once
constexpr int kMaxDevices = 64;
void* g_static_ptr[kMaxDevices] = {nullptr};
std::mutex g_static_mu;

dp_status static_scratch(unsigned char** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return DP_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_static_mu);
  if (!g_static_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess || !p) return DP_ERR_CUDA;
    g_static_ptr[dev] = p;
  }
  *out = static_cast<unsigned char*>(g_static_ptr[dev]);
  return DP_OK;
}

// row offsets of the atoms' pair rows: start[i] = sum of cnt[k < i] and
// start[n] = the total, in 64-bit integers (65536 atoms in a box of edge
// rlist see 27 images of every atom: ~1.2e11 rows, past any 32-bit offset).
// One block; thread t scans its contiguous run of atoms, the runs' totals
// are scanned across the block, then each run is written.
constexpr int kScanThreads = 1024;
__global__ void __launch_bounds__(kScanThreads) k_static_scan64(const int32_t* __restrict__ cnt,
                                                                int n,
                                                                int64_t* __restrict__ start) {
  __shared__ int64_t warp_tot[kScanThreads / 32];
  const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
  const int per = (n + kScanThreads - 1) / kScanThreads;
  const int b = min(n, t * per), e = min(n, b + per);
  int64_t run = 0;
  for (int k = b; k < e; ++k) run += cnt[k];
  // inclusive scan of the runs within the warp, then across the warps
  int64_t inc = run;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const int64_t v = __shfl_up_sync(0xffffffffu, inc, d);
    if (lane >= d) inc += v;
  }
  if (lane == 31) warp_tot[wid] = inc;
  __syncthreads();
  if (wid == 0) {
    int64_t w = warp_tot[lane];
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const int64_t v = __shfl_up_sync(0xffffffffu, w, d);
      if (lane >= d) w += v;
    }
    warp_tot[lane] = w;  // inclusive totals of warps 0..lane
  }
  __syncthreads();
  int64_t acc = inc - run + (wid > 0 ? warp_tot[wid - 1] : 0);
  for (int k = b; k < e; ++k) {
    start[k] = acc;
    acc += cnt[k];
  }
  if (t == kScanThreads - 1) start[n] = warp_tot[kScanThreads / 32 - 1];
}

// pairs of atom i within rlist, counted (rows == nullptr) or written as
// (i, j, n0, n1, n2) rows from row_start[i] on (rows past cap are dropped);
// one warp per atom in cell order, the same tests as the list build
__global__ void __launch_bounds__(128) k_static_pairs(
    int n, const double* __restrict__ x, const int32_t* __restrict__ cellc,
    const float4* __restrict__ off, const int32_t* __restrict__ cell_start,
    const int32_t* __restrict__ cell_atoms, CellGeom g, double rlist, int32_t* __restrict__ cnt,
    const int64_t* __restrict__ row_start, int64_t cap, int32_t* __restrict__ rows) {
  const int lane = threadIdx.x & 31;
  const int w = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  if (w >= n) return;
  const int i = cell_atoms[w];
  const int id = cellc[i];
  const int ci[3] = {id / (g.nc[2] * g.nc[1]), (id / g.nc[2]) % g.nc[1], id % g.nc[2]};
  const float4 oi = off[i];
  const double rl2 = rlist * rlist;
  const float rl2f = (float)rl2;
  const float lo = rl2f * (1.0f - 1e-4f), hi = rl2f * (1.0f + 1e-4f);
  const unsigned below = (1u << lane) - 1u;
  int c = 0;
  for (int slot = 0; slot < 27; ++slot) {
    const int o[3] = {slot / 9 - 1, (slot / 3) % 3 - 1, slot % 3 - 1};
    int cc[3], img[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const int v = ci[a] + o[a];
      img[a] = v < 0 ? -1 : (v >= g.nc[a] ? 1 : 0);
      cc[a] = v - img[a] * g.nc[a];
    }
    const int cid = (cc[0] * g.nc[1] + cc[1]) * g.nc[2] + cc[2];
    const int s = cell_start[cid], e = cell_start[cid + 1];
    const float sx = o[0] * g.edgef[0], sy = o[1] * g.edgef[1], sz = o[2] * g.edgef[2];
    for (int base = s; base < e; base += 32) {
      const int k = base + lane;
      bool in = false;
      int j = 0;
      if (k < e) {
        j = cell_atoms[k];
        const float4 oj = off[j];
        const float dx = (oj.x - oi.x) + sx, dy = (oj.y - oi.y) + sy, dz = (oj.z - oi.z) + sz;
        const float r2 = dx * dx + dy * dy + dz * dz;
        if (!((j == i) && slot == 13)) {
          if (r2 < lo) {
            in = true;
          } else if (r2 <= hi) {
            double r2d = 0.0;
#pragma unroll
            for (int a = 0; a < 3; ++a) {
              const double d = __dadd_rn(__dsub_rn(x[(size_t)j * 3 + a], x[(size_t)i * 3 + a]),
                                         __dmul_rn((double)img[a], g.L[a]));
              r2d = __dadd_rn(r2d, __dmul_rn(d, d));
            }
            in = r2d < rl2;
          }
        }
      }
      const unsigned m = __ballot_sync(0xffffffffu, in);
      if (in && rows) {
        const int64_t r = row_start[i] + c + __popc(m & below);
        if (r >= 0 && r < cap) {
          int32_t* q = rows + r * 5;
          q[0] = i;
          q[1] = j;
          q[2] = img[0];
          q[3] = img[1];
          q[4] = img[2];
        }
      }
      c += __popc(m);
    }
  }
  if (lane == 0 && !rows) cnt[i] = c;
}

}  // namespace

extern "C" dp_status dp_neighbor_pairs_static(int64_t natoms, const double* coords,
                                              const double* box, double rlist, int64_t cap,
                                              int32_t* out5, int64_t* count, void* stream) {
  if (natoms < 0 || !box || !count || !(rlist > 0) || (natoms > 0 && !coords) || cap < 0 ||
      (cap > 0 && !out5))
    return DP_ERR_ARG;
  if (natoms > kStaticMaxAtoms) return DP_ERR_CAPACITY;
  CellGeom g{};
  long long ncell = 1;
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b)
      if (a != b && box[a * 3 + b] != 0.0) return DP_ERR_BOX;
  for (int a = 0; a < 3; ++a) {
    const double L = box[a * 4];
    if (!(L > 0.0) || L < rlist) return DP_ERR_BOX;
    g.L[a] = L;
    // compared as a double first: a huge L / rlist must not reach the int
    const double ncd = std::floor(L / rlist);
    if (!(ncd <= (double)kStaticMaxCells)) return DP_ERR_CAPACITY;
    const int nc = (int)ncd;
    g.nc[a] = nc < 1 ? 1 : nc;
    g.edge[a] = L / g.nc[a];
    g.edgef[a] = (float)g.edge[a];
    ncell *= g.nc[a];
  }
  if (ncell > kStaticMaxCells) return DP_ERR_CAPACITY;
  g.ncell = ncell;
  *count = 0;
  if (natoms == 0) return DP_OK;
  unsigned char* sc = nullptr;
  dp_status st = static_scratch(&sc);
  if (st != DP_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int n = (int)natoms;
  double* xw = reinterpret_cast<double*>(sc + kOffX);
  int32_t* cellc = reinterpret_cast<int32_t*>(sc + kOffCellc);
  int32_t* tmp = reinterpret_cast<int32_t*>(sc + kOffTmp);
  int32_t* atoms = reinterpret_cast<int32_t*>(sc + kOffAtoms);
  float4* off = reinterpret_cast<float4*>(sc + kOffOff);
  int32_t* types = reinterpret_cast<int32_t*>(sc + kOffTypes);
  int32_t* cnt = reinterpret_cast<int32_t*>(sc + kOffCnt);
  int64_t* row = reinterpret_cast<int64_t*>(sc + kOffRow);
  int32_t* ccount = reinterpret_cast<int32_t*>(sc + kOffCellCount);
  int32_t* cfill = reinterpret_cast<int32_t*>(sc + kOffCellFill);
  int32_t* cstart = reinterpret_cast<int32_t*>(sc + kOffCellStart);
  // the parts the kernels accumulate into start from zero on every call
  if (cudaMemsetAsync(ccount, 0, sizeof(int32_t) * (ncell + 1), s) != cudaSuccess ||
      cudaMemsetAsync(cfill, 0, sizeof(int32_t) * (ncell + 1), s) != cudaSuccess ||
      cudaMemsetAsync(types, 0, sizeof(int32_t) * n, s) != cudaSuccess ||
      cudaMemcpyAsync(xw, coords, sizeof(double) * 3 * n, cudaMemcpyDeviceToDevice, s) !=
          cudaSuccess)
    return DP_ERR_CUDA;
  launch_wrap_bin(s, n, xw, g, cellc, ccount);
  launch_scan(s, ccount, cstart, ncell);
  launch_scatter(s, n, cellc, cstart, cfill, tmp);
  launch_cell_sort(s, ncell, cstart, tmp, atoms);
  launch_mirror(s, n, xw, cellc, types, g, off);
  const int blocks = (int)(((int64_t)n * 32 + 127) / 128);
  k_static_pairs<<<blocks, 128, 0, s>>>(n, xw, cellc, off, cstart, atoms, g, rlist, cnt, nullptr, 0,
                                       nullptr);
  k_static_scan64<<<1, kScanThreads, 0, s>>>(cnt, n, row);
  k_static_pairs<<<blocks, 128, 0, s>>>(n, xw, cellc, off, cstart, atoms, g, rlist, cnt, row, cap,
                                       out5);
  DP_LAUNCHED(3);
  int64_t total = 0;
  if (cudaGetLastError() != cudaSuccess ||
      cudaMemcpyAsync(&total, row + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return DP_ERR_CUDA;
  *count = total;
  return DP_OK;
}
