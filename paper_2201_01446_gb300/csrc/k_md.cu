// Velocity-Verlet integration (paper Sec. 4), force finalisation and the
// deterministic reductions for energy, virial and kinetic energy.
#include "dp_internal.h"

unsigned long long g_dp_launches = 0;
thread_local unsigned long long g_dp_launches_tl = 0;

namespace {

__global__ void k_force_finalize(int64_t n, const unsigned long long* __restrict__ ffix,
                                 double* __restrict__ f, int32_t* __restrict__ status) {
  int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n * 3) return;
  f[k] = (double)(long long)ffix[k] * DP_FINV;
}

// stage 1 of a fixed-order sum: block b adds rows [b*chunk, (b+1)*chunk)
__global__ void k_sum_stage1(int64_t rows, int width, int64_t chunk, const double* __restrict__ in,
                             double* __restrict__ part) {
  __shared__ double sm[256];
  const int64_t r0 = blockIdx.x * chunk;
  const int64_t r1 = min(rows, r0 + chunk);
  for (int c = 0; c < width; ++c) {
    double s = 0.0;
    for (int64_t r = r0 + threadIdx.x; r < r1; r += blockDim.x) s += in[r * width + c];
    sm[threadIdx.x] = s;
    __syncthreads();
    for (int o = 128; o >= 1; o >>= 1) {
      if (threadIdx.x < o) sm[threadIdx.x] += sm[threadIdx.x + o];
      __syncthreads();
    }
    if (threadIdx.x == 0) part[(int64_t)blockIdx.x * width + c] = sm[0];
    __syncthreads();
  }
}

__global__ void k_sum_stage2(int nblk, int width, const double* __restrict__ part,
                             double* __restrict__ out) {
  const int c = threadIdx.x;
  if (c >= width) return;
  double s = 0.0;
  for (int b = 0; b < nblk; ++b) s += part[b * width + c];
  out[c] = s;
}

constexpr int kSumBlocks = 512;

// the same two stages for several segments at once (segment q: rows
// [off[q], off[q] + rows[q]) of in): every segment gets exactly the
// additions launch_sum_rows would make on it alone
__global__ void k_sum_stage1_seg(const int64_t* __restrict__ seg_rows,
                                 const int64_t* __restrict__ seg_off, int width,
                                 const double* __restrict__ in, double* __restrict__ part) {
  __shared__ double sm[256];
  const int q = blockIdx.y;
  const int64_t rows = seg_rows[q];
  int64_t chunk = (rows + kSumBlocks - 1) / kSumBlocks;
  if (chunk < 1) chunk = 1;
  const double* src = in + seg_off[q] * width;
  const int64_t r0 = blockIdx.x * chunk;
  const int64_t r1 = min(rows, r0 + chunk);
  for (int c = 0; c < width; ++c) {
    double s = 0.0;
    for (int64_t r = r0 + threadIdx.x; r < r1; r += blockDim.x) s += src[r * width + c];
    sm[threadIdx.x] = s;
    __syncthreads();
    for (int o = 128; o >= 1; o >>= 1) {
      if (threadIdx.x < o) sm[threadIdx.x] += sm[threadIdx.x + o];
      __syncthreads();
    }
    if (threadIdx.x == 0) part[((int64_t)q * kSumBlocks + blockIdx.x) * width + c] = sm[0];
    __syncthreads();
  }
}

__global__ void k_sum_stage2_seg(int nseg, int width, const double* __restrict__ part,
                                 double* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nseg * width) return;
  const int q = i / width, c = i - q * width;
  double s = 0.0;
  for (int b = 0; b < kSumBlocks; ++b) s += part[((int64_t)q * kSumBlocks + b) * width + c];
  out[i] = s;
}

// out[c] = in[0][c] + in[1][c] + ... (sequential from 0)
__global__ void k_add_rows(int nrows, int width, const double* __restrict__ in,
                           double* __restrict__ out) {
  const int c = threadIdx.x;
  if (c >= width) return;
  double s = 0.0;
  for (int r = 0; r < nrows; ++r) s += in[r * width + c];
  out[c] = s;
}

__global__ void k_kick_drift(int64_t n, double* __restrict__ x, double* __restrict__ v,
                             const double* __restrict__ f, const int32_t* __restrict__ types,
                             const double* __restrict__ inv_mass_acc, double dt,
                             const double* __restrict__ xref, double half_skin2,
                             int32_t* __restrict__ status) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double a = 0.5 * dt * inv_mass_acc[types[i]];
  double d2 = 0.0;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    double vv = v[i * 3 + c] + a * f[i * 3 + c];
    v[i * 3 + c] = vv;
    double xx = x[i * 3 + c] + dt * vv;
    x[i * 3 + c] = xx;
    double d = xx - xref[i * 3 + c];
    d2 += d * d;
  }
  if (d2 > half_skin2) atomicAdd(&status[ST_SKIN], 1);
}

__global__ void k_kick(int64_t n, double* __restrict__ v, const double* __restrict__ f,
                       const int32_t* __restrict__ types, const double* __restrict__ inv_mass_acc,
                       const double* __restrict__ mass, double dt, double* __restrict__ ke) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int t = types[i];
  const double a = 0.5 * dt * inv_mass_acc[t];
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    double vv = v[i * 3 + c] + a * f[i * 3 + c];
    v[i * 3 + c] = vv;
    s += vv * vv;
  }
  if (ke) ke[i] = 0.5 * mass[t] * s;
}

__global__ void k_check_energy(int64_t n, const double* __restrict__ e, int32_t* __restrict__ status) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (!isfinite(e[i])) atomicAdd(&status[ST_NONFINITE], 1);
}

__global__ void k_map_types(int64_t n, const int32_t* __restrict__ in, const int32_t* __restrict__ map,
                            int nmap, int32_t* __restrict__ out, int32_t* __restrict__ status) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int t = in[i];
  if (t < 0 || t >= nmap) {
    atomicAdd(&status[ST_BADTYPE], 1);
    t = 0;
  }
  out[i] = map[t];
}

inline int nblk(int64_t n, int t) { return (int)((n + t - 1) / t); }

}  // namespace

void launch_zero_forces(cudaStream_t st, int64_t n, unsigned long long* ffix) {
  if (n > 0) cudaMemsetAsync(ffix, 0, sizeof(unsigned long long) * 3 * (size_t)n, st);
}

void launch_force_finalize(cudaStream_t st, int64_t n, const unsigned long long* ffix, double* f,
                           int32_t* status) {
  if (n > 0) DP_LAUNCHED(1), k_force_finalize<<<nblk(n * 3, 256), 256, 0, st>>>(n, ffix, f, status);
}

int sum_rows_part_size(int64_t rows, int width) { return kSumBlocks * width; }

void launch_sum_rows(cudaStream_t st, int64_t rows, int width, const double* in, double* part,
                     double* out) {
  int64_t chunk = (rows + kSumBlocks - 1) / kSumBlocks;
  if (chunk < 1) chunk = 1;
  DP_LAUNCHED(2);
  k_sum_stage1<<<kSumBlocks, 256, 0, st>>>(rows, width, chunk, in, part);
  k_sum_stage2<<<1, 32, 0, st>>>(kSumBlocks, width, part, out);
}

int64_t sum_rows_seg_part_size(int nseg, int width) { return (int64_t)nseg * kSumBlocks * width; }

void launch_sum_rows_seg(cudaStream_t st, int nseg, const int64_t* seg_rows, const int64_t* seg_off,
                         int width, const double* in, double* part, double* out) {
  if (nseg <= 0) return;
  DP_LAUNCHED(2);
  k_sum_stage1_seg<<<dim3(kSumBlocks, nseg), 256, 0, st>>>(seg_rows, seg_off, width, in, part);
  k_sum_stage2_seg<<<(nseg * width + 127) / 128, 128, 0, st>>>(nseg, width, part, out);
}

void launch_add_rows(cudaStream_t st, int nrows, int width, const double* in, double* out) {
  DP_LAUNCHED(1);
  k_add_rows<<<1, 32, 0, st>>>(nrows, width, in, out);
}

void launch_kick_drift(cudaStream_t st, int64_t n, double* x, double* v, const double* f,
                       const int32_t* types, const double* inv_mass_acc, double dt,
                       const double* xref, double half_skin2, int32_t* status) {
  if (n > 0)
    DP_LAUNCHED(1), k_kick_drift<<<nblk(n, 256), 256, 0, st>>>(n, x, v, f, types, inv_mass_acc, dt, xref,
                                               half_skin2, status);
}

void launch_kick(cudaStream_t st, int64_t n, double* v, const double* f, const int32_t* types,
                 const double* inv_mass_acc, const double* mass, double dt, double* ke) {
  if (n > 0) DP_LAUNCHED(1), k_kick<<<nblk(n, 256), 256, 0, st>>>(n, v, f, types, inv_mass_acc, mass, dt, ke);
}

void launch_check_energy(cudaStream_t st, int64_t n, const double* e, int32_t* status) {
  if (n > 0) DP_LAUNCHED(1), k_check_energy<<<nblk(n, 256), 256, 0, st>>>(n, e, status);
}

void launch_map_types(cudaStream_t st, int64_t n, const int32_t* in, const int32_t* map, int nmap,
                      int32_t* out, int32_t* status) {
  if (n > 0) DP_LAUNCHED(1), k_map_types<<<nblk(n, 256), 256, 0, st>>>(n, in, map, nmap, out, status);
}
