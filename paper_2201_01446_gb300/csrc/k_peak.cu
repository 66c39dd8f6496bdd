// FP32 FMA throughput probe: the denominator of the FP32 CUDA-core
// rooflines (the tabulated embedding's per-pair arithmetic and the plain
// comparator), measured on the GPU at the clock it runs at, since no measured
// FP32 peak is published for GB300.  Every thread runs kChains independent
// FMA chains and 64 warps are resident per SM (16 per scheduler), so the
// FMA latency is covered and every FP32 lane can issue one FMA per cycle.
// The result is written only if it equals a value the chains cannot
// produce, so the compiler keeps every FMA.
#include "dp_internal.h"

namespace {

constexpr int kChains = 8;
constexpr int kPeakThreads = 256;
constexpr int kInner = 64;  // unrolled FMAs per chain per outer iteration

__device__ float g_fma_sink[kPeakThreads];

__global__ void __launch_bounds__(kPeakThreads) k_fma_peak(int64_t outer, float a, float b) {
  float v[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) v[c] = (float)(threadIdx.x + c) * 1e-3f;
  for (int64_t it = 0; it < outer; ++it) {
#pragma unroll
    for (int k = 0; k < kInner; ++k)
#pragma unroll
      for (int c = 0; c < kChains; ++c) v[c] = fmaf(v[c], a, b);
  }
  float s = 0.0f;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += v[c];
  if (s == -12345.678f) g_fma_sink[threadIdx.x] = s;  // never true for the inputs given
}

}  // namespace

extern "C" dp_status dp_fma_peak_run(int64_t outer, void* stream, double* flops) {
  if (outer < 1 || !flops) return DP_ERR_ARG;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return DP_ERR_CUDA;
  const int blocks = sms * 8;  // 8 CTAs of 256 threads = 64 warps per SM
  // a = 1 - 2^-20, b = 2^-20: v stays bounded in (0, 1], finite and normal
  k_fma_peak<<<blocks, kPeakThreads, 0, static_cast<cudaStream_t>(stream)>>>(
      outer, 1.0f - 9.5367431640625e-7f, 9.5367431640625e-7f);
  DP_LAUNCHED(1);
  if (cudaGetLastError() != cudaSuccess) return DP_ERR_CUDA;
  *flops = 2.0 * (double)blocks * kPeakThreads * (double)outer * kInner * kChains;
  return DP_OK;
}
