// The fitting net's activation, shared by the CUDA-core and tensor-core
// fitting kernels: tanh (the CUDA math library's tanhf) or the tanh table of
// Sec. 3.5 (second order on [0, 8) in 1024 intervals of 1/128, odd symmetry,
// 1 beyond 8).  Returns t and stores dt/da in d: 1 - t^2 for tanhf, the
// table polynomial's own derivative for the table (so the forces remain the
// exact gradient of the energy the table gives).
#pragma once
#include <cuda_runtime.h>

// the table path, kept out of line so that the epilogues' default (tanhf)
// path stays as short as it was
static __device__ __noinline__ float act_tanh_table(float a, const float4* __restrict__ tab, float* d) {
  const float ax = fabsf(a);
  if (ax >= 8.0f) {
    *d = 0.0f;
    return copysignf(1.0f, a);
  }
  const int k = min((int)(ax * 128.0f), 1023);
  const float u = ax - (float)k * (1.0f / 128.0f);  // exact: both within a factor 2
  const float4 c = __ldg(tab + k);                   // (a0, a1, a2, 0)
  *d = fmaf(2.0f * c.z, u, c.y);
  return copysignf(fmaf(fmaf(c.z, u, c.y), u, c.x), a);
}

__device__ __forceinline__ float act_tanh(float a, const float4* __restrict__ tab, float& d) {
  if (tab) return act_tanh_table(a, tab, &d);
  const float t = tanhf(a);
  d = 1.0f - t * t;
  return t;
}

// compile-time choice for the tensor-core epilogues: the default instantiation
// carries no table code at all
template <bool TAB>
__device__ __forceinline__ float act_tanh_t(float a, const float4* __restrict__ tab, float& d) {
  if constexpr (TAB) {
    return act_tanh_table(a, tab, &d);
  } else {
    const float t = tanhf(a);
    d = 1.0f - t * t;
    return t;
  }
}
