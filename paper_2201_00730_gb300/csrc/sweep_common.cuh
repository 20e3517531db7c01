// Helpers shared by the fused point-cloud sweeps: exp2 on the MUFU, packed
// f32x2 arithmetic (one issue slot for two lanes) and the exact one-row
// softmin used to recompute rows whose fixed reference missed.
#pragma once

#include <cuda_runtime.h>

#include "uot_internal.cuh"

namespace uot {
namespace simd {

typedef unsigned long long u64;

__device__ __forceinline__ float ex2f(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float max3f(float a, float b, float c) {
  float d;
  asm("max.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
  return d;
}
__device__ __forceinline__ u64 pk(float a, float b) {
  u64 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ void upk(u64 v, float& a, float& b) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
}
__device__ __forceinline__ u64 fma2(u64 a, u64 b, u64 c) {
  u64 d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
__device__ __forceinline__ u64 add2(u64 a, u64 b) {
  u64 d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ u64 mul2(u64 a, u64 b) {
  u64 d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}

// Neumaier's compensated addition s + y (running sum s, compensation c).
__device__ __forceinline__ void neu_add(float& s, float& c, float y) {
  const float t = s + y;
  c += (fabsf(s) >= fabsf(y)) ? ((s - t) + y) : ((y - t) + s);
  s = t;
}

// Softmin partial of one query row over all keys in the direct form, one warp
// with a running max per lane; the lanes' pairs are combined on every lane.
template <int D>
__device__ inline void exact_row(const float* __restrict__ xq, const float* __restrict__ kp, int nk,
                          const float* __restrict__ l2w, const float* __restrict__ pot, float sf, int lane,
                          float& Mo, float& So) {
  float x[D];
#pragma unroll
  for (int d = 0; d < D; ++d) x[d] = xq[d];
  float Mx = kInitMax, Sx = 0.f;
  for (int j = lane; j < nk; j += 32) {
    float r2 = 0.f;
#pragma unroll
    for (int d = 0; d < D; ++d) { const float dd = x[d] - kp[(size_t)j * D + d]; r2 = fmaf(dd, dd, r2); }
    const float lw = l2w[j];
    if (lw <= 0.5f * kZeroW) continue;
    const float t = fmaf(-sf, r2, fmaf(sf, pot ? pot[j] : 0.f, lw));
    const float mn = fmaxf(Mx, t);
    Sx = Sx * ex2f(Mx - mn) + ex2f(t - mn);
    Mx = mn;
  }
  for (int off = 16; off > 0; off >>= 1) {
    const float M2 = __shfl_xor_sync(0xffffffffu, Mx, off);
    const float S2 = __shfl_xor_sync(0xffffffffu, Sx, off);
    const float mn = fmaxf(Mx, M2);
    Sx = Sx * ex2f(Mx - mn) + S2 * ex2f(M2 - mn);
    Mx = mn;
  }
  Mo = Mx;
  So = Sx;
}

}  // namespace simd
}  // namespace uot
