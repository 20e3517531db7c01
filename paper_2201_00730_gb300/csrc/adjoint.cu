// Adjoint sweeps of the softmin, for the unrolled backward pass.
//
// A softmin over keys k with known normaliser (the key's own softmin value h_k)
//     h_k = -eps log sum_q w_q exp((pot_q - C_qk)/eps)
// has softmax weights P_qk = w_q exp((pot_q - C_qk + h_k)/eps).  Its vector-
// Jacobian product with a cotangent c_k on h needs, for every query q,
//     R_q   = sum_k c_k exp((pot_q - C_qk + h_k)/eps)        (pot_bar_q -= w_q R_q, w_bar_q -= eps R_q)
//     Mo_q  = sum_k c_k exp((pot_q - C_qk + h_k)/eps) (q - k) (q_bar += 2 w_q Mo_q, for C = |q - k|^2)
// i.e. one more O(NM) pass with signed coefficients.  The exponent is taken
// relative to a running max (base 2), as in the forward sweeps, and chunks of
// keys write partials (max, sums) merged in FP64 by k_adjoint_merge.
#include <cuda_runtime.h>
#include <math.h>

#include "uot_internal.cuh"

namespace uot {
namespace {

constexpr int kThreads = 256;
constexpr int kTile = 64;

__device__ __forceinline__ float ex2f(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

template <int DMAX>
__global__ void __launch_bounds__(kThreads)
k_adjoint(const float* __restrict__ q, int nq, const float* __restrict__ kp, int nk, int dim,
          const float* __restrict__ pot_q, const float* __restrict__ h_k, const float* __restrict__ c_k, double s,
          int kps, float* __restrict__ part) {
  extern __shared__ float sk[];  // [kTile][dim + 2]: coords, s*h_k, c_k
  const int split = blockIdx.y;
  const int j0 = split * kps;
  const int j1 = min(nk, j0 + kps);
  const int ld = dim + 2;
  const int i = blockIdx.x * kThreads + threadIdx.x;
  const float sf = (float)s;
  float xq[DMAX];
#pragma unroll
  for (int d = 0; d < DMAX; ++d) xq[d] = (i < nq && d < dim) ? q[(size_t)i * dim + d] : 0.f;
  const float zq = (i < nq) ? sf * pot_q[i] : 0.f;
  float mx = kInitMax, acc = 0.f;
  float mom[DMAX];
#pragma unroll
  for (int d = 0; d < DMAX; ++d) mom[d] = 0.f;
  for (int jt = j0; jt < j1; jt += kTile) {
    const int cnt = min(kTile, j1 - jt);
    __syncthreads();
    for (int e = threadIdx.x; e < kTile * ld; e += kThreads) {
      const int u = e / ld, d = e - u * ld;
      float v = 0.f;
      if (u < cnt) {
        const int j = jt + u;
        v = (d < dim) ? kp[(size_t)j * dim + d] : (d == dim ? (float)(s * (double)h_k[j]) : c_k[j]);
      } else if (d == dim) {
        v = kZeroW;
      }
      sk[e] = v;
    }
    __syncthreads();
    for (int u = 0; u < cnt; ++u) {
      const float* kv = sk + u * ld;
      float r2 = 0.f;
#pragma unroll
      for (int d = 0; d < DMAX; ++d)
        if (d < dim) { const float dd = xq[d] - kv[d]; r2 = fmaf(dd, dd, r2); }
      const float z = fmaf(-sf, r2, zq + kv[dim]);
      const float mn = fmaxf(mx, z);
      const float sc = ex2f(mx - mn);
      const float e = kv[dim + 1] * ex2f(z - mn);
      acc = fmaf(acc, sc, e);
#pragma unroll
      for (int d = 0; d < DMAX; ++d)
        if (d < dim) mom[d] = fmaf(mom[d], sc, e * (xq[d] - kv[d]));
      mx = mn;
    }
  }
  if (i < nq) {
    const int CH = 2 + dim;
    float* base = part + (size_t)split * CH * nq;
    base[i] = mx;
    base[(size_t)nq + i] = acc;
#pragma unroll
    for (int d = 0; d < DMAX; ++d)
      if (d < dim) base[(size_t)(2 + d) * nq + i] = mom[d];
  }
}

// value_q = 2^M sum; moments alike; FP64 assembly of the key chunks.
// One thread per (row, channel c): c = 0 the value, c = 1 + d moment d (rows fastest:
// coalesced partial loads).  Chunk weights 2^(M_k - M) in FP32 (relative error ~1e-7), the
// sums and the common factor 2^M in FP64.
__global__ void k_adjoint_merge(const float* part, int nq, int dim, int splits, double* val, double* mom) {
  const int CH = 2 + dim;
  const int c = blockIdx.y;
  const int ch = c == 0 ? 1 : 1 + c;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nq; i += gridDim.x * blockDim.x) {
    float M = kInitMax;
    for (int k = 0; k < splits; ++k) M = fmaxf(M, __ldg(part + (size_t)k * CH * nq + i));
    double v = 0.0;
    for (int k = 0; k < splits; ++k) {
      const float* b = part + (size_t)k * CH * nq;
      v += (double)__ldg(b + (size_t)ch * nq + i) * (double)ex2f(__ldg(b + i) - M);
    }
    v *= exp2((double)M);
    if (c == 0) val[i] = v;
    else mom[(size_t)i * dim + (c - 1)] = v;
  }
}

}  // namespace

SweepGeom adjoint_geom(int nq, int nk) {
  SweepGeom g{};
  g.threads = kThreads;
  g.rows = 1;
  g.row_blocks = (nq + kThreads - 1) / kThreads;
  const long long target = (long long)device_sm_count() * 2;
  long long splits = (target + g.row_blocks - 1) / g.row_blocks;
  const long long cap = (nk + kTile - 1) / kTile;
  if (splits > cap) splits = cap;
  if (splits > 256) splits = 256;
  if (splits < 1) splits = 1;
  g.keys_per_split = (int)((nk + splits - 1) / splits);
  g.splits = (nk + g.keys_per_split - 1) / g.keys_per_split;
  return g;
}

cudaError_t launch_adjoint(const float* q, int nq, const float* kp, int nk, int dim, const float* pot_q,
                           const float* h_k, const float* c_k, double s, float* part, double* val, double* mom,
                           const float* center, const int* maxbits, const MomOperands& mo, cudaStream_t st) {
  if (center && dim >= 32) {
    const SweepGeom gf = mom_geom(nq, nk);
    cudaError_t e = launch_mom_sweep(mo.opq, mo.nq2, nq, mo.opk, mo.nk2, nk, q, kp, dim, center, maxbits, nullptr,
                                     nullptr, nullptr, pot_q, h_k, c_k, s, 1.0f, mo.zt, mo.multbits, part, gf,
                                     mo.status, st);
    if (e != cudaSuccess) return e;
    k_adjoint_merge<<<dim3((nq + 255) / 256, dim + 1), 256, 0, st>>>(part, nq, dim, gf.splits, val, mom);
    note_launch();
    return cudaGetLastError();
  }
  const SweepGeom g = adjoint_geom(nq, nk);
  dim3 grid(g.row_blocks, g.splits);
  const size_t smem = sizeof(float) * kTile * (dim + 2);
  if (dim <= 4)
    k_adjoint<4><<<grid, kThreads, smem, st>>>(q, nq, kp, nk, dim, pot_q, h_k, c_k, s, g.keys_per_split, part);
  else if (dim <= 16)
    k_adjoint<16><<<grid, kThreads, smem, st>>>(q, nq, kp, nk, dim, pot_q, h_k, c_k, s, g.keys_per_split, part);
  else
    k_adjoint<64><<<grid, kThreads, smem, st>>>(q, nq, kp, nk, dim, pot_q, h_k, c_k, s, g.keys_per_split, part);
  note_launch();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_adjoint_merge<<<dim3((nq + 255) / 256, dim + 1), 256, 0, st>>>(part, nq, dim, g.splits, val, mom);
  note_launch();
  return cudaGetLastError();
}

}  // namespace uot
