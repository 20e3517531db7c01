// Softmin sweeps over a stored FP32 cost matrix C (N x M, row-major).
//
// Both directions read C once per sweep, coalesced, with streaming 128-bit
// loads; C is never transposed:
//  * row sweep (axis 0): one warp per row, lanes stride the row by float4,
//    per-lane online max + sum-exp, warp-shuffle merge at the end of the row;
//  * column sweep (axis 1): one thread per 4 consecutive columns, rows of a
//    slab streamed in groups of 8 (512 contiguous bytes per warp per row),
//    per-column online max + sum-exp.
// Each CTA covers one chunk of the reduced index and writes (max, sum)
// partials like the points sweep.
#include <cuda_runtime.h>

#include "uot_internal.cuh"

namespace uot {
namespace {

constexpr int kThreads = 256;
constexpr int kRowChunk = 8192;  // max columns per CTA in the row sweep (shared h)
constexpr int kRowsPerCta = 32;  // rows per CTA in the row sweep
constexpr int kColSlabTile = 1024;

__device__ __forceinline__ float ex2f(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__device__ __forceinline__ float key_bias(const float* l2w, const float* pot, int j, double s,
                                          double shift) {
  const float lw = l2w[j];
  if (lw <= 0.5f * kZeroW) return kZeroW;
  const double pj = pot ? (double)pot[j] : 0.0;
  return (float)((double)lw + s * (pj + shift));
}

__device__ __forceinline__ void lse_merge(float& m, float& a, float m2, float a2) {
  const float mn = fmaxf(m, m2);
  a = a * ex2f(m - mn) + a2 * ex2f(m2 - mn);
  m = mn;
}

template <bool VEC>
__global__ void __launch_bounds__(kThreads)
k_dense_rows(const float* __restrict__ C, int n, int m, const float* __restrict__ l2w,
             const float* __restrict__ pot, const double* __restrict__ shift, double s, int kps,
             float* __restrict__ part) {
  __shared__ float hs[kRowChunk];
  const int split = blockIdx.y;
  const int j0 = split * kps;
  const int j1 = min(m, j0 + kps);
  const int cnt = j1 - j0;
  const double sh = shift ? *shift : 0.0;
  for (int u = threadIdx.x; u < cnt; u += kThreads) hs[u] = key_bias(l2w, pot, j0 + u, s, sh);
  __syncthreads();
  const float sf = (float)s;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int r0 = blockIdx.x * kRowsPerCta;
  const int r1 = min(n, r0 + kRowsPerCta);
  for (int row = r0 + warp; row < r1; row += kThreads / 32) {
    const float* crow = C + (size_t)row * m + j0;
    float mx = kInitMax, acc = 0.f;
    int tail = 0;
    if constexpr (VEC) {
      const int cnt512 = cnt & ~511, cnt4 = cnt & ~3;
      // 4 float4 per lane per step: 512 columns per warp step
      for (int base = 0; base < cnt512; base += 512) {
        float4 c[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) c[k] = __ldcs(reinterpret_cast<const float4*>(crow + base + k * 128 + lane * 4));
        float t[16];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const int col = base + k * 128 + lane * 4;
          t[4 * k + 0] = fmaf(-sf, c[k].x, hs[col + 0]);
          t[4 * k + 1] = fmaf(-sf, c[k].y, hs[col + 1]);
          t[4 * k + 2] = fmaf(-sf, c[k].z, hs[col + 2]);
          t[4 * k + 3] = fmaf(-sf, c[k].w, hs[col + 3]);
        }
        float tm = t[0];
#pragma unroll
        for (int k = 1; k < 16; ++k) tm = fmaxf(tm, t[k]);
        const float mn = fmaxf(mx, tm);
        float a = acc * ex2f(mx - mn);
#pragma unroll
        for (int k = 0; k < 16; ++k) a += ex2f(t[k] - mn);
        acc = a;
        mx = mn;
      }
      for (int u = cnt512; u < cnt4; u += 128) {  // leftover whole float4 groups
        const int col = u + lane * 4;
        if (col < cnt4) {
          const float4 c = __ldcs(reinterpret_cast<const float4*>(crow + col));
          const float t0 = fmaf(-sf, c.x, hs[col]), t1 = fmaf(-sf, c.y, hs[col + 1]);
          const float t2 = fmaf(-sf, c.z, hs[col + 2]), t3 = fmaf(-sf, c.w, hs[col + 3]);
          const float mn = fmaxf(mx, fmaxf(fmaxf(t0, t1), fmaxf(t2, t3)));
          acc = acc * ex2f(mx - mn) + ex2f(t0 - mn) + ex2f(t1 - mn) + ex2f(t2 - mn) + ex2f(t3 - mn);
          mx = mn;
        }
      }
      tail = cnt4;
    }
    for (int col = tail + lane; col < cnt; col += 32) {  // scalar tail (or whole row if !VEC)
      const float t = fmaf(-sf, __ldcs(crow + col), hs[col]);
      const float mn = fmaxf(mx, t);
      acc = acc * ex2f(mx - mn) + ex2f(t - mn);
      mx = mn;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      const float m2 = __shfl_xor_sync(0xffffffffu, mx, off);
      const float a2 = __shfl_xor_sync(0xffffffffu, acc, off);
      lse_merge(mx, acc, m2, a2);
    }
    if (lane == 0) {
      float* base = part + (size_t)split * 2 * n;
      base[row] = mx;
      base[(size_t)n + row] = acc;
    }
  }
}

template <bool VEC>
__global__ void __launch_bounds__(kThreads)
k_dense_cols(const float* __restrict__ C, int n, int m, const float* __restrict__ l2w,
             const float* __restrict__ pot, const double* __restrict__ shift, double s, int rps,
             float* __restrict__ part) {
  constexpr int W = VEC ? 4 : 1;
  constexpr int G = 8;
  __shared__ float hs[kColSlabTile];
  const int split = blockIdx.y;
  const int i0 = split * rps;
  const int i1 = min(n, i0 + rps);
  const double sh = shift ? *shift : 0.0;
  const float sf = (float)s;
  const int col = (blockIdx.x * kThreads + threadIdx.x) * W;
  const bool active = col < m;  // with VEC, m % 4 == 0 so the whole float4 is in range
  float mx[W], acc[W];
#pragma unroll
  for (int w = 0; w < W; ++w) { mx[w] = kInitMax; acc[w] = 0.f; }
  for (int it = i0; it < i1; it += kColSlabTile) {
    const int cnt = min(kColSlabTile, i1 - it);
    __syncthreads();
    for (int u = threadIdx.x; u < kColSlabTile; u += kThreads)
      hs[u] = (u < cnt) ? key_bias(l2w, pot, it + u, s, sh) : kZeroW;
    __syncthreads();
    if (!active) continue;
    const float* cbase = C + (size_t)it * m + col;
    for (int u0 = 0; u0 < cnt; u0 += G) {
      float t[G][W];
#pragma unroll
      for (int g = 0; g < G; ++g) {
        const int u = u0 + g;
        const float h = hs[u];  // kZeroW beyond cnt
        if (u < cnt) {
          if constexpr (VEC) {
            const float4 c = __ldcs(reinterpret_cast<const float4*>(cbase + (size_t)u * m));
            t[g][0] = fmaf(-sf, c.x, h);
            t[g][1] = fmaf(-sf, c.y, h);
            t[g][2] = fmaf(-sf, c.z, h);
            t[g][3] = fmaf(-sf, c.w, h);
          } else {
            t[g][0] = fmaf(-sf, __ldcs(cbase + (size_t)u * m), h);
          }
        } else {
#pragma unroll
          for (int w = 0; w < W; ++w) t[g][w] = kZeroW;
        }
      }
#pragma unroll
      for (int w = 0; w < W; ++w) {
        float tm = t[0][w];
#pragma unroll
        for (int g = 1; g < G; ++g) tm = fmaxf(tm, t[g][w]);
        const float mn = fmaxf(mx[w], tm);
        float a = acc[w] * ex2f(mx[w] - mn);
#pragma unroll
        for (int g = 0; g < G; ++g) a += ex2f(t[g][w] - mn);
        acc[w] = a;
        mx[w] = mn;
      }
    }
  }
  if (active) {
    float* base = part + (size_t)split * 2 * m;
#pragma unroll
    for (int w = 0; w < W; ++w) {
      base[col + w] = mx[w];
      base[(size_t)m + col + w] = acc[w];
    }
  }
}

}  // namespace

SweepGeom dense_row_geom(int nrows, int ncols, bool tuned) {
  SweepGeom g{};
  g.threads = kThreads;
  g.rows = 1;
  g.row_blocks = (nrows + kRowsPerCta - 1) / kRowsPerCta;
  // columns per CTA (at most kRowChunk: the shared copy of h)
  const int chunk = tuned ? (int)tune_value("dense.row_chunk", -1, (long long)nrows * ncols, kRowChunk) : kRowChunk;
  int splits = (ncols + chunk - 1) / chunk;
  int kps = (ncols + splits - 1) / splits;
  kps = (kps + 3) & ~3;  // keeps every chunk start 16-byte aligned
  g.keys_per_split = kps;
  g.splits = (ncols + kps - 1) / kps;
  return g;
}

SweepGeom dense_col_geom(int nrows, int ncols, bool tuned) {
  SweepGeom g{};
  g.threads = kThreads;
  g.rows = 1;
  const int W = (ncols % 4 == 0) ? 4 : 1;
  const int cols_per_cta = kThreads * W;
  g.row_blocks = (ncols + cols_per_cta - 1) / cols_per_cta;
  const long long target =
      (long long)device_sm_count() * (tuned ? tune_value("dense.col_ctas", -1, (long long)nrows * ncols, 4) : 4);
  long long splits = (target + g.row_blocks - 1) / g.row_blocks;
  const long long cap = (nrows + 63) / 64;  // at least 64 rows per slab
  if (splits > cap) splits = cap;
  if (splits > 256) splits = 256;
  if (splits < 1) splits = 1;
  g.keys_per_split = (int)((nrows + splits - 1) / splits);
  g.splits = (nrows + g.keys_per_split - 1) / g.keys_per_split;
  return g;
}

cudaError_t launch_dense_sweep(int axis, const float* C, int n, int m, const float* l2w_k,
                               const float* pot_k, const double* shift_k, double s, float* part,
                               const SweepGeom& g, cudaStream_t st) {
  // C is 16-byte aligned (checked by the API), so float4 rows need only m % 4 == 0.
  const bool aligned = (m % 4 == 0);
  dim3 grid(g.row_blocks, g.splits);
  if (axis == 0) {
    if (aligned) k_dense_rows<true><<<grid, kThreads, 0, st>>>(C, n, m, l2w_k, pot_k, shift_k, s, g.keys_per_split, part);
    else k_dense_rows<false><<<grid, kThreads, 0, st>>>(C, n, m, l2w_k, pot_k, shift_k, s, g.keys_per_split, part);
  } else {
    if (aligned) k_dense_cols<true><<<grid, kThreads, 0, st>>>(C, n, m, l2w_k, pot_k, shift_k, s, g.keys_per_split, part);
    else k_dense_cols<false><<<grid, kThreads, 0, st>>>(C, n, m, l2w_k, pot_k, shift_k, s, g.keys_per_split, part);
  }
  note_launch();
  return cudaGetLastError();
}

}  // namespace uot
