// Fused softmin sweeps over point clouds: the cost |q_i - k_j|^p is evaluated on
// the fly from shared-memory key tiles and never stored.
//
// For every query point i (a row of C for the row sweep, a column for the
// column sweep) and every key chunk, the kernel produces the partial
// log2-sum-exp of
//     t_ij = log2 w_j + s (pot_j + shift) - s C_ij,      s = log2(e) / eps,
// as a pair (max_j t_ij, sum_j 2^(t_ij - max)).  The softmin of Sec. 3 is then
//     Smin_w^eps(C_i. - pot) = -(max + log2 sum) / s,
// formed by the combine kernel in FP64 after all chunks are merged.
//
// Fast path (dim <= 3, p = 2): coordinates are pre-scaled by sqrt(s) so that
// t = h_j - |q'_i - k'_j|^2 costs dim FADD + dim FFMA per entry; one ex2 per
// entry on the MUFU pipe; the running max is updated once per group of U keys.
// Each thread owns R query points; keys are read from shared memory as float4
// broadcasts.  Optional "moment" channels accumulate sum 2^(t-max) (q'-k')_d,
// used by the envelope gradient.
#include <cuda_runtime.h>

#include "uot_internal.cuh"

namespace uot {
namespace {

constexpr int kThreads = 256;
constexpr int kTile = 512;  // keys staged per shared-memory tile

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

// Key bias h_j = log2 w_j + s (pot_j + shift), formed in FP64 and rounded once.
__device__ __forceinline__ float key_bias(const float* l2w, const float* pot, int j, double s,
                                          double shift) {
  const float lw = l2w[j];
  if (lw <= 0.5f * kZeroW) return kZeroW;
  const double pj = pot ? (double)pot[j] : 0.0;
  return (float)((double)lw + s * (pj + shift));
}

template <int D, int R, int U, bool MOM>
__global__ void __launch_bounds__(kThreads)
k_sweep_small(const float* __restrict__ q, int nq, const float* __restrict__ kp, int nk,
              const float* __restrict__ l2w, const float* __restrict__ pot,
              const double* __restrict__ shift, double s, float rs, int kps,
              float* __restrict__ part) {
  static_assert(D >= 1 && D <= 3, "fast path covers dim 1..3");
  __shared__ float4 sk[kTile];
  const int split = blockIdx.y;
  const int j0 = split * kps;
  const int j1 = min(nk, j0 + kps);
  const double sh = shift ? *shift : 0.0;

  float xq[R][D];
  float mx[R], acc[R];
  float mom[R][MOM ? D : 1];
  const int ibase = blockIdx.x * (kThreads * R) + threadIdx.x;
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int i = ibase + r * kThreads;
#pragma unroll
    for (int d = 0; d < D; ++d) xq[r][d] = (i < nq) ? rs * q[(size_t)i * D + d] : 0.f;
    mx[r] = kInitMax;
    acc[r] = 0.f;
#pragma unroll
    for (int d = 0; d < (MOM ? D : 1); ++d) mom[r][d] = 0.f;
  }

  for (int jt = j0; jt < j1; jt += kTile) {
    const int cnt = min(kTile, j1 - jt);
    __syncthreads();
    for (int u = threadIdx.x; u < kTile; u += kThreads) {
      float4 v = make_float4(0.f, 0.f, 0.f, kZeroW);
      if (u < cnt) {
        const int j = jt + u;
        v.x = rs * kp[(size_t)j * D + 0];
        if constexpr (D > 1) v.y = rs * kp[(size_t)j * D + 1];
        if constexpr (D > 2) v.z = rs * kp[(size_t)j * D + 2];
        v.w = key_bias(l2w, pot, j, s, sh);
      }
      sk[u] = v;
    }
    __syncthreads();
    const int cntU = (cnt + U - 1) / U * U;  // tail keys are zero-weight sentinels
    for (int u0 = 0; u0 < cntU; u0 += U) {
      float t[R][U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const float4 kv = sk[u0 + u];
#pragma unroll
        for (int r = 0; r < R; ++r) {
          const float d0 = xq[r][0] - kv.x;
          float c = fmaf(-d0, d0, kv.w);
          if constexpr (D > 1) { const float d1 = xq[r][1] - kv.y; c = fmaf(-d1, d1, c); }
          if constexpr (D > 2) { const float d2 = xq[r][2] - kv.z; c = fmaf(-d2, d2, c); }
          t[r][u] = c;
        }
      }
#pragma unroll
      for (int r = 0; r < R; ++r) {
        float tm = t[r][0];
#pragma unroll
        for (int u = 1; u + 1 < U; u += 2) tm = max3f(tm, t[r][u], t[r][u + 1]);
        if ((U % 2) == 0) tm = fmaxf(tm, t[r][U - 1]);
        const float mn = fmaxf(mx[r], tm);
        const float sc = ex2f(mx[r] - mn);
        mx[r] = mn;
        float a = acc[r] * sc;
        if constexpr (MOM) {
#pragma unroll
          for (int d = 0; d < D; ++d) mom[r][d] *= sc;
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const float e = ex2f(t[r][u] - mn);
          a += e;
          if constexpr (MOM) {
            const float4 kv = sk[u0 + u];
            mom[r][0] = fmaf(e, xq[r][0] - kv.x, mom[r][0]);
            if constexpr (D > 1) mom[r][1] = fmaf(e, xq[r][1] - kv.y, mom[r][1]);
            if constexpr (D > 2) mom[r][2] = fmaf(e, xq[r][2] - kv.z, mom[r][2]);
          }
        }
        acc[r] = a;
      }
    }
  }

  constexpr int CH = 2 + (MOM ? D : 0);
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int i = ibase + r * kThreads;
    if (i < nq) {
      float* base = part + (size_t)split * CH * nq;
      base[i] = mx[r];
      base[(size_t)nq + i] = acc[r];
      if constexpr (MOM) {
#pragma unroll
        for (int d = 0; d < D; ++d) base[(size_t)(2 + d) * nq + i] = mom[r][d];
      }
    }
  }
}

// Generic path: any dim <= DMAX, any exponent p >= 1, unscaled coordinates.
// One query point per thread; keys staged in shared memory as [tile][dim + 1].
// Moments accumulate sum 2^(t-max) dC/dq (= p |q-k|^(p-2) (q-k)).
constexpr int kGenTile = 64;

template <int DMAX, bool MOM>
__global__ void __launch_bounds__(kThreads)
k_sweep_generic(const float* __restrict__ q, int nq, const float* __restrict__ kp, int nk, int dim,
                float p, const float* __restrict__ l2w, const float* __restrict__ pot,
                const double* __restrict__ shift, double s, int kps, float* __restrict__ part) {
  extern __shared__ float skg[];  // [kGenTile][dim + 1]
  const int split = blockIdx.y;
  const int j0 = split * kps;
  const int j1 = min(nk, j0 + kps);
  const double sh = shift ? *shift : 0.0;
  const float sf = (float)s;
  const int i = blockIdx.x * kThreads + threadIdx.x;
  const int ld = dim + 1;

  float xq[DMAX];
#pragma unroll
  for (int d = 0; d < DMAX; ++d) xq[d] = (i < nq && d < dim) ? q[(size_t)i * dim + d] : 0.f;
  float mx = kInitMax, acc = 0.f;
  float mom[MOM ? DMAX : 1];
#pragma unroll
  for (int d = 0; d < (MOM ? DMAX : 1); ++d) mom[d] = 0.f;
  const bool p2 = (p == 2.0f);
  const float hp = 0.5f * p;

  for (int jt = j0; jt < j1; jt += kGenTile) {
    const int cnt = min(kGenTile, j1 - jt);
    __syncthreads();
    for (int e = threadIdx.x; e < kGenTile * ld; e += kThreads) {
      const int u = e / ld, d = e - u * ld;
      float v;
      if (u < cnt) {
        const int j = jt + u;
        v = (d < dim) ? kp[(size_t)j * dim + d] : key_bias(l2w, pot, j, s, sh);
      } else {
        v = (d < dim) ? 0.f : kZeroW;
      }
      skg[e] = v;
    }
    __syncthreads();
    for (int u = 0; u < cnt; ++u) {
      const float* kv = skg + u * ld;
      float r2 = 0.f;
#pragma unroll
      for (int d = 0; d < DMAX; ++d) {
        if (d < dim) {
          const float dd = xq[d] - kv[d];
          r2 = fmaf(dd, dd, r2);
        }
      }
      float c = p2 ? r2 : ((r2 > 0.f) ? ex2f(hp * __log2f(r2)) : 0.f);
      const float t = fmaf(-sf, c, kv[dim]);
      const float mn = fmaxf(mx, t);
      const float sc = ex2f(mx - mn);
      const float e = ex2f(t - mn);
      acc = fmaf(acc, sc, e);
      if (MOM) {
        float w = e * 2.0f;
        if (!p2) w = (r2 > 0.f) ? e * p * ex2f((hp - 1.0f) * __log2f(r2)) : 0.f;
#pragma unroll
        for (int d = 0; d < DMAX; ++d)
          if (d < dim) mom[d] = fmaf(mom[d], sc, w * (xq[d] - kv[d]));
      }
      mx = mn;
    }
  }
  if (i < nq) {
    const int CH = 2 + (MOM ? dim : 0);
    float* base = part + (size_t)split * CH * nq;
    base[i] = mx;
    base[(size_t)nq + i] = acc;
    if (MOM) {
#pragma unroll
      for (int d = 0; d < DMAX; ++d)
        if (d < dim) base[(size_t)(2 + d) * nq + i] = mom[d];
    }
  }
}

template <int D, int R, bool MOM>
cudaError_t run_small(const SideDesc& q, const SideDesc& k, const float* pot, const double* shift,
                      double s, float* part, const SweepGeom& g, cudaStream_t st) {
  dim3 grid(g.row_blocks, g.splits);
  k_sweep_small<D, R, 8, MOM><<<grid, kThreads, 0, st>>>(q.pts, q.n, k.pts, k.n, k.l2w, pot, shift, s,
                                                        (float)sqrt(s), g.keys_per_split, part);
  note_launch();
  return cudaGetLastError();
}

template <int D, bool MOM>
cudaError_t run_small_r(const SideDesc& q, const SideDesc& k, const float* pot, const double* shift,
                        double s, float* part, const SweepGeom& g, cudaStream_t st) {
  switch (g.rows) {
    case 1: return run_small<D, 1, MOM>(q, k, pot, shift, s, part, g, st);
    case 2: return run_small<D, 2, MOM>(q, k, pot, shift, s, part, g, st);
    default: return run_small<D, 4, MOM>(q, k, pot, shift, s, part, g, st);
  }
}

template <int DMAX, bool MOM>
cudaError_t run_generic(const SideDesc& q, const SideDesc& k, int dim, float p, const float* pot,
                        const double* shift, double s, float* part, const SweepGeom& g,
                        cudaStream_t st) {
  dim3 grid(g.row_blocks, g.splits);
  const size_t smem = sizeof(float) * kGenTile * (dim + 1);
  k_sweep_generic<DMAX, MOM><<<grid, kThreads, smem, st>>>(q.pts, q.n, k.pts, k.n, dim, p, k.l2w, pot,
                                                           shift, s, g.keys_per_split, part);
  note_launch();
  return cudaGetLastError();
}

template <bool MOM>
cudaError_t dispatch(const SideDesc& q, const SideDesc& k, int dim, float p, const float* pot,
                     const double* shift, double s, float* part, const SweepGeom& g, cudaStream_t st) {
  if (p == 2.0f && dim <= 3) {
    if (dim == 1) return run_small_r<1, MOM>(q, k, pot, shift, s, part, g, st);
    if (dim == 2) return run_small_r<2, MOM>(q, k, pot, shift, s, part, g, st);
    return run_small_r<3, MOM>(q, k, pot, shift, s, part, g, st);
  }
  if (dim <= 4) return run_generic<4, MOM>(q, k, dim, p, pot, shift, s, part, g, st);
  if (dim <= 16) return run_generic<16, MOM>(q, k, dim, p, pot, shift, s, part, g, st);
  return run_generic<64, MOM>(q, k, dim, p, pot, shift, s, part, g, st);
}

}  // namespace

cudaError_t launch_points_sweep(const SideDesc& q, const SideDesc& k, int dim, float p,
                                const float* pot_k, const double* shift_k, double s, bool moments,
                                float* part, const SweepGeom& g, cudaStream_t st) {
  return moments ? dispatch<true>(q, k, dim, p, pot_k, shift_k, s, part, g, st)
                 : dispatch<false>(q, k, dim, p, pot_k, shift_k, s, part, g, st);
}

SweepGeom points_geom(int nq, int nk, int dim, bool moments, bool tuned) {
  SweepGeom g{};
  g.threads = kThreads;
  const bool fast = dim <= 3;
  const long long entries = (long long)nq * nk;
  int R = 1;
  if (fast) {
    if (nq >= 64 * kThreads * 4) R = 4;
    else if (nq >= 16 * kThreads * 2) R = 2;
    if (tuned) R = (int)tune_value("points.rows", dim, entries, R);
  }
  if (moments && dim == 3 && R > 2) R = 2;
  g.rows = R;
  const int rows_per_cta = kThreads * R;
  g.row_blocks = (nq + rows_per_cta - 1) / rows_per_cta;
  const int sms = device_sm_count();
  const int resident = (fast && tuned) ? (int)tune_value("points.resident", dim, entries, 3) : (fast ? 3 : 2);
  const long long target = (long long)sms * resident;
  // At least one wave of CTAs, and no CTA larger than ~16M entries.
  long long splits = (target + g.row_blocks - 1) / g.row_blocks;
  const long long work = (long long)rows_per_cta * nk;
  const long long by_work = (work + (16ll << 20) - 1) / (16ll << 20);
  if (by_work > splits) {
    // round up to whole waves of the SMs
    long long total = by_work * g.row_blocks;
    total = (total + target - 1) / target * target;
    splits = (total + g.row_blocks - 1) / g.row_blocks;
  }
  const long long min_keys = fast ? 64 : kGenTile;
  const long long cap = (nk + min_keys - 1) / min_keys;
  if (splits > cap) splits = cap;
  if (splits > 256) splits = 256;
  if (splits < 1) splits = 1;
  g.keys_per_split = (int)((nk + splits - 1) / splits);
  g.splits = (nk + g.keys_per_split - 1) / g.keys_per_split;
  return g;
}

}  // namespace uot
