// Batched ragged solver: many independent UOT problems (points cost, dim <= 3,
// p = 2), each with its own N, M, eps, rho1, rho2, advanced together.
//
// One kernel launch per half-step covers every problem still running.  Its CTAs
// are persistent workers that pull work units (problem k, block of 128 query
// rows) from a global queue ordered longest-first (key count), so ragged sizes
// balance across the 152 SMs.  A unit sweeps all keys of its problem, so each
// row's softmin is complete inside the unit and its half-step is applied at
// once; the unit's FP64 mass and residual partials go to a slot of its own and
// the last unit of a problem to arrive finishes that problem's scalars
// (translation, lambda*, residual, convergence).  The iteration index lives in
// device memory, so a chunk of iterations can be captured once as a CUDA graph
// and replayed; converged problems stop themselves on the device.  No block
// ever waits for another.
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>
#include <vector>

#include "batched.cuh"
#include "uot_internal.cuh"

namespace uot {
namespace {

constexpr int kThreads = 128;   // rows per unit (one per thread)
constexpr int kKeyTile = 256;
constexpr int kGroup = 8;

__device__ __forceinline__ float ex2f(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__device__ __forceinline__ void lse_add(double& m, double& s, double m2, double s2) {
  if (m2 == -INFINITY) return;
  if (m == -INFINITY) { m = m2; s = s2; return; }
  if (m2 > m) { s = s * exp(m - m2) + s2; m = m2; }
  else { s += s2 * exp(m2 - m); }
}

__device__ __forceinline__ double shfl_d(double v, int off) { return __shfl_xor_sync(0xffffffffu, v, off); }

// (lse pair, max, flag) reduction over the CTA; result valid in thread 0.
__device__ void cta_reduce(double& m, double& s, double& r, double& bad) {
  __shared__ double sm[kThreads / 32], ss[kThreads / 32], sr[kThreads / 32], sb[kThreads / 32];
  double M = m;
  for (int off = 16; off > 0; off >>= 1) M = fmax(M, shfl_d(M, off));
  double S = (m == -INFINITY) ? 0.0 : s * exp(m - M);
  for (int off = 16; off > 0; off >>= 1) {
    S += shfl_d(S, off);
    r = fmax(r, shfl_d(r, off));
    bad = fmax(bad, shfl_d(bad, off));
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) { sm[warp] = M; ss[warp] = S; sr[warp] = r; sb[warp] = bad; }
  __syncthreads();
  if (threadIdx.x == 0) {
    m = -INFINITY; s = 0.0; r = 0.0; bad = 0.0;
    for (int w = 0; w < kThreads / 32; ++w) {
      lse_add(m, s, sm[w], ss[w]);
      r = fmax(r, sr[w]);
      bad = fmax(bad, sb[w]);
    }
  }
  __syncthreads();
}

// Softmin partial (max, sum of 2^(t - max)) of query row i of a unit over all keys.
template <int D>
__device__ __forceinline__ void unit_lse(float4* sk, const float* qp, int i, bool live, const float* kp, int nk,
                                         const float* kl2, const float* kpot, double s, float& mx, float& acc) {
  const float rs = (float)sqrt(s);
  float xq[3] = {0.f, 0.f, 0.f};
  if (live)
    for (int d = 0; d < D; ++d) xq[d] = rs * qp[(size_t)i * D + d];
  mx = kInitMax;
  acc = 0.f;
  for (int j0 = 0; j0 < nk; j0 += kKeyTile) {
    const int cnt = min(kKeyTile, nk - j0);
    __syncthreads();
    for (int uu = threadIdx.x; uu < kKeyTile; uu += kThreads) {
      float4 v = make_float4(0.f, 0.f, 0.f, kZeroW);
      if (uu < cnt) {
        const int j = j0 + uu;
        v.x = rs * kp[(size_t)j * D];
        if (D > 1) v.y = rs * kp[(size_t)j * D + 1];
        if (D > 2) v.z = rs * kp[(size_t)j * D + 2];
        const float lw = kl2[j];
        if (lw > 0.5f * kZeroW) v.w = (float)((double)lw + s * (double)kpot[j]);
      }
      sk[uu] = v;
    }
    __syncthreads();
    const int cntg = (cnt + kGroup - 1) / kGroup * kGroup;
    for (int g0 = 0; g0 < cntg; g0 += kGroup) {
      float tv[kGroup];
#pragma unroll
      for (int q = 0; q < kGroup; ++q) {
        const float4 kv = sk[g0 + q];
        const float d0 = xq[0] - kv.x;
        float c = fmaf(-d0, d0, kv.w);
        if (D > 1) { const float d1 = xq[1] - kv.y; c = fmaf(-d1, d1, c); }
        if (D > 2) { const float d2 = xq[2] - kv.z; c = fmaf(-d2, d2, c); }
        tv[q] = c;
      }
      float tm = tv[0];
#pragma unroll
      for (int q = 1; q < kGroup; ++q) tm = fmaxf(tm, tv[q]);
      const float mn = fmaxf(mx, tm);
      float a = acc * ex2f(mx - mn);
#pragma unroll
      for (int q = 0; q < kGroup; ++q) a += ex2f(tv[q] - mn);
      acc = a;
      mx = mn;
    }
  }
}

__global__ void __launch_bounds__(kThreads)
k_batch_half(BHalf h) {
  __shared__ float4 sk[kKeyTile];
  __shared__ int s_unit;
  __shared__ bool s_last;
  const int t = *h.iter;  // this half-step belongs to iteration t + 1
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) s_unit = (int)atomicAdd(h.next, 1u);
    __syncthreads();
    const int qi = s_unit;
    if (qi >= h.nunits) break;
    const int u = h.queue[qi];                 // partial slot (problem-contiguous numbering)
    const int2 un = h.units[u];                // (problem, first row)
    const int k = un.x, r0 = un.y;
    BState& st = h.st[k];
    if (st.status != 0) continue;              // retired problem (uniform over the CTA)
    const BProb pr = h.probs[k];
    const bool f_side = (h.side == 0);
    const int nq = f_side ? pr.n : pr.m, nk = f_side ? pr.m : pr.n;
    const float* qp = (f_side ? h.x + pr.x_off : h.y + pr.y_off);
    const float* kp = (f_side ? h.y + pr.y_off : h.x + pr.x_off);
    const float* kl2 = (f_side ? h.l2b + pr.b_off : h.l2a + pr.a_off);
    const int so = (t + 1) & 1, si = t & 1;
    // key potential: f side keys are g_hat_{t+1}; g side keys are f_hat_t
    const float* kpot = f_side ? (so ? h.g1 : h.g0) + pr.b_off : h.f + pr.a_off;
    const double s = pr.s;
    const int i = r0 + threadIdx.x;
    const bool live = i < nq;
    float mx, acc;
    if (pr.dim == 1) unit_lse<1>(sk, qp, i, live, kp, nk, kl2, kpot, s, mx, acc);
    else if (pr.dim == 2) unit_lse<2>(sk, qp, i, live, kp, nk, kl2, kpot, s, mx, acc);
    else unit_lse<3>(sk, qp, i, live, kp, nk, kl2, kpot, s, mx, acc);
    // half-step of this row
    const Slot& sl = st.slot[f_side ? so : si];
    const double eps = pr.eps;
    const double rho_o = f_side ? pr.rho1 : pr.rho2, rho_i = f_side ? pr.rho2 : pr.rho1;
    const double key_shift = h.ti ? (f_side ? sl.cg : sl.cf) : 0.0;
    double um = -INFINITY, us = 0.0, ur = 0.0, ubad = 0.0;
    if (live) {
      const double lse2 = (double)mx + (double)log2f(acc);
      if (lse2 < 0.25 * (double)kZeroW) ubad = 1.0;
      const double S = -lse2 / s - key_shift;
      double v;
      float* out = f_side ? h.f + pr.a_off : (so ? h.g1 : h.g0) + pr.b_off;
      const float* old = f_side ? nullptr : (si ? h.g1 : h.g0) + pr.b_off;
      if (h.ti) {
        const double Xin = f_side ? sl.B : sl.A;
        v = rho_o / (rho_o + eps) * S - eps / (eps + rho_o) * rho_o / (rho_o + rho_i) * Xin;
        const double lw = f_side ? h.lna[pr.a_off + i] : h.lnb[pr.b_off + i];
        if (lw != -INFINITY) { um = lw - v / rho_o; us = 1.0; }
        if (!f_side && t >= 1) {
          const Slot& sp = st.slot[si];
          ur = fabs((double)old[i] + sp.cg - v - eps / (eps + rho_o) * rho_i / (rho_o + rho_i) * sp.B);
        }
      } else {
        v = rho_o / (rho_o + eps) * S;
        if (!f_side && t >= 1) ur = fabs((double)old[i] - v);
      }
      if (!isfinite(v)) ubad = 1.0;
      out[i] = (float)v;
    }
    cta_reduce(um, us, ur, ubad);
    if (threadIdx.x == 0) {
      double* o = h.upart + 4 * (size_t)u;
      o[0] = um; o[1] = us; o[2] = ur; o[3] = ubad;
      __threadfence();
      const unsigned nunits_k = f_side ? (unsigned)pr.units_f : (unsigned)pr.units_g;
      s_last = (atomicAdd(&st.cnt, 1u) == nunits_k - 1);
    }
    __syncthreads();
    if (!s_last || threadIdx.x != 0) continue;
    // last unit of problem k: finish its half-step
    __threadfence();
    st.cnt = 0;
    const int base = f_side ? pr.ubase_f : pr.ubase_g;
    const int nu = f_side ? pr.units_f : pr.units_g;
    double M = -INFINITY, Sm = 0.0, R = 0.0, B = 0.0;
    for (int q = 0; q < nu; ++q) {
      const double* o = h.upart + 4 * (size_t)(base + q);
      lse_add(M, Sm, __ldcg(o), __ldcg(o + 1));
      R = fmax(R, __ldcg(o + 2));
      B = fmax(B, __ldcg(o + 3));
    }
    int status = 0;
    if (B != 0.0 || isnan(R)) status = 2;
    if (h.ti) {
      const double Xhat = -rho_o * (M + log(Sm));
      const double kk = eps / (eps + rho_o) * rho_i / (rho_o + rho_i);
      const double c = kk / (1.0 - kk) * Xhat;
      const double X = Xhat + c;
      if (!isfinite(X)) status = 2;
      Slot& sw = st.slot[so];
      if (f_side) {
        sw.A = X; sw.cf = c;
        sw.lam = pr.rho1 / (pr.rho1 + pr.rho2) * sw.B - pr.rho2 / (pr.rho1 + pr.rho2) * X;
      } else {
        sw.B = X; sw.cg = c;
      }
    }
    if (!f_side && t >= 1) {
      st.resid = (float)R;
      const bool check = (t == h.max_iter) || (h.tol > 0.0 && t % h.check_every == 0);
      if (status == 0 && check && (t == h.max_iter || R <= h.tol)) {
        st.conv_iter = t;
        status = (R <= h.tol) ? 1 : 3;
      }
    }
    if (status != 0) {
      if (status == 2) st.conv_iter = t;
      st.status = status;
      atomicSub(h.active, 1u);
    }
  }
  // the last CTA to leave resets the queue (and advances the iteration after an f half-step)
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(h.finished, 1u) == gridDim.x - 1) {
      *h.next = 0;
      *h.finished = 0;
      if (h.side == 0) *h.iter = t + 1;
    }
  }
}

// Per problem: TI slot init A_0 = Smin_a^rho1(0) = -rho1 log m(a); zero the rest.
__global__ void k_batch_init(const BProb* probs, BState* st, const float* a, int count, int ti,
                             unsigned int* active) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= count) return;
  const BProb pr = probs[k];
  double ma = 0.0;
  for (int i = 0; i < pr.n; ++i) ma += (double)a[pr.a_off + i];
  BState z{};
  const double A = ti ? -pr.rho1 * log(ma) : 0.0;
  z.slot[0].A = A;
  z.slot[1].A = A;
  z.status = (ma > 0.0 && isfinite(ma)) ? 0 : 2;
  z.conv_iter = 0;
  st[k] = z;
  if (z.status != 0) atomicSub(active, 1u);
}

// Output map per problem from the slot of its returned iterate; also counts live problems.
__global__ void k_batch_phi(const BProb* probs, const BState* st, float* f, float* g0, const float* g1,
                            int count, int ti) {
  const int k = blockIdx.x;
  if (k >= count) return;
  const BProb pr = probs[k];
  const int T = st[k].conv_iter;
  const Slot& sl = st[k].slot[T & 1];
  const double sf = ti ? sl.cf + sl.lam : 0.0, sg = ti ? sl.cg - sl.lam : 0.0;
  const float* gsrc = ((T & 1) ? g1 : g0) + pr.b_off;
  float* gdst = g0 + pr.b_off;
  for (int i = threadIdx.x; i < pr.n; i += blockDim.x)
    if (ti) f[pr.a_off + i] = (float)((double)f[pr.a_off + i] + sf);
  for (int j = threadIdx.x; j < pr.m; j += blockDim.x) gdst[j] = (float)((double)gsrc[j] + sg);
}

}  // namespace

int batch_rows_per_unit() { return kThreads; }

cudaError_t launch_batch_half(const BHalf& h, int grid, cudaStream_t st) {
  k_batch_half<<<grid, kThreads, 0, st>>>(h);
  note_launch();
  return cudaGetLastError();
}

int batch_grid() {
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_batch_half, kThreads, 0) != cudaSuccess || occ < 1)
    occ = 4;
  // the persistent grid: occupancy-many CTAs per SM, or fewer when tuned so
  const long long t = tune_value("batch.ctas_per_sm", -1, 0, occ);
  return device_sm_count() * (int)(t < occ ? t : occ);
}

cudaError_t launch_batch_init(const BProb* probs, BState* st, const float* a, int count, int ti,
                              unsigned int* active, cudaStream_t s) {
  k_batch_init<<<(count + 127) / 128, 128, 0, s>>>(probs, st, a, count, ti, active);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_batch_phi(const BProb* probs, const BState* st, float* f, float* g0, const float* g1, int count,
                             int ti, cudaStream_t s) {
  k_batch_phi<<<count, 128, 0, s>>>(probs, st, f, g0, g1, count, ti);
  note_launch();
  return cudaGetLastError();
}

}  // namespace uot
