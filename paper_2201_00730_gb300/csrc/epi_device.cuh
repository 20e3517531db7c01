// Device-side half-step epilogue shared by the standalone combine kernel and
// the sweeps that finish their own rows (last CTA of a row block).
//
// Per query row i: merge the key-chunk partials into the softmin
// S_i = -(max + log2 sum)/s, then apply the half-step of the mode:
//   softmin : out_i = S_i
//   plain   : out_i = rho_o/(rho_o+eps) S_i                          (aprox for rho KL, Sec. 3)
//   TI      : out_i = rho_o/(rho_o+eps) S_i - eps/(eps+rho_o) rho_o/(rho_o+rho_i) X_in
//             with FP64 accumulation of log sum_i w_i e^{-out_i/rho_o}   (proof of Prop. 4, App. B)
// and the residual against the previous vector.  Grid-level results are
// reduced by the last block to arrive (no block ever waits on another).
#pragma once

#include <cuda_runtime.h>
#include <math.h>

#include "uot_internal.cuh"

namespace uot {
namespace epi {

__device__ __forceinline__ float ex2f(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// log2 sum_k 2^(pm_k) ps_k over the key chunks of query i (FP32, max taken out),
// in one pass over groups of 8 chunks whose 16 loads are all issued up front.
__device__ __forceinline__ double merge_lse2(const float* part, int CH, int nq, int splits, int i) {
  float M = kInitMax, S = 0.f;
  const size_t stride = (size_t)CH * nq;
  for (int k0 = 0; k0 < splits; k0 += 8) {
    float mv[8], sv[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int k = k0 + u;
      if (k < splits) {
        const float* b = part + (size_t)k * stride;
        mv[u] = __ldcg(b + i);
        sv[u] = __ldcg(b + (size_t)nq + i);
      } else {
        mv[u] = kInitMax;
        sv[u] = 0.f;
      }
    }
    float cm = M;
#pragma unroll
    for (int u = 0; u < 8; ++u) cm = fmaxf(cm, mv[u]);
    float acc = S * ex2f(M - cm);
#pragma unroll
    for (int u = 0; u < 8; ++u) acc = fmaf(sv[u], ex2f(mv[u] - cm), acc);
    S = acc;
    M = cm;
  }
  return (double)M + (double)log2f(S);
}

struct Acc {
  double m, s;  // log-sum-exp pair: sum = s * e^m (m = -inf: empty)
  double r;     // residual max
  double bad;   // non-finite flag
};

__device__ __forceinline__ Acc acc_empty() { return Acc{-INFINITY, 0.0, 0.0, 0.0}; }

__device__ __forceinline__ void lse_add(double& m, double& s, double m2, double s2) {
  if (m2 == -INFINITY) return;
  if (m == -INFINITY) { m = m2; s = s2; return; }
  if (m2 > m) { s = s * exp(m - m2) + s2; m = m2; }
  else { s += s2 * exp(m2 - m); }
}

struct Consts {
  double Xin, cS, cX, base_old, cR, inv_s, inv_rho, key_shift;
};

__device__ __forceinline__ Consts consts(const EpiParams& e) {
  const Slot& si = e.state->slot[e.slot_in];
  Consts c;
  c.Xin = e.out_is_f ? si.B : si.A;                                   // key-side Smin^rho scalar
  c.cS = e.rho_o / (e.rho_o + e.eps);                                 // aprox factor
  c.cX = e.eps / (e.eps + e.rho_o) * e.rho_o / (e.rho_o + e.rho_i);
  c.base_old = e.out_is_f ? si.cf : si.cg;                            // stored hat + shift = bar
  c.cR = e.eps / (e.eps + e.rho_o) * e.rho_i / (e.rho_o + e.rho_i) * (e.out_is_f ? si.A : si.B);
  c.inv_s = 1.0 / e.s;
  c.inv_rho = 1.0 / e.rho_o;
  c.key_shift = e.key_shift ? *e.key_shift : 0.0;
  return c;
}

// Half-step of one query row.
__device__ __forceinline__ void row(const EpiParams& e, const Consts& c, int i, Acc& acc) {
  const double lse2 = merge_lse2(e.part, 2 + e.moments, e.nq, e.splits, i);
  if (lse2 < 0.25 * (double)kZeroW) acc.bad = 1.0;  // every key had zero weight
  // Smin in cost units; a shift tau of the key potential moves it by -tau exactly
  const double S = -lse2 * c.inv_s - c.key_shift;
  double v;
  if (e.mode == EPI_SOFTMIN) {
    v = S;
  } else if (e.mode == EPI_PLAIN) {
    v = c.cS * S;
    if (e.old_out) acc.r = fmax(acc.r, fabs((double)e.old_out[i] - v));
  } else {
    v = c.cS * S - c.cX * c.Xin;
    const double lw = e.lnw_o[i];
    if (lw != -INFINITY) lse_add(acc.m, acc.s, lw - v * c.inv_rho, 1.0);
    if (e.old_out) acc.r = fmax(acc.r, fabs((double)e.old_out[i] + c.base_old - v - c.cR));
  }
  if (!isfinite(v)) acc.bad = 1.0;
  e.out[e.perm_out ? e.perm_out[i] : i] = (float)v;
}

__device__ __forceinline__ double shfl_d(double v, int off) {
  return __shfl_xor_sync(0xffffffffu, v, off);
}

// Block reduction: max of m first, one exp per thread, then sums (no exp per tree level).
__device__ inline Acc block_reduce(Acc v) {
  __shared__ double sm[32], ss[32], sr[32], sb[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  double M = v.m;
  for (int off = 16; off > 0; off >>= 1) M = fmax(M, shfl_d(M, off));
  double s = (v.m == -INFINITY) ? 0.0 : v.s * exp(v.m - M);
  double r = v.r, b = v.bad;
  for (int off = 16; off > 0; off >>= 1) {
    s += shfl_d(s, off);
    r = fmax(r, shfl_d(r, off));
    b = fmax(b, shfl_d(b, off));
  }
  if (lane == 0) { sm[warp] = M; ss[warp] = s; sr[warp] = r; sb[warp] = b; }
  __syncthreads();
  Acc out = acc_empty();
  if (threadIdx.x == 0) {
    for (int w = 0; w < nw; ++w) {
      lse_add(out.m, out.s, sm[w], ss[w]);
      out.r = fmax(out.r, sr[w]);
      out.bad = fmax(out.bad, sb[w]);
    }
  }
  __syncthreads();
  return out;  // valid in thread 0
}

__device__ __forceinline__ bool arrive_last(unsigned int* counter, unsigned int total) {
  __shared__ bool last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = (atomicAdd(counter, 1u) == total - 1);
  __syncthreads();
  if (last) __threadfence();
  return last;
}

// Thread 0 of the last block: scalars of the half-step, residual, status.
__device__ inline void finalize(const EpiParams& e, const Acc& t) {
  DevState* st = e.state;
  int status = st->status;
  if (t.bad != 0.0 || isnan(t.r)) status |= kStatusNonfinite;
  if (e.mode == EPI_TI) {
    const double lse = t.m + log(t.s);               // log <w, e^{-hat/rho_o}>
    const double Xhat = -e.rho_o * lse;              // Smin_w^rho_o(hat)
    const double k = e.eps / (e.eps + e.rho_o) * e.rho_i / (e.rho_o + e.rho_i);
    const double c = k / (1.0 - k) * Xhat;           // closed-form translation
    const double X = Xhat + c;                       // Smin(hat + c) = Smin(hat) + c
    if (!isfinite(X)) status |= kStatusNonfinite;
    Slot& so = st->slot[e.slot_out];
    if (e.out_is_f) {
      so.A = X; so.cf = c;
      const double tau1 = e.rho_o / (e.rho_o + e.rho_i), tau2 = e.rho_i / (e.rho_o + e.rho_i);
      so.lam = tau1 * so.B - tau2 * X;               // lambda* = tau1 Smin_b(gb) - tau2 Smin_a(fb)
    } else {
      so.B = X; so.cg = c;
    }
  }
  if (e.old_out) {
    st->resid = (float)t.r;
    if (e.resid_hist) e.resid_hist[e.hist_index] = (float)t.r;
  }
  st->status = status;
}

// Grid-level tail: block partial -> blk[slot]; the last of `nblocks` arrivals
// reduces all partials and finalises.
__device__ inline void grid_tail(const EpiParams& e, const Acc& mine, int slot, int nblocks) {
  if (threadIdx.x == 0) {
    double* o = e.blk + 4 * (size_t)slot;
    o[0] = mine.m; o[1] = mine.s; o[2] = mine.r; o[3] = mine.bad;
  }
  if (!arrive_last(&e.state->counter, (unsigned)nblocks)) return;
  Acc t = acc_empty();
  for (int k = threadIdx.x; k < nblocks; k += blockDim.x) {
    const double* o = e.blk + 4 * (size_t)k;
    lse_add(t.m, t.s, __ldcg(o), __ldcg(o + 1));
    t.r = fmax(t.r, __ldcg(o + 2));
    t.bad = fmax(t.bad, __ldcg(o + 3));
  }
  t = block_reduce(t);
  if (threadIdx.x == 0) {
    finalize(e, t);
    e.state->counter = 0;
  }
}

}  // namespace epi
}  // namespace uot
