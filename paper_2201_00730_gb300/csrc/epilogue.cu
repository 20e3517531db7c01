// O(N + M) kernels around the sweeps: merging sweep partials into the softmin,
// the affine half-step updates (aprox for rho*KL, Sec. 3), the FP64 mass
// reductions and closed-form translation of TI-Sinkhorn (Prop. 2 and the
// proof of Prop. 4, App. B), the output map Phi, the dual/primal objective
// sums and the envelope-gradient epilogue.
//
// Grid-wide reductions use the last-block-done pattern: every block writes its
// partial, fences, and increments a counter; the block that sees the final
// count reduces all partials and resets the counter.  Nothing ever waits on
// another block, so no launch can hang.
#include <cuda_runtime.h>
#include <math.h>

#include "epi_device.cuh"
#include "uot_internal.cuh"

namespace uot {
namespace {

constexpr int kBlk = 256;

__device__ __forceinline__ float ex2f(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// log2 sum_k 2^(pm_k) ps_k over the key chunks of query i, in FP32 with the
// max taken out; returned in FP64.
__device__ __forceinline__ double merge_lse2(const float* part, int CH, int nq, int splits, int i) {
  float M = kInitMax;
  for (int k = 0; k < splits; ++k) M = fmaxf(M, part[(size_t)k * CH * nq + i]);
  float S = 0.f;
  for (int k = 0; k < splits; ++k) {
    const float* b = part + (size_t)k * CH * nq;
    S += b[(size_t)nq + i] * ex2f(b[i] - M);
  }
  return (double)M + (double)log2f(S);
}

// (max, sum) log-sum-exp pair merge in FP64; an empty pair has m = -inf, s = 0.
__device__ __forceinline__ void lse_add(double& m, double& s, double m2, double s2) {
  if (m2 == -INFINITY) return;
  if (m == -INFINITY) { m = m2; s = s2; return; }
  if (m2 > m) { s = s * exp(m - m2) + s2; m = m2; }
  else { s += s2 * exp(m2 - m); }
}

__device__ __forceinline__ bool last_block(unsigned int* counter) {
  __shared__ bool am_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) am_last = (atomicAdd(counter, 1u) == gridDim.x - 1);
  __syncthreads();
  if (am_last) __threadfence();
  return am_last;
}

// Block reduction of (lse pair, max, flag) through shared memory.
struct Red4 { double m, s, r, bad; };

__device__ Red4 block_reduce(Red4 v) {
  __shared__ Red4 sh[kBlk];
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int off = blockDim.x / 2; off > 0; off >>= 1) {
    if (threadIdx.x < off) {
      Red4 o = sh[threadIdx.x + off];
      Red4 me = sh[threadIdx.x];
      lse_add(me.m, me.s, o.m, o.s);
      me.r = fmax(me.r, o.r);
      me.bad = fmax(me.bad, o.bad);
      sh[threadIdx.x] = me;
    }
    __syncthreads();
  }
  Red4 out = sh[0];
  __syncthreads();
  return out;
}

__global__ void __launch_bounds__(kBlk) k_combine(EpiParams e) {
  const epi::Consts& c = epi::block_consts(e);
  epi::RowAcc acc = epi::rowacc_empty();
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < e.nq; i += gridDim.x * blockDim.x) epi::row(e, c, i, acc);
  epi::block_finish(e, acc, blockIdx.x, gridDim.x);
}

// only < 0: both slots <- {A = Smin_a^rho1(f0) = -rho1 log sum_i a_i e^{-f0_i/rho1}, B = cf = cg = lam = 0};
// only = q >= 0: slot q's A <- Smin_a^rho1(f0) and cf <- 0, the rest of the state kept (a new fb
// stored in full, e.g. after an Anderson extrapolation)
__global__ void __launch_bounds__(kBlk) k_ti_init(const float* f0, const double* ln_a, int n, double rho1,
                                                  DevState* st, double* blk, int only) {
  Red4 acc{-INFINITY, 0.0, 0.0, 0.0};
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const double lw = ln_a[i];
    const double f = f0 ? (double)f0[i] : 0.0;
    if (!isfinite(f)) acc.bad = 1.0;
    if (lw != -INFINITY) lse_add(acc.m, acc.s, lw - f / rho1, 1.0);
  }
  const Red4 b = block_reduce(acc);
  if (threadIdx.x == 0) {
    double* o = blk + 4 * (size_t)blockIdx.x;
    o[0] = b.m; o[1] = b.s; o[2] = 0.0; o[3] = b.bad;
  }
  if (!last_block(&st->counter)) return;
  Red4 t{-INFINITY, 0.0, 0.0, 0.0};
  for (int k = threadIdx.x; k < (int)gridDim.x; k += blockDim.x) {
    const double* o = blk + 4 * (size_t)k;
    lse_add(t.m, t.s, __ldcg(o), __ldcg(o + 1));
    t.bad = fmax(t.bad, __ldcg(o + 3));
  }
  t = block_reduce(t);
  if (threadIdx.x == 0) {
    const double A = -rho1 * (t.m + log(t.s));
    const float Ah = (float)A, Al = (float)(A - (double)Ah);
    if (only >= 0) {
      Slot& o = st->slot[only];
      o.A = A; o.cf = 0.0;
      o.Af[0] = Ah; o.Af[1] = Al;
      o.cff[0] = o.cff[1] = 0.f;
    } else {
      for (int q = 0; q < 2; ++q) {
        Slot& o = st->slot[q];
        o.A = A; o.B = 0.0; o.cf = 0.0; o.cg = 0.0; o.lam = 0.0;
        o.Af[0] = Ah; o.Af[1] = Al;
        o.Bf[0] = o.Bf[1] = o.cff[0] = o.cff[1] = o.cgf[0] = o.cgf[1] = o.lamf[0] = o.lamf[1] = 0.f;
      }
    }
    if (!isfinite(A) || t.bad != 0.0) st->status |= kStatusNonfinite;
    st->counter = 0;
  }
}

__global__ void k_finalize(int ti, const float* f_hat, const float* g_hat, float* f, float* g, int n,
                           int m, const DevState* st, int slot, const int* pf, const int* pg) {
  // ti = 1: Phi(fb, gb) with fb = f_hat + cf; ti = 2 (G-Sinkhorn): (fb + lambda, gb - lambda)
  const Slot& s = st->slot[slot];
  const double sf = ti == 1 ? s.cf + s.lam : ti == 2 ? s.lam : 0.0;
  const double sg = ti == 1 ? s.cg - s.lam : ti == 2 ? -s.lam : 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n + m; i += gridDim.x * blockDim.x) {
    if (i < n) {
      if (ti) f[pf ? pf[i] : i] = (float)((double)f_hat[i] + sf);
      else if (pf || f_hat != f) f[pf ? pf[i] : i] = f_hat[i];
    } else {
      const int j = i - n;
      if (ti) g[pg ? pg[j] : j] = (float)((double)g_hat[j] + sg);
      else if (pg || g_hat != g) g[pg ? pg[j] : j] = g_hat[j];
    }
  }
}

__global__ void k_log_weights(const float* w, int n, double* lnw, float* l2w, float* l2lo, int* flags) {
  int bad = 0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const float v = w[i];
    if (!(v >= 0.f) || !isfinite(v)) bad = 1;
    if (v > 0.f) {
      const double l = log((double)v);
      const double l2 = l * kLog2e;
      const float hi = (float)l2;
      lnw[i] = l;
      l2w[i] = hi;
      if (l2lo) l2lo[i] = (float)(l2 - (double)hi);
    } else {
      lnw[i] = -INFINITY;
      l2w[i] = kZeroW;
      if (l2lo) l2lo[i] = 0.f;
    }
  }
  if (bad && flags) atomicOr(flags, kStatusBadWeights);
}

// ---- dual / primal objective ------------------------------------------------
// Sums over i (rows, S from the row sweep) and j (columns, S' from the column sweep):
//  0 m(a)   1 sum a e^{-f/rho1}   2 m(pi1)=sum a e^{(f-S)/eps}   3 sum pi1 f   4 sum pi1 (f-S)/eps
//  5 m(b)   6 sum b e^{-g/rho2}   7 m(pi2)                       8 sum pi2 g   9 sum pi2 (g-S')/eps
constexpr int kDualSums = 10;

__global__ void __launch_bounds__(kBlk) k_dual(DualParams d) {
  __shared__ double sh[kDualSums][kBlk];
  double acc[kDualSums];
#pragma unroll
  for (int q = 0; q < kDualSums; ++q) acc[q] = 0.0;
  const int total = d.n + (d.part_c ? d.m : 0);
  const int total_w = d.n + d.m;  // masses of b always needed
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < total_w; idx += gridDim.x * blockDim.x) {
    if (idx < d.n) {
      const int i = idx;
      const double a = d.a[i], f = d.f[i];
      acc[0] += a;
      acc[1] += a * exp(-f / d.rho1);
      const double S = -merge_lse2(d.part_r, 2, d.n, d.splits_r, i) / d.s;
      const double z = (f - S) / d.eps;
      const double pi1 = (a > 0.0) ? exp(d.ln_a[i] + z) : 0.0;
      acc[2] += pi1;
      acc[3] += pi1 * f;
      acc[4] += pi1 * z;
    } else {
      const int j = idx - d.n;
      const double b = d.b[j], g = d.g[j];
      acc[5] += b;
      acc[6] += b * exp(-g / d.rho2);
      if (idx < total) {
        const double Sp = -merge_lse2(d.part_c, 2, d.m, d.splits_c, j) / d.s;
        const double z = (g - Sp) / d.eps;
        const double pi2 = (b > 0.0) ? exp(d.ln_b[j] + z) : 0.0;
        acc[7] += pi2;
        acc[8] += pi2 * g;
        acc[9] += pi2 * z;
      }
    }
  }
#pragma unroll
  for (int q = 0; q < kDualSums; ++q) sh[q][threadIdx.x] = acc[q];
  __syncthreads();
  for (int off = blockDim.x / 2; off > 0; off >>= 1) {
    if (threadIdx.x < off)
      for (int q = 0; q < kDualSums; ++q) sh[q][threadIdx.x] += sh[q][threadIdx.x + off];
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int q = 0; q < kDualSums; ++q) d.blk[(size_t)blockIdx.x * kDualSums + q] = sh[q][0];
  if (!last_block(&d.state->counter)) return;
  if (threadIdx.x == 0) {
    double t[kDualSums];
    for (int q = 0; q < kDualSums; ++q) t[q] = 0.0;
    for (int k = 0; k < (int)gridDim.x; ++k)
      for (int q = 0; q < kDualSums; ++q) t[q] += __ldcg(d.blk + (size_t)k * kDualSums + q);
    const double ma = t[0], mb = t[5];
    // F_eps(f, g) of Eq. (eq-dual-uot-kl)
    const double dual = d.rho1 * (ma - t[1]) + d.rho2 * (mb - t[6]) - d.eps * t[2] + d.eps * ma * mb;
    d.out[0] = dual;
    if (d.want_primal && d.part_c) {
      // <pi,C> + eps KL(pi|a(x)b) = sum pi1 f + sum pi2 g - eps m(pi) + eps m(a) m(b)
      // KL(pi1|a) = sum pi1 (f - S)/eps - m(pi1) + m(a), likewise for pi2
      const double kl1 = t[4] - t[2] + ma, kl2 = t[9] - t[7] + mb;
      const double primal = t[3] + t[8] - d.eps * t[2] + d.eps * ma * mb + d.rho1 * kl1 + d.rho2 * kl2;
      d.out[1] = primal;
      d.out[2] = t[2];
    }
    if (!isfinite(dual)) d.state->status |= kStatusNonfinite;
    d.state->counter = 0;
  }
}

// ---- envelope gradients -------------------------------------------------------
__global__ void __launch_bounds__(kBlk) k_grad(GradParams gp) {
  const int CH = 2 + gp.moments;
  const double m_other = gp.state->dual[0];
  const bool fast = (gp.dim <= 3 && gp.p == 2.0f);
  const double pts_scale = fast ? 2.0 / sqrt(gp.s) : 1.0;  // fast path moments are sqrt(s)-scaled
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < gp.nq; i += gridDim.x * blockDim.x) {
    const double lse2 = merge_lse2(gp.part, CH, gp.nq, gp.splits, i);
    const double S = -lse2 / gp.s;
    const double f = gp.pot_o[i];
    const double z = (f - S) / gp.eps;
    const int io = gp.perm ? gp.perm[i] : i;
    if (gp.grad_w)
      gp.grad_w[io] = (float)(gp.rho_o * (1.0 - exp(-f / gp.rho_o)) - gp.eps * (exp(z) - m_other));
    if (gp.grad_pts) {
      const double lw = gp.lnw_o[i];
      const double pi1 = (lw == -INFINITY) ? 0.0 : exp(lw + z);
      // merge the moment channels with the same max as the sums
      float M = kInitMax;
      for (int k = 0; k < gp.splits; ++k) M = fmaxf(M, gp.part[(size_t)k * CH * gp.nq + i]);
      float sum = 0.f;
      for (int k = 0; k < gp.splits; ++k) {
        const float* b = gp.part + (size_t)k * CH * gp.nq;
        sum += b[(size_t)gp.nq + i] * ex2f(b[i] - M);
      }
      for (int dd = 0; dd < gp.dim; ++dd) {
        float mo = 0.f;
        for (int k = 0; k < gp.splits; ++k) {
          const float* b = gp.part + (size_t)k * CH * gp.nq;
          mo += b[(size_t)(2 + dd) * gp.nq + i] * ex2f(b[i] - M);
        }
        gp.grad_pts[(size_t)io * gp.dim + dd] = (float)(pi1 * pts_scale * (double)mo / (double)sum);
      }
    }
  }
}

__global__ void __launch_bounds__(kBlk) k_mass(const float* w, int n, double* blk, DevState* st, int idx) {
  __shared__ double sh[kBlk];
  double acc = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) acc += w[i];
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int off = blockDim.x / 2; off > 0; off >>= 1) {
    if (threadIdx.x < off) sh[threadIdx.x] += sh[threadIdx.x + off];
    __syncthreads();
  }
  if (threadIdx.x == 0) blk[blockIdx.x] = sh[0];
  if (!last_block(&st->counter)) return;
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int k = 0; k < (int)gridDim.x; ++k) t += __ldcg(blk + k);
    st->dual[idx] = t;
    st->counter = 0;
  }
}

int grid_for(int n) {
  int g = (n + kBlk - 1) / kBlk;
  if (g < 1) g = 1;
  if (g > 1024) g = 1024;
  return g;
}

}  // namespace

cudaError_t launch_combine(const EpiParams& e0, cudaStream_t st) {
  EpiParams e = e0;
  epi_finish_params(e);
  k_combine<<<grid_for(e.nq), kBlk, 0, st>>>(e);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_ti_init(const float* f0, const double* ln_a, int n, double rho1, DevState* s,
                           double* blk, cudaStream_t st, int only) {
  k_ti_init<<<grid_for(n), kBlk, 0, st>>>(f0, ln_a, n, rho1, s, blk, only);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_finalize(int ti, const float* f_hat, const float* g_hat, float* f, float* g, int n,
                            int m, const DevState* s, int slot, const int* perm_f, const int* perm_g,
                            cudaStream_t st) {
  k_finalize<<<grid_for(n + m), kBlk, 0, st>>>(ti, f_hat, g_hat, f, g, n, m, s, slot, perm_f, perm_g);
  note_launch();
  return cudaGetLastError();
}

namespace {
void split2(double d, float* o) {
  o[0] = (float)d;
  o[1] = (float)(d - (double)o[0]);
}
}  // namespace

void epi_finish_params(EpiParams& e) {
  const double k = e.eps / (e.eps + e.rho_o) * e.rho_i / (e.rho_o + e.rho_i);
  split2(1.0 / e.s, e.U2);
  split2(e.rho_o / (e.rho_o + e.eps), e.CS2);
  split2(e.eps / (e.eps + e.rho_o) * e.rho_o / (e.rho_o + e.rho_i), e.CX2);
  split2(k, e.CR2);
  split2(kLog2e / e.rho_o, e.RL2);
  split2(-e.rho_o, e.NR2);
  split2(k / (1.0 - k), e.KK2);
  split2(e.rho_o / (e.rho_o + e.rho_i), e.T12);
  split2(e.rho_i / (e.rho_o + e.rho_i), e.T22);
}

cudaError_t launch_log_weights(const float* w, int n, double* lnw, float* l2w, float* l2lo, int* flags,
                               cudaStream_t st) {
  k_log_weights<<<grid_for(n), kBlk, 0, st>>>(w, n, lnw, l2w, l2lo, flags);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_dual(const DualParams& d, cudaStream_t st) {
  k_dual<<<grid_for(d.n + d.m), kBlk, 0, st>>>(d);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_grad_epilogue(const GradParams& gp, cudaStream_t st) {
  k_grad<<<grid_for(gp.nq), kBlk, 0, st>>>(gp);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_mass(const float* w, int n, double* blk, DevState* s, int idx, cudaStream_t st) {
  k_mass<<<grid_for(n), kBlk, 0, st>>>(w, n, blk, s, idx);
  note_launch();
  return cudaGetLastError();
}

}  // namespace uot

namespace uot {
namespace {

// Phi of the iterate that a device-driven loop stopped at (index state->loop_t,
// or state->iters after the resident solver; its scalars in the slot and its g
// in g0 or g1 of that index's parity).
__global__ void k_finalize_loop(int ti, const float* f_hat, const float* g0, const float* g1, float* f, float* g,
                                int n, int m, const DevState* st, const int* pf, const int* pg, int small) {
  const int slot = (small ? st->iters : st->loop_t) & 1;
  const float* g_hat = slot ? g1 : g0;
  const Slot& s = st->slot[slot];
  const double sf = ti == 1 ? s.cf + s.lam : ti == 2 ? s.lam : 0.0;
  const double sg = ti == 1 ? s.cg - s.lam : ti == 2 ? -s.lam : 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n + m; i += gridDim.x * blockDim.x) {
    if (i < n) {
      if (ti) f[pf ? pf[i] : i] = (float)((double)f_hat[i] + sf);
      else if (pf || f_hat != f) f[pf ? pf[i] : i] = f_hat[i];
    } else {
      const int j = i - n;
      if (ti) g[pg ? pg[j] : j] = (float)((double)g_hat[j] + sg);
      else if (pg || g_hat != g) g[pg ? pg[j] : j] = g_hat[j];
    }
  }
}

// The outcome of a solve from the device state, the way the host driver
// reports it; small = 1 when the resident solver ran the loop (iteration
// count in st->iters, scalars in slot iters & 1).
__global__ void k_write_result(const DevState* st, int ti, int small, double tol, uot_result* out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const int it = small ? st->iters : st->loop_t;
  const float r = st->resid;
  const int flags = st->status;
  const bool conv = !isnan(r) && (double)r <= tol;
  int code = UOT_OK;
  if (flags & kStatusTimeout) code = UOT_ERR_TIMEOUT;
  else if (flags & kStatusBadWeights) code = UOT_ERR_NONFINITE;
  else if (flags != 0 || isnan(r)) code = UOT_ERR_NONFINITE;
  else if (tol > 0.0 && !conv) code = UOT_NOT_CONVERGED;
  out->iters = it;
  out->converged = conv ? 1 : 0;
  out->status = code;
  const unsigned int miss = st->lse_miss;
  out->lse_misses = (int32_t)(miss > 0x7fffffffu ? 0x7fffffffu : miss);
  out->residual = (double)r;
  out->lambda = ti ? st->slot[it & 1].lam : 0.0;
}

}  // namespace

cudaError_t launch_finalize_loop(int ti, const float* f_hat, const float* g0, const float* g1, float* f, float* g,
                                 int n, int m, const DevState* s, const int* perm_f, const int* perm_g, int small,
                                 cudaStream_t st) {
  k_finalize_loop<<<grid_for(n + m), kBlk, 0, st>>>(ti, f_hat, g0, g1, f, g, n, m, s, perm_f, perm_g, small);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_write_result(const DevState* s, int ti, int small, double tol, uot_result* out, cudaStream_t st) {
  k_write_result<<<1, 32, 0, st>>>(s, ti, small, tol, out);
  note_launch();
  return cudaGetLastError();
}

}  // namespace uot
