// Half-step maps and the translation lambda* of F- and G-Sinkhorn for a
// general smooth phi^* (Sec. 3), here rho KL and the Berg entropy.
//
// The softmin S of a half-step comes from the ordinary sweeps (softmin mode,
// the key shift applied exactly); this file adds
//  * the map out = -aprox_{phi^*}(-S) (+ the G-Sinkhorn shift), where
//    aprox_{phi^*}(x) = argmin_y eps e^{(x - y)/eps} + phi^*(y) solves
//    (x - y)/eps = log phi^*'(y) (Sec. 3).  For rho KL it is rho/(rho + eps) x.
//    For the Berg entropy, phi^*(q) = -rho log(1 - q/rho) (q < rho), so
//    phi^*'(y) = rho/(rho - y); with u = (rho - y)/eps the equation becomes
//    u + log u = L, L = log(rho/eps) + (rho - x)/eps, i.e. u = omega(L) (the
//    Wright omega function, W_0(e^L)) and aprox(x) = rho - eps omega(L).
//    omega is found by Newton's method on u + log u - L in FP64 (the map is
//    O(N + M) work per half-step);
//  * lambda*(fb, gb) = argmax_lambda <a, -phi_1^*(-fb - lambda)> + <b, -phi_2^*(-gb + lambda)>
//    (Prop. 1: the entropic term does not depend on lambda), the root of the
//    decreasing derivative F'(lambda) = <a, phi_1^*'(-fb - lambda)> - <b, phi_2^*'(-gb + lambda)>,
//    by Newton steps F'/F'' kept inside a bracket of the root (bisection when a
//    step leaves it; the bracket starts as the domain of the Berg terms,
//    lambda > -rho1 - min fb and lambda < rho2 + min gb over the live points,
//    and grows by doubling on a KL side).  Each step is one launch: FP64 sums
//    over the grid, the last block to finish updates lambda (no block waits on
//    another).
#include <cuda_runtime.h>
#include <math.h>

#include "uot_internal.cuh"

namespace uot {
namespace {

constexpr int kBlk = 256;

// omega(L): the root u > 0 of u + log u = L.
__device__ double wright_omega(double L) {
  double u = (L > 1.0) ? L - log(L) : exp(L);
  if (!(u > 0.0)) u = 1e-300;
  for (int it = 0; it < 40; ++it) {
    // Newton: u <- u - (u + log u - L) u / (1 + u) = u (1 + L - log u) / (1 + u)
    const double nu = u * (1.0 + L - log(u)) / (1.0 + u);
    const double d = fabs(nu - u);
    u = nu > 0.0 ? nu : 0.5 * u;
    if (d <= 1e-16 * u) break;
  }
  return u;
}

// -aprox_{phi^*}(-S)
__device__ double neg_aprox(int phi, double rho, double eps, double S) {
  if (phi == UOT_PHI_BERG) {
    const double L = log(rho / eps) + (rho + S) / eps;
    return eps * wright_omega(L) - rho;
  }
  return rho / (rho + eps) * S;
}

__device__ void atomic_max_nonneg(float* p, float v) {
  // non-negative floats order like their bit patterns
  atomicMax(reinterpret_cast<int*>(p), __float_as_int(v));
}

__global__ void __launch_bounds__(kBlk) k_phi_half(const float* S, float* out, int n, int phi, double rho,
                                                   double eps, const double* shift, double sign, float* resid,
                                                   int* status) {
  const double sh = shift ? sign * *shift : 0.0;
  float r = 0.f;
  bool bad = false;
  for (int i = blockIdx.x * kBlk + threadIdx.x; i < n; i += gridDim.x * kBlk) {
    const double v = neg_aprox(phi, rho, eps, (double)S[i]) + sh;
    const float vf = (float)v;
    if (!isfinite(vf)) bad = true;
    r = fmaxf(r, fabsf(vf - out[i]));
    out[i] = vf;
  }
  for (int o = 16; o > 0; o >>= 1) r = fmaxf(r, __shfl_xor_sync(0xffffffffu, r, o));
  if ((threadIdx.x & 31) == 0 && resid) atomic_max_nonneg(resid, isnan(r) ? INFINITY : r);
  if (bad) atomicOr(status, kStatusNonfinite);
}

// phi^*'(q) and phi^*''(q)
__device__ void dphi(int phi, double rho, double q, double& d1, double& d2) {
  if (phi == UOT_PHI_BERG) {
    const double t = rho / (rho - q);
    d1 = t;
    d2 = t * t / rho;
  } else {
    d1 = exp(q / rho);
    d2 = d1 / rho;
  }
}

// Partial sums of one block, reduced in FP64.
template <int K>
__device__ void block_sum(double (&v)[K], double* sh) {
  for (int k = 0; k < K; ++k)
    for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0)
    for (int k = 0; k < K; ++k) sh[k * (kBlk / 32) + w] = v[k];
  __syncthreads();
  if (threadIdx.x < 32)
    for (int k = 0; k < K; ++k) {
      double x = threadIdx.x < kBlk / 32 ? sh[k * (kBlk / 32) + threadIdx.x] : 0.0;
      for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
      v[k] = x;
    }
}

__device__ bool last_block(unsigned int* counter) {
  __shared__ bool last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    last = atomicAdd(counter, 1u) == gridDim.x - 1;
    if (last) __threadfence();
  }
  __syncthreads();
  return last;
}

struct LamArgs {
  const float* fb;  // internal order
  const float* gb;
  const float* a;
  const float* b;
  int n, m, phi1, phi2;
  double rho1, rho2;
  LamState* ls;
  double* blk;  // [gridDim.x * 2] partials
  DevState* st;
  int slot;     // the slot whose shifts follow lambda
};

__device__ void publish(const LamArgs& q, double lam) {
  LamState* s = q.ls;
  s->lam = lam;
  Slot& sl = q.st->slot[q.slot];
  sl.lam = lam;
  sl.cf = lam;
  sl.cg = -lam;
  const float h = (float)lam, lo = (float)(lam - (double)h);
  sl.lamf[0] = h; sl.lamf[1] = lo;
  sl.cff[0] = h; sl.cff[1] = lo;
  sl.cgf[0] = -h; sl.cgf[1] = -lo;
}

// Bracket from the domain: the live minima of fb and gb.
__global__ void __launch_bounds__(kBlk) k_lam_init(LamArgs q) {
  __shared__ double sh[2 * (kBlk / 32)];
  double mf = INFINITY, mg = INFINITY;
  for (int i = blockIdx.x * kBlk + threadIdx.x; i < q.n + q.m; i += gridDim.x * kBlk) {
    if (i < q.n) {
      if (q.a[i] > 0.f) mf = fmin(mf, (double)q.fb[i]);
    } else if (q.b[i - q.n] > 0.f) {
      mg = fmin(mg, (double)q.gb[i - q.n]);
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    mf = fmin(mf, __shfl_xor_sync(0xffffffffu, mf, o));
    mg = fmin(mg, __shfl_xor_sync(0xffffffffu, mg, o));
  }
  if ((threadIdx.x & 31) == 0) { sh[threadIdx.x >> 5] = mf; sh[kBlk / 32 + (threadIdx.x >> 5)] = mg; }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < kBlk / 32; ++w) { mf = fmin(mf, sh[w]); mg = fmin(mg, sh[kBlk / 32 + w]); }
    q.blk[2 * blockIdx.x] = mf;
    q.blk[2 * blockIdx.x + 1] = mg;
  }
  if (!last_block(&q.ls->counter)) return;
  if (threadIdx.x != 0) return;
  mf = INFINITY; mg = INFINITY;
  for (int k = 0; k < (int)gridDim.x; ++k) {
    mf = fmin(mf, __ldcg(q.blk + 2 * k));
    mg = fmin(mg, __ldcg(q.blk + 2 * k + 1));
  }
  LamState* s = q.ls;
  s->counter = 0;
  s->lo = (q.phi1 == UOT_PHI_BERG && isfinite(mf)) ? -q.rho1 - mf : -INFINITY;
  s->hi = (q.phi2 == UOT_PHI_BERG && isfinite(mg)) ? q.rho2 + mg : INFINITY;
  s->done = 0;
  double lam = s->lam;  // start from the previous lambda when it lies in the bracket
  if (!(lam > s->lo && lam < s->hi)) {
    if (isfinite(s->lo) && isfinite(s->hi)) lam = 0.5 * (s->lo + s->hi);
    else if (isfinite(s->lo)) lam = s->lo + 1.0;
    else if (isfinite(s->hi)) lam = s->hi - 1.0;
    else lam = 0.0;
    if (!(lam > s->lo && lam < s->hi)) lam = 0.5 * (s->lo + s->hi);
  }
  publish(q, lam);
}

// One safeguarded Newton step.
__global__ void __launch_bounds__(kBlk) k_lam_step(LamArgs q) {
  __shared__ double sh[2 * (kBlk / 32)];
  if (q.ls->done) return;  // uniform: read once per block before any barrier
  const double lam = q.ls->lam;
  double v[2] = {0.0, 0.0};  // F'(lam), F''(lam)
  for (int i = blockIdx.x * kBlk + threadIdx.x; i < q.n + q.m; i += gridDim.x * kBlk) {
    double d1, d2;
    if (i < q.n) {
      const double w = q.a[i];
      if (w > 0.0) {
        dphi(q.phi1, q.rho1, -(double)q.fb[i] - lam, d1, d2);
        v[0] += w * d1;
        v[1] -= w * d2;
      }
    } else {
      const double w = q.b[i - q.n];
      if (w > 0.0) {
        dphi(q.phi2, q.rho2, -(double)q.gb[i - q.n] + lam, d1, d2);
        v[0] -= w * d1;
        v[1] -= w * d2;
      }
    }
  }
  block_sum<2>(v, sh);
  if (threadIdx.x == 0) {
    q.blk[2 * blockIdx.x] = v[0];
    q.blk[2 * blockIdx.x + 1] = v[1];
  }
  if (!last_block(&q.ls->counter)) return;
  if (threadIdx.x != 0) return;
  double g = 0.0, h = 0.0;
  for (int k = 0; k < (int)gridDim.x; ++k) {
    g += __ldcg(q.blk + 2 * k);
    h += __ldcg(q.blk + 2 * k + 1);
  }
  LamState* s = q.ls;
  s->counter = 0;
  if (!isfinite(g) || !(h < 0.0)) {
    s->done = 1;
    if (!isfinite(g)) atomicOr(&q.st->status, kStatusNonfinite);
    return;
  }
  if (g == 0.0) { s->done = 1; return; }
  if (g > 0.0) s->lo = lam;  // F' decreasing: the root lies above
  else s->hi = lam;
  double nx = lam - g / h;
  if (!(nx > s->lo && nx < s->hi)) {
    if (isfinite(s->lo) && isfinite(s->hi)) nx = 0.5 * (s->lo + s->hi);
    else if (g > 0.0) nx = lam + fmax(1.0, 2.0 * fabs(lam));
    else nx = lam - fmax(1.0, 2.0 * fabs(lam));
  }
  if (fabs(nx - lam) <= 4e-16 * fmax(1.0, fabs(lam)) || s->hi - s->lo <= 4e-16 * fmax(1.0, fabs(lam))) s->done = 1;
  publish(q, nx);
}

// Caller-order outputs f = fb + sf * lambda, g = gb - sg * lambda.
__global__ void k_phi_out(const float* fb, const float* gb, const int* pf, const int* pg, float* f, float* g, int n,
                          int m, const double* lam, int g_mode) {
  const double l = g_mode ? *lam : 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n + m; i += gridDim.x * blockDim.x) {
    if (i < n) f[pf ? pf[i] : i] = (float)((double)fb[i] + l);
    else g[pg ? pg[i - n] : i - n] = (float)((double)gb[i - n] - l);
  }
}

int grid_for(int n) {
  const int b = (n + kBlk - 1) / kBlk;
  const int cap = 2 * device_sm_count();
  return b < 1 ? 1 : (b > cap ? cap : b);
}

}  // namespace

cudaError_t launch_phi_half(const float* S, float* out, int n, int phi, double rho, double eps, const double* shift,
                            double sign, float* resid, int* status, cudaStream_t st) {
  k_phi_half<<<grid_for(n), kBlk, 0, st>>>(S, out, n, phi, rho, eps, shift, sign, resid, status);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_lambda_star(const float* fb, const float* gb, const float* a, const float* b, int n, int m,
                               int phi1, int phi2, double rho1, double rho2, LamState* ls, double* blk, DevState* st,
                               int slot, int steps, cudaStream_t s) {
  LamArgs q{fb, gb, a, b, n, m, phi1, phi2, rho1, rho2, ls, blk, st, slot};
  const int grid = grid_for(n + m);
  k_lam_init<<<grid, kBlk, 0, s>>>(q);
  note_launch();
  for (int k = 0; k < steps; ++k) {
    k_lam_step<<<grid, kBlk, 0, s>>>(q);
    note_launch();
  }
  return cudaGetLastError();
}

cudaError_t launch_phi_out(const float* fb, const float* gb, const int* pf, const int* pg, float* f, float* g, int n,
                           int m, const double* lam, int g_mode, cudaStream_t st) {
  k_phi_out<<<grid_for(n + m), kBlk, 0, st>>>(fb, gb, pf, pg, f, g, n, m, lam, g_mode);
  note_launch();
  return cudaGetLastError();
}

}  // namespace uot
