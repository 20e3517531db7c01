// 1-D unbalanced multi-marginal OT and barycenters (Sec. 5) by Frank-Wolfe on
// the translation-invariant functional H, batched: one warp per problem, FP64.
//
// A problem has K measures (x_k, alpha_k) on the line with sorted points,
// barycentric weights omega_k >= 0 summing to one, the rho KL penalties and
// the squared-distance ground cost, whose multi-marginal form is
//   C(z_1..z_K) = sum_k omega_k (z_k - B(z))^2,  B(z) = sum_k omega_k z_k.
// Each Frank-Wolfe step computes, with all lanes,
//   q_k = log <alpha_k, e^{-fb_k / (omega_k rho)}>,
//   lambda_k = omega_k rho q_k - omega_k / (sum_l omega_l) sum_l omega_l rho q_l
//     (the optimal translation of the K-marginal dual, Sec. 5, rho KL setting),
//   alpha~_k = alpha_k e^{-(fb_k + lambda_k) / (omega_k rho)}
// then lane 0 runs SolveMOT (Alg. 3) between the re-weighted measures: the
// measure with the least remaining mass among those not at their last point
// moves to its next point (lowest index on ties), every measure's remaining
// mass drops by that amount, and the new point's potential is the cost of the
// current index tuple minus the other measures' current potentials; the last
// tuple takes the mass left.  All lanes then step
//   fb_k <- (1 - tau_t) fb_k + tau_t r_k,  tau_t = 2 / (2 + t).
// The output is the translated pair f_k = fb_k + lambda_k and the barycenter of
// the plan that SolveMOT returns at the final iterate: the points B(tuple) of
// its tuples of positive mass, with those masses as weights.  The walk runs in
// FP64 with the oracle's order of operations, so its branches are the same.
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>
#include <string>
#include <vector>

#include "uot_internal.cuh"

namespace uot {
namespace {

constexpr int kMMWarps = 4;  // problems per CTA
constexpr int kMMMaxK = 8;   // measures per problem

struct MMProb {
  long long off[kMMMaxK];  // first point of each measure (x, alpha, f and the workspace vectors)
  long long bofs;          // first barycenter entry
  int n[kMMMaxK];
  double omega[kMMMaxK];
  double rho;
};

__device__ __forceinline__ double mm_warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double mm_warp_max(double v) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// log <w, e^{-v / c}> over the entries with w > 0 (largest exponent taken out first)
__device__ double mm_log_dot_exp(const float* __restrict__ w, const double* v, int n, double c, int lane) {
  double mx = -INFINITY;
  for (int i = lane; i < n; i += 32)
    if (w[i] > 0.f) mx = fmax(mx, -v[i] / c);
  mx = mm_warp_max(mx);
  double sm = 0.0;
  for (int i = lane; i < n; i += 32)
    if (w[i] > 0.f) sm += (double)w[i] * exp(-v[i] / c - mx);
  sm = mm_warp_sum(sm);
  return mx + log(sm);
}

// lambda_k of the K-marginal rho KL dual at the potentials v (all lanes get them)
template <int K>
__device__ void mm_lambda(const MMProb& P, const float* __restrict__ alpha, double* const (&v)[K], int lane,
                          double (&lam)[K]) {
  double q[K], wsum = 0.0, s = 0.0;
#pragma unroll
  for (int k = 0; k < K; ++k) q[k] = mm_log_dot_exp(alpha + P.off[k], v[k], P.n[k], P.omega[k] * P.rho, lane);
#pragma unroll
  for (int k = 0; k < K; ++k) {
    wsum += P.omega[k];
    s += P.omega[k] * P.rho * q[k];
  }
#pragma unroll
  for (int k = 0; k < K; ++k) lam[k] = P.omega[k] * P.rho * q[k] - P.omega[k] / wsum * s;
}

// C(z) = sum_k omega_k (z_k - B(z))^2 and B(z), in the oracle's order of operations
template <int K>
__device__ __forceinline__ double mm_cost(const double (&z)[K], const double (&w)[K], double* bary) {
  double b = 0.0;
#pragma unroll
  for (int k = 0; k < K; ++k) b += w[k] * z[k];
  double c = 0.0;
#pragma unroll
  for (int k = 0; k < K; ++k) c += w[k] * ((z[k] - b) * (z[k] - b));
  if (bary) *bary = b;
  return c;
}

// SolveMOT (Alg. 3) on lane 0 between the re-weighted measures at[k]; writes the
// potentials r[k]; with bx / bw (nullable) also the plan's barycenter points and
// masses (tuples of positive mass, in plan order), returning their number.
template <int K>
__device__ int mm_walk(const MMProb& P, const float* __restrict__ x, double* const (&at)[K], double* const (&r)[K],
                       double* bx, double* bw) {
  double w[K], z[K], rem[K], cur[K];
  int idx[K];
#pragma unroll
  for (int k = 0; k < K; ++k) {
    w[k] = P.omega[k];
    idx[k] = 0;
    z[k] = (double)x[P.off[k]];
    rem[k] = at[k][0];
    r[k][0] = 0.0;
    cur[k] = 0.0;
  }
  double b = 0.0;
  r[0][0] = mm_cost<K>(z, w, &b);
  cur[0] = r[0][0];
  int nb = 0;
  for (;;) {
    // the measure with the least remaining mass among those that can still move
    int p = -1;
#pragma unroll
    for (int k = 0; k < K; ++k)
      if (idx[k] < P.n[k] - 1 && (p < 0 || rem[k] < rem[p])) p = k;
    if (p < 0) break;
    const double mass = rem[p];
    if (bx && mass > 0.0) {
      bx[nb] = b;
      bw[nb] = mass;
      ++nb;
    }
#pragma unroll
    for (int k = 0; k < K; ++k) rem[k] = rem[k] - mass;
    // the new point of measure p; the potentials of the others stay where they are
    int np = 0;
#pragma unroll
    for (int k = 0; k < K; ++k)
      if (k == p) np = ++idx[k];
    const long long op = P.off[p];
#pragma unroll
    for (int k = 0; k < K; ++k)
      if (k == p) z[k] = (double)x[op + np];
    const double c = mm_cost<K>(z, w, &b);
    double others = 0.0;
#pragma unroll
    for (int k = 0; k < K; ++k)
      if (k != p) others += cur[k];
    const double v = c - others;
#pragma unroll
    for (int k = 0; k < K; ++k)
      if (k == p) {
        cur[k] = v;
        rem[k] = at[k][np];
      }
    r[p][np] = v;
  }
  if (bx && rem[0] > 0.0) {
    bx[nb] = b;  // the last tuple takes the mass left
    bw[nb] = rem[0];
    ++nb;
  }
  return nb;
}

template <int K>
__global__ void __launch_bounds__(32 * kMMWarps)
k_mmot1d(const MMProb* __restrict__ probs, int count, int n_iter, const float* __restrict__ x,
         const float* __restrict__ alpha, double* fb_all, double* at_all, double* r_all, double* __restrict__ f,
         double* __restrict__ bx, double* __restrict__ bw, int* __restrict__ blen, int* __restrict__ status) {
  const int lane = threadIdx.x & 31;
  const int pk = blockIdx.x * kMMWarps + (threadIdx.x >> 5);
  if (pk >= count) return;  // whole warp
  const MMProb P = probs[pk];
  double* FB[K];
  double* AT[K];
  double* R[K];
  bool bad_w = false, bad_x = false;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    FB[k] = fb_all + P.off[k];
    AT[k] = at_all + P.off[k];
    R[k] = r_all + P.off[k];
    const float* X = x + P.off[k];
    const float* A = alpha + P.off[k];
    double tot = 0.0;
    for (int i = lane; i < P.n[k]; i += 32) {
      const float wv = A[i], xi = X[i];
      if (!(wv >= 0.f) || !isfinite(wv)) bad_w = true; else tot += wv;
      if (!isfinite(xi) || (i + 1 < P.n[k] && !(xi <= X[i + 1]))) bad_x = true;
    }
    tot = mm_warp_sum(tot);
    if (!(tot > 0.0)) bad_w = true;
  }
  bad_w = __any_sync(0xffffffffu, bad_w);
  bad_x = __any_sync(0xffffffffu, bad_x);
  if (bad_w || bad_x) {
#pragma unroll
    for (int k = 0; k < K; ++k)
      for (int i = lane; i < P.n[k]; i += 32) f[P.off[k] + i] = __longlong_as_double(0x7ff8000000000000LL);
    if (lane == 0) {
      status[pk] = bad_w ? UOT_ERR_NONFINITE : UOT_ERR_INVALID_ARG;
      blen[pk] = 0;
    }
    return;
  }
#pragma unroll
  for (int k = 0; k < K; ++k)
    for (int i = lane; i < P.n[k]; i += 32) FB[k][i] = 0.0;
  __syncwarp();
  double lam[K];
  auto reweight = [&]() {
    mm_lambda<K>(P, alpha, FB, lane, lam);
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const float* A = alpha + P.off[k];
      const double c = P.omega[k] * P.rho;
      for (int i = lane; i < P.n[k]; i += 32) AT[k][i] = (double)A[i] * exp(-(FB[k][i] + lam[k]) / c);
    }
    __syncwarp();
  };
  for (int t = 0; t < n_iter; ++t) {
    reweight();
    if (lane == 0) (void)mm_walk<K>(P, x, AT, R, nullptr, nullptr);
    __syncwarp();
    const double tau = 2.0 / (2.0 + (double)t);
#pragma unroll
    for (int k = 0; k < K; ++k)
      for (int i = lane; i < P.n[k]; i += 32) FB[k][i] = (1.0 - tau) * FB[k][i] + tau * R[k][i];
    __syncwarp();
  }
  // the translated potentials, and the barycenter of the plan at the final iterate
  reweight();
#pragma unroll
  for (int k = 0; k < K; ++k)
    for (int i = lane; i < P.n[k]; i += 32) f[P.off[k] + i] = FB[k][i] + lam[k];
  if (lane == 0) {
    blen[pk] = mm_walk<K>(P, x, AT, R, bx + P.bofs, bw + P.bofs);
    status[pk] = UOT_OK;
  }
}

size_t mm_align256(size_t v) { return (v + 255) & ~size_t(255); }

struct MMLayout {
  size_t probs, status, blen, fb, at, r, total;
  long long lx;    // length of the packed point arrays
  long long lb;    // length of the packed barycenter arrays
};

uot_status mmfail(uot_status s, const char* msg) {
  set_last_error(msg);
  return s;
}

uot_status validate_mm(const uot_mmot1d_batch* b, MMLayout* L) {
  if (!b) return mmfail(UOT_ERR_INVALID_ARG, "batch is NULL");
  if (b->count < 1) return mmfail(UOT_ERR_INVALID_ARG, "batch count must be >= 1");
  if (b->K < 2 || b->K > kMMMaxK) return mmfail(UOT_ERR_INVALID_ARG, "K must be in 2..8");
  if (b->n_iter < 1) return mmfail(UOT_ERR_INVALID_ARG, "n_iter must be >= 1");
  if (!b->n || !b->off || !b->rho || !b->omega) return mmfail(UOT_ERR_INVALID_ARG, "batch host arrays must not be NULL");
  if (!b->x || !b->alpha) return mmfail(UOT_ERR_INVALID_ARG, "batch device arrays must not be NULL");
  long long lx = 0, lb = 0;
  for (int p = 0; p < b->count; ++p) {
    if (!(b->rho[p] > 0) || !isfinite(b->rho[p])) return mmfail(UOT_ERR_INVALID_ARG, "every problem needs finite rho > 0");
    double ws = 0.0;
    long long tot = 0;
    for (int k = 0; k < b->K; ++k) {
      const int n = b->n[p * b->K + k];
      const long long o = b->off[p * b->K + k];
      const double w = b->omega[p * b->K + k];
      if (n < 1) return mmfail(UOT_ERR_INVALID_ARG, "every measure needs at least one point");
      if (o < 0) return mmfail(UOT_ERR_INVALID_ARG, "offsets must be >= 0");
      if (!(w > 0) || !isfinite(w)) return mmfail(UOT_ERR_INVALID_ARG, "barycentric weights must be finite and > 0");
      ws += w;
      tot += n;
      lx = std::max(lx, o + n);
    }
    if (!(fabs(ws - 1.0) <= 1e-12)) return mmfail(UOT_ERR_INVALID_ARG, "barycentric weights must sum to one");
    lb += tot;
  }
  size_t off = 0;
  auto take = [&](size_t bytes) { size_t o = off; off = mm_align256(off + bytes); return o; };
  L->probs = take(sizeof(MMProb) * b->count);
  L->status = take(sizeof(int) * b->count);
  L->blen = take(sizeof(int) * b->count);
  L->fb = take(sizeof(double) * lx);
  L->at = take(sizeof(double) * lx);
  L->r = take(sizeof(double) * lx);
  L->total = off;
  L->lx = lx;
  L->lb = lb;
  return UOT_OK;
}

#define MMCUDA(call)                                                   \
  do {                                                                 \
    cudaError_t e_ = (call);                                           \
    if (e_ != cudaSuccess) {                                           \
      std::string m_ = std::string(#call) + ": " + cudaGetErrorString(e_); \
      return mmfail(UOT_ERR_CUDA, m_.c_str());                         \
    }                                                                  \
  } while (0)

template <int K>
void launch_mm(int blocks, cudaStream_t st, const MMProb* probs, int count, int n_iter, const float* x,
               const float* alpha, double* fb, double* at, double* r, double* f, double* bx, double* bw, int* blen,
               int* status) {
  k_mmot1d<K><<<blocks, 32 * kMMWarps, 0, st>>>(probs, count, n_iter, x, alpha, fb, at, r, f, bx, bw, blen, status);
}

}  // namespace
}  // namespace uot

using namespace uot;

extern "C" {

size_t uot_mmot1d_workspace_size(const uot_mmot1d_batch* batch) {
  MMLayout L;
  if (validate_mm(batch, &L) != UOT_OK) return 0;
  return L.total;
}

size_t uot_mmot1d_barycenter_size(const uot_mmot1d_batch* batch) {
  MMLayout L;
  if (validate_mm(batch, &L) != UOT_OK) return 0;
  return (size_t)L.lb;
}

uot_status uot_mmot1d_batched(const uot_mmot1d_batch* b, double* f, double* bary_x, double* bary_w,
                              int32_t* bary_len, int32_t* status, void* ws, size_t ws_bytes, void* stream) {
  MMLayout L;
  uot_status v = validate_mm(b, &L);
  if (v != UOT_OK) return v;
  if (!f || !bary_x || !bary_w) return mmfail(UOT_ERR_INVALID_ARG, "f, bary_x and bary_w must not be NULL");
  if (!ws) return mmfail(UOT_ERR_WORKSPACE, "workspace is NULL");
  if (reinterpret_cast<uintptr_t>(ws) & 255) return mmfail(UOT_ERR_WORKSPACE, "workspace must be 256-byte aligned");
  if (ws_bytes < L.total) return mmfail(UOT_ERR_WORKSPACE, "workspace too small for the batch");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  char* base = static_cast<char*>(ws);
  const int count = b->count, K = b->K;
  std::vector<MMProb> probs(count);
  long long bofs = 0;
  for (int p = 0; p < count; ++p) {
    MMProb& P = probs[p];
    P = MMProb{};
    P.rho = b->rho[p];
    P.bofs = bofs;
    for (int k = 0; k < K; ++k) {
      P.off[k] = b->off[p * K + k];
      P.n[k] = b->n[p * K + k];
      P.omega[k] = b->omega[p * K + k];
      bofs += P.n[k];
    }
  }
  MMProb* d_probs = reinterpret_cast<MMProb*>(base + L.probs);
  int* d_status = reinterpret_cast<int*>(base + L.status);
  int* d_blen = reinterpret_cast<int*>(base + L.blen);
  double* fb = reinterpret_cast<double*>(base + L.fb);
  double* at = reinterpret_cast<double*>(base + L.at);
  double* r = reinterpret_cast<double*>(base + L.r);
  MMCUDA(cudaMemcpyAsync(d_probs, probs.data(), sizeof(MMProb) * count, cudaMemcpyHostToDevice, st));
  const int blocks = (count + kMMWarps - 1) / kMMWarps;
  switch (K) {
    case 2: launch_mm<2>(blocks, st, d_probs, count, b->n_iter, b->x, b->alpha, fb, at, r, f, bary_x, bary_w, d_blen, d_status); break;
    case 3: launch_mm<3>(blocks, st, d_probs, count, b->n_iter, b->x, b->alpha, fb, at, r, f, bary_x, bary_w, d_blen, d_status); break;
    case 4: launch_mm<4>(blocks, st, d_probs, count, b->n_iter, b->x, b->alpha, fb, at, r, f, bary_x, bary_w, d_blen, d_status); break;
    case 5: launch_mm<5>(blocks, st, d_probs, count, b->n_iter, b->x, b->alpha, fb, at, r, f, bary_x, bary_w, d_blen, d_status); break;
    case 6: launch_mm<6>(blocks, st, d_probs, count, b->n_iter, b->x, b->alpha, fb, at, r, f, bary_x, bary_w, d_blen, d_status); break;
    case 7: launch_mm<7>(blocks, st, d_probs, count, b->n_iter, b->x, b->alpha, fb, at, r, f, bary_x, bary_w, d_blen, d_status); break;
    default: launch_mm<8>(blocks, st, d_probs, count, b->n_iter, b->x, b->alpha, fb, at, r, f, bary_x, bary_w, d_blen, d_status);
  }
  note_launch();
  MMCUDA(cudaGetLastError());
  std::vector<int> hs(count), hl(count);
  MMCUDA(cudaMemcpyAsync(hs.data(), d_status, sizeof(int) * count, cudaMemcpyDeviceToHost, st));
  MMCUDA(cudaMemcpyAsync(hl.data(), d_blen, sizeof(int) * count, cudaMemcpyDeviceToHost, st));
  MMCUDA(cudaStreamSynchronize(st));
  uot_status out = UOT_OK;
  for (int p = 0; p < count; ++p) {
    if (status) status[p] = hs[p];
    if (bary_len) bary_len[p] = hl[p];
    if (out == UOT_OK && hs[p] != UOT_OK) out = static_cast<uot_status>(hs[p]);
  }
  if (out != UOT_OK) set_last_error("some problems have invalid points or weights (see status)");
  return out;
}

}  // extern "C"
