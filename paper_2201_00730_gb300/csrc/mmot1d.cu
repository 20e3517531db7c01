// 1-D unbalanced multi-marginal OT and barycenters (Sec. 5) by Frank-Wolfe on
// the translation-invariant functional H, batched: one warp per problem, in
// float pairs (about 44 bits; FP64 runs at a small fraction of the FP32 rate on
// this GPU, and the walk's dependent FP64 chain bounded the kernel).
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
// its tuples of positive mass, with those masses as weights.  The walk keeps the
// oracle's order of operations on float pairs and the re-weighted masses divided
// by their common mass (no comparison sees the factor; the output masses are
// multiplied back), so its branches are the oracle's except within about 1e-13
// of a tie.
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>
#include <string>
#include <vector>

#include "ffloat.cuh"
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

using ffl::ff;

__device__ __forceinline__ ff ld_ff(const float2* p, long long i) {
  const float2 v = p[i];
  return ff{v.x, v.y};
}
__device__ __forceinline__ void st_ff(float2* p, long long i, ff v) { p[i] = make_float2(v.hi, v.lo); }
// a < b and a > 0 for normalised float pairs
__device__ __forceinline__ bool ff_lt(ff a, ff b) { return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo); }
__device__ __forceinline__ bool ff_pos(ff a) { return a.hi > 0.f || (a.hi == 0.f && a.lo > 0.f); }
__device__ __forceinline__ ff ff_max(ff a, ff b) { return ff_lt(a, b) ? b : a; }
__device__ __forceinline__ ff mm_warp_sum_ff(ff v) {
  for (int o = 16; o > 0; o >>= 1)
    v = ffl::add(v, ff{__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o)});
  return v;
}
__device__ __forceinline__ ff mm_warp_max_ff(ff v) {
  for (int o = 16; o > 0; o >>= 1)
    v = ff_max(v, ff{__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o)});
  return v;
}

constexpr double kMMLog2e = 1.44269504088896340736;
constexpr ff kMMLog2eff{(float)kMMLog2e, (float)(kMMLog2e - (double)(float)kMMLog2e)};

// w e^y for w >= 0 and a float pair y with w e^y <= 1 (y may be large when w is tiny): the power
// of two is split off first so that the table exp2 stays within its range
__device__ __forceinline__ ff mm_w_exp(float w, ff y) {
  ff z = ffl::mul(y, kMMLog2eff);
  float sc = 1.f;
  if (z.hi > 60.f) {
    const float k = ceilf(z.hi) - 60.f;
    z = ffl::add(z, -k);
    sc = ffl::pow2f((int)k);
  }
  return ffl::mul(ffl::exp2(z), w * sc);
}

// log <w, e^{-v cinv}> over the entries with w > 0 (largest exponent taken out first)
__device__ ff mm_log_dot_exp(const float* __restrict__ w, const float2* v, int n, ff cinv, int lane) {
  ff mx{-INFINITY, 0.f};
  for (int i = lane; i < n; i += 32)
    if (w[i] > 0.f) mx = ff_max(mx, ffl::neg(ffl::mul(ld_ff(v, i), cinv)));
  mx = mm_warp_max_ff(mx);
  ff sm{0.f, 0.f};
  for (int i = lane; i < n; i += 32)
    if (w[i] > 0.f) {
      const ff e = ffl::add(ffl::neg(ffl::mul(ld_ff(v, i), cinv)), ffl::neg(mx));
      sm = ffl::add(sm, ffl::mul(ffl::exp2(ffl::mul(e, kMMLog2eff)), w[i]));
    }
  sm = mm_warp_sum_ff(sm);
  return ffl::add(mx, ffl::log_ff(sm));
}

// Per-problem constants as float pairs (the FP64 work done once): omega_k, 1 / (omega_k rho),
// omega_k rho and omega_k / sum_l omega_l.
template <int K>
struct MMConst {
  ff w[K], cinv[K], orho[K], ofrac[K];
};

// lambda_k of the K-marginal rho KL dual at the potentials v (all lanes get them), and q_k
template <int K>
__device__ void mm_lambda(const MMProb& P, const MMConst<K>& C, const float* __restrict__ alpha,
                          float2* const (&v)[K], int lane, ff (&lam)[K], ff (&q)[K]) {
  ff s{0.f, 0.f};
#pragma unroll
  for (int k = 0; k < K; ++k) {
    q[k] = mm_log_dot_exp(alpha + P.off[k], v[k], P.n[k], C.cinv[k], lane);
    s = ffl::add(s, ffl::mul(C.orho[k], q[k]));
  }
#pragma unroll
  for (int k = 0; k < K; ++k) lam[k] = ffl::add(ffl::mul(C.orho[k], q[k]), ffl::neg(ffl::mul(C.ofrac[k], s)));
}

// C(z) = sum_k omega_k (z_k - B(z))^2 and B(z), in the oracle's order of operations (float pairs)
template <int K>
__device__ __forceinline__ ff mm_cost(const float (&z)[K], const ff (&w)[K], ff* bary) {
  ff b{0.f, 0.f};
#pragma unroll
  for (int k = 0; k < K; ++k) b = ffl::add(b, ffl::mul(w[k], z[k]));
  ff c{0.f, 0.f};
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const ff d = ffl::add(ffl::neg(b), z[k]);
    c = ffl::add(c, ffl::mul(w[k], ffl::mul(d, d)));
  }
  *bary = b;
  return c;
}

// SolveMOT (Alg. 3) on lane 0 between the re-weighted measures at[k] (divided by their common mass,
// which no comparison sees); writes the potentials r[k]; with bx / bw (nullable) also the plan's
// barycenter points and masses (tuples of positive mass, in plan order; the masses times mscale,
// the common mass), returning their number.  Float pairs: the branches are the oracle's except
// within about 1e-13 of a tie between remaining masses.
template <int K>
__device__ int mm_walk(const MMProb& P, const MMConst<K>& C, const float* __restrict__ x, float2* const (&at)[K],
                       float2* const (&r)[K], double* bx, double* bw, ff mscale) {
  float z[K];
  ff rem[K], cur[K];
  int idx[K];
#pragma unroll
  for (int k = 0; k < K; ++k) {
    idx[k] = 0;
    z[k] = x[P.off[k]];
    rem[k] = ld_ff(at[k], 0);
    st_ff(r[k], 0, ff{0.f, 0.f});
    cur[k] = ff{0.f, 0.f};
  }
  ff b;
  cur[0] = mm_cost<K>(z, C.w, &b);
  st_ff(r[0], 0, cur[0]);
  int nb = 0;
  for (;;) {
    // the measure with the least remaining mass among those that can still move
    int p = -1;
    ff mass{0.f, 0.f};
#pragma unroll
    for (int k = 0; k < K; ++k)
      if (idx[k] < P.n[k] - 1 && (p < 0 || ff_lt(rem[k], mass))) {
        p = k;
        mass = rem[k];
      }
    if (p < 0) break;
    if (bx && ff_pos(mass)) {
      bx[nb] = ffl::to_double(b);
      bw[nb] = ffl::to_double(ffl::mul(mass, mscale));
      ++nb;
    }
    const ff nm = ffl::neg(mass);
#pragma unroll
    for (int k = 0; k < K; ++k) rem[k] = ffl::add(rem[k], nm);
    // the new point of measure p; the potentials of the others stay where they are
    int np = 0;
#pragma unroll
    for (int k = 0; k < K; ++k)
      if (k == p) np = ++idx[k];
    const long long op = P.off[p];
#pragma unroll
    for (int k = 0; k < K; ++k)
      if (k == p) z[k] = x[op + np];
    const ff c = mm_cost<K>(z, C.w, &b);
    ff others{0.f, 0.f};
#pragma unroll
    for (int k = 0; k < K; ++k)
      if (k != p) others = ffl::add(others, cur[k]);
    const ff v = ffl::add(c, ffl::neg(others));
#pragma unroll
    for (int k = 0; k < K; ++k)
      if (k == p) {
        cur[k] = v;
        rem[k] = ld_ff(at[k], np);
      }
    st_ff(r[p], np, v);
  }
  if (bx && ff_pos(rem[0])) {
    bx[nb] = ffl::to_double(b);  // the last tuple takes the mass left
    bw[nb] = ffl::to_double(ffl::mul(rem[0], mscale));
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
  // working vectors as float pairs in the double-sized slots of the workspace
  float2* FB[K];
  float2* AT[K];
  float2* R[K];
  bool bad_w = false, bad_x = false;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    FB[k] = reinterpret_cast<float2*>(fb_all + P.off[k]);
    AT[k] = reinterpret_cast<float2*>(at_all + P.off[k]);
    R[k] = reinterpret_cast<float2*>(r_all + P.off[k]);
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
  MMConst<K> C;
  {
    double wsum = 0.0;
#pragma unroll
    for (int k = 0; k < K; ++k) wsum += P.omega[k];
#pragma unroll
    for (int k = 0; k < K; ++k) {
      C.w[k] = ffl::from_double(P.omega[k]);
      C.cinv[k] = ffl::from_double(1.0 / (P.omega[k] * P.rho));
      C.orho[k] = ffl::from_double(P.omega[k] * P.rho);
      C.ofrac[k] = ffl::from_double(P.omega[k] / wsum);
    }
  }
#pragma unroll
  for (int k = 0; k < K; ++k)
    for (int i = lane; i < P.n[k]; i += 32) st_ff(FB[k], i, ff{0.f, 0.f});
  __syncwarp();
  ff lam[K], q[K], lnm{0.f, 0.f};
  // a~_k = alpha_k e^{-(fb_k + lambda_k) / (omega_k rho)} divided by their common mass m
  // (ln m = q_0 - lambda_0 / (omega_0 rho)), which keeps them <= 1
  auto reweight = [&]() {
    mm_lambda<K>(P, C, alpha, FB, lane, lam, q);
    lnm = ffl::add(q[0], ffl::neg(ffl::mul(lam[0], C.cinv[0])));
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const float* A = alpha + P.off[k];
      for (int i = lane; i < P.n[k]; i += 32) {
        ff v{0.f, 0.f};
        if (A[i] > 0.f) {
          const ff e = ffl::add(ffl::neg(ffl::mul(ffl::add(ld_ff(FB[k], i), lam[k]), C.cinv[k])), ffl::neg(lnm));
          v = mm_w_exp(A[i], e);
        }
        st_ff(AT[k], i, v);
      }
    }
    __syncwarp();
  };
  for (int t = 0; t < n_iter; ++t) {
    reweight();
    if (lane == 0) (void)mm_walk<K>(P, C, x, AT, R, nullptr, nullptr, ff{1.f, 0.f});
    __syncwarp();
    const ff tau = ffl::from_double(2.0 / (2.0 + (double)t));
    const ff t1 = ffl::add(ffl::neg(tau), 1.f);
#pragma unroll
    for (int k = 0; k < K; ++k)
      for (int i = lane; i < P.n[k]; i += 32)
        st_ff(FB[k], i, ffl::add(ffl::mul(ld_ff(FB[k], i), t1), ffl::mul(ld_ff(R[k], i), tau)));
    __syncwarp();
  }
  // the translated potentials, and the barycenter of the plan at the final iterate
  reweight();
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const double lk = ffl::to_double(lam[k]);
    for (int i = lane; i < P.n[k]; i += 32) f[P.off[k] + i] = ffl::to_double(ld_ff(FB[k], i)) + lk;
  }
  if (lane == 0) {
    const ff m = ffl::exp2(ffl::mul(lnm, kMMLog2eff));
    blen[pk] = mm_walk<K>(P, C, x, AT, R, bx + P.bofs, bw + P.bofs, m);
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
