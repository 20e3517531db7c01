// 1-D unbalanced multi-marginal OT and barycenters (Sec. 5) by Frank-Wolfe on
// the translation-invariant functional H, batched: one warp per problem, in
// float pairs (about 44 bits; FP64 runs at a small fraction of the FP32 rate on
// this GPU, and the walk's dependent FP64 chain bounded the kernel).
//
// A problem has K measures (x_k, alpha_k) on the line with sorted points,
// barycentric weights omega_k >= 0 summing to one, the rho KL penalties and
// the squared-distance ground cost, whose multi-marginal form is
//   C(z_1..z_K) = sum_k omega_k (z_k - B(z))^2,  B(z) = sum_k omega_k z_k.
// Each Frank-Wolfe step computes, with all lanes (the SolveMOT walk too: a
// merge path over the warp, see mm_walk),
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
#include <mutex>
#include <string>
#include <vector>

#include "ffloat.cuh"
#include "uot_internal.cuh"

namespace uot {
namespace {

constexpr int kMMWarps = 4;  // problems per CTA
constexpr int kMMMaxK = 8;   // measures per problem
// a problem with at most this many points in all keeps its re-weighted masses (and their partial
// sums and the ranks of the walk's events) in shared memory
constexpr int kMMSmemPoints = 2048;

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

// v[0..n) <- its inclusive prefix sums, float pairs, on one warp (a contiguous chunk per lane,
// the chunk totals scanned across the lanes).  A point of zero weight (w[i] == 0) then gets
// exactly its predecessor's sum: the scan's association differs between chunks, and a sum that
// differed in its last bits would turn that point's zero mass into a tiny positive one.
__device__ void mm_prefix_sum(float2* v, const float* __restrict__ w, int n, int lane) {
  const int c = (n + 31) / 32, b = min(n, lane * c), e = min(n, b + c);
  ff t{0.f, 0.f};
  int lnz = -1;  // the last point of nonzero weight in this lane's chunk
  for (int k = b; k < e; ++k) {
    t = ffl::add(t, ld_ff(v, k));
    if (w[k] != 0.f) lnz = k;
  }
  for (int o = 1; o < 32; o <<= 1) {
    const float h = __shfl_up_sync(0xffffffffu, t.hi, o), l = __shfl_up_sync(0xffffffffu, t.lo, o);
    const int z = __shfl_up_sync(0xffffffffu, lnz, o);
    if (lane >= o) {
      t = ffl::add(t, ff{h, l});
      lnz = max(lnz, z);
    }
  }
  const float h = __shfl_up_sync(0xffffffffu, t.hi, 1), l = __shfl_up_sync(0xffffffffu, t.lo, 1);
  int carry = __shfl_up_sync(0xffffffffu, lnz, 1);  // the last nonzero point before this chunk
  if (lane == 0) carry = -1;
  ff run = lane == 0 ? ff{0.f, 0.f} : ff{h, l};
  for (int k = b; k < e; ++k) {
    run = ffl::add(run, ld_ff(v, k));
    if (w[k] != 0.f) st_ff(v, k, run);
  }
  __syncwarp();
  for (int k = b; k < e; ++k) {
    if (w[k] == 0.f) st_ff(v, k, carry >= 0 ? ld_ff(v, carry) : ff{0.f, 0.f});
    else carry = k;
  }
}

// number of entries of the sorted a[0..n) that are <= v (le) or < v (!le)
__device__ __forceinline__ int mm_count(const float2* a, int n, ff v, bool le) {
  int lo = 0, hi = n;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    const ff x = ld_ff(a, mid);
    if (le ? !ff_lt(v, x) : ff_lt(x, v)) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

// SolveMOT (Alg. 3) on the whole warp between the re-weighted measures (at[k]: the masses divided
// by their common mass; replaced here by their partial sums A^k).  Every step takes the movable
// measure of least A^k_{idx_k} (lowest index on ties), so the walk is the stable K-way merge of the
// partial-sum sequences: the lanes rank every event of that merge together, each lane takes an
// equal share of the steps, reads its starting tuple off the ranks, and walks it.  The current potentials always sum to the current
// tuple's cost, so a newly reached point's potential is its measure's previous one plus the
// change of that cost: a share shifts each measure's potential by a sum of cost changes, and a
// warp scan of those K sums gives every share its starting potentials for the second walk, which
// writes them.  With bx / bw (nullable) also the plan's barycenter points and masses (tuples of
// positive mass in plan order, the masses times mscale; their places from a warp scan of the
// shares' counts); returns their number (on every lane).  Float pairs: the branches are the
// oracle's except within about 1e-13 of a tie between partial sums.
template <int K>
__device__ int mm_walk(const MMProb& P, const MMConst<K>& C, const float* __restrict__ x,
                       const float* __restrict__ alpha, float2* const (&at)[K], int* const (&rk)[K],
                       float2* const (&r)[K], double* bx, double* bw, ff mscale, int lane) {
#pragma unroll
  for (int k = 0; k < K; ++k) mm_prefix_sum(at[k], alpha + P.off[k], P.n[k], lane);
  __syncwarp();
  int total = 0;
#pragma unroll
  for (int k = 0; k < K; ++k) total += P.n[k] - 1;
  const int s0 = (int)((long long)lane * total / 32), s1 = (int)((long long)(lane + 1) * total / 32);
  // the rank of every event in the merge, all lanes over all events (uniform work): event (k, i)
  // comes after i events of its own measure, the events of lower measures of value <= its own and
  // those of higher measures of smaller value
#pragma unroll
  for (int k = 0; k < K; ++k)
    for (int i = lane; i < P.n[k] - 1; i += 32) {
      const ff v = ld_ff(at[k], i);
      int rnk = i;
#pragma unroll
      for (int q = 0; q < K; ++q)
        if (q != k) rnk += mm_count(at[q], P.n[q] - 1, v, q < k);
      rk[k][i] = rnk;
    }
  __syncwarp();
  // the lane's starting tuple: per measure, the number of its events of rank below s0
  int idx0[K];
#pragma unroll
  for (int k = 0; k < K; ++k) {
    int lo = 0, hi = P.n[k] - 1;
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (rk[k][mid] < s0) lo = mid + 1;
      else hi = mid;
    }
    idx0[k] = lo;
  }
  // the value of event s0 - 1 (the largest value among the events taken), 0 at the start
  ff prev0{0.f, 0.f};
#pragma unroll
  for (int k = 0; k < K; ++k)
    if (idx0[k] > 0) prev0 = ff_max(prev0, ld_ff(at[k], idx0[k] - 1));
  // first walk: each measure's summed cost changes, and the count of positive masses
  ff d[K];
  int npos = 0;
  {
    int idx[K];
    float z[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
      idx[k] = idx0[k];
      z[k] = x[P.off[k] + idx[k]];
      d[k] = ff{0.f, 0.f};
    }
    ff b, Cc = mm_cost<K>(z, C.w, &b), prev = prev0;
    for (int st = s0; st < s1; ++st) {
      int p = -1;
      ff v{0.f, 0.f};
#pragma unroll
      for (int k = 0; k < K; ++k)
        if (idx[k] < P.n[k] - 1) {
          const ff a = ld_ff(at[k], idx[k]);
          if (p < 0 || ff_lt(a, v)) { p = k; v = a; }
        }
      if (ff_pos(ffl::add(v, ffl::neg(prev)))) ++npos;
      prev = v;
#pragma unroll
      for (int k = 0; k < K; ++k)
        if (k == p) {
          ++idx[k];
          z[k] = x[P.off[k] + idx[k]];
        }
      const ff Cn = mm_cost<K>(z, C.w, &b);
      const ff dc = ffl::add(Cn, ffl::neg(Cc));
#pragma unroll
      for (int k = 0; k < K; ++k)
        if (k == p) d[k] = ffl::add(d[k], dc);
      Cc = Cn;
    }
  }
  // exclusive scans over the lanes: starting potentials and output places
  ff cur[K];
  {
    float z0[K];
#pragma unroll
    for (int k = 0; k < K; ++k) z0[k] = x[P.off[k]];
    ff b0;
    const ff c00 = mm_cost<K>(z0, C.w, &b0);
#pragma unroll
    for (int k = 0; k < K; ++k) {
      ff t = d[k];
      for (int o = 1; o < 32; o <<= 1) {
        const float h = __shfl_up_sync(0xffffffffu, t.hi, o), l = __shfl_up_sync(0xffffffffu, t.lo, o);
        if (lane >= o) t = ffl::add(t, ff{h, l});
      }
      const float h = __shfl_up_sync(0xffffffffu, t.hi, 1), l = __shfl_up_sync(0xffffffffu, t.lo, 1);
      const ff ex = lane == 0 ? ff{0.f, 0.f} : ff{h, l};
      cur[k] = k == 0 ? ffl::add(c00, ex) : ex;
    }
    if (lane == 0) {
#pragma unroll
      for (int k = 0; k < K; ++k) st_ff(r[k], 0, k == 0 ? c00 : ff{0.f, 0.f});
    }
  }
  int cnt = npos;
  for (int o = 1; o < 32; o <<= 1) {
    const int v = __shfl_up_sync(0xffffffffu, cnt, o);
    if (lane >= o) cnt += v;
  }
  const int all = __shfl_sync(0xffffffffu, cnt, 31);
  int out = cnt - npos;
  // second walk: the potentials (and the barycenter entries)
  {
    int idx[K];
    float z[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
      idx[k] = idx0[k];
      z[k] = x[P.off[k] + idx[k]];
    }
    ff b, Cc = mm_cost<K>(z, C.w, &b), prev = prev0;
    for (int st = s0; st < s1; ++st) {
      int p = -1;
      ff v{0.f, 0.f};
#pragma unroll
      for (int k = 0; k < K; ++k)
        if (idx[k] < P.n[k] - 1) {
          const ff a = ld_ff(at[k], idx[k]);
          if (p < 0 || ff_lt(a, v)) { p = k; v = a; }
        }
      const ff mass = ffl::add(v, ffl::neg(prev));
      if (ff_pos(mass)) {
        if (bx) {
          bx[out] = ffl::to_double(b);
          bw[out] = ffl::to_double(ffl::mul(mass, mscale));
        }
        ++out;
      }
      prev = v;
      int np = 0;
#pragma unroll
      for (int k = 0; k < K; ++k)
        if (k == p) {
          np = ++idx[k];
          z[k] = x[P.off[k] + idx[k]];
        }
      const ff Cn = mm_cost<K>(z, C.w, &b);
      const ff dc = ffl::add(Cn, ffl::neg(Cc));
      Cc = Cn;
#pragma unroll
      for (int k = 0; k < K; ++k)
        if (k == p) {
          cur[k] = ffl::add(cur[k], dc);
          st_ff(r[k], np, cur[k]);
        }
    }
  }
  // the last tuple takes the mass left: A^0 at its last point minus the last event's value
  int nb = all;
  {
    ff last{0.f, 0.f};
#pragma unroll
    for (int k = 0; k < K; ++k)
      if (P.n[k] > 1) last = ff_max(last, ld_ff(at[k], P.n[k] - 2));
    const ff mass = ffl::add(ld_ff(at[0], P.n[0] - 1), ffl::neg(last));
    if (ff_pos(mass)) {
      if (bx && lane == 0) {
        float z[K];
#pragma unroll
        for (int k = 0; k < K; ++k) z[k] = x[P.off[k] + P.n[k] - 1];
        ff b;
        (void)mm_cost<K>(z, C.w, &b);
        bx[all] = ffl::to_double(b);
        bw[all] = ffl::to_double(ffl::mul(mass, mscale));
      }
      ++nb;
    }
  }
  __syncwarp();
  return nb;
}

template <int K>
__global__ void __launch_bounds__(32 * kMMWarps)
k_mmot1d(const MMProb* __restrict__ probs, int count, int n_iter, const float* __restrict__ x,
         const float* __restrict__ alpha, double* fb_all, double* at_all, double* r_all, int* rk_all,
         double* __restrict__ f,
         double* __restrict__ bx, double* __restrict__ bw, int* __restrict__ blen, int* __restrict__ status) {
  const int lane = threadIdx.x & 31;
  const int pk = blockIdx.x * kMMWarps + (threadIdx.x >> 5);
  if (pk >= count) return;  // whole warp
  const MMProb P = probs[pk];
  // working vectors as float pairs in the double-sized slots of the workspace
  extern __shared__ float2 mm_smem[];
  float2* FB[K];
  float2* AT[K];
  float2* R[K];
  int* RK[K];
  bool bad_w = false, bad_x = false;
  int npts = 0;
#pragma unroll
  for (int k = 0; k < K; ++k) npts += P.n[k];
  const bool in_smem = npts <= kMMSmemPoints;
  int soff = 0;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    FB[k] = reinterpret_cast<float2*>(fb_all + P.off[k]);
    AT[k] = in_smem ? mm_smem + (threadIdx.x >> 5) * kMMSmemPoints + soff : reinterpret_cast<float2*>(at_all + P.off[k]);
    RK[k] = in_smem ? reinterpret_cast<int*>(mm_smem + kMMWarps * kMMSmemPoints) + (threadIdx.x >> 5) * kMMSmemPoints + soff
                    : rk_all + P.off[k];
    soff += P.n[k];
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
    (void)mm_walk<K>(P, C, x, alpha, AT, RK, R, nullptr, nullptr, ff{1.f, 0.f}, lane);
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
  const ff m = ffl::exp2(ffl::mul(lnm, kMMLog2eff));
  const int nb = mm_walk<K>(P, C, x, alpha, AT, RK, R, bx + P.bofs, bw + P.bofs, m, lane);
  if (lane == 0) {
    blen[pk] = nb;
    status[pk] = UOT_OK;
  }
}

size_t mm_align256(size_t v) { return (v + 255) & ~size_t(255); }

struct MMLayout {
  size_t probs, status, blen, fb, at, r, rk, total;
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
  L->rk = take(sizeof(int) * lx);
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
cudaError_t launch_mm(int blocks, cudaStream_t st, const MMProb* probs, int count, int n_iter, const float* x,
                      const float* alpha, double* fb, double* at, double* r, int* rk, double* f, double* bx,
                      double* bw, int* blen, int* status) {
  constexpr size_t smem = (sizeof(float2) + sizeof(int)) * kMMWarps * kMMSmemPoints;
  static std::once_flag once;
  static cudaError_t attr = cudaSuccess;
  std::call_once(once, [] {
    attr = cudaFuncSetAttribute(k_mmot1d<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  });
  if (attr != cudaSuccess) return attr;
  k_mmot1d<K><<<blocks, 32 * kMMWarps, smem, st>>>(probs, count, n_iter, x, alpha, fb, at, r, rk, f, bx, bw,
                                                   blen, status);
  return cudaSuccess;
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
  int* rk = reinterpret_cast<int*>(base + L.rk);
  MMCUDA(cudaMemcpyAsync(d_probs, probs.data(), sizeof(MMProb) * count, cudaMemcpyHostToDevice, st));
  const int blocks = (count + kMMWarps - 1) / kMMWarps;
  cudaError_t le = cudaSuccess;
  switch (K) {
    case 2: le = launch_mm<2>(blocks, st, d_probs, count, b->n_iter, b->x, b->alpha, fb, at, r, rk, f, bary_x, bary_w, d_blen, d_status); break;
    case 3: le = launch_mm<3>(blocks, st, d_probs, count, b->n_iter, b->x, b->alpha, fb, at, r, rk, f, bary_x, bary_w, d_blen, d_status); break;
    case 4: le = launch_mm<4>(blocks, st, d_probs, count, b->n_iter, b->x, b->alpha, fb, at, r, rk, f, bary_x, bary_w, d_blen, d_status); break;
    case 5: le = launch_mm<5>(blocks, st, d_probs, count, b->n_iter, b->x, b->alpha, fb, at, r, rk, f, bary_x, bary_w, d_blen, d_status); break;
    case 6: le = launch_mm<6>(blocks, st, d_probs, count, b->n_iter, b->x, b->alpha, fb, at, r, rk, f, bary_x, bary_w, d_blen, d_status); break;
    case 7: le = launch_mm<7>(blocks, st, d_probs, count, b->n_iter, b->x, b->alpha, fb, at, r, rk, f, bary_x, bary_w, d_blen, d_status); break;
    default: le = launch_mm<8>(blocks, st, d_probs, count, b->n_iter, b->x, b->alpha, fb, at, r, rk, f, bary_x, bary_w, d_blen, d_status);
  }
  MMCUDA(le);
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
