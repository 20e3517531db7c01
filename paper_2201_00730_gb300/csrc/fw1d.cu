// 1-D unregularised UOT by Frank-Wolfe on H_0 (Sec. 4, Alg. 2), batched: one
// warp per problem, in float pairs (about 44 bits: FP64 runs at a small
// fraction of the FP32 rate on this GPU).  Per step the warp computes
//   lambda* = rho1 rho2 / (rho1 + rho2) (log<a, e^{-fb/rho1}> - log<b, e^{-gb/rho2}>)   (Prop. 2)
//   a~ = a e^{-(fb + lambda*)/rho1},  b~ = b e^{-(gb - lambda*)/rho2}              (Eq. fw-updated-histo)
// with all lanes (a~ and b~ divided by their common mass, which the walk does
// not see), then the warp walks the two sorted point lists to get the duals
// (r, s) of the balanced 1-D OT between a~ and b~ (SolveOT1D, Alg. 1: the point
// whose remaining mass is smaller is exhausted first, and each newly reached
// point's potential is the current pair's cost minus the other side's current
// potential) as a merge path split over the lanes, and all lanes take the step
//   (fb, gb) <- (1 - gamma_t)(fb, gb) + gamma_t (r, s),  gamma_t = 2 / (2 + t).
// The batch supplies the rest of the parallelism.  Working vectors live in the
// workspace, indexed by the problems' offsets (a~ and b~ in shared memory when
// the problem is small enough).
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>
#include <string>
#include <vector>

#include "ffloat.cuh"
#include "uot_internal.cuh"

namespace uot {
namespace {

constexpr int kFWWarps = 4;         // problems per CTA
constexpr int kFWSmemPoints = 1536;  // a problem with N + M <= this keeps a~, b~ in shared memory

struct FWProb {
  long long xo, yo;
  int n, m;
  double rho1, rho2;
};

__device__ __forceinline__ double warp_sum_d(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// float-pair warp reductions (the pair is rounded after each combination)
__device__ __forceinline__ ffl::ff warp_sum_ff(ffl::ff v) {
  for (int o = 16; o > 0; o >>= 1)
    v = ffl::add(v, ffl::ff{__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o)});
  return v;
}
__device__ __forceinline__ ffl::ff ff_max(ffl::ff a, ffl::ff b) {
  return (a.hi > b.hi || (a.hi == b.hi && a.lo >= b.lo)) ? a : b;
}
__device__ __forceinline__ ffl::ff warp_max_ff(ffl::ff v) {
  for (int o = 16; o > 0; o >>= 1)
    v = ff_max(v, ffl::ff{__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o)});
  return v;
}

// log2(e) as a float pair
constexpr double kLog2e = 1.44269504088896340736;
constexpr ffl::ff kLog2eff{(float)kLog2e, (float)(kLog2e - (double)(float)kLog2e)};

// e^y for a float pair y <= 0 (or of moderate size): 2^(y log2 e)
__device__ __forceinline__ ffl::ff exp_ff(ffl::ff y) { return ffl::exp2(ffl::mul(y, kLog2eff)); }

// w e^y for w >= 0 and a float pair y with w e^y <= 1 (y itself may be large when w is tiny): the
// power of two is split off first so that the table exp2 stays within its range
__device__ __forceinline__ ffl::ff w_exp_ff(float w, ffl::ff y) {
  ffl::ff z = ffl::mul(y, kLog2eff);
  float sc = 1.f;
  if (z.hi > 60.f) {
    const float k = ceilf(z.hi) - 60.f;  // w 2^k <= 1 since w 2^z <= 1
    z = ffl::add(z, -k);
    sc = ffl::pow2f((int)k);
  }
  return ffl::mul(ffl::exp2(z), w * sc);
}

// log <w, e^{-v rinv}> over the entries with w > 0 (largest exponent taken out first), float pairs
__device__ ffl::ff log_dot_exp_neg(const float* __restrict__ w, const float2* v, int n, ffl::ff rinv, int lane) {
  ffl::ff mx{-INFINITY, 0.f};
  for (int i = lane; i < n; i += 32)
    if (w[i] > 0.f) mx = ff_max(mx, ffl::neg(ffl::mul(ffl::ff{v[i].x, v[i].y}, rinv)));
  mx = warp_max_ff(mx);
  ffl::ff sm{0.f, 0.f};
  for (int i = lane; i < n; i += 32)
    if (w[i] > 0.f) {
      const ffl::ff e = ffl::add(ffl::neg(ffl::mul(ffl::ff{v[i].x, v[i].y}, rinv)), ffl::neg(mx));
      sm = ffl::add(sm, ffl::mul(exp_ff(e), w[i]));
    }
  sm = warp_sum_ff(sm);
  return ffl::add(mx, ffl::log_ff(sm));
}

// |x - y|^p as a float pair: x - y exactly (two_sum), then its square (p = 2),
// its magnitude (p = 1), or an FP64 power for other p
// (pmode: 2 for p = 2, 1 for p = 1, 0 otherwise, decided once outside the walk, whose every
// comparison of the FP64 p would otherwise take the slow FP64 pipe)
__device__ __forceinline__ ffl::ff cost_ff(float xi, float yj, int pmode, double p) {
  const ffl::ff d = ffl::two_sum(xi, -yj);
  if (pmode == 2) return ffl::mul(d, d);
  if (pmode == 1) return d.hi < 0.f ? ffl::neg(d) : d;
  return ffl::from_double(pow(fabs((double)d.hi + (double)d.lo), p));
}

// a < b for normalised float pairs
__device__ __forceinline__ bool ff_lt(float2 a, float2 b) { return a.x < b.x || (a.x == b.x && a.y < b.y); }

// v[0..n) <- its inclusive prefix sums, float pairs, on one warp (a contiguous chunk per lane,
// the chunk totals scanned across the lanes)
__device__ void prefix_sum_ff(float2* v, int n, int lane) {
  const int c = (n + 31) / 32, b = min(n, lane * c), e = min(n, b + c);
  ffl::ff t{0.f, 0.f};
  for (int k = b; k < e; ++k) t = ffl::add(t, ffl::ff{v[k].x, v[k].y});
  for (int o = 1; o < 32; o <<= 1) {
    const float h = __shfl_up_sync(0xffffffffu, t.hi, o), l = __shfl_up_sync(0xffffffffu, t.lo, o);
    if (lane >= o) t = ffl::add(t, ffl::ff{h, l});
  }
  // the sum of the chunks before this lane's
  const float h = __shfl_up_sync(0xffffffffu, t.hi, 1), l = __shfl_up_sync(0xffffffffu, t.lo, 1);
  ffl::ff run = lane == 0 ? ffl::ff{0.f, 0.f} : ffl::ff{h, l};
  for (int k = b; k < e; ++k) {
    run = ffl::add(run, ffl::ff{v[k].x, v[k].y});
    v[k] = make_float2(run.hi, run.lo);
  }
}

// The number of A-events among the first s events of the merge of A_0..A_{n-2} and B_0..B_{m-2}
// (ties to A): the largest i in [max(0, s - (m-1)), min(s, n-1)] with A_{i-1} <= B_{s-i}, a B index
// past m - 2 counting as +infinity (the predicate holds at the lower end and falls with i).
__device__ int merge_i(const float2* A, int n, const float2* B, int m, int s) {
  int lo = max(0, s - (m - 1)), hi = min(s, n - 1);
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    const bool ok = (s - mid >= m - 1) || !ff_lt(B[s - mid], A[mid - 1]);
    if (ok) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

__global__ void __launch_bounds__(32 * kFWWarps)
k_fw1d(const FWProb* __restrict__ probs, int count, int n_iter, double p, const float* __restrict__ x,
       const float* __restrict__ a, const float* __restrict__ y, const float* __restrict__ b, double* fb_all,
       double* gb_all, double* at_all, double* bt_all, double* r_all, double* s_all, double* __restrict__ f,
       double* __restrict__ g, int* __restrict__ status) {
  extern __shared__ double fw_smem[];
  const int lane = threadIdx.x & 31;
  const int k = blockIdx.x * kFWWarps + (threadIdx.x >> 5);
  if (k >= count) return;  // whole warp
  const FWProb P = probs[k];
  const int n = P.n, m = P.m;
  const float *X = x + P.xo, *A = a + P.xo, *Y = y + P.yo, *B = b + P.yo;
  double *FB = fb_all + P.xo, *AT = at_all + P.xo, *R = r_all + P.xo, *F = f + P.xo;
  double *GB = gb_all + P.yo, *BT = bt_all + P.yo, *S = s_all + P.yo, *G = g + P.yo;
  if (n + m <= kFWSmemPoints) {
    // the walk reads a~ and b~ right after the other lanes wrote them: keep them on chip
    AT = fw_smem + (threadIdx.x >> 5) * kFWSmemPoints;
    BT = AT + n;
  }

  // inputs: weights finite and >= 0 with positive totals, points finite and ascending
  bool bad_w = false, bad_x = false;
  double ta = 0.0, tb = 0.0;
  for (int i = lane; i < n; i += 32) {
    const float w = A[i], xi = X[i];
    if (!(w >= 0.f) || !isfinite(w)) bad_w = true; else ta += w;
    if (!isfinite(xi) || (i + 1 < n && !(xi <= X[i + 1]))) bad_x = true;
  }
  for (int j = lane; j < m; j += 32) {
    const float w = B[j], yj = Y[j];
    if (!(w >= 0.f) || !isfinite(w)) bad_w = true; else tb += w;
    if (!isfinite(yj) || (j + 1 < m && !(yj <= Y[j + 1]))) bad_x = true;
  }
  ta = warp_sum_d(ta);
  tb = warp_sum_d(tb);
  bad_w = __any_sync(0xffffffffu, bad_w) || !(ta > 0.0) || !(tb > 0.0);
  bad_x = __any_sync(0xffffffffu, bad_x);
  if (bad_w || bad_x) {
    for (int i = lane; i < n; i += 32) F[i] = __longlong_as_double(0x7ff8000000000000LL);
    for (int j = lane; j < m; j += 32) G[j] = __longlong_as_double(0x7ff8000000000000LL);
    if (lane == 0) status[k] = bad_w ? UOT_ERR_NONFINITE : UOT_ERR_INVALID_ARG;
    return;
  }

  // working vectors as float pairs (about 44 bits) in the double-sized slots of the workspace: FP64
  // runs at a small fraction of the FP32 rate on this GPU, and the exponentials of every step were
  // the kernel's FP64 bound
  float2 *FB2 = reinterpret_cast<float2*>(FB), *GB2 = reinterpret_cast<float2*>(GB);
  float2 *AT2 = reinterpret_cast<float2*>(AT), *BT2 = reinterpret_cast<float2*>(BT);
  for (int i = lane; i < n; i += 32) FB2[i] = make_float2(0.f, 0.f);
  for (int j = lane; j < m; j += 32) GB2[j] = make_float2(0.f, 0.f);
  __syncwarp();
  const double r1 = P.rho1, r2 = P.rho2;
  const ffl::ff ri1 = ffl::from_double(1.0 / r1), ri2 = ffl::from_double(1.0 / r2);
  const ffl::ff kappa = ffl::from_double(r1 * r2 / (r1 + r2));
  ffl::ff lam{0.f, 0.f};
  for (int t = 0;; ++t) {
    const ffl::ff la = log_dot_exp_neg(A, FB2, n, ri1, lane), lb = log_dot_exp_neg(B, GB2, m, ri2, lane);
    lam = ffl::mul(kappa, ffl::add(la, ffl::neg(lb)));
    if (t == n_iter) break;
    // a~ and b~ divided by their common mass m (Prop. 1): ln m = la - lambda / rho1.  The walk
    // depends on the masses only through comparisons of their partial sums, which the common
    // factor leaves unchanged; it keeps every a~_i, b~_j <= 1
    const ffl::ff lnm = ffl::add(la, ffl::neg(ffl::mul(lam, ri1)));
    for (int i = lane; i < n; i += 32) {
      ffl::ff v{0.f, 0.f};
      if (A[i] > 0.f) {
        const ffl::ff e = ffl::add(ffl::neg(ffl::mul(ffl::add(ffl::ff{FB2[i].x, FB2[i].y}, lam), ri1)), ffl::neg(lnm));
        v = w_exp_ff(A[i], e);
      }
      AT2[i] = make_float2(v.hi, v.lo);
    }
    for (int j = lane; j < m; j += 32) {
      ffl::ff v{0.f, 0.f};
      if (B[j] > 0.f) {
        const ffl::ff e =
            ffl::add(ffl::neg(ffl::mul(ffl::add(ffl::ff{GB2[j].x, GB2[j].y}, ffl::neg(lam)), ri2)), ffl::neg(lnm));
        v = w_exp_ff(B[j], e);
      }
      BT2[j] = make_float2(v.hi, v.lo);
    }
    __syncwarp();
    // SolveOT1D, the duals of the north-west corner coupling, on the whole warp.  With A_i, B_j
    // the partial sums of a~ and b~, the untransported masses at (i, j) differ by B_j - A_i, so
    // "point i is exhausted first" is A_i <= B_j: the walk's path is the merge of the sorted
    // sequences A_0..A_{N-2} and B_0..B_{M-2} (ties to A).  Each lane takes an equal share of
    // the N + M - 2 steps, finds its starting point by a binary search on that merge, and walks
    // it; a newly reached point's potential is the current pair's cost minus the other side's
    // potential, so a share maps its starting i-potential x to c + sigma x (sigma = +-1), and a
    // warp scan of those maps gives every share its starting value before the second walk,
    // which writes the potentials.  Branches are the oracle's except within ~1e-13 of a tie.
    prefix_sum_ff(AT2, n, lane);
    prefix_sum_ff(BT2, m, lane);
    __syncwarp();
    {
      const int pmode = p == 2.0 ? 2 : (p == 1.0 ? 1 : 0);
      const int steps = (n - 1) + (m - 1);
      const int s0 = (int)((long long)lane * steps / 32), s1 = (int)((long long)(lane + 1) * steps / 32);
      const int i0 = merge_i(AT2, n, BT2, m, s0), j0 = s0 - i0;
      // first walk: the share's map of its starting i-potential
      ffl::ff cR{0.f, 0.f}, cS = cost_ff(X[i0], Y[j0], pmode, p);
      float sgR = 1.f, sgS = -1.f;
      {
        int i = i0, j = j0;
        for (int st = s0; st < s1; ++st) {
          if (i < n - 1 && (j == m - 1 || !ff_lt(BT2[j], AT2[i]))) {
            ++i;
            cR = ffl::add(cost_ff(X[i], Y[j], pmode, p), ffl::neg(cS));
            sgR = -sgS;
          } else {
            ++j;
            cS = ffl::add(cost_ff(X[i], Y[j], pmode, p), ffl::neg(cR));
            sgS = -sgR;
          }
        }
      }
      // inclusive scan of the maps x -> c + sigma x, composed in walk order
      ffl::ff c = cR;
      float sg = sgR;
      for (int o = 1; o < 32; o <<= 1) {
        const float ch = __shfl_up_sync(0xffffffffu, c.hi, o), cl = __shfl_up_sync(0xffffffffu, c.lo, o);
        const float sp = __shfl_up_sync(0xffffffffu, sg, o);
        if (lane >= o) {
          c = ffl::add(c, ffl::ff{sg * ch, sg * cl});
          sg *= sp;
        }
      }
      // the share's starting i-potential: the composition over the lanes before it, applied to r_0 = 0
      float rh = __shfl_up_sync(0xffffffffu, c.hi, 1), rl = __shfl_up_sync(0xffffffffu, c.lo, 1);
      if (lane == 0) rh = rl = 0.f;
      // second walk: the potentials
      float2* R2 = reinterpret_cast<float2*>(R);
      float2* S2 = reinterpret_cast<float2*>(S);
      ffl::ff ri{rh, rl}, sj = ffl::add(cost_ff(X[i0], Y[j0], pmode, p), ffl::ff{-rh, -rl});
      if (lane == 0) {
        R2[0] = make_float2(0.f, 0.f);
        S2[0] = make_float2(sj.hi, sj.lo);
      }
      int i = i0, j = j0;
      for (int st = s0; st < s1; ++st) {
        if (i < n - 1 && (j == m - 1 || !ff_lt(BT2[j], AT2[i]))) {
          ++i;
          ri = ffl::add(cost_ff(X[i], Y[j], pmode, p), ffl::neg(sj));
          R2[i] = make_float2(ri.hi, ri.lo);
        } else {
          ++j;
          sj = ffl::add(cost_ff(X[i], Y[j], pmode, p), ffl::neg(ri));
          S2[j] = make_float2(sj.hi, sj.lo);
        }
      }
    }
    __syncwarp();
    // (fb, gb) <- (1 - gamma) (fb, gb) + gamma (r, s), gamma = 2 / (2 + t)
    const ffl::ff gm = ffl::from_double(2.0 / (2.0 + (double)t));
    const ffl::ff g1 = ffl::add(ffl::neg(gm), 1.f);
    const float2* R2 = reinterpret_cast<const float2*>(R);
    const float2* S2 = reinterpret_cast<const float2*>(S);
    for (int i = lane; i < n; i += 32) {
      const ffl::ff v = ffl::add(ffl::mul(ffl::ff{FB2[i].x, FB2[i].y}, g1), ffl::mul(ffl::ff{R2[i].x, R2[i].y}, gm));
      FB2[i] = make_float2(v.hi, v.lo);
    }
    for (int j = lane; j < m; j += 32) {
      const ffl::ff v = ffl::add(ffl::mul(ffl::ff{GB2[j].x, GB2[j].y}, g1), ffl::mul(ffl::ff{S2[j].x, S2[j].y}, gm));
      GB2[j] = make_float2(v.hi, v.lo);
    }
    __syncwarp();
  }
  const double ld = ffl::to_double(lam);
  for (int i = lane; i < n; i += 32) F[i] = ffl::to_double(ffl::ff{FB2[i].x, FB2[i].y}) + ld;
  for (int j = lane; j < m; j += 32) G[j] = ffl::to_double(ffl::ff{GB2[j].x, GB2[j].y}) - ld;
  if (lane == 0) status[k] = UOT_OK;
}

size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

struct FWLayout {
  size_t probs, status, fb, gb, at, bt, r, s, total;
  long long lx, ly;
};

uot_status fwfail(uot_status s, const char* msg) {
  set_last_error(msg);
  return s;
}

uot_status validate_fw(const uot_fw1d_batch* b, FWLayout* L) {
  if (!b) return fwfail(UOT_ERR_INVALID_ARG, "batch is NULL");
  if (b->count < 1) return fwfail(UOT_ERR_INVALID_ARG, "batch count must be >= 1");
  if (b->n_iter < 1) return fwfail(UOT_ERR_INVALID_ARG, "n_iter must be >= 1");
  if (!(b->p >= 1.0) || !isfinite(b->p)) return fwfail(UOT_ERR_INVALID_ARG, "p must be finite and >= 1");
  if (!b->n || !b->m || !b->x_off || !b->y_off || !b->rho1 || !b->rho2)
    return fwfail(UOT_ERR_INVALID_ARG, "batch host arrays must not be NULL");
  if (!b->x || !b->a || !b->y || !b->b) return fwfail(UOT_ERR_INVALID_ARG, "batch device arrays must not be NULL");
  long long lx = 0, ly = 0;
  for (int k = 0; k < b->count; ++k) {
    if (b->n[k] < 1 || b->m[k] < 1) return fwfail(UOT_ERR_INVALID_ARG, "every problem needs n, m >= 1");
    if (!(b->rho1[k] > 0) || !(b->rho2[k] > 0) || !isfinite(b->rho1[k]) || !isfinite(b->rho2[k]))
      return fwfail(UOT_ERR_INVALID_ARG, "every problem needs finite rho1, rho2 > 0");
    if (b->x_off[k] < 0 || b->y_off[k] < 0) return fwfail(UOT_ERR_INVALID_ARG, "offsets must be >= 0");
    lx = std::max(lx, (long long)(b->x_off[k] + b->n[k]));
    ly = std::max(ly, (long long)(b->y_off[k] + b->m[k]));
  }
  size_t off = 0;
  auto take = [&](size_t bytes) { size_t o = off; off = align256(off + bytes); return o; };
  L->probs = take(sizeof(FWProb) * b->count);
  L->status = take(sizeof(int) * b->count);
  L->fb = take(sizeof(double) * lx);
  L->at = take(sizeof(double) * lx);
  L->r = take(sizeof(double) * lx);
  L->gb = take(sizeof(double) * ly);
  L->bt = take(sizeof(double) * ly);
  L->s = take(sizeof(double) * ly);
  L->total = off;
  L->lx = lx;
  L->ly = ly;
  return UOT_OK;
}

#define FWCUDA(call)                                                   \
  do {                                                                 \
    cudaError_t e_ = (call);                                           \
    if (e_ != cudaSuccess) {                                           \
      std::string m_ = std::string(#call) + ": " + cudaGetErrorString(e_); \
      return fwfail(UOT_ERR_CUDA, m_.c_str());                         \
    }                                                                  \
  } while (0)

}  // namespace
}  // namespace uot

using namespace uot;

extern "C" {

size_t uot_fw1d_workspace_size(const uot_fw1d_batch* batch) {
  FWLayout L;
  if (validate_fw(batch, &L) != UOT_OK) return 0;
  return L.total;
}

uot_status uot_fw1d_batched(const uot_fw1d_batch* b, double* f, double* g, int32_t* status, void* ws,
                            size_t ws_bytes, void* stream) {
  FWLayout L;
  uot_status v = validate_fw(b, &L);
  if (v != UOT_OK) return v;
  if (!f || !g) return fwfail(UOT_ERR_INVALID_ARG, "f and g must not be NULL");
  if (!ws) return fwfail(UOT_ERR_WORKSPACE, "workspace is NULL");
  if (reinterpret_cast<uintptr_t>(ws) & 255) return fwfail(UOT_ERR_WORKSPACE, "workspace must be 256-byte aligned");
  if (ws_bytes < L.total) return fwfail(UOT_ERR_WORKSPACE, "workspace too small for the batch");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  char* base = static_cast<char*>(ws);
  const int count = b->count;
  std::vector<FWProb> probs(count);
  for (int k = 0; k < count; ++k)
    probs[k] = FWProb{b->x_off[k], b->y_off[k], b->n[k], b->m[k], b->rho1[k], b->rho2[k]};
  FWProb* d_probs = reinterpret_cast<FWProb*>(base + L.probs);
  int* d_status = reinterpret_cast<int*>(base + L.status);
  FWCUDA(cudaMemcpyAsync(d_probs, probs.data(), sizeof(FWProb) * count, cudaMemcpyHostToDevice, st));
  const int blocks = (count + kFWWarps - 1) / kFWWarps;
  k_fw1d<<<blocks, 32 * kFWWarps, sizeof(double) * kFWWarps * kFWSmemPoints, st>>>(
      d_probs, count, b->n_iter, b->p, b->x, b->a, b->y, b->b, reinterpret_cast<double*>(base + L.fb),
      reinterpret_cast<double*>(base + L.gb), reinterpret_cast<double*>(base + L.at),
      reinterpret_cast<double*>(base + L.bt), reinterpret_cast<double*>(base + L.r),
      reinterpret_cast<double*>(base + L.s), f, g, d_status);
  note_launch();
  FWCUDA(cudaGetLastError());
  std::vector<int> hs(count);
  FWCUDA(cudaMemcpyAsync(hs.data(), d_status, sizeof(int) * count, cudaMemcpyDeviceToHost, st));
  FWCUDA(cudaStreamSynchronize(st));
  uot_status out = UOT_OK;
  for (int k = 0; k < count; ++k) {
    if (status) status[k] = hs[k];
    if (out == UOT_OK && hs[k] != UOT_OK) out = static_cast<uot_status>(hs[k]);
  }
  if (out != UOT_OK) set_last_error("some problems have invalid points or weights (see status)");
  return out;
}

}  // extern "C"
