// 1-D unregularised UOT by Frank-Wolfe on H_0 (Sec. 4, Alg. 2), batched: one
// warp per problem; FP64 except the walk's potentials (float pairs).  Per step
// the warp computes
//   lambda* = rho1 rho2 / (rho1 + rho2) (log<a, e^{-fb/rho1}> - log<b, e^{-gb/rho2}>)   (Prop. 2)
//   a~ = a e^{-(fb + lambda*)/rho1},  b~ = b e^{-(gb - lambda*)/rho2}              (Eq. fw-updated-histo)
// with all lanes, then lane 0 walks the two sorted point lists once to get the
// duals (r, s) of the balanced 1-D OT between a~ and b~ (SolveOT1D, Alg. 1:
// the point whose remaining mass is smaller is exhausted first, and each newly
// reached point's potential is the current pair's cost minus the other side's
// current potential), and all lanes take the step
//   (fb, gb) <- (1 - gamma_t)(fb, gb) + gamma_t (r, s),  gamma_t = 2 / (2 + t).
// The walk is sequential by nature (O(N + M) dependent steps, one FP64 add
// each); the batch supplies the parallelism.  Working vectors live in the
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
__device__ __forceinline__ double warp_max_d(double v) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// log <w, e^{-v / rho}> over the entries with w > 0 (largest exponent taken out first)
__device__ double log_dot_exp_neg(const float* __restrict__ w, const double* v, int n, double rho, int lane) {
  double mx = -INFINITY;
  for (int i = lane; i < n; i += 32)
    if (w[i] > 0.f) mx = fmax(mx, -v[i] / rho);
  mx = warp_max_d(mx);
  double sm = 0.0;
  for (int i = lane; i < n; i += 32)
    if (w[i] > 0.f) sm += (double)w[i] * exp(-v[i] / rho - mx);
  sm = warp_sum_d(sm);
  return mx + log(sm);
}

// |x - y|^p as a float pair: x - y exactly (two_sum), then its square (p = 2),
// its magnitude (p = 1), or an FP64 power for other p
__device__ __forceinline__ ffl::ff cost_ff(float xi, float yj, double p) {
  const ffl::ff d = ffl::two_sum(xi, -yj);
  if (p == 2.0) return ffl::mul(d, d);
  if (p == 1.0) return d.hi < 0.f ? ffl::neg(d) : d;
  return ffl::from_double(pow(fabs((double)d.hi + (double)d.lo), p));
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

  for (int i = lane; i < n; i += 32) FB[i] = 0.0;
  for (int j = lane; j < m; j += 32) GB[j] = 0.0;
  __syncwarp();
  const double r1 = P.rho1, r2 = P.rho2, kappa = r1 * r2 / (r1 + r2);
  double lam = 0.0;
  for (int t = 0;; ++t) {
    lam = kappa * (log_dot_exp_neg(A, FB, n, r1, lane) - log_dot_exp_neg(B, GB, m, r2, lane));
    if (t == n_iter) break;
    for (int i = lane; i < n; i += 32) AT[i] = A[i] > 0.f ? (double)A[i] * exp(-(FB[i] + lam) / r1) : 0.0;
    for (int j = lane; j < m; j += 32) BT[j] = B[j] > 0.f ? (double)B[j] * exp(-(GB[j] - lam) / r2) : 0.0;
    __syncwarp();
    if (lane == 0) {
      // SolveOT1D, the duals of the north-west corner coupling.  The masses not yet
      // transported enter only through dm = fl(m_j - m_i): "point i is exhausted first"
      // is m_i <= m_j, i.e. dm >= 0, and the next dm is fl(dm - a~_{i+1}) after i moves,
      // fl(dm + b~_{j+1}) after j moves, the same roundings as tracking (m_i, m_j) in FP64,
      // so the walk takes the same branches with one dependent FP64 add a step.  The
      // potentials run in float pairs on the FP32 pipes; the next point and mass of both
      // sides are loaded ahead of each decision.
      float2* R2 = reinterpret_cast<float2*>(R);
      float2* S2 = reinterpret_cast<float2*>(S);
      int i = 0, j = 0;
      float xi = X[0], yj = Y[0];
      ffl::ff ri{0.f, 0.f}, sj = cost_ff(xi, yj, p);
      R2[0] = make_float2(0.f, 0.f);
      S2[0] = make_float2(sj.hi, sj.lo);
      double dm = BT[0] - AT[0];
      double na = n > 1 ? AT[1] : 0.0, nb = m > 1 ? BT[1] : 0.0;
      float nx = n > 1 ? X[1] : 0.f, ny = m > 1 ? Y[1] : 0.f;
      while (i < n - 1 || j < m - 1) {
        // dm is never -0 (masses are >= +0), so its sign bit decides dm >= 0 without an FP64 compare
        if ((__double_as_longlong(dm) >= 0 && i < n - 1) || j == m - 1) {
          ++i;
          dm -= na;
          xi = nx;
          if (i + 1 < n) { na = AT[i + 1]; nx = X[i + 1]; }
          ri = ffl::add(cost_ff(xi, yj, p), ffl::neg(sj));
          R2[i] = make_float2(ri.hi, ri.lo);
        } else {
          ++j;
          dm += nb;
          yj = ny;
          if (j + 1 < m) { nb = BT[j + 1]; ny = Y[j + 1]; }
          sj = ffl::add(cost_ff(xi, yj, p), ffl::neg(ri));
          S2[j] = make_float2(sj.hi, sj.lo);
        }
      }
    }
    __syncwarp();
    const double gm = 2.0 / (2.0 + (double)t);
    const float2* R2 = reinterpret_cast<const float2*>(R);
    const float2* S2 = reinterpret_cast<const float2*>(S);
    for (int i = lane; i < n; i += 32) FB[i] = (1.0 - gm) * FB[i] + gm * ((double)R2[i].x + (double)R2[i].y);
    for (int j = lane; j < m; j += 32) GB[j] = (1.0 - gm) * GB[j] + gm * ((double)S2[j].x + (double)S2[j].y);
    __syncwarp();
  }
  for (int i = lane; i < n; i += 32) F[i] = FB[i] + lam;
  for (int j = lane; j < m; j += 32) G[j] = GB[j] - lam;
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
