// O(N + M) kernels of the unrolled backward pass through T H-Sinkhorn
// iterations (reverse mode of the updates of Sec. 3 / App. B, proof of Prop. 4):
//
//   g half-step   S'_j = Smin_a^eps(C_.j - fb),  g_hat = a2 S' - b2 A(fb),  gb = g_hat + kg Bhat(g_hat)
//   f half-step   S_i  = Smin_b^eps(C_i. - gb),  f_hat = a1 S  - b1 B(gb),  fb = f_hat + kf Ahat(f_hat)
//   output        lambda = tau1 B(gb_T) - tau2 A(fb_T),  L = F_eps(fb_T + lambda, gb_T - lambda)
//
// with A = Smin_a^rho1, B = Smin_b^rho2, a1 = rho1/(rho1+eps), b1 = eps/(eps+rho1) rho1/(rho1+rho2),
// a2, b2 likewise, kf = k_f/(1-k_f), kg = k_g/(1-k_g).  The derivative of Smin_w^rho(u) is the
// softmax p_i = w_i exp((Smin - u_i)/rho) (and -rho exp((Smin - u_i)/rho) with respect to w_i); the
// O(NM) parts are the adjoint sweeps (adjoint.cu).  Each kernel below is one elementwise step
// of that chain; the reductions it needs (sums of cotangents) are FP64 and finished by the last
// block, whose result the next kernel reads.
#include <cuda_runtime.h>
#include <math.h>

#include "sweep_common.cuh"
#include "uot_internal.cuh"

namespace uot {
namespace {

constexpr int kBlk = 256;

__device__ __forceinline__ bool last_block_done(unsigned int* counter) {
  __shared__ bool am_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) am_last = (atomicAdd(counter, 1u) == gridDim.x - 1);
  __syncthreads();
  if (am_last) __threadfence();
  return am_last;
}

// Block sum of v, then grid sum into *out by the last block.
__device__ void grid_sum(double v, double* blk, unsigned int* counter, double* out) {
  __shared__ double sh[kBlk];
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int off = blockDim.x / 2; off > 0; off >>= 1) {
    if (threadIdx.x < off) sh[threadIdx.x] += sh[threadIdx.x + off];
    __syncthreads();
  }
  if (threadIdx.x == 0) blk[blockIdx.x] = sh[0];
  if (!last_block_done(counter)) return;
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int k = 0; k < (int)gridDim.x; ++k) t += __ldcg(blk + k);
    *out = t;
    *counter = 0;
  }
}

int grid_for(int n) {
  int g = (n + kBlk - 1) / kBlk;
  return g < 1 ? 1 : (g > 1024 ? 1024 : g);
}

// p_i = w_i e^{(X - u_i)/rho} and d Smin / d w_i = -rho e^{(X - u_i)/rho}
__device__ __forceinline__ double soft_p(double lnw, double X, double u, double rho) {
  return lnw == -INFINITY ? 0.0 : exp(lnw + (X - u) / rho);
}

// out_i = base_i + add_i (FP32 vectors + scalar): v_i = u_i + c
__global__ void k_add_scalar(const float* u, const double* c, int n, float* v) {
  const double cc = *c;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    v[i] = (float)((double)u[i] + cc);
}

// Normalised gradient moments G_q = sum_k w_qk dC/dq / sum_k w_qk from sweep partials with moments:
// one thread per (row, coordinate) (rows fastest: coalesced partial loads); the chunk weights
// 2^(M_k - M) in FP32 (relative error ~1e-7), the sums in FP64.
__global__ void k_moments(const float* part, int nq, int dim, int splits, double scale, float* G) {
  const int CH = 2 + dim;
  const int d = blockIdx.y;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nq; i += gridDim.x * blockDim.x) {
    float M = kInitMax;
    for (int k = 0; k < splits; ++k) M = fmaxf(M, __ldg(part + (size_t)k * CH * nq + i));
    double sum = 0.0, mo = 0.0;
    for (int k = 0; k < splits; ++k) {
      const float* b = part + (size_t)k * CH * nq;
      const double w = (double)simd::ex2f(__ldg(b + i) - M);
      sum += (double)__ldg(b + (size_t)nq + i) * w;
      mo += (double)__ldg(b + (size_t)(2 + d) * nq + i) * w;
    }
    G[(size_t)i * dim + d] = (float)(scale * mo / sum);
  }
}

// Final stage, one side: dL/dpot_i = w_i e^{-pot_i/rho} - w_i e^{(pot_i - S_i)/eps} from the plain
// sweep partials at the output pair; sum of it into *sum.
__global__ void k_final_side(const float* part, int CH, int nq, int splits, double s, double eps, double rho,
                             const float* pot, const double* lnw, float* cot, double* blk, unsigned int* ctr,
                             double* sum) {
  double acc = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nq; i += gridDim.x * blockDim.x) {
    float M = kInitMax;
    for (int k = 0; k < splits; ++k) M = fmaxf(M, part[(size_t)k * CH * nq + i]);
    double S = 0.0;
    for (int k = 0; k < splits; ++k) {
      const float* b = part + (size_t)k * CH * nq;
      S += (double)b[(size_t)nq + i] * exp2((double)b[i] - (double)M);
    }
    const double Smin = -((double)M + log2(S)) / s;
    const double u = pot[i], lw = lnw[i];
    const double v = (lw == -INFINITY) ? 0.0 : exp(lw - u / rho) - exp(lw + (u - Smin) / eps);
    cot[i] = (float)v;
    acc += v;
  }
  grid_sum(acc, blk, ctr, sum);
}

// Final stage, Smin terms of lambda: cot_i += Xbar p_i(u), gw_i += Xbar (-rho) e^{(X-u_i)/rho},
// with Xbar = coef * (sum_f - sum_g); optional grid sum of the updated cot into *sum.
__global__ void k_final_lambda(int n, const float* u, const double* lnw, const double* X, double rho, double coef,
                               const double* sum_f, const double* sum_g, float* cot, float* gw, double* blk,
                               unsigned int* ctr, double* sum) {
  const double Xbar = coef * (*sum_f - *sum_g);
  const double Xv = *X;
  double acc = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const double e = exp((Xv - (double)u[i]) / rho);
    const double c = (double)cot[i] + Xbar * soft_p(lnw[i], Xv, u[i], rho);
    cot[i] = (float)c;
    gw[i] = (float)((double)gw[i] - Xbar * rho * e);
    acc += c;
  }
  if (sum) grid_sum(acc, blk, ctr, sum);
}

// f-step backward, first part (over i): f_hat_bar = fbb + Ahat_bar p(f_hat), Ahat_bar = kf * sum(fbb);
// ga += Ahat_bar (-rho1) e^{(Ahat - f_hat)/rho1}; Sb = a1 f_hat_bar; gx += Sb * G; sum(f_hat_bar) -> *sum_out.
__global__ void k_bw_f1(int n, int dim, const float* fbb, const float* fhat, const double* lna, const double* Ahat,
                        const double* sum_fbb, double kf, double rho1, double a1, const float* G, float* ga,
                        float* gx, float* Sb, double* blk, unsigned int* ctr, double* sum_out) {
  const double Abar = kf * (*sum_fbb), A = *Ahat;
  double acc = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const double fh = fhat[i];
    const double fhb = (double)fbb[i] + Abar * soft_p(lna[i], A, fh, rho1);
    ga[i] = (float)((double)ga[i] - Abar * rho1 * exp((A - fh) / rho1));
    const double sb = a1 * fhb;
    Sb[i] = (float)sb;
    for (int d = 0; d < dim; ++d) gx[(size_t)i * dim + d] += (float)(sb * (double)G[(size_t)i * dim + d]);
    acc += fhb;
  }
  grid_sum(acc, blk, ctr, sum_out);
}

// g-side init from the B(gb) term of f_hat: gbb += Bbar p(gb), Bbar = coef * sum_in; gb_w += Bbar (-rho2) e^{...}.
__global__ void k_bw_smin_init(int n, const float* u, const double* lnw, const double* X, double rho, double coef,
                               const double* sum_in, float* cot, float* gw) {
  const double Xbar = coef * (*sum_in), Xv = *X;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const double e = exp((Xv - (double)u[i]) / rho);
    cot[i] = (float)((double)cot[i] + Xbar * soft_p(lnw[i], Xv, u[i], rho));
    gw[i] = (float)((double)gw[i] - Xbar * rho * e);
  }
}

// After an adjoint sweep on side q: cot_i -= w_i val_i (d Smin / d pot = -P), gw_i += -eps val_i
// (d Smin / d w), gpts_i += 2 w_i mom_i (d Smin / d C = +P); optional grid sum of cot into *sum.
__global__ void k_bw_adj(int n, int dim, const double* val, const double* mom, const double* lnw, double eps,
                         float* cot, float* gw, float* gpts, double* blk, unsigned int* ctr, double* sum) {
  double acc = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const double w = lnw[i] == -INFINITY ? 0.0 : exp(lnw[i]);
    const double c = (double)cot[i] - w * val[i];
    cot[i] = (float)c;
    gw[i] = (float)((double)gw[i] - eps * val[i]);
    for (int d = 0; d < dim; ++d) gpts[(size_t)i * dim + d] += (float)(2.0 * w * mom[(size_t)i * dim + d]);
    acc += c;
  }
  if (sum) grid_sum(acc, blk, ctr, sum);
}

// g-step backward (over j): g_hat_bar = gbb + Bhat_bar p(g_hat), Bhat_bar = kg * sum(gbb);
// gb += Bhat_bar (-rho2) e^{(Bhat - g_hat)/rho2}; Spb = a2 g_hat_bar; gy += Spb * Gp; gbb <- 0;
// sum(g_hat_bar) -> *sum_out.
__global__ void k_bw_g1(int m, int dim, float* gbb, const float* ghat, const double* lnb, const double* Bhat,
                        const double* sum_gbb, double kg, double rho2, double a2, const float* Gp, float* gb,
                        float* gy, float* Spb, double* blk, unsigned int* ctr, double* sum_out) {
  const double Bbar = kg * (*sum_gbb), B = *Bhat;
  double acc = 0.0;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < m; j += gridDim.x * blockDim.x) {
    const double gh = ghat[j];
    const double ghb = (double)gbb[j] + Bbar * soft_p(lnb[j], B, gh, rho2);
    gb[j] = (float)((double)gb[j] - Bbar * rho2 * exp((B - gh) / rho2));
    const double spb = a2 * ghb;
    Spb[j] = (float)spb;
    for (int d = 0; d < dim; ++d) gy[(size_t)j * dim + d] += (float)(spb * (double)Gp[(size_t)j * dim + d]);
    gbb[j] = 0.f;
    acc += ghb;
  }
  grid_sum(acc, blk, ctr, sum_out);
}

// f-side init from the A(fb_t) term of g_hat: fbb = Abar p(fb_t), Abar = coef * sum_in; ga += Abar (-rho1) e^{...}.
__global__ void k_bw_fset(int n, const float* fb, const double* lna, const double* A, double rho1, double coef,
                          const double* sum_in, float* fbb, float* ga) {
  const double Abar = coef * (*sum_in), Av = *A;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    fbb[i] = (float)(Abar * soft_p(lna[i], Av, fb[i], rho1));
    ga[i] = (float)((double)ga[i] - Abar * rho1 * exp((Av - (double)fb[i]) / rho1));
  }
}

// copies of the slot scalars of one iteration into the per-iteration record
__global__ void k_record_scalars(const DevState* st, int slot_t, int slot_t1, double* rec) {
  const Slot& a = st->slot[slot_t];
  const Slot& b = st->slot[slot_t1];
  rec[0] = a.A;           // A_t     = Smin_a^rho1(fb_t)
  rec[1] = b.B - b.cg;    // Bhat    = Smin_b^rho2(g_hat_{t+1})
  rec[2] = b.B;           // B_{t+1} = Smin_b^rho2(gb_{t+1})
  rec[3] = b.A - b.cf;    // Ahat    = Smin_a^rho1(f_hat_{t+1})
  rec[4] = b.cg;
  rec[5] = b.cf;
  rec[6] = a.cf;
  rec[7] = b.A;           // A_{t+1}
}

}  // namespace

#define UOT_LAUNCH(kernel, n, ...)                                   \
  do {                                                               \
    kernel<<<grid_for(n), kBlk, 0, st>>>(__VA_ARGS__);               \
    note_launch();                                                   \
    cudaError_t e_ = cudaGetLastError();                             \
    if (e_ != cudaSuccess) return e_;                                \
  } while (0)

cudaError_t launch_add_scalar(const float* u, const double* c, int n, float* v, cudaStream_t st) {
  UOT_LAUNCH(k_add_scalar, n, u, c, n, v);
  return cudaSuccess;
}
cudaError_t launch_moments(const float* part, int nq, int dim, int splits, double scale, float* G, cudaStream_t st) {
  k_moments<<<dim3((nq + kBlk - 1) / kBlk, dim), kBlk, 0, st>>>(part, nq, dim, splits, scale, G);
  note_launch();
  return cudaGetLastError();
}
cudaError_t launch_final_side(const float* part, int CH, int nq, int splits, double s, double eps, double rho,
                              const float* pot, const double* lnw, float* cot, double* blk, unsigned int* ctr,
                              double* sum, cudaStream_t st) {
  UOT_LAUNCH(k_final_side, nq, part, CH, nq, splits, s, eps, rho, pot, lnw, cot, blk, ctr, sum);
  return cudaSuccess;
}
cudaError_t launch_final_lambda(int n, const float* u, const double* lnw, const double* X, double rho, double coef,
                                const double* sum_f, const double* sum_g, float* cot, float* gw, double* blk,
                                unsigned int* ctr, double* sum, cudaStream_t st) {
  UOT_LAUNCH(k_final_lambda, n, n, u, lnw, X, rho, coef, sum_f, sum_g, cot, gw, blk, ctr, sum);
  return cudaSuccess;
}
cudaError_t launch_bw_f1(int n, int dim, const float* fbb, const float* fhat, const double* lna, const double* Ahat,
                         const double* sum_fbb, double kf, double rho1, double a1, const float* G, float* ga,
                         float* gx, float* Sb, double* blk, unsigned int* ctr, double* sum_out, cudaStream_t st) {
  UOT_LAUNCH(k_bw_f1, n, n, dim, fbb, fhat, lna, Ahat, sum_fbb, kf, rho1, a1, G, ga, gx, Sb, blk, ctr, sum_out);
  return cudaSuccess;
}
cudaError_t launch_bw_smin_init(int n, const float* u, const double* lnw, const double* X, double rho, double coef,
                                const double* sum_in, float* cot, float* gw, cudaStream_t st) {
  UOT_LAUNCH(k_bw_smin_init, n, n, u, lnw, X, rho, coef, sum_in, cot, gw);
  return cudaSuccess;
}
cudaError_t launch_bw_adj(int n, int dim, const double* val, const double* mom, const double* lnw, double eps,
                          float* cot, float* gw, float* gpts, double* blk, unsigned int* ctr, double* sum,
                          cudaStream_t st) {
  UOT_LAUNCH(k_bw_adj, n, n, dim, val, mom, lnw, eps, cot, gw, gpts, blk, ctr, sum);
  return cudaSuccess;
}
cudaError_t launch_bw_g1(int m, int dim, float* gbb, const float* ghat, const double* lnb, const double* Bhat,
                         const double* sum_gbb, double kg, double rho2, double a2, const float* Gp, float* gb,
                         float* gy, float* Spb, double* blk, unsigned int* ctr, double* sum_out, cudaStream_t st) {
  UOT_LAUNCH(k_bw_g1, m, m, dim, gbb, ghat, lnb, Bhat, sum_gbb, kg, rho2, a2, Gp, gb, gy, Spb, blk, ctr, sum_out);
  return cudaSuccess;
}
cudaError_t launch_bw_fset(int n, const float* fb, const double* lna, const double* A, double rho1, double coef,
                           const double* sum_in, float* fbb, float* ga, cudaStream_t st) {
  UOT_LAUNCH(k_bw_fset, n, n, fb, lna, A, rho1, coef, sum_in, fbb, ga);
  return cudaSuccess;
}
cudaError_t launch_record_scalars(const DevState* s, int slot_t, int slot_t1, double* rec, cudaStream_t st) {
  k_record_scalars<<<1, 1, 0, st>>>(s, slot_t, slot_t1, rec);
  note_launch();
  return cudaGetLastError();
}

}  // namespace uot
