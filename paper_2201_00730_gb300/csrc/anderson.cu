// Anderson extrapolation of the Sinkhorn iterates (appendix, "Combining
// Sinkhorn with Anderson acceleration"): from the last K + 1 iterates
// x_0..x_K of a block (a ring of K + 1 device vectors), the residuals
// u_k = x_{k+1} - x_k, the Gram matrix G = U^T U in FP64, its trace-relative
// regularisation G / trace(G) + r I, the weights c = (..)^{-1} 1 / 1^T (..)^{-1} 1
// (one thread, Gaussian elimination with partial pivoting) and the new iterate
// sum_{k<K} c_k x_k.
#include <cuda_runtime.h>
#include <math.h>

#include "uot_internal.cuh"

namespace uot {
namespace {

constexpr int kT = 256;
constexpr int kMaxK = 6;
constexpr int kAndBlocks = 608;
constexpr int kMaxNE = kMaxK * (kMaxK + 1) / 2;

struct AndLayout {
  size_t hist, lam, c, blk, counter, total;
  size_t stride;  // floats between ring entries
};

AndLayout and_layout(int n, int K) {
  AndLayout L{};
  auto up = [](size_t v) { return (v + 255) / 256 * 256; };
  L.stride = ((size_t)n + 63) / 64 * 64;
  L.hist = 0;
  L.lam = up(L.hist + sizeof(float) * L.stride * (K + 1));
  L.c = up(L.lam + sizeof(double) * (K + 1));
  L.blk = up(L.c + sizeof(double) * K);
  L.counter = up(L.blk + sizeof(double) * kAndBlocks * kMaxNE);
  L.total = up(L.counter + sizeof(unsigned int));
  return L;
}

int blocks_for(int n) {
  const int b = (n + kT - 1) / kT;
  return b < 1 ? 1 : (b > kAndBlocks ? kAndBlocks : b);
}

__global__ void k_and_store(const float* __restrict__ f, int n, int mode, const Slot* slot, float* __restrict__ dst,
                            double* lam_dst) {
  float hi = 0.f, lo = 0.f;
  if (mode == 1) { hi = slot->cff[0]; lo = slot->cff[1]; }
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    dst[i] = (mode == 1) ? (f[i] + hi) + lo : f[i];
  if (blockIdx.x == 0 && threadIdx.x == 0) *lam_dst = (mode == 2) ? slot->lam : 0.0;
}

__device__ __forceinline__ double warp_sum(double v) {
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  return v;
}

// Gram matrix of the residuals (upper triangle, row by row), block partials,
// the last block solves for the weights.
template <int K>
__global__ void __launch_bounds__(kT) k_and_gram(const float* __restrict__ hist, size_t stride, int n, int p0,
                                                 double r, double* blk, unsigned int* counter, double* c_out,
                                                 int* status) {
  constexpr int NE = K * (K + 1) / 2;
  double acc[NE];
#pragma unroll
  for (int e = 0; e < NE; ++e) acc[e] = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    double x[K + 1];
#pragma unroll
    for (int k = 0; k <= K; ++k) x[k] = (double)hist[(size_t)((p0 + k) % (K + 1)) * stride + i];
    double u[K];
#pragma unroll
    for (int k = 0; k < K; ++k) u[k] = x[k + 1] - x[k];
    int e = 0;
#pragma unroll
    for (int a = 0; a < K; ++a)
#pragma unroll
      for (int b = a; b < K; ++b) acc[e++] += u[a] * u[b];
  }
  __shared__ double red[NE][kT / 32];
  __shared__ bool last;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int e = 0; e < NE; ++e) {
    const double v = warp_sum(acc[e]);
    if (lane == 0) red[e][warp] = v;
  }
  __syncthreads();
  if (threadIdx.x < NE) {
    double v = 0.0;
    for (int w = 0; w < kT / 32; ++w) v += red[threadIdx.x][w];
    blk[(size_t)blockIdx.x * NE + threadIdx.x] = v;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    last = atomicAdd(counter, 1u) == gridDim.x - 1;
    if (last) __threadfence();
  }
  __syncthreads();
  if (!last || threadIdx.x != 0) return;
  // the blocks' partials in a fixed order
  double G[K][K];
  {
    double g[NE];
    for (int e = 0; e < NE; ++e) g[e] = 0.0;
    for (int b = 0; b < (int)gridDim.x; ++b)
      for (int e = 0; e < NE; ++e) g[e] += __ldcg(blk + (size_t)b * NE + e);
    int e = 0;
    for (int a = 0; a < K; ++a)
      for (int b = a; b < K; ++b) { G[a][b] = g[e]; G[b][a] = g[e]; ++e; }
  }
  double tr = 0.0;
  for (int a = 0; a < K; ++a) tr += G[a][a];
  const double sc = tr > 0.0 ? 1.0 / tr : 1.0;
  double M[K][K + 1];
  for (int a = 0; a < K; ++a) {
    for (int b = 0; b < K; ++b) M[a][b] = G[a][b] * sc + (a == b ? r : 0.0);
    M[a][K] = 1.0;
  }
  bool ok = true;
  for (int col = 0; col < K; ++col) {
    int piv = col;
    for (int a = col + 1; a < K; ++a)
      if (fabs(M[a][col]) > fabs(M[piv][col])) piv = a;
    if (!(fabs(M[piv][col]) > 0.0)) { ok = false; break; }
    if (piv != col)
      for (int b = 0; b <= K; ++b) { const double tmp = M[col][b]; M[col][b] = M[piv][b]; M[piv][b] = tmp; }
    for (int a = col + 1; a < K; ++a) {
      const double fct = M[a][col] / M[col][col];
      for (int b = col; b <= K; ++b) M[a][b] -= fct * M[col][b];
    }
  }
  double z[K], zs = 0.0;
  if (ok) {
    for (int a = K - 1; a >= 0; --a) {
      double v = M[a][K];
      for (int b = a + 1; b < K; ++b) v -= M[a][b] * z[b];
      z[a] = v / M[a][a];
      zs += z[a];
    }
    ok = isfinite(zs) && zs != 0.0;
  }
  for (int a = 0; a < K; ++a) {
    const double ca = ok ? z[a] / zs : (a == K - 1 ? 1.0 : 0.0);  // failure: keep the last iterate
    c_out[a] = ca;
    if (!isfinite(ca)) ok = false;
  }
  if (!ok) atomicOr(status, kStatusNonfinite);
  *counter = 0;
}

template <int K>
__global__ void k_and_combine(float* __restrict__ f, const float* hist_ro, float* hist, size_t stride,
                              int n, int p0, const double* __restrict__ c) {
  double cc[K];
#pragma unroll
  for (int k = 0; k < K; ++k) cc[k] = c[k];
  const int pn = (p0 + K) % (K + 1);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    double v = 0.0;
#pragma unroll
    for (int k = 0; k < K; ++k) v = fma(cc[k], (double)hist_ro[(size_t)((p0 + k) % (K + 1)) * stride + i], v);
    const float fv = (float)v;
    f[i] = fv;
    hist[(size_t)pn * stride + i] = fv;
  }
}

// G-Sinkhorn: lambda takes the same combination; it is the next g half-step's key shift
template <int K>
__global__ void k_and_lambda(double* lam, int p0, const double* __restrict__ c, Slot* slot) {
  double v = 0.0;
  for (int k = 0; k < K; ++k) v += c[k] * lam[(p0 + k) % (K + 1)];
  lam[(p0 + K) % (K + 1)] = v;
  const float hi = (float)v, lo = (float)(v - (double)hi);
  slot->cf = v;
  slot->lam = v;
  slot->cff[0] = hi; slot->cff[1] = lo;
  slot->lamf[0] = hi; slot->lamf[1] = lo;
}

template <int K>
cudaError_t extrapolate(float* f, int n, int p0, double r, void* buf, Slot* slot_g, int* status, cudaStream_t st) {
  const AndLayout L = and_layout(n, K);
  char* b = static_cast<char*>(buf);
  float* hist = reinterpret_cast<float*>(b + L.hist);
  double* lam = reinterpret_cast<double*>(b + L.lam);
  double* c = reinterpret_cast<double*>(b + L.c);
  const int nb = blocks_for(n);
  k_and_gram<K><<<nb, kT, 0, st>>>(hist, L.stride, n, p0, r, reinterpret_cast<double*>(b + L.blk),
                                   reinterpret_cast<unsigned int*>(b + L.counter), c, status);
  note_launch();
  k_and_combine<K><<<nb, kT, 0, st>>>(f, hist, hist, L.stride, n, p0, c);
  note_launch();
  if (slot_g) {
    k_and_lambda<K><<<1, 1, 0, st>>>(lam, p0, c, slot_g);
    note_launch();
  }
  return cudaGetLastError();
}

}  // namespace

size_t anderson_bytes(int n, int K) { return and_layout(n, K).total; }

cudaError_t anderson_reset(void* buf, int n, int K, cudaStream_t st) {
  const AndLayout L = and_layout(n, K);
  return cudaMemsetAsync(static_cast<char*>(buf) + L.counter, 0, sizeof(unsigned int), st);
}

cudaError_t launch_anderson_store(const float* f, int n, int K, int pos, int mode, const Slot* slot, void* buf,
                                  cudaStream_t st) {
  const AndLayout L = and_layout(n, K);
  char* b = static_cast<char*>(buf);
  k_and_store<<<blocks_for(n), kT, 0, st>>>(f, n, mode, slot, reinterpret_cast<float*>(b + L.hist) + (size_t)pos * L.stride,
                                            reinterpret_cast<double*>(b + L.lam) + pos);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_anderson_extrapolate(float* f, int n, int K, int p0, double r, void* buf, Slot* slot_g,
                                        int* status, cudaStream_t st) {
  switch (K) {
    case 2: return extrapolate<2>(f, n, p0, r, buf, slot_g, status, st);
    case 3: return extrapolate<3>(f, n, p0, r, buf, slot_g, status, st);
    case 4: return extrapolate<4>(f, n, p0, r, buf, slot_g, status, st);
    case 5: return extrapolate<5>(f, n, p0, r, buf, slot_g, status, st);
    default: return extrapolate<6>(f, n, p0, r, buf, slot_g, status, st);
  }
}

}  // namespace uot

extern "C" size_t uot_anderson_workspace(int32_t n, int32_t k) {
  if (n < 1 || k < 2 || k > 6) return 0;
  return uot::anderson_bytes(n, k);
}
