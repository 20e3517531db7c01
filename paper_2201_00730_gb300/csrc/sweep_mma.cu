// Gradient and adjoint sweeps for high-dimensional point clouds (dim >= 32,
// p = 2) with the contractions on mma.sync tensor-core fragments (the
// non-moment sweeps run on tcgen05, sweep_umma.cu):
//
//   t_ij = h_j - s |x_i - y_j|^2 = (h_j - s |y_j|^2) + (-s |x_i|^2) + 2 s x_i . y_j
//
// (coordinates taken relative to a common centre c, so the two squared norms
// stay small).  The dot products x_i . y_j are evaluated with mma.sync
// m16n8k8 TF32 in three passes (hi.hi + hi.lo + lo.hi with x = hi + lo,
// hi = tf32(x)), which keeps the product at about FP32 accuracy (one TF32
// pass would cost ~1e-3 relative), with the online log-sum-exp on the
// accumulator fragments in registers as in fused attention kernels.
#include <cuda_runtime.h>
#include <stdint.h>

#include "uot_internal.cuh"

namespace uot {
namespace {

constexpr int kWarps = 8;
constexpr int kThreads = kWarps * 32;
constexpr int kRows = 16 * kWarps;  // 128 query rows per CTA
constexpr int kKeys = 64;           // keys per tile
constexpr int kDMax = 64;           // dim <= 64, padded to a multiple of 8
constexpr int kLd = kDMax + 4;      // padded row stride (words): conflict-free fragment loads

__device__ __forceinline__ float ex2f(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__device__ __forceinline__ uint32_t tf32_hi(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

// split x = hi + lo with both parts representable in TF32
__device__ __forceinline__ void split_tf32(float x, uint32_t& hi, uint32_t& lo) {
  hi = tf32_hi(x);
  lo = tf32_hi(x - __uint_as_float(hi));
}

__device__ __forceinline__ void mma_tf32(float (&c)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                         uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// Softmin sweep with moments on the tensor cores (dim >= 32, p = 2): the
// partials of the plain sweep plus, per row, the moment channels
//     mom_d = momscale * sum_j mult_j 2^(t_ij - max) (x_i - y_j)_d
// of the gradient sweeps (forward: mult = 1, momscale = 2, the dC/dx factor)
// and of the unrolled backward's adjoint sweeps (mult = the signed key
// cotangent, momscale = 1).  As in fused attention, the moment is a second
// contraction: x_i sum_j P_ij - sum_j P_ij y_j with P the (scaled) exponential
// weights, so O = P.Y runs on the tensor cores too (3xTF32 again), with the
// keys of an 8-key block taken in the order (0, 2, 4, 6, 1, 3, 5, 7): the
// accumulator fragment of S = X.Y^T then is the A fragment of P.Y as it stands.
// The exponent is t_ij = H_j + Z_i - s |x_i - y_j|^2 with
//   forward: H_j = log2 w_j + s (pot_j + shift), Z_i = 0;
//   adjoint: H_j = s h_j, Z_i = s pot_i.
__global__ void __launch_bounds__(kThreads, 1)
k_sweep_flash(const float* __restrict__ q, int nq, const float* __restrict__ kp, int nk, int dim,
              const float* __restrict__ center, const float* __restrict__ l2w, const float* __restrict__ pot,
              const double* __restrict__ shift, const float* __restrict__ zrow, const float* __restrict__ hk,
              const float* __restrict__ mk, double s, float momscale, int kps, float* __restrict__ part) {
  extern __shared__ uint32_t smem[];
  uint32_t* khi = smem;                      // [kKeys][kLd]
  uint32_t* klo = khi + kKeys * kLd;         // [kKeys][kLd]
  float* kH = reinterpret_cast<float*>(klo + kKeys * kLd);  // [kKeys]
  float* kM = kH + kKeys;                                   // [kKeys] key multipliers
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = lane >> 2, tg = lane & 3;
  const int split = blockIdx.y;
  const int j0 = split * kps, j1 = min(nk, j0 + kps);
  const int dim8 = (dim + 7) & ~7;
  const double sh = shift ? *shift : 0.0;
  const float sf = (float)s, s2 = (float)(2.0 * s);

  const int rbase = blockIdx.x * kRows + warp * 16;
  const int rA = rbase + g, rB = rbase + g + 8;
  uint32_t ahi[kDMax / 8][4], alo[kDMax / 8][4];
  float qn[2] = {0.f, 0.f};
#pragma unroll
  for (int ks = 0; ks < kDMax / 8; ++ks) {
    if (ks * 8 < dim8) {
      const int c0 = ks * 8 + tg, c1 = ks * 8 + tg + 4;
      float v[4];
      v[0] = (rA < nq && c0 < dim) ? q[(size_t)rA * dim + c0] - center[c0] : 0.f;
      v[1] = (rB < nq && c0 < dim) ? q[(size_t)rB * dim + c0] - center[c0] : 0.f;
      v[2] = (rA < nq && c1 < dim) ? q[(size_t)rA * dim + c1] - center[c1] : 0.f;
      v[3] = (rB < nq && c1 < dim) ? q[(size_t)rB * dim + c1] - center[c1] : 0.f;
      qn[0] = fmaf(v[0], v[0], fmaf(v[2], v[2], qn[0]));
      qn[1] = fmaf(v[1], v[1], fmaf(v[3], v[3], qn[1]));
#pragma unroll
      for (int e = 0; e < 4; ++e) split_tf32(v[e], ahi[ks][e], alo[ks][e]);
    } else {
#pragma unroll
      for (int e = 0; e < 4; ++e) { ahi[ks][e] = 0u; alo[ks][e] = 0u; }
    }
  }
  qn[0] += __shfl_xor_sync(0xffffffffu, qn[0], 1);
  qn[0] += __shfl_xor_sync(0xffffffffu, qn[0], 2);
  qn[1] += __shfl_xor_sync(0xffffffffu, qn[1], 1);
  qn[1] += __shfl_xor_sync(0xffffffffu, qn[1], 2);
  const float ZA = (zrow && rA < nq) ? sf * zrow[rA] : 0.f, ZB = (zrow && rB < nq) ? sf * zrow[rB] : 0.f;
  const float Rr[2] = {fmaf(-sf, qn[0], ZA), fmaf(-sf, qn[1], ZB)};  // row constants, added at the end
  float mu[2] = {kInitMax, kInitMax}, acc[2] = {0.f, 0.f};
  float o[kDMax / 8][4];  // P.Y: rows (g, g + 8) x dims (8 db + 2 tg, + 1)
#pragma unroll
  for (int db = 0; db < kDMax / 8; ++db) o[db][0] = o[db][1] = o[db][2] = o[db][3] = 0.f;

  for (int jt = j0; jt < j1; jt += kKeys) {
    const int cnt = min(kKeys, j1 - jt);
    __syncthreads();
    for (int e = threadIdx.x; e < kKeys * dim8; e += kThreads) {
      const int u = e / dim8, d = e - u * dim8;
      float v = 0.f;
      if (u < cnt && d < dim) v = kp[(size_t)(jt + u) * dim + d] - center[d];
      uint32_t hi, lo;
      split_tf32(v, hi, lo);
      khi[u * kLd + d] = hi;
      klo[u * kLd + d] = lo;
    }
    __syncthreads();
    if (threadIdx.x < kKeys) {
      const int u = threadIdx.x;
      float H = kZeroW, mult = 0.f;
      if (u < cnt) {
        const int j = jt + u;
        float y2 = 0.f;
#pragma unroll 8
        for (int d = 0; d < dim8; ++d) {
          const float v = __uint_as_float(khi[u * kLd + d]) + __uint_as_float(klo[u * kLd + d]);
          y2 = fmaf(v, v, y2);
        }
        if (hk) {
          H = (float)(s * (double)hk[j] - s * (double)y2);
          mult = mk ? mk[j] : 1.f;
        } else {
          const float lw = l2w[j];
          if (lw > 0.5f * kZeroW) {
            const double pj = pot ? (double)pot[j] : 0.0;
            H = (float)((double)lw + s * (pj + sh) - s * (double)y2);
            mult = mk ? mk[j] : 1.f;
          }
        }
      }
      kH[u] = H;
      kM[u] = mult;
    }
    __syncthreads();
    // S = X.Y^T on 16 rows x 64 keys per warp
    float c[kKeys / 8][4];
#pragma unroll
    for (int nb = 0; nb < kKeys / 8; ++nb) {
      c[nb][0] = c[nb][1] = c[nb][2] = c[nb][3] = 0.f;
#pragma unroll
      for (int ks = 0; ks < kDMax / 8; ++ks) {
        if (ks * 8 < dim8) {
          const int key = nb * 8 + g;
          const uint32_t bh0 = khi[key * kLd + ks * 8 + tg], bh1 = khi[key * kLd + ks * 8 + tg + 4];
          const uint32_t bl0 = klo[key * kLd + ks * 8 + tg], bl1 = klo[key * kLd + ks * 8 + tg + 4];
          mma_tf32(c[nb], alo[ks][0], alo[ks][1], alo[ks][2], alo[ks][3], bh0, bh1);
          mma_tf32(c[nb], ahi[ks][0], ahi[ks][1], ahi[ks][2], ahi[ks][3], bl0, bl1);
          mma_tf32(c[nb], ahi[ks][0], ahi[ks][1], ahi[ks][2], ahi[ks][3], bh0, bh1);
        }
      }
    }
    float tmA = kInitMax, tmB = kInitMax;
#pragma unroll
    for (int nb = 0; nb < kKeys / 8; ++nb) {
      const float H0 = kH[nb * 8 + 2 * tg], H1 = kH[nb * 8 + 2 * tg + 1];
      c[nb][0] = fmaf(s2, c[nb][0], H0);
      c[nb][1] = fmaf(s2, c[nb][1], H1);
      c[nb][2] = fmaf(s2, c[nb][2], H0);
      c[nb][3] = fmaf(s2, c[nb][3], H1);
      tmA = fmaxf(tmA, fmaxf(c[nb][0], c[nb][1]));
      tmB = fmaxf(tmB, fmaxf(c[nb][2], c[nb][3]));
    }
    tmA = fmaxf(tmA, __shfl_xor_sync(0xffffffffu, tmA, 1));
    tmA = fmaxf(tmA, __shfl_xor_sync(0xffffffffu, tmA, 2));
    tmB = fmaxf(tmB, __shfl_xor_sync(0xffffffffu, tmB, 1));
    tmB = fmaxf(tmB, __shfl_xor_sync(0xffffffffu, tmB, 2));
    const float mA = fmaxf(mu[0], tmA), mB = fmaxf(mu[1], tmB);
    const float scA = ex2f(mu[0] - mA), scB = ex2f(mu[1] - mB);
    float sA = acc[0] * scA, sB = acc[1] * scB;
#pragma unroll
    for (int db = 0; db < kDMax / 8; ++db) {
      o[db][0] *= scA; o[db][1] *= scA;
      o[db][2] *= scB; o[db][3] *= scB;
    }
    // P (weighted exponentials) in place of S, then O += P.Y with the key order (2 tg, 2 tg + 1)
#pragma unroll
    for (int nb = 0; nb < kKeys / 8; ++nb) {
      const float M0 = kM[nb * 8 + 2 * tg], M1 = kM[nb * 8 + 2 * tg + 1];
      c[nb][0] = M0 * ex2f(c[nb][0] - mA);
      c[nb][1] = M1 * ex2f(c[nb][1] - mA);
      c[nb][2] = M0 * ex2f(c[nb][2] - mB);
      c[nb][3] = M1 * ex2f(c[nb][3] - mB);
      sA += c[nb][0] + c[nb][1];
      sB += c[nb][2] + c[nb][3];
      uint32_t ph[4], pl[4];
      split_tf32(c[nb][0], ph[0], pl[0]);  // (row g,     key 2 tg)     -> a0
      split_tf32(c[nb][2], ph[1], pl[1]);  // (row g + 8, key 2 tg)     -> a1
      split_tf32(c[nb][1], ph[2], pl[2]);  // (row g,     key 2 tg + 1) -> a2
      split_tf32(c[nb][3], ph[3], pl[3]);  // (row g + 8, key 2 tg + 1) -> a3
      const int k0 = nb * 8 + 2 * tg, k1 = k0 + 1;
#pragma unroll
      for (int db = 0; db < kDMax / 8; ++db) {
        if (db * 8 < dim8) {
          const int d = db * 8 + g;
          const uint32_t vh0 = khi[k0 * kLd + d], vh1 = khi[k1 * kLd + d];
          const uint32_t vl0 = klo[k0 * kLd + d], vl1 = klo[k1 * kLd + d];
          mma_tf32(o[db], pl[0], pl[1], pl[2], pl[3], vh0, vh1);
          mma_tf32(o[db], ph[0], ph[1], ph[2], ph[3], vl0, vl1);
          mma_tf32(o[db], ph[0], ph[1], ph[2], ph[3], vh0, vh1);
        }
      }
    }
    mu[0] = mA; mu[1] = mB;
    acc[0] = sA; acc[1] = sB;
  }
  acc[0] += __shfl_xor_sync(0xffffffffu, acc[0], 1);
  acc[0] += __shfl_xor_sync(0xffffffffu, acc[0], 2);
  acc[1] += __shfl_xor_sync(0xffffffffu, acc[1], 1);
  acc[1] += __shfl_xor_sync(0xffffffffu, acc[1], 2);
  const int CH = 2 + dim;
  float* base = part + (size_t)split * CH * nq;
  if (tg == 0) {
    if (rA < nq) { base[rA] = mu[0] + Rr[0]; base[(size_t)nq + rA] = acc[0]; }
    if (rB < nq) { base[rB] = mu[1] + Rr[1]; base[(size_t)nq + rB] = acc[1]; }
  }
  // moments: momscale (x_i acc - O_i), each (row, dim) held by one thread of the quad
#pragma unroll
  for (int db = 0; db < kDMax / 8; ++db) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int d = db * 8 + 2 * tg + h;
      if (d < dim) {
        const float cd = center[d];
        if (rA < nq) base[(size_t)(2 + d) * nq + rA] = momscale * fmaf(q[(size_t)rA * dim + d] - cd, acc[0], -o[db][h]);
        if (rB < nq) base[(size_t)(2 + d) * nq + rB] = momscale * fmaf(q[(size_t)rB * dim + d] - cd, acc[1], -o[db][2 + h]);
      }
    }
  }
}

// centre = mean of the two clouds, one block per coordinate: keeps |x - c|, |y - c| small in the expansion
__global__ void k_center(const float* x, int n, const float* y, int m, int dim, float* center) {
  __shared__ double sh[256];
  const int d = blockIdx.x;
  double acc = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) acc += x[(size_t)i * dim + d];
  for (int j = threadIdx.x; j < m; j += blockDim.x) acc += y[(size_t)j * dim + d];
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int off = blockDim.x / 2; off > 0; off >>= 1) {
    if (threadIdx.x < off) sh[threadIdx.x] += sh[threadIdx.x + off];
    __syncthreads();
  }
  if (threadIdx.x == 0) center[d] = (float)(sh[0] / (double)(n + m));
}

size_t flash_smem_bytes() { return sizeof(uint32_t) * 2 * kKeys * kLd + sizeof(float) * 2 * kKeys; }

}  // namespace

cudaError_t launch_center(const float* x, int n, const float* y, int m, int dim, float* center, cudaStream_t st) {
  k_center<<<dim, 256, 0, st>>>(x, n, y, m, dim, center);
  note_launch();
  return cudaGetLastError();
}

// One CTA of 8 warps per SM at most (the kernel holds ~200 registers a thread):
// key chunks so that row blocks x chunks fill the SMs.
SweepGeom flash_geom(int nq, int nk) {
  SweepGeom g{};
  g.threads = kThreads;
  g.rows = 1;
  g.row_blocks = (nq + kRows - 1) / kRows;
  const long long target = device_sm_count();
  const int max_tiles = (nk + kKeys - 1) / kKeys;
  double best = 1e300;
  int best_k = 1;
  for (int k = 1; k <= 256 && k <= max_tiles; ++k) {
    const int tiles_per = (max_tiles + k - 1) / k;
    const int kk = (max_tiles + tiles_per - 1) / tiles_per;
    if (kk != k) continue;
    const long long ctas = (long long)g.row_blocks * kk;
    const long long waves = (ctas + target - 1) / target;
    const double est = (double)waves * (tiles_per + 1.0);
    if (est < best * 0.999) { best = est; best_k = kk; }
  }
  const int tiles_per = (max_tiles + best_k - 1) / best_k;
  g.keys_per_split = tiles_per * kKeys;
  g.splits = (nk + g.keys_per_split - 1) / g.keys_per_split;
  return g;
}

cudaError_t launch_flash_sweep(const float* q, int nq, const float* kp, int nk, int dim, const float* center,
                               const float* l2w, const float* pot, const double* shift, const float* zrow,
                               const float* hk, const float* mk, double s, float momscale, float* part,
                               const SweepGeom& g, cudaStream_t st) {
  static bool attr_set = false;
  const size_t smem = flash_smem_bytes();
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(k_sweep_flash, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  dim3 grid(g.row_blocks, g.splits);
  k_sweep_flash<<<grid, kThreads, smem, st>>>(q, nq, kp, nk, dim, center, l2w, pot, shift, zrow, hk, mk, s, momscale,
                                              g.keys_per_split, part);
  note_launch();
  return cudaGetLastError();
}

}  // namespace uot
