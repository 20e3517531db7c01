// Gradient and adjoint sweeps for high-dimensional point clouds (dim >= 32,
// p = 2) with both contractions on mma.sync tensor-core fragments (the
// non-moment sweeps run on tcgen05, sweep_umma.cu):
//
//   t_ij = h_j - s |x_i - y_j|^2 = (h_j - s |y'_j|^2) + (-s |x'_i|^2) + 2 s x'_i . y'_j,
//
// x' = x - c, y' = y - c with c the clouds' common centre.  As in the tcgen05
// sweep, every coordinate is scaled by a power of two 2^e shared by both
// clouds (the largest |x - c| 2^e in [2^14, 2^15)) and split into FP16 parts
// hi + lo (11 significant bits each); x'.y' is hi.hi + lo.hi + hi.lo on
// mma.sync m16n8k16 FP16 with FP32 accumulation (the dropped lo.lo is below
// 2^-22 of |x'||y'|) and the squared norms use the same represented values.
// The moments are a second contraction, as in fused attention:
//     mom_d = momscale * sum_j mult_j 2^(t_ij - max) (x_i - y_j)_d
//           = momscale (x'_i,d sum_j P_ij - O_i,d),  O = P . Z,  Z_j = mult_j y'_j,
// with P the exponential weights of the running max (in [0, 1], split into
// FP16 hi + lo) and Z scaled once more by a power of two 2^k per CTA (the
// largest |mult_j| of the CTA's keys in [1/2, 1]) so that it fits FP16; O runs
// on the same m16n8k16 instruction (Ph.Zh + Pl.Zh + Ph.Zl), its accumulator
// fragments rescaled with the running max, and P comes from the S accumulator
// fragments as they stand (the accumulator of two 8-key tiles is the A
// fragment of one 16-key step).  The exponent is t_ij = H_j + Z_i - s |x_i - y_j|^2 with
//   forward: H_j = log2 w_j + s (pot_j + shift), Z_i = 0, mult = 1 (live keys);
//   adjoint: H_j = s h_j, Z_i = s pot_i, mult = the signed key cotangent.
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "uot_internal.cuh"

namespace uot {
namespace {

constexpr int kWarps = 8;
constexpr int kThreads = kWarps * 32;
constexpr int kRows = 16 * kWarps;  // 128 query rows per CTA
constexpr int kKeys = 64;           // keys per tile
constexpr int kLdT = kKeys / 2 + 4; // words per dimension row of Z^T (conflict-free fragment loads)

__device__ __forceinline__ float ex2f(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float p2f(int e) { return __int_as_float((127 + e) << 23); }

// Scale exponent of the coordinates: the largest |x - c| (float bits) times 2^e in [2^14, 2^15).
__device__ __forceinline__ int coord_exp(const int* maxbits) {
  const int mb = maxbits ? *maxbits : 0;
  if (mb <= 0) return 0;
  const int e = 14 - (((mb >> 23) & 255) - 127);
  return e < -40 ? -40 : (e > 40 ? 40 : e);
}

__device__ __forceinline__ void split_h(float v, __half& hi, __half& lo) {
  hi = __float2half_rn(v);
  lo = __float2half_rn(v - __half2float(hi));
}
__device__ __forceinline__ uint32_t pack_h(__half a, __half b) {
  return (uint32_t)__half_as_ushort(a) | ((uint32_t)__half_as_ushort(b) << 16);
}
// a = hi + lo of two values, packed (first value in the low half)
__device__ __forceinline__ void split_pack(float v0, float v1, uint32_t& hi, uint32_t& lo) {
  __half h0, l0, h1, l1;
  split_h(v0, h0, l0);
  split_h(v1, h1, l1);
  hi = pack_h(h0, h1);
  lo = pack_h(l0, l1);
}

__device__ __forceinline__ void mma16(float (&c)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3, uint32_t b0,
                                      uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// Shared memory of one CTA (KS = dim16 / 16 K-steps of 16 coordinates).
template <int KS>
struct FlashSmem {
  static constexpr int kLdK = 8 * KS + 4;  // words per key row of Y (pairs of coordinates), padded
  uint32_t xh[kRows * kLdK], xl[kRows * kLdK];  // X' 2^e of the CTA's rows, row-major, hi / lo
  uint32_t yh[kKeys * kLdK], yl[kKeys * kLdK];  // Y' 2^e, key-major, hi / lo
  uint32_t zh[16 * KS * kLdT], zl[16 * KS * kLdT];  // Z 2^(e+k), coordinate-major (pairs of keys), hi / lo
  float kH[kKeys], kM[kKeys];
  float red[kWarps];
  float cen[16 * KS];
  // the next key tile, copied ahead (cp.async) while the current one computes:
  // coordinates (row-major, dim a key) and the per-key scalars l2w, pot, hk, mk
  float raw[kKeys * 16 * KS];
  float rs[4][kKeys];
};

__device__ __forceinline__ void cp4(void* s, const void* g) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"((unsigned)__cvta_generic_to_shared(s)), "l"(g)
               : "memory");
}
__device__ __forceinline__ void cp16(void* s, const void* g) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((unsigned)__cvta_generic_to_shared(s)), "l"(g)
               : "memory");
}

// One CTA: 128 query rows (8 warps of 16) against the keys [split kps, + kps).
template <int KS>
__global__ void __launch_bounds__(kThreads, 2)
k_sweep_flash(const float* __restrict__ q, int nq, const float* __restrict__ kp, int nk, int dim,
              const float* __restrict__ center, const int* __restrict__ maxbits, const float* __restrict__ l2w,
              const float* __restrict__ pot, const double* __restrict__ shift, const float* __restrict__ zrow,
              const float* __restrict__ hk, const float* __restrict__ mk, double s, float momscale, int kps,
              float* __restrict__ part) {
  constexpr int D16 = 16 * KS;
  constexpr int LDK = FlashSmem<KS>::kLdK;
  extern __shared__ __align__(16) unsigned char smraw[];
  FlashSmem<KS>& sm = *reinterpret_cast<FlashSmem<KS>*>(smraw);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = lane >> 2, t = lane & 3;
  const int split = blockIdx.y;
  const int j0 = split * kps, j1 = min(nk, j0 + kps);
  const int ce = coord_exp(maxbits);
  const float csc = p2f(ce), icsc = p2f(-ce);
  const double sh = shift ? *shift : 0.0;
  const float sf = (float)s;
  const float s2 = (float)(2.0 * s) * icsc * icsc;  // the products carry 2^2e

  // the CTA's multiplier scale 2^k: the largest |mult_j| of its keys times 2^k in [1/2, 1)
  float mmax = 0.f;
  if (mk) {
    for (int j = j0 + (int)threadIdx.x; j < j1; j += kThreads) mmax = fmaxf(mmax, fabsf(mk[j]));
  } else {
    mmax = 1.f;
  }
  for (int o = 16; o > 0; o >>= 1) mmax = fmaxf(mmax, __shfl_xor_sync(0xffffffffu, mmax, o));
  if (lane == 0) sm.red[warp] = mmax;
  __syncthreads();
  mmax = sm.red[0];
#pragma unroll
  for (int w = 1; w < kWarps; ++w) mmax = fmaxf(mmax, sm.red[w]);
  int kz = 0;
  if (mmax > 0.f && mmax < INFINITY) {
    kz = -(((__float_as_int(mmax) >> 23) & 255) - 127) - 1;
    kz = kz < -120 ? -120 : (kz > 120 ? 120 : kz);
  }
  const float zsc = p2f(kz), izsc = p2f(-kz);

  for (int d = threadIdx.x; d < D16; d += kThreads) sm.cen[d] = d < dim ? center[d] : 0.f;
  // copies of key tile [jn, jn + 64) into raw / rs (the caller commits and waits)
  const bool al16 = ((reinterpret_cast<uintptr_t>(kp) & 15u) == 0) && ((dim & 3) == 0);
  auto issue = [&](int jn) {
    const int cn = min(kKeys, j1 - jn);
    const float* src = kp + (size_t)jn * dim;
    const int nf = cn * dim;
    if (al16) {
      for (int k = threadIdx.x; k < (nf >> 2); k += kThreads) cp16(sm.raw + 4 * k, src + 4 * k);
    } else {
      for (int k = threadIdx.x; k < nf; k += kThreads) cp4(sm.raw + k, src + k);
    }
    if ((int)threadIdx.x < cn) {
      const int j = jn + threadIdx.x;
      if (l2w) cp4(&sm.rs[0][threadIdx.x], l2w + j);
      if (pot) cp4(&sm.rs[1][threadIdx.x], pot + j);
      if (hk) cp4(&sm.rs[2][threadIdx.x], hk + j);
      if (mk) cp4(&sm.rs[3][threadIdx.x], mk + j);
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  };
  if (j0 < j1) issue(j0);
  // the CTA's rows: X' 2^e split, row-major, pairs of coordinates per word (the A fragments of
  // S = X.Y^T are read from here: rows g and g + 8 of a warp's 16, coordinates (2t, 2t+1) and
  // (2t+8, 2t+9) of a 16-coordinate step)
  for (int u2 = threadIdx.x; u2 < kRows * (D16 / 2); u2 += kThreads) {
    const int u = u2 / (D16 / 2), w = u2 - u * (D16 / 2), d = 2 * w;
    const int r = blockIdx.x * kRows + u;
    float v0 = 0.f, v1 = 0.f;
    if (r < nq) {
      const float* xr = q + (size_t)r * dim;
      if (d < dim) v0 = (xr[d] - center[d]) * csc;
      if (d + 1 < dim) v1 = (xr[d + 1] - center[d + 1]) * csc;
    }
    uint32_t hi, lo;
    split_pack(v0, v1, hi, lo);
    sm.xh[u * LDK + w] = hi;
    sm.xl[u * LDK + w] = lo;
  }
  __syncthreads();
  const int rbase = blockIdx.x * kRows + warp * 16;
  const int rA = rbase + g, rB = rbase + g + 8;
  const uint32_t* xhA = sm.xh + (warp * 16 + g) * LDK;
  const uint32_t* xhB = xhA + 8 * LDK;
  const uint32_t* xlA = sm.xl + (warp * 16 + g) * LDK;
  const uint32_t* xlB = xlA + 8 * LDK;
  // |x'|^2 of the represented coordinates, per row (each of the quad's threads a quarter of the words)
  float qn[2] = {0.f, 0.f};
  for (int w = t; w < D16 / 2; w += 4) {
    const uint32_t hw[2] = {xhA[w], xhB[w]}, lw[2] = {xlA[w], xlB[w]};
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const float2 fh = __half22float2(*reinterpret_cast<const __half2*>(&hw[k]));
      const float2 fl = __half22float2(*reinterpret_cast<const __half2*>(&lw[k]));
      const float y0 = fh.x + fl.x, y1 = fh.y + fl.y;
      qn[k] = fmaf(y0, y0, fmaf(y1, y1, qn[k]));
    }
  }
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    qn[k] += __shfl_xor_sync(0xffffffffu, qn[k], 1);
    qn[k] += __shfl_xor_sync(0xffffffffu, qn[k], 2);
  }
  const float ZA = (zrow && rA < nq) ? sf * zrow[rA] : 0.f, ZB = (zrow && rB < nq) ? sf * zrow[rB] : 0.f;
  const float Rr[2] = {fmaf(-sf, qn[0] * icsc * icsc, ZA), fmaf(-sf, qn[1] * icsc * icsc, ZB)};
  float mu[2] = {kInitMax, kInitMax}, acc[2] = {0.f, 0.f};
  float o[2 * KS][4];  // O = P.Z: rows (g, g + 8) x coordinates (8 db + 2 t, + 1)
#pragma unroll
  for (int db = 0; db < 2 * KS; ++db) o[db][0] = o[db][1] = o[db][2] = o[db][3] = 0.f;

  for (int jt = j0; jt < j1; jt += kKeys) {
    const int cnt = min(kKeys, j1 - jt);
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    __syncthreads();
    // Y' 2^e split, key-major, pairs of coordinates per word
    for (int u2 = threadIdx.x; u2 < kKeys * (D16 / 2); u2 += kThreads) {
      const int u = u2 / (D16 / 2), w = u2 - u * (D16 / 2), d = 2 * w;
      float v0 = 0.f, v1 = 0.f;
      if (u < cnt) {
        const float* kr = sm.raw + u * dim;
        if (d < dim) v0 = (kr[d] - sm.cen[d]) * csc;
        if (d + 1 < dim) v1 = (kr[d + 1] - sm.cen[d + 1]) * csc;
      }
      uint32_t hi, lo;
      split_pack(v0, v1, hi, lo);
      sm.yh[u * LDK + w] = hi;
      sm.yl[u * LDK + w] = lo;
    }
    __syncthreads();
    // key constants, and Z = mult Y' 2^(e + k) split, coordinate-major, pairs of keys per word
    if (threadIdx.x < kKeys) {
      const int u = threadIdx.x;
      float H = kZeroW, mult = 0.f;
      if (u < cnt) {
        const int j = jt + u;
        float y2 = 0.f;
        for (int w = 0; w < D16 / 2; ++w) {
          const uint32_t hh = sm.yh[u * LDK + w], ll = sm.yl[u * LDK + w];
          const float2 fh = __half22float2(*reinterpret_cast<const __half2*>(&hh));
          const float2 fl = __half22float2(*reinterpret_cast<const __half2*>(&ll));
          const float y0 = fh.x + fl.x, y1 = fh.y + fl.y;
          y2 = fmaf(y0, y0, fmaf(y1, y1, y2));
        }
        (void)j;
        const double y2u = (double)y2 * (double)icsc * (double)icsc;
        if (hk) {
          H = (float)(s * (double)sm.rs[2][u] - s * y2u);
          mult = mk ? sm.rs[3][u] : 1.f;
        } else {
          const float lw = sm.rs[0][u];
          if (lw > 0.5f * kZeroW) {
            const double pj = pot ? (double)sm.rs[1][u] : 0.0;
            H = (float)((double)lw + s * (pj + sh) - s * y2u);
            mult = mk ? sm.rs[3][u] : 1.f;
          }
        }
      }
      sm.kH[u] = H;
      sm.kM[u] = mult;
    }
    // coordinates fastest: the reads of Y' are consecutive halves
    for (int idx = threadIdx.x; idx < D16 * (kKeys / 2); idx += kThreads) {
      const int w = idx / D16, d = idx - w * D16;
      float z[2];
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        const int u = 2 * w + k;
        const float mult = (u < cnt) ? (mk ? sm.rs[3][u] : 1.f) * zsc : 0.f;
        const __half* ph = reinterpret_cast<const __half*>(sm.yh + u * LDK);
        const __half* pl = reinterpret_cast<const __half*>(sm.yl + u * LDK);
        z[k] = mult * (__half2float(ph[d]) + __half2float(pl[d]));
      }
      uint32_t hi, lo;
      split_pack(z[0], z[1], hi, lo);
      sm.zh[d * kLdT + w] = hi;
      sm.zl[d * kLdT + w] = lo;
    }
    __syncthreads();
    // raw and rs are free (read before the barrier): copy the next tile while this one computes
    if (jt + kKeys < j1) issue(jt + kKeys);
    // S = X.Y^T on 16 rows x 64 keys per warp (K-steps outside: one step's A fragments live)
    float c[kKeys / 8][4];
#pragma unroll
    for (int nb = 0; nb < kKeys / 8; ++nb) c[nb][0] = c[nb][1] = c[nb][2] = c[nb][3] = 0.f;
#pragma unroll
    for (int ks = 0; ks < KS; ++ks) {
      const uint32_t ah0 = xhA[8 * ks + t], ah1 = xhB[8 * ks + t], ah2 = xhA[8 * ks + 4 + t], ah3 = xhB[8 * ks + 4 + t];
      const uint32_t al0 = xlA[8 * ks + t], al1 = xlB[8 * ks + t], al2 = xlA[8 * ks + 4 + t], al3 = xlB[8 * ks + 4 + t];
#pragma unroll
      for (int nb = 0; nb < kKeys / 8; ++nb) {
        const uint32_t* yh = sm.yh + (8 * nb + g) * LDK;
        const uint32_t* yl = sm.yl + (8 * nb + g) * LDK;
        const uint32_t bh0 = yh[8 * ks + t], bh1 = yh[8 * ks + 4 + t];
        const uint32_t bl0 = yl[8 * ks + t], bl1 = yl[8 * ks + 4 + t];
        mma16(c[nb], ah0, ah1, ah2, ah3, bh0, bh1);
        mma16(c[nb], al0, al1, al2, al3, bh0, bh1);
        mma16(c[nb], ah0, ah1, ah2, ah3, bl0, bl1);
      }
    }
    float tmA = kInitMax, tmB = kInitMax;
#pragma unroll
    for (int nb = 0; nb < kKeys / 8; ++nb) {
      const float H0 = sm.kH[8 * nb + 2 * t], H1 = sm.kH[8 * nb + 2 * t + 1];
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
    for (int db = 0; db < 2 * KS; ++db) {
      o[db][0] *= scA; o[db][1] *= scA;
      o[db][2] *= scB; o[db][3] *= scB;
    }
    // P in place of S (weights in [0, 1]); the sums carry the multipliers, O carries them in Z
#pragma unroll
    for (int nb = 0; nb < kKeys / 8; ++nb) {
      const float M0 = sm.kM[8 * nb + 2 * t], M1 = sm.kM[8 * nb + 2 * t + 1];
      c[nb][0] = ex2f(c[nb][0] - mA);
      c[nb][1] = ex2f(c[nb][1] - mA);
      c[nb][2] = ex2f(c[nb][2] - mB);
      c[nb][3] = ex2f(c[nb][3] - mB);
      sA = fmaf(M0, c[nb][0], fmaf(M1, c[nb][1], sA));
      sB = fmaf(M0, c[nb][2], fmaf(M1, c[nb][3], sB));
    }
    // O += P.Z, 16 keys a step: the S accumulators of two 8-key tiles are the A fragment
#pragma unroll
    for (int kk = 0; kk < kKeys / 16; ++kk) {
      uint32_t ph[4], pl[4];
      split_pack(c[2 * kk][0], c[2 * kk][1], ph[0], pl[0]);
      split_pack(c[2 * kk][2], c[2 * kk][3], ph[1], pl[1]);
      split_pack(c[2 * kk + 1][0], c[2 * kk + 1][1], ph[2], pl[2]);
      split_pack(c[2 * kk + 1][2], c[2 * kk + 1][3], ph[3], pl[3]);
#pragma unroll
      for (int db = 0; db < 2 * KS; ++db) {
        const uint32_t* zh = sm.zh + (8 * db + g) * kLdT;
        const uint32_t* zl = sm.zl + (8 * db + g) * kLdT;
        const uint32_t bh0 = zh[8 * kk + t], bh1 = zh[8 * kk + 4 + t];
        const uint32_t bl0 = zl[8 * kk + t], bl1 = zl[8 * kk + 4 + t];
        mma16(o[db], ph[0], ph[1], ph[2], ph[3], bh0, bh1);
        mma16(o[db], pl[0], pl[1], pl[2], pl[3], bh0, bh1);
        mma16(o[db], ph[0], ph[1], ph[2], ph[3], bl0, bl1);
      }
    }
    mu[0] = mA; mu[1] = mB;
    acc[0] = sA; acc[1] = sB;
  }
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    acc[k] += __shfl_xor_sync(0xffffffffu, acc[k], 1);
    acc[k] += __shfl_xor_sync(0xffffffffu, acc[k], 2);
  }
  const int CH = 2 + dim;
  float* base = part + (size_t)split * CH * nq;
  if (t == 0) {
    if (rA < nq) { base[rA] = mu[0] + Rr[0]; base[(size_t)nq + rA] = acc[0]; }
    if (rB < nq) { base[rB] = mu[1] + Rr[1]; base[(size_t)nq + rB] = acc[1]; }
  }
  // moments: momscale (x'_d sum_j P_ij mult_j - O_d 2^-(e + k)), each (row, coordinate) on one thread of the quad
  const float osc = icsc * izsc;
#pragma unroll
  for (int db = 0; db < 2 * KS; ++db) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int d = db * 8 + 2 * t + h;
      if (d < dim) {
        const float cd = center[d];
        if (rA < nq)
          base[(size_t)(2 + d) * nq + rA] = momscale * fmaf(q[(size_t)rA * dim + d] - cd, acc[0], -o[db][h] * osc);
        if (rB < nq)
          base[(size_t)(2 + d) * nq + rB] = momscale * fmaf(q[(size_t)rB * dim + d] - cd, acc[1], -o[db][2 + h] * osc);
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

}  // namespace

cudaError_t launch_center(const float* x, int n, const float* y, int m, int dim, float* center, cudaStream_t st) {
  k_center<<<dim, 256, 0, st>>>(x, n, y, m, dim, center);
  note_launch();
  return cudaGetLastError();
}

// Two CTAs of 8 warps per SM (about 128 registers a thread): key chunks so
// that row blocks x chunks fill them.
SweepGeom flash_geom(int nq, int nk) {
  SweepGeom g{};
  g.threads = kThreads;
  g.rows = 1;
  g.row_blocks = (nq + kRows - 1) / kRows;
  const long long target = 2LL * device_sm_count();
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

namespace {
template <int KS>
cudaError_t run_flash(const float* q, int nq, const float* kp, int nk, int dim, const float* center,
                      const int* maxbits, const float* l2w, const float* pot, const double* shift, const float* zrow,
                      const float* hk, const float* mk, double s, float momscale, float* part, const SweepGeom& g,
                      cudaStream_t st) {
  const size_t smem = sizeof(FlashSmem<KS>);
  static bool attr_set = false;  // per instantiation
  if (!attr_set) {
    const cudaError_t e = cudaFuncSetAttribute(k_sweep_flash<KS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  dim3 grid(g.row_blocks, g.splits);
  k_sweep_flash<KS><<<grid, kThreads, smem, st>>>(q, nq, kp, nk, dim, center, maxbits, l2w, pot, shift, zrow, hk,
                                                  mk, s, momscale, g.keys_per_split, part);
  note_launch();
  return cudaGetLastError();
}
}  // namespace

cudaError_t launch_flash_sweep(const float* q, int nq, const float* kp, int nk, int dim, const float* center,
                               const int* maxbits, const float* l2w, const float* pot, const double* shift,
                               const float* zrow, const float* hk, const float* mk, double s, float momscale,
                               float* part, const SweepGeom& g, cudaStream_t st) {
  if (dim < 17 || dim > 64) return cudaErrorInvalidValue;
  const int KS = (dim + 15) / 16;
  if (KS == 2) return run_flash<2>(q, nq, kp, nk, dim, center, maxbits, l2w, pot, shift, zrow, hk, mk, s, momscale, part, g, st);
  if (KS == 3) return run_flash<3>(q, nq, kp, nk, dim, center, maxbits, l2w, pot, shift, zrow, hk, mk, s, momscale, part, g, st);
  return run_flash<4>(q, nq, kp, nk, dim, center, maxbits, l2w, pot, shift, zrow, hk, mk, s, momscale, part, g, st);
}

}  // namespace uot
