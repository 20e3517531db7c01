// Moment and adjoint sweeps for high-dimensional point clouds (dim >= 32,
// p = 2) on the fifth-generation tensor cores: both contractions of
//     mom_d = momscale * sum_j mult_j 2^(t_ij - m_i) (x_i - y_j)_d
//           = momscale (x'_i,d sum_j mult_j P_ij - O_i,d),   O = P . Z,   Z_j = mult_j y'_j
// run as tcgen05 kind::f16 MMAs with FP32 accumulators in TMEM:
//   S = X'.Y'^T from the operands of the plain tcgen05 sweep (the power-of-two
//     scaled coordinates split into FP16 hi + lo, three passes), and
//   O = P.Z with P in [0, 1] split into FP16 hi + lo and written by the
//     consumer warps into TMEM (the A operand of the MMA), Z^T an operand
//     built once per launch (split FP16 hi + lo of mult_j y'_j 2^(e + k),
//     2^k putting the largest |mult| in [1/2, 1)), three passes again.
// Each CTA's part of a row block is swept twice: the first pass takes the row
// maxima m_i of its keys, the second forms P = 2^(t - m) <= 1 against them, so
// O accumulates in TMEM without any rescaling.  Output: the partials of the
// moment sweeps, (m_i + R_i, sum_j mult_j P_ij, moments) per (row, slot).
//
// Roles (one CTA per SM, 18 warps): lane 0 of warp 16 issues the MMAs, lane 0
// of warp 17 the copies (each buffer refilled once the MMAs that read it have
// completed, which the MMAs signal through tcgen05.commit); warps 0..15 read the
// S accumulators (warp w: TMEM lanes 32 (w % 4) .. +31, key quarter w / 4 of
// each 128-key tile), keep the maxima, form P and the value sums, write P, and
// at the end of a segment read O.  Handoffs on mbarriers, every wait bounded (a
// wait that gives up stops every role; each issuing role then lets its own
// copies or MMAs in flight land).
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <mutex>

#include "ffloat.cuh"
#include "sweep_common.cuh"
#include "tc_ptx.cuh"
#include "uot_internal.cuh"

namespace uot {
namespace {

using namespace simd;

constexpr int kRows = 128;     // MMA M
constexpr int kKeys = 128;     // keys per tile (N of S, K of O)
constexpr int kStages = 2;     // key-tile and Z-tile buffers
constexpr int kMaxChunk = 4096;  // keys per CTA (H and mult in shared memory)
constexpr int kConsWarps = 16;
constexpr int kMmaWarp = kConsWarps, kCopyWarp = kConsWarps + 1;  // the MMA and copy issuers
constexpr int kAllThreads = 32 * (kConsWarps + 2);
constexpr uint32_t kColS = 0;      // two 128-column S accumulators
constexpr uint32_t kColPh = 256;   // P hi: 64 columns (128 keys, two FP16 a column)
constexpr uint32_t kColPl = 320;   // P lo
constexpr uint32_t kColO = 384;    // O: dim16 columns
constexpr uint32_t kTmemCols = 512;
constexpr long long kSpin = kWaitPolls;
constexpr uint32_t kPiece = 65536;
constexpr int kZK = 2 * kKeys;     // Z^T rows hold [hi of 128 keys | lo of 128 keys]

__host__ __device__ constexpr int kmajor_off(int r, int k, int sbo) {
  return (r >> 3) * sbo + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2;
}
__device__ __forceinline__ float p2f(int e) { return __int_as_float((127 + e) << 23); }

// Scale exponent of the split: the largest |x - c| (float bits) times 2^e in [2^14, 2^15).
__device__ __forceinline__ int coord_exp(const int* maxbits) {
  const int mb = *maxbits;
  if (mb <= 0) return 0;
  const int e = 14 - (((mb >> 23) & 255) - 127);
  return e < -40 ? -40 : (e > 40 ? 40 : e);
}
// Exponent k with max |mult| 2^k in [1/2, 1) (multbits: the largest |mult| as float bits, or 0).
__device__ __forceinline__ int mult_exp(const int* multbits) {
  if (!multbits) return 0;
  const int mb = *multbits;
  if (mb <= 0 || mb >= 0x7f800000) return 0;
  const int k = -(((mb >> 23) & 255) - 127) - 1;
  return k < -120 ? -120 : (k > 120 ? 120 : k);
}

__global__ void k_mult_max(const float* __restrict__ mk, int n, int* multbits) {
  float mx = 0.f;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) mx = fmaxf(mx, fabsf(mk[j]));
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0 && mx > 0.f) atomicMax(multbits, __float_as_int(mx));
}

// Z^T operand of the key cloud: per 128-key tile a [dim16 x 256] FP16 block in
// the canonical K-major layout (row d: the hi parts of the tile's keys, then
// their lo parts), mult_j (y_j - c) 2^(e + k); keys past nk (and, without mk,
// zero-weight keys) are zero.
__global__ void k_zt_operand(const float* __restrict__ kp, int nk, int TT, int dim, int dim16,
                             const float* __restrict__ center, const int* __restrict__ maxbits,
                             const float* __restrict__ l2w, const float* __restrict__ mk,
                             const int* __restrict__ multbits, __half* __restrict__ zt) {
  const int sbo = kZK * 16;
  const size_t tile_bytes = (size_t)(dim16 / 8) * sbo;
  const float sc = p2f(coord_exp(maxbits) + mult_exp(mk ? multbits : nullptr));
  const long long total = (long long)TT * kKeys * dim16;
  for (long long u = (long long)blockIdx.x * blockDim.x + threadIdx.x; u < total;
       u += (long long)gridDim.x * blockDim.x) {
    const int j = (int)(u / dim16), d = (int)(u - (long long)j * dim16);
    float v = 0.f;
    if (j < nk && d < dim) {
      const float mult = mk ? mk[j] : (l2w[j] > 0.5f * kZeroW ? 1.f : 0.f);
      v = mult * ((kp[(size_t)j * dim + d] - center[d]) * sc);
    }
    const __half hi = __float2half_rn(v), lo = __float2half_rn(v - __half2float(hi));
    char* tb = reinterpret_cast<char*>(zt) + (size_t)(j / kKeys) * tile_bytes;
    const int kk = j % kKeys;
    *reinterpret_cast<__half*>(tb + kmajor_off(d, kk, sbo)) = hi;
    *reinterpret_cast<__half*>(tb + kmajor_off(d, kKeys + kk, sbo)) = lo;
  }
}

struct MBars {
  uint64_t a_full;
  uint64_t b_full[kStages];   // key tile landed
  uint64_t z_full[kStages];   // Z^T tile landed
  uint64_t s_done[2];         // S MMAs of an accumulator completed
  uint64_t s_empty[2];        // the consumers read an S accumulator
  uint64_t p_full;            // the consumers wrote P
  uint64_t o_done[2];         // O MMAs of a pass-2 tile completed (by parity of the pass-2 count)
  uint64_t a_free;            // the S MMAs of a row block's last job completed (A may be replaced)
  uint64_t b_free[kStages];   // the S MMAs that read a key stage completed
  uint64_t z_free[kStages];   // the O MMAs that read a Z^T stage completed
  uint32_t tmem;
  int err;
  float hq[3][kRows];         // column quarters 1..3 of a row: maxima, then sums
};

__device__ __forceinline__ void copy_pieces(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  tc::mbar_arrive_expect_tx(bar, bytes);
  for (uint32_t o = 0; o < bytes; o += kPiece) {
    const uint32_t len = bytes - o < kPiece ? bytes - o : kPiece;
    tc::bulk_g2s(static_cast<char*>(dst) + o, static_cast<const char*>(src) + o, len, bar);
  }
}

__host__ __device__ __forceinline__ long long cta_of_unit(long long x, long long U, long long G) {
  return ((x + 1) * G + U - 1) / U - 1;
}

// Job table of a CTA: its units in order, each row-block segment twice (pass 1
// then pass 2).  jt: key tile, jf: flags (bit 0 pass 2, bit 1 last job of its
// pass in the segment, bit 2 first job of the segment, bit 3 the segment holds
// the row block's last tile), js: the unit's H slot, jr: row block.
struct Jobs {
  short jt[64], js[64], jr[64];
  unsigned char jf[64];
  short ztile[32];  // key tile of the n-th pass-2 job
  int njobs, npass2;
};

template <int KS>
__global__ void __launch_bounds__(kAllThreads, 1)
k_sweep_umma_mom(const __half* __restrict__ opq, const float* __restrict__ nq2, int nq, const __half* __restrict__ opk,
                 const float* __restrict__ nk2, int nk, const __half* __restrict__ zt, const float* __restrict__ q,
                 const float* __restrict__ center, int dim, const int* __restrict__ maxbits,
                 const int* __restrict__ multbits, const float* __restrict__ l2w, const float* __restrict__ pot,
                 const double* __restrict__ shift, const float* __restrict__ zrow, const float* __restrict__ hk,
                 const float* __restrict__ mk, double s, float momscale, int TT, int splits, float* __restrict__ part,
                 long long spin, int* __restrict__ status) {
  extern __shared__ __align__(1024) unsigned char smraw[];
  constexpr int dim16 = 16 * KS;
  constexpr int KA = 2 * dim16;
  const uint32_t sbo = (uint32_t)KA * 16u, sboZ = (uint32_t)kZK * 16u;
  const uint32_t bytesA = 16u * sbo, bytesB = (uint32_t)(kKeys / 8) * sbo, bytesZ = (uint32_t)(dim16 / 8) * sboZ;
  unsigned char* A = smraw;
  unsigned char* B = A + bytesA;                   // [kStages][bytesB]
  unsigned char* Z = B + kStages * bytesB;         // [kStages][bytesZ]
  float* Hs = reinterpret_cast<float*>(Z + kStages * bytesZ);
  float* Ms = Hs + kMaxChunk;
  MBars& br = *reinterpret_cast<MBars*>(Ms + kMaxChunk);
  Jobs& jb = *reinterpret_cast<Jobs*>(&br + 1);
  float* hq4 = reinterpret_cast<float*>(&jb + 1);  // [4][kRows]
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const long long U = (long long)((nq + kRows - 1) / kRows) * TT, G = gridDim.x;
  const long long u0 = (long long)blockIdx.x * U / G, u1 = ((long long)blockIdx.x + 1) * U / G;
  const int L = (int)(u1 - u0);
  const int t0 = (int)(u0 % TT);
  const int nslot = L < TT ? L : TT;
  const int ce = coord_exp(maxbits), ke = mult_exp(mk ? multbits : nullptr);
  const float s2 = (float)(2.0 * s) * p2f(-ce) * p2f(-ce);  // S carries 2^2e
  const float osc = p2f(-ce - ke);                           // O carries 2^(e + k)
  const double sh = shift ? *shift : 0.0;

  if (warp == 0) tc::tmem_alloc(&br.tmem, kTmemCols);
  if (tid == 32 * kConsWarps) {
    // job table
    int j = 0, np = 0, t = 0;
    while (t < L) {
      const int rb = (int)((u0 + t) / TT), ta = (int)((u0 + t) % TT);
      const int n = (L - t) < (TT - ta) ? (L - t) : (TT - ta);
      for (int pass = 0; pass < 2; ++pass)
        for (int k = 0; k < n; ++k, ++j) {
          jb.jt[j] = (short)(ta + k);
          jb.js[j] = (short)((t + k) % TT);
          jb.jr[j] = (short)rb;
          jb.jf[j] = (unsigned char)(pass | (k == n - 1 ? 2 : 0) | (pass == 0 && k == 0 ? 4 : 0) |
                                     (ta + n == TT ? 8 : 0));
          if (pass == 1) jb.ztile[np++] = (short)(ta + k);
        }
      t += n;
    }
    jb.njobs = j;
    jb.npass2 = np;
    tc::mbar_init(&br.a_full, 1);
    for (int b = 0; b < kStages; ++b) {
      tc::mbar_init(&br.b_full[b], 1);
      tc::mbar_init(&br.z_full[b], 1);
    }
    for (int b = 0; b < 2; ++b) {
      tc::mbar_init(&br.s_done[b], 1);
      tc::mbar_init(&br.s_empty[b], kConsWarps);
      tc::mbar_init(&br.o_done[b], 1);
    }
    tc::mbar_init(&br.p_full, kConsWarps);
    tc::mbar_init(&br.a_free, 1);
    for (int b = 0; b < kStages; ++b) {
      tc::mbar_init(&br.b_free[b], 1);
      tc::mbar_init(&br.z_free[b], 1);
    }
    tc::fence_mbar_init();
    br.err = 0;
  }
  // key constants and multipliers of the CTA's key tiles (zero weight and padding: kZeroW, 0), in
  // float pairs (about 44 bits, rounded once to FP32; FP64 here is slow on this GPU)
  // (all of a thread's loads are issued before any is used: one L2 round trip, not one a key)
  {
    const ffl::ff s_ff = ffl::from_double(s), sh_ff = ffl::from_double(sh);
    constexpr int kPer = (kMaxChunk + kAllThreads - 1) / kAllThreads;
    const int nu = nslot * kKeys;
    float hw[kPer], pj[kPer], n2[kPer], mm[kPer];
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
      const int u = tid + k * kAllThreads;
      const int j = ((t0 + u / kKeys) % TT) * kKeys + u % kKeys;
      const bool in = u < nu && j < nk;
      hw[k] = in ? (hk ? hk[j] : l2w[j]) : kZeroW;  // hk_j, or log2 w_j
      pj[k] = (in && !hk && pot) ? pot[j] : 0.f;
      n2[k] = in ? nk2[j] : 0.f;
      mm[k] = (in && mk) ? mk[j] : 1.f;
    }
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
      const int u = tid + k * kAllThreads;
      if (u < nu) {
        const int j = ((t0 + u / kKeys) % TT) * kKeys + u % kKeys;
        float H = kZeroW, m = 0.f;
        if (j < nk) {
          const ffl::ff sn = ffl::neg(ffl::mul(s_ff, n2[k]));
          if (hk) {
            const ffl::ff h = ffl::add(ffl::mul(s_ff, hw[k]), sn);
            H = h.hi + h.lo;
            m = mm[k];
          } else if (hw[k] > 0.5f * kZeroW) {
            const ffl::ff sp = ffl::mul(ffl::add(sh_ff, pj[k]), s_ff);
            const ffl::ff h = ffl::add(ffl::add(sp, sn), hw[k]);
            H = h.hi + h.lo;
            m = mm[k];
          }
        }
        Hs[u] = H;
        Ms[u] = m;
      }
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = br.tmem;
  volatile int* err = &br.err;
  const int NJ = jb.njobs;

  if (warp == kCopyWarp) {
    // --------------------------------------------------------------- producer
    // (copies in job order: job j's query block, key tile and, in pass 2, Z^T tile, each once the
    // MMAs that read its buffer before have completed; all of those belong to earlier jobs)
    if (lane == 0) {
      int b_arm[kStages] = {}, z_arm[kStages] = {};
      int a_arm = 0, nfree = 0, np = 0;
      for (int j = 0; j < NJ && !*err; ++j) {
        const bool pass2 = jb.jf[j] & 1;
        bool ok = true;
        if (j == 0 || jb.jr[j] != jb.jr[j - 1]) {
          if (j > 0) {
            ok = tc::mbar_wait(&br.a_free, (uint32_t)(nfree & 1), spin);
            ++nfree;
          }
          if (!ok) { *err = 1; break; }
          copy_pieces(A, reinterpret_cast<const char*>(opq) + (size_t)jb.jr[j] * bytesA, bytesA, &br.a_full);
          ++a_arm;
        }
        {
          const int st = j % kStages;
          if (j >= kStages && !tc::mbar_wait(&br.b_free[st], (uint32_t)(((j - kStages) / kStages) & 1), spin)) {
            *err = 1;
            break;
          }
          copy_pieces(B + (size_t)st * bytesB, reinterpret_cast<const char*>(opk) + (size_t)jb.jt[j] * bytesB, bytesB,
                      &br.b_full[st]);
          ++b_arm[st];
        }
        if (pass2) {
          const int zs = np % kStages;
          if (np >= kStages && !tc::mbar_wait(&br.z_free[zs], (uint32_t)(((np - kStages) / kStages) & 1), spin)) {
            *err = 1;
            break;
          }
          copy_pieces(Z + (size_t)zs * bytesZ, reinterpret_cast<const char*>(zt) + (size_t)jb.ztile[np] * bytesZ,
                      bytesZ, &br.z_full[zs]);
          ++z_arm[zs];
          ++np;
        }
      }
      // this role's copies land before the CTA ends, whoever stopped (each barrier's latest phase; bounded)
      if (a_arm > 0) (void)tc::mbar_wait(&br.a_full, (uint32_t)((a_arm - 1) & 1), kSpin);
      for (int st = 0; st < kStages; ++st) {
        if (b_arm[st] > 0) (void)tc::mbar_wait(&br.b_full[st], (uint32_t)((b_arm[st] - 1) & 1), kSpin);
        if (z_arm[st] > 0) (void)tc::mbar_wait(&br.z_full[st], (uint32_t)((z_arm[st] - 1) & 1), kSpin);
      }
    }
    __syncwarp();
  } else if (warp == kMmaWarp) {
    // -------------------------------------------------------------------- MMA
    if (lane == 0) {
      int a_use = 0, s_commit = -1, o_commit = -1;
      const uint64_t dAh = tc::smem_desc(tc::smem_addr(A), 128, sbo);
      const uint64_t dAl = dAh + (uint64_t)(KS * 16);
      const uint32_t idS = tc::idesc_f16(kRows, kKeys), idO = tc::idesc_f16(kRows, dim16);
      int np = 0;
      for (int j = 0; j < NJ && !*err; ++j) {
        const int st = j % kStages, b = j % 2;
        const bool pass2 = jb.jf[j] & 1;
        bool ok = true;
        if (j == 0 || jb.jr[j] != jb.jr[j - 1]) {
          ok = tc::mbar_wait(&br.a_full, (uint32_t)(a_use & 1), spin);
          ++a_use;
        }
        ok = ok && tc::mbar_wait(&br.b_full[st], (uint32_t)((j / kStages) & 1), spin);
        ok = ok && (j < 2 || tc::mbar_wait(&br.s_empty[b], (uint32_t)(((j - 2) / 2) & 1), spin));
        if (!ok) { *err = 1; break; }
        tc::fence_after_sync();
        {
          const uint32_t d = tmem + kColS + (uint32_t)(b * kKeys);
          const uint64_t dBh = tc::smem_desc(tc::smem_addr(B + (size_t)st * bytesB), 128, sbo);
          const uint64_t dBl = dBh + (uint64_t)(KS * 16);
#pragma unroll
          for (int k = 0; k < KS; ++k) tc::mma_f16(d, dAh + 16 * k, dBh + 16 * k, idS, k > 0);
#pragma unroll
          for (int k = 0; k < KS; ++k) tc::mma_f16(d, dAl + 16 * k, dBh + 16 * k, idS, true);
#pragma unroll
          for (int k = 0; k < KS; ++k) tc::mma_f16(d, dAh + 16 * k, dBl + 16 * k, idS, true);
          tc::commit(&br.s_done[b]);
          tc::commit(&br.b_free[st]);
          if (j == NJ - 1 || jb.jr[j + 1] != jb.jr[j]) tc::commit(&br.a_free);
          s_commit = j;
        }
        if (pass2) {
          const int zs = np % kStages;
          ok = tc::mbar_wait(&br.z_full[zs], (uint32_t)((np / kStages) & 1), spin);
          ok = ok && tc::mbar_wait(&br.p_full, (uint32_t)(np & 1), spin);
          if (!ok) { *err = 1; break; }
          tc::fence_after_sync();
          const bool first = (j == 0) || !(jb.jf[j - 1] & 1);  // first pass-2 job of the segment
          const uint32_t d = tmem + kColO;
          const uint64_t dZh = tc::smem_desc(tc::smem_addr(Z + (size_t)zs * bytesZ), 128, sboZ);
          const uint64_t dZl = dZh + (uint64_t)(kKeys / 8 * 8);  // lo parts: kKeys keys further (16 B units)
#pragma unroll
          for (int k = 0; k < kKeys / 16; ++k)
            tc::mma_f16_tmem_a(d, tmem + kColPh + 8 * k, dZh + 16 * k, idO, !(first && k == 0));
#pragma unroll
          for (int k = 0; k < kKeys / 16; ++k) tc::mma_f16_tmem_a(d, tmem + kColPl + 8 * k, dZh + 16 * k, idO, true);
#pragma unroll
          for (int k = 0; k < kKeys / 16; ++k) tc::mma_f16_tmem_a(d, tmem + kColPh + 8 * k, dZl + 16 * k, idO, true);
          tc::commit(&br.o_done[np % 2]);
          tc::commit(&br.z_free[zs]);
          o_commit = np;
          ++np;
        }
      }
      // the MMAs committed complete before the CTA ends, whoever stopped (the latest phase of each
      // barrier; immediate when the consumers saw them; bounded)
      for (int j = s_commit - 1; j <= s_commit; ++j)
        if (j >= 0) (void)tc::mbar_wait(&br.s_done[j % 2], (uint32_t)((j / 2) & 1), kSpin);
      for (int n = o_commit - 1; n <= o_commit; ++n)
        if (n >= 0) (void)tc::mbar_wait(&br.o_done[n % 2], (uint32_t)((n / 2) & 1), kSpin);
    }
    __syncwarp();
  } else {
    // --------------------------------------------------------------- consumers
    const int qd = warp & 3, h = warp >> 2;  // TMEM lane quarter, key quarter
    const int row = 32 * qd + lane;
    const uint32_t lane_base = tmem + ((uint32_t)(32 * qd) << 16);
    float M = kInitMax, acc = 0.f;
    bool dead = false;  // warp-uniform: a wait gave up, the remaining jobs are skipped
    int np = 0;
    const int CH = 2 + dim;
    for (int j = 0; j < NJ; ++j) {
      const int b = j % 2;
      const unsigned f = jb.jf[j];
      const bool pass2 = f & 1, last = f & 2;
      if (!dead) {
        bool done = !*err && tc::mbar_wait(&br.s_done[b], (uint32_t)((j / 2) & 1), spin);
        done = __all_sync(0xffffffffu, done);  // tcgen05.ld is warp-wide
        if (!done) {
          if (lane == 0) *err = 1;
          dead = true;
        }
      }
      float v[32];
      if (!dead) {
        tc::fence_after_sync();
        tc::ld32(lane_base + kColS + (uint32_t)(b * kKeys) + (uint32_t)(32 * h), v);
        tc::fence_before_sync();
        __syncwarp();
        if (lane == 0) tc::mbar_arrive(&br.s_empty[b]);
        const float* H = Hs + jb.js[j] * kKeys + 32 * h;
#pragma unroll
        for (int e = 0; e < 32; ++e) v[e] = fmaf(s2, v[e], H[e]);
      }
      if (!pass2) {
        if (!dead) {
#pragma unroll
          for (int e = 0; e < 32; ++e) M = fmaxf(M, v[e]);
        }
        if (last) {
          // the row's maximum over the four key quarters, on every one of them
          hq4[h * kRows + row] = M;
          asm volatile("bar.sync 1, %0;" ::"n"(32 * kConsWarps) : "memory");
          M = fmaxf(fmaxf(hq4[row], hq4[kRows + row]), fmaxf(hq4[2 * kRows + row], hq4[3 * kRows + row]));
          asm volatile("bar.sync 1, %0;" ::"n"(32 * kConsWarps) : "memory");
        }
        continue;
      }
      // pass 2: P = 2^(t - M) <= 1 into TMEM (hi and lo FP16 parts), value sums
      if (!dead) {
        const float* Mu = Ms + jb.js[j] * kKeys + 32 * h;
        uint32_t ph[16], pl[16];
#pragma unroll
        for (int w = 0; w < 16; ++w) {
          const float p0 = ex2f(v[2 * w] - M), p1 = ex2f(v[2 * w + 1] - M);
          acc = fmaf(Mu[2 * w], p0, fmaf(Mu[2 * w + 1], p1, acc));
          const __half h0 = __float2half_rn(p0), h1 = __float2half_rn(p1);
          const __half l0 = __float2half_rn(p0 - __half2float(h0)), l1 = __float2half_rn(p1 - __half2float(h1));
          ph[w] = (uint32_t)__half_as_ushort(h0) | ((uint32_t)__half_as_ushort(h1) << 16);
          pl[w] = (uint32_t)__half_as_ushort(l0) | ((uint32_t)__half_as_ushort(l1) << 16);
        }
        // the O MMAs of the previous pass-2 job read P: wait for them
        bool ok = np == 0 || tc::mbar_wait(&br.o_done[(np - 1) % 2], (uint32_t)(((np - 1) / 2) & 1), spin);
        ok = __all_sync(0xffffffffu, ok && !*err);
        if (!ok) {
          if (lane == 0) *err = 1;
          dead = true;
        } else {
          tc::fence_after_sync();
          tc::st16(lane_base + kColPh + (uint32_t)(16 * h), ph);
          tc::st16(lane_base + kColPl + (uint32_t)(16 * h), pl);
          tc::fence_before_sync();
          __syncwarp();
          if (lane == 0) tc::mbar_arrive(&br.p_full);
        }
      }
      if (last) {
        // end of this CTA's part of the row block: O, the value sums of the four quarters, the partials
        float o[4 * KS];
        if (!dead) {
          bool ok = tc::mbar_wait(&br.o_done[np % 2], (uint32_t)((np / 2) & 1), spin);
          ok = __all_sync(0xffffffffu, ok && !*err);
          if (!ok) {
            if (lane == 0) *err = 1;
            dead = true;
          } else {
            tc::fence_after_sync();
#pragma unroll
            for (int c = 0; c < KS; ++c) {
              float t4[4];
              tc::ld4(lane_base + kColO + (uint32_t)(4 * KS * h + 4 * c), t4);
#pragma unroll
              for (int e = 0; e < 4; ++e) o[4 * c + e] = t4[e];
            }
            tc::fence_before_sync();
          }
        }
        hq4[h * kRows + row] = acc;
        asm volatile("bar.sync 1, %0;" ::"n"(32 * kConsWarps) : "memory");
        const float at = (hq4[row] + hq4[kRows + row]) + (hq4[2 * kRows + row] + hq4[3 * kRows + row]);
        asm volatile("bar.sync 1, %0;" ::"n"(32 * kConsWarps) : "memory");
        const int rb = jb.jr[j];
        const int i = rb * kRows + row;
        if (i < nq) {
          const int slot = (int)((long long)blockIdx.x - cta_of_unit((long long)rb * TT, U, G));
          float* base = part + (size_t)slot * CH * nq;
          const bool bad = *err != 0;
          const float nan = __int_as_float(0x7fc00000);
          if (h == 0) {
            const float Rr = -(float)s * nq2[i] + (zrow ? (float)s * zrow[i] : 0.f);
            base[i] = bad ? nan : M + Rr;
            base[(size_t)nq + i] = bad ? nan : at;
          }
#pragma unroll
          for (int c = 0; c < 4 * KS; ++c) {
            const int d = 4 * KS * h + c;
            if (d < dim) {
              const float xd = q[(size_t)i * dim + d] - center[d];
              base[(size_t)(2 + d) * nq + i] = bad ? nan : momscale * fmaf(xd, at, -o[c] * osc);
            }
          }
          if (f & 8)
            for (int k = slot + 1; k < splits; ++k) {
              float* e = part + (size_t)k * CH * nq;
              if (h == 0) { e[i] = kInitMax; e[(size_t)nq + i] = 0.f; }
              for (int c = 0; c < 4 * KS; ++c) {
                const int d = 4 * KS * h + c;
                if (d < dim) e[(size_t)(2 + d) * nq + i] = 0.f;
              }
            }
        }
        M = kInitMax;
        acc = 0.f;
      }
      if (pass2) ++np;
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, kTmemCols);
  if (tid == 0 && br.err && status) atomicOr(status, kStatusTimeout);
}

size_t mom_smem_bytes(int dim16) {
  const size_t KA = 2 * (size_t)dim16;
  const size_t bytesA = 16 * KA * 16, bytesB = (kKeys / 8) * KA * 16, bytesZ = (size_t)(dim16 / 8) * kZK * 16;
  return bytesA + kStages * (bytesB + bytesZ) + 2 * sizeof(float) * kMaxChunk + sizeof(MBars) + sizeof(Jobs) +
         sizeof(float) * 4 * kRows + 64;
}

template <int KS>
cudaError_t run_mom(const __half* opq, const float* nq2, int nq, const __half* opk, const float* nk2, int nk,
                    const __half* zt, const float* q, const float* center, int dim, const int* maxbits,
                    const int* multbits, const float* l2w, const float* pot, const double* shift, const float* zrow,
                    const float* hk, const float* mk, double s, float momscale, float* part, const SweepGeom& g,
                    int* status, cudaStream_t st) {
  const size_t smem = mom_smem_bytes(16 * KS);
  static std::mutex mu;
  static bool attr = false;
  {
    std::lock_guard<std::mutex> lk(mu);
    if (!attr) {
      cudaError_t e = cudaFuncSetAttribute(k_sweep_umma_mom<KS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
      attr = true;
    }
  }
  const int TT = (nk + kKeys - 1) / kKeys;
  k_sweep_umma_mom<KS><<<g.ctas, kAllThreads, smem, st>>>(opq, nq2, nq, opk, nk2, nk, zt, q, center, dim, maxbits,
                                                          multbits, l2w, pot, shift, zrow, hk, mk, s, momscale, TT,
                                                          g.splits, part, wait_limit(), status);
  note_launch();
  return cudaGetLastError();
}

}  // namespace

size_t mom_zt_bytes(int n, int dim) {
  const int dim16 = (dim + 15) & ~15;
  const size_t TT = ((size_t)n + kKeys - 1) / kKeys;
  return TT * (size_t)(dim16 / 8) * kZK * 16;
}

SweepGeom mom_geom(int nq, int nk) {
  SweepGeom g{};
  g.threads = kAllThreads;
  g.rows = 1;
  g.row_blocks = (nq + kRows - 1) / kRows;
  const long long TT = (nk + kKeys - 1) / kKeys;
  g.keys_per_split = (int)TT * kKeys;
  // the (row block, key tile) units spread evenly over one CTA per SM (a multiple of the SM
  // count when a CTA would otherwise hold more than kMaxChunk keys)
  const long long U = (long long)g.row_blocks * TT;
  const long long sms = device_sm_count(), per = kMaxChunk / kKeys;
  long long G = sms * ((U + sms * per - 1) / (sms * per));
  if (G > U) G = U;
  g.ctas = (int)G;
  // partial slots: the CTAs one row block's TT units are spread over
  const long long lmin = U / G;
  long long splits = TT < 2 ? 1 : 2 + (TT - 2) / lmin;
  if (splits > G) splits = G;
  g.splits = (int)splits;
  return g;
}

// Moment sweep on tcgen05: opq / nq2 and opk / nk2 are the plain sweep's
// operands and squared norms of the query and key clouds, zt (mom_zt_bytes of
// the key cloud) and multbits (one int) scratch for the Z^T operand.
cudaError_t launch_mom_sweep(const void* opq, const float* nq2, int nq, const void* opk, const float* nk2, int nk,
                             const float* q, const float* kp, int dim, const float* center, const int* maxbits,
                             const float* l2w, const float* pot, const double* shift, const float* zrow,
                             const float* hk, const float* mk, double s, float momscale, void* zt, int* multbits,
                             float* part, const SweepGeom& g, int* status, cudaStream_t st) {
  if (dim < 17 || dim > 64) return cudaErrorInvalidValue;
  const int dim16 = (dim + 15) & ~15, KS = dim16 / 16;
  const int TT = (nk + kKeys - 1) / kKeys;
  const int sms = device_sm_count();
  if (mk) {
    cudaError_t e = cudaMemsetAsync(multbits, 0, sizeof(int), st);
    if (e != cudaSuccess) return e;
    int blocks = (nk + 255) / 256;
    if (blocks > 4 * sms) blocks = 4 * sms;
    k_mult_max<<<blocks, 256, 0, st>>>(mk, nk, multbits);
    note_launch();
  }
  {
    const long long total = (long long)TT * kKeys * dim16;
    long long blocks = (total + 255) / 256;
    if (blocks > 8LL * sms) blocks = 8LL * sms;
    k_zt_operand<<<(int)blocks, 256, 0, st>>>(kp, nk, TT, dim, dim16, center, maxbits, l2w, mk, multbits,
                                              static_cast<__half*>(zt));
    note_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  const __half* A = static_cast<const __half*>(opq);
  const __half* Bk = static_cast<const __half*>(opk);
  const __half* Z = static_cast<const __half*>(zt);
  switch (KS) {
    case 2: return run_mom<2>(A, nq2, nq, Bk, nk2, nk, Z, q, center, dim, maxbits, multbits, l2w, pot, shift, zrow, hk, mk, s, momscale, part, g, status, st);
    case 3: return run_mom<3>(A, nq2, nq, Bk, nk2, nk, Z, q, center, dim, maxbits, multbits, l2w, pot, shift, zrow, hk, mk, s, momscale, part, g, status, st);
    default: return run_mom<4>(A, nq2, nq, Bk, nk2, nk, Z, q, center, dim, maxbits, multbits, l2w, pot, shift, zrow, hk, mk, s, momscale, part, g, status, st);
  }
}

}  // namespace uot
