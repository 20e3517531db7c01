// Softmin sweep for high-dimensional point clouds (dim >= 32, p = 2) on the
// fifth-generation tensor cores (tcgen05, accumulators in TMEM):
//
//   t_ij = h_j - s |x_i - y_j|^2 = H_j + R_i + 2 s x'_i . y'_j,
//   x' = x - c, y' = y - c (c the clouds' common centre),
//   H_j = h_j - s |y'_j|^2,  R_i = -s |x'_i|^2,
//
// with the dot products x'.y' a dense (rows x dim) x (dim x keys)
// contraction.  Each coordinate, scaled by a power of two 2^e common to both
// clouds (so that the largest is below 2^15), is split into FP16 parts
// hi + lo, and the product is hi.hi + lo.hi + hi.lo (three kind::f16 MMA
// passes with FP32 accumulation; hi and lo carry 11 significant bits each,
// the dropped lo.lo is below 2^-22 of |x'||y'|), rescaled by 2^-2e.  The
// split operands of both clouds are built once per call in the canonical
// K-major layout (8-row x 16-byte core matrices, no swizzle), so that a tile
// of 8k rows is one contiguous block: a CTA copies its 128 query rows and
// each 256-key tile into shared memory with bulk asynchronous copies
// completing on mbarriers (two key stages); one lane issues the MMAs of a
// tile (N = 256) into a pair of TMEM accumulators while sixteen consumer warps read
// the earlier ones (four threads per row, one per column quarter; tcgen05.ld), add
// H_j and keep a running (max, sum of 2^(t - max)) per row.  Output: the
// (max + R_i, sum) partials per (row, key chunk) of the other sweeps.  The
// grid holds one CTA per SM, each taking an equal contiguous range of the
// (row block, key tile) units, so that no SM idles when the row blocks do
// not divide the SM count.
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

constexpr int kRows = 128;                    // MMA M
constexpr int kKeys = 256;                    // MMA N (keys per tile)
constexpr int kPad = 256;                     // operand rows padded to a multiple of this
constexpr int kStages = 2;                    // key-tile buffers
constexpr int kAccCols = kKeys;               // TMEM columns per accumulator (N fp32)
constexpr int kAcc = 2;                       // accumulators in TMEM (a ring)
constexpr int kTmemCols = kAcc * kAccCols;
constexpr int kMaxChunk = 4096;               // keys per CTA (H_j kept in shared memory)
constexpr long long kSpin = kWaitPolls;       // drain waits: mbarrier polls before giving up
constexpr uint32_t kIdesc = tc::idesc_f16(kRows, kKeys);  // N = 256, the largest for M = 128
constexpr uint32_t kPiece = 65536;            // bytes per bulk copy
constexpr size_t kOneCtaSmem = 120 * 1024;

// Byte offset of element (r, k) of a 2-byte K-major operand with SBO bytes
// between 8-row groups: core matrices of 8 rows x 8 elements, 128 bytes each.
__host__ __device__ constexpr int kmajor_offset_h(int r, int k, int sbo) {
  return (r >> 3) * sbo + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2;
}

// 2^e as a float / double (|e| well inside the normal range).
__device__ __forceinline__ float pow2f(int e) { return __int_as_float((127 + e) << 23); }
__device__ __forceinline__ double pow2d(int e) { return __longlong_as_double((long long)(1023 + e) << 52); }

// Scale exponent e of the split: the largest |x - c| (its bit pattern, a
// non-negative float) times 2^e lies in [2^14, 2^15); e within [-40, 40].
__device__ __forceinline__ int scale_exp(int maxbits) {
  if (maxbits <= 0) return 0;
  const int E = ((maxbits >> 23) & 255) - 127;
  const int e = 14 - E;
  return e < -40 ? -40 : (e > 40 ? 40 : e);
}

// Largest |x_rd - c_d| over both clouds, as the bit pattern of a non-negative
// float (ordered like the value) in *maxbits (zeroed by the caller).
__global__ void k_umma_maxabs(const float* __restrict__ x, int n, const float* __restrict__ y, int m, int dim,
                              const float* __restrict__ center, int* maxbits) {
  float mx = 0.f;
  const long long tx = (long long)n * dim, total = tx + (long long)m * dim;
  for (long long u = (long long)blockIdx.x * blockDim.x + threadIdx.x; u < total;
       u += (long long)gridDim.x * blockDim.x) {
    const float v = u < tx ? x[u] - center[u % dim] : y[u - tx] - center[(u - tx) % dim];
    mx = fmaxf(mx, fabsf(v));
  }
  for (int off = 16; off > 0; off >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, off));
  if ((threadIdx.x & 31) == 0 && mx > 0.f) atomicMax(maxbits, __float_as_int(mx));
}

// Operand matrix of one cloud: row r, the split scaled coordinates of r - c as
// [hi (dim16) | lo (dim16)] FP16 in the canonical K-major layout, KA = 2 dim16
// values a row, rows padded with zeros to a multiple of 256; norm2[r] = |w_r|^2
// with w = (hi + lo) 2^-e, the coordinates the products see.
__global__ void k_umma_operand(const float* __restrict__ pts, int n, int npad, int dim, int dim16,
                               const float* __restrict__ center, const int* __restrict__ maxbits,
                               __half* __restrict__ op, float* __restrict__ norm2) {
  const int KA = 2 * dim16;
  const int sbo = KA * 16;
  const int e = scale_exp(*maxbits);
  const float sc = pow2f(e), isc = pow2f(-e);
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < npad; r += gridDim.x * blockDim.x) {
    float acc = 0.f;
    for (int d0 = 0; d0 < dim16; d0 += 8) {
      __align__(16) __half hi[8];
      __align__(16) __half lo[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int d = d0 + j;
        const float v = (r < n && d < dim) ? (pts[(size_t)r * dim + d] - center[d]) * sc : 0.f;
        hi[j] = __float2half_rn(v);
        lo[j] = __float2half_rn(v - __half2float(hi[j]));
        const float w = (__half2float(hi[j]) + __half2float(lo[j])) * isc;
        acc = fmaf(w, w, acc);
      }
      char* base = reinterpret_cast<char*>(op);
      *reinterpret_cast<uint4*>(base + kmajor_offset_h(r, d0, sbo)) = *reinterpret_cast<const uint4*>(hi);
      *reinterpret_cast<uint4*>(base + kmajor_offset_h(r, dim16 + d0, sbo)) = *reinterpret_cast<const uint4*>(lo);
    }
    if (r < n) norm2[r] = acc;
  }
}

struct Bars {
  uint64_t a_full;
  uint64_t a_free;            // the MMAs of a row block's last tile completed (A may be replaced)
  uint64_t b_full[kStages];   // key stage landed (bulk copies)
  uint64_t b_free[kStages];   // the MMAs that read a key stage completed
  uint64_t m_done[kAcc];      // the MMAs of an accumulator completed
  uint64_t empty[kAcc];       // the consumer warps read an accumulator
  uint32_t tmem;
  int err;
  float s_hi, s_lo, sh_hi, sh_lo, s2;  // s and the potential shift as float pairs; s 2^-2e
  float hm[2][3][kRows];      // column quarters 1..3: (max, sum) per row, by segment parity
  float hs[2][3][kRows];
};

__device__ __forceinline__ void copy_pieces(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  tc::mbar_arrive_expect_tx(bar, bytes);
  for (uint32_t o = 0; o < bytes; o += kPiece) {
    const uint32_t len = bytes - o < kPiece ? bytes - o : kPiece;
    tc::bulk_g2s(static_cast<char*>(dst) + o, static_cast<const char*>(src) + o, len, bar);
  }
}

// First CTA whose unit range [c U / G, (c + 1) U / G) holds unit x.
__host__ __device__ __forceinline__ long long cta_of_unit(long long x, long long U, long long G) {
  return ((x + 1) * G + U - 1) / U - 1;
}

// Roles: warps 0..15 read the accumulators (warp w: TMEM lane quarter w % 4,
// i.e. rows 32 (w % 4) .. + 31, and column quarter w / 4 of every tile, one
// 64-column TMEM load a tile); lane 0 of warp 16 issues the MMAs; lane 0 of
// warp 17 issues the copies.  Handoffs: a_full / b_full (query rows / key
// tile landed: producer -> MMA), a_free / b_free (the MMAs that read them
// completed: MMA -> producer, which refills them), m_done (MMAs ->
// consumers), empty (consumers -> MMA, accumulator free again).  The two
// single-thread roles are kept apart so that neither waits behind the other's
// waits.  Every wait is bounded; a wait that gives up sets err, which stops
// every role, and each issuing role then lets its own copies or MMAs in flight
// land before the CTA ends.
constexpr int kConsWarps = 16;
constexpr int kMmaWarp = kConsWarps, kCopyWarp = kConsWarps + 1;
constexpr int kAllThreads = 32 * (kConsWarps + 2);

// Work units are the pairs (row block of 128 queries, key tile of 256 keys),
// numbered row-block-major, U = row blocks x TT of them; CTA c of the G in
// the grid takes the contiguous units [c U / G, (c + 1) U / G), at most
// kMaxChunk / kKeys of them.  A row block's units are split over consecutive
// CTAs; the k-th of them writes its (max, sum) partials to slot k of part, and
// the last one fills the slots it leaves unused with (kInitMax, 0), which the
// merge ignores.  KS = dim16 / 16 MMA K-steps per pass.
template <int KS>
__global__ void __launch_bounds__(kAllThreads, 1)
k_sweep_umma(const __half* __restrict__ opq, const float* __restrict__ nq2, int nq, const __half* __restrict__ opk,
             const float* __restrict__ nk2, int nk, const float* __restrict__ l2w, const float* __restrict__ pot,
             const double* __restrict__ shift, double s, const int* __restrict__ maxbits, int TT, int splits,
             float* __restrict__ part, long long spin, int* __restrict__ status) {
  extern __shared__ __align__(1024) unsigned char smraw[];
  constexpr int dim16 = 16 * KS;
  constexpr int KA = 2 * dim16;  // FP16 values a row
  const uint32_t sbo = (uint32_t)KA * 16u;
  const uint32_t bytesA = 16u * sbo, bytesB = (uint32_t)(kKeys / 8) * sbo;
  unsigned char* A = smraw;
  unsigned char* B = smraw + bytesA;  // [kStages][kKeys x KA]
  float* Hs = reinterpret_cast<float*>(smraw + bytesA + kStages * bytesB);
  Bars& br = *reinterpret_cast<Bars*>(smraw + bytesA + kStages * bytesB + sizeof(float) * kMaxChunk);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const long long U = (long long)((nq + kRows - 1) / kRows) * TT, G = gridDim.x;
  const long long u0 = (long long)blockIdx.x * U / G, u1 = ((long long)blockIdx.x + 1) * U / G;
  const int L = (int)(u1 - u0);
  const int rb0 = (int)(u0 / TT), t0 = (int)(u0 % TT);
  // H slots: slot v holds key tile (t0 + v) % TT, and unit u0 + t reads slot t % TT
  const int nslot = L < TT ? L : TT;
  if (warp == 0) tc::tmem_alloc(&br.tmem, kTmemCols);
  if (tid == 32 * kMmaWarp) {
    tc::mbar_init(&br.a_full, 1);
    tc::mbar_init(&br.a_free, 1);
    for (int b = 0; b < kStages; ++b) {
      tc::mbar_init(&br.b_full[b], 1);
      tc::mbar_init(&br.b_free[b], 1);
    }
    for (int b = 0; b < kAcc; ++b) {
      tc::mbar_init(&br.m_done[b], 1);
      tc::mbar_init(&br.empty[b], kConsWarps);
    }
    tc::fence_mbar_init();
    br.err = 0;
    // the CTA's FP64 work (slow on this GPU), done once: s and the shift as float pairs
    const double sh = shift ? *shift : 0.0;
    br.s_hi = (float)s;
    br.s_lo = (float)(s - (double)br.s_hi);
    br.sh_hi = (float)sh;
    br.sh_lo = (float)(sh - (double)br.sh_hi);
    br.s2 = (float)(2.0 * s * pow2d(-2 * scale_exp(*maxbits)));  // products carry 2^2e
  }
  // key constants H_j = h_j - s |y'_j|^2 of the CTA's key tiles (zero-weight and padding keys: kZeroW),
  // in float pairs (about 44 bits, then rounded once to FP32); all of a thread's loads are issued
  // before the barrier, so that they take one L2 round trip
  constexpr int kPer = (kMaxChunk + kAllThreads - 1) / kAllThreads;
  const int nu = nslot * kKeys;
  float lw[kPer], pj[kPer], n2[kPer];
#pragma unroll
  for (int k = 0; k < kPer; ++k) {
    const int u = tid + k * kAllThreads;
    const int j = ((t0 + u / kKeys) % TT) * kKeys + u % kKeys;
    const bool in = u < nu && j < nk;
    lw[k] = in ? l2w[j] : kZeroW;
    pj[k] = (in && pot) ? pot[j] : 0.f;
    n2[k] = in ? nk2[j] : 0.f;
  }
  __syncthreads();  // barriers initialised, constants written
  if (tid == 32 * kCopyWarp) {
    // the first copies start before the key constants are computed
    copy_pieces(A, reinterpret_cast<const char*>(opq) + (size_t)rb0 * bytesA, bytesA, &br.a_full);
    for (int t = 0; t < L && t < kStages; ++t)
      copy_pieces(reinterpret_cast<char*>(B) + (size_t)t * bytesB,
                  reinterpret_cast<const char*>(opk) + (size_t)((t0 + t) % TT) * bytesB, bytesB, &br.b_full[t]);
  }
  {
    const ffl::ff s_ff{br.s_hi, br.s_lo}, sh_ff{br.sh_hi, br.sh_lo};
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
      const int u = tid + k * kAllThreads;
      if (u < nu) {
        float H = kZeroW;
        if (lw[k] > 0.5f * kZeroW) {
          const ffl::ff sp = ffl::mul(ffl::add(sh_ff, pj[k]), s_ff);
          const ffl::ff h = ffl::add(ffl::add(sp, ffl::neg(ffl::mul(s_ff, n2[k]))), lw[k]);
          H = h.hi + h.lo;
        }
        Hs[u] = H;
      }
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = br.tmem;
  const float s2 = br.s2, s_f = br.s_hi;
  volatile int* err = &br.err;

  if (warp == kCopyWarp) {
    // --------------------------------------------------------------- producer
    if (lane == 0) {
      int armed[kStages] = {}, a_armed = 1, nfree = 0;
      for (int t = 0; t < L && t < kStages; ++t) armed[t] = 1;
      int rb = rb0, tile = t0;
      for (int t = 1; t < L && !*err; ++t) {
        if (++tile == TT) { tile = 0; ++rb; }
        if (tile == 0) {
          // next row block: its rows replace A once the MMAs of the previous row block completed
          if (!tc::mbar_wait(&br.a_free, (uint32_t)(nfree & 1), spin)) { *err = 1; break; }
          ++nfree;
          copy_pieces(A, reinterpret_cast<const char*>(opq) + (size_t)rb * bytesA, bytesA, &br.a_full);
          ++a_armed;
        }
        if (t >= kStages) {
          // key tile t goes to stage t % kStages once the MMAs of tile t - kStages completed
          const int st = t % kStages;
          if (!tc::mbar_wait(&br.b_free[st], (uint32_t)(((t - kStages) / kStages) & 1), spin)) { *err = 1; break; }
          copy_pieces(reinterpret_cast<char*>(B) + (size_t)st * bytesB,
                      reinterpret_cast<const char*>(opk) + (size_t)((t0 + t) % TT) * bytesB, bytesB,
                      &br.b_full[st]);
          ++armed[st];
        }
      }
      // this role's copies land before the CTA ends, whoever stopped (each barrier's latest phase;
      // immediate when the MMAs consumed them; bounded)
      (void)tc::mbar_wait(&br.a_full, (uint32_t)((a_armed - 1) & 1), kSpin);
      for (int st = 0; st < kStages; ++st)
        if (armed[st] > 0) (void)tc::mbar_wait(&br.b_full[st], (uint32_t)((armed[st] - 1) & 1), kSpin);
    }
    __syncwarp();
  } else if (warp == kMmaWarp) {
    // -------------------------------------------------------------------- MMA
    if (lane == 0) {
      int committed = -1;
      // descriptors: one K-step (16 values: two 16-byte core-matrix columns, 256 bytes) adds 16 to the
      // start field, the lo parts start dim16 / 8 core-matrix columns (16 KS in the field) further
      const uint64_t dAh = tc::smem_desc(tc::smem_addr(A), 128, sbo);
      const uint64_t dAl = dAh + (uint64_t)(KS * 16);
      int tile = t0, a_used = 0;
      for (int t = 0; t < L && !*err; ++t) {
        const int st = t % kStages, b = t % kAcc;
        if (t > 0 && ++tile == TT) tile = 0;
        bool ok = true;
        if (t == 0 || tile == 0) {
          ok = tc::mbar_wait(&br.a_full, (uint32_t)(a_used & 1), spin);
          ++a_used;
        }
        ok = ok && tc::mbar_wait(&br.b_full[st], (uint32_t)((t / kStages) & 1), spin);
        // accumulator b was last read for tile t - kAcc
        ok = ok && (t < kAcc || tc::mbar_wait(&br.empty[b], (uint32_t)(((t - kAcc) / kAcc) & 1), spin));
        if (!ok) { *err = 1; break; }
        tc::fence_after_sync();
        const uint32_t d = tmem + (uint32_t)(b * kAccCols);
        const uint64_t dBh = tc::smem_desc(tc::smem_addr(reinterpret_cast<char*>(B) + (size_t)st * bytesB), 128, sbo);
        const uint64_t dBl = dBh + (uint64_t)(KS * 16);
        // hi.hi, then lo.hi (lo parts of x), then hi.lo (lo parts of y)
#pragma unroll
        for (int k = 0; k < KS; ++k) tc::mma_f16(d, dAh + 16 * k, dBh + 16 * k, kIdesc, k > 0);
#pragma unroll
        for (int k = 0; k < KS; ++k) tc::mma_f16(d, dAl + 16 * k, dBh + 16 * k, kIdesc, true);
#pragma unroll
        for (int k = 0; k < KS; ++k) tc::mma_f16(d, dAh + 16 * k, dBl + 16 * k, kIdesc, true);
        tc::commit(&br.m_done[b]);
        tc::commit(&br.b_free[st]);
        if (tile == TT - 1 || t == L - 1) tc::commit(&br.a_free);
        committed = t;
      }
      // the MMAs committed complete before the CTA ends, whoever stopped (the latest phase of each
      // accumulator; immediate when the consumers saw them; bounded)
      for (int t = committed - kAcc + 1; t <= committed; ++t)
        if (t >= 0) (void)tc::mbar_wait(&br.m_done[t % kAcc], (uint32_t)((t / kAcc) & 1), kSpin);
    }
    __syncwarp();
  } else {
    // --------------------------------------------------------------- consumers
    const int q = warp & 3, h = warp >> 2;  // TMEM lane quarter, column quarter
    const int row = 32 * q + lane;
    const uint32_t tl = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)((kKeys / 4) * h);
    float M = kInitMax, S = 0.f;
    bool dead = false;  // warp-uniform: a wait gave up, the remaining units are skipped
    int rb = rb0, tile = t0, seg = 0;
    for (int t = 0; t < L; ++t) {
      if (t > 0 && ++tile == TT) { tile = 0; ++rb; }
      if (!dead) {
        const int b = t % kAcc;
        // one lane polls the barrier (sixteen warps of pollers slow every shared-memory access of the
        // issuer); the warp-synchronous broadcast orders the others' tcgen05.ld after it
        bool done = false;
        if (lane == 0) done = !*err && tc::mbar_wait(&br.m_done[b], (uint32_t)((t / kAcc) & 1), spin);
        done = __shfl_sync(0xffffffffu, done ? 1 : 0, 0) != 0;  // tcgen05.ld is warp-wide
        if (!done) {
          if (lane == 0) *err = 1;
          dead = true;
        }
      }
      if (!dead) {
        const int b = t % kAcc;
        tc::fence_after_sync();
        // this thread's quarter of the tile's columns
        float v[kKeys / 4];
        tc::ld64(tl + (uint32_t)(b * kAccCols), v);
        tc::fence_before_sync();
        __syncwarp();
        if (lane == 0) tc::mbar_arrive(&br.empty[b]);
        const float* H = Hs + (t % TT) * kKeys + (kKeys / 4) * h;
#pragma unroll
        for (int c0 = 0; c0 < 64; c0 += 32) {
          float* vv = v + c0;
          const float* HH = H + c0;
#pragma unroll
          for (int e = 0; e < 32; e += 4) {
            const float4 hv = *reinterpret_cast<const float4*>(HH + e);
            vv[e] = fmaf(s2, vv[e], hv.x);
            vv[e + 1] = fmaf(s2, vv[e + 1], hv.y);
            vv[e + 2] = fmaf(s2, vv[e + 2], hv.z);
            vv[e + 3] = fmaf(s2, vv[e + 3], hv.w);
          }
          float cm = vv[0];
#pragma unroll
          for (int e = 1; e < 31; e += 2) cm = max3f(cm, vv[e], vv[e + 1]);
          cm = fmaxf(cm, vv[31]);
          const float mn = fmaxf(M, cm);
          const u64 nm = pk(-mn, -mn);
          u64 a2[4] = {pk(0.f, 0.f), pk(0.f, 0.f), pk(0.f, 0.f), pk(0.f, 0.f)};
#pragma unroll
          for (int e = 0; e < 32; e += 2) {
            float w0, w1;
            upk(add2(pk(vv[e], vv[e + 1]), nm), w0, w1);
            a2[(e >> 1) & 3] = add2(a2[(e >> 1) & 3], pk(ex2f(w0), ex2f(w1)));
          }
          float s0, s1;
          upk(add2(add2(a2[0], a2[1]), add2(a2[2], a2[3])), s0, s1);
          S = S * ex2f(M - mn) + (s0 + s1);
          M = mn;
        }
      }
      if (tile == TT - 1 || t == L - 1) {
        // end of this CTA's part of row block rb: the four column quarters of a row meet
        if (h > 0) {
          br.hm[seg & 1][h - 1][row] = M;
          br.hs[seg & 1][h - 1][row] = S;
        }
        asm volatile("bar.sync 1, %0;" ::"n"(32 * kConsWarps) : "memory");
        if (h == 0) {
          float mn = M;
#pragma unroll
          for (int k = 0; k < 3; ++k) mn = fmaxf(mn, br.hm[seg & 1][k][row]);
          float St = S * ex2f(M - mn);
#pragma unroll
          for (int k = 0; k < 3; ++k) St += br.hs[seg & 1][k][row] * ex2f(br.hm[seg & 1][k][row] - mn);
          const int i = rb * kRows + row;
          if (i < nq) {
            const int slot = (int)((long long)blockIdx.x - cta_of_unit((long long)rb * TT, U, G));
            float* base = part + (size_t)slot * 2 * nq;
            const bool bad = *err != 0;
            base[i] = bad ? __int_as_float(0x7fc00000) : mn - s_f * nq2[i];
            base[(size_t)nq + i] = bad ? __int_as_float(0x7fc00000) : St;
            if (tile == TT - 1)
              for (int k = slot + 1; k < splits; ++k) {
                part[(size_t)k * 2 * nq + i] = kInitMax;
                part[(size_t)k * 2 * nq + nq + i] = 0.f;
              }
          }
        }
        M = kInitMax;
        S = 0.f;
        ++seg;
      }
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, kTmemCols);
  if (tid == 0 && br.err && status) atomicOr(status, kStatusTimeout);
}

size_t umma_smem_bytes(int dim16) {
  const size_t KA = 2 * (size_t)dim16;
  const size_t need = 16 * KA * 16 + kStages * (kKeys / 8) * KA * 16 + sizeof(float) * kMaxChunk + sizeof(Bars);
  // more than half of an SM's shared memory: one CTA per SM, so that no CTA waits for TMEM
  return need < kOneCtaSmem ? kOneCtaSmem : need;
}

template <int KS>
cudaError_t run_umma(const __half* opq, const float* nq2, int nq, const __half* opk, const float* nk2, int nk,
                     const float* l2w, const float* pot, const double* shift, double s, const int* maxbits,
                     float* part, const SweepGeom& g, int* status, cudaStream_t st) {
  const size_t smem = umma_smem_bytes(16 * KS);
  static std::mutex mu;
  static bool attr = false;
  {
    std::lock_guard<std::mutex> lk(mu);
    if (!attr) {
      cudaError_t e = cudaFuncSetAttribute(k_sweep_umma<KS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
      attr = true;
    }
  }
  k_sweep_umma<KS><<<g.ctas, kAllThreads, smem, st>>>(opq, nq2, nq, opk, nk2, nk, l2w, pot, shift, s, maxbits,
                                                      g.keys_per_split / kKeys, g.splits, part, wait_limit(), status);
  note_launch();
  return cudaGetLastError();
}

}  // namespace

int umma_dim16(int dim) { return (dim + 15) & ~15; }

size_t umma_operand_floats(int n, int dim) {
  // FP16 hi and lo parts: dim16 floats' worth of bytes a row
  const size_t npad = ((size_t)n + kPad - 1) / kPad * kPad;
  return npad * (size_t)umma_dim16(dim);
}

cudaError_t launch_umma_scale(const float* x, int n, const float* y, int m, int dim, const float* center,
                              int* maxbits, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(maxbits, 0, sizeof(int), st);
  if (e != cudaSuccess) return e;
  const long long total = ((long long)n + m) * dim;
  long long blocks = (total + 255) / 256;
  if (blocks > 4 * (long long)device_sm_count()) blocks = 4 * (long long)device_sm_count();
  k_umma_maxabs<<<(int)blocks, 256, 0, st>>>(x, n, y, m, dim, center, maxbits);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_umma_operand(const float* pts, int n, int dim, const float* center, const int* maxbits,
                                void* op, float* norm2, cudaStream_t st) {
  const int npad = (n + kPad - 1) / kPad * kPad;
  const int blocks = (npad + 255) / 256;
  k_umma_operand<<<blocks, 256, 0, st>>>(pts, n, npad, dim, umma_dim16(dim), center, maxbits,
                                         static_cast<__half*>(op), norm2);
  note_launch();
  return cudaGetLastError();
}

SweepGeom umma_geom(int nq, int nk) {
  SweepGeom g{};
  g.threads = kAllThreads;
  g.rows = 1;
  g.row_blocks = (nq + kRows - 1) / kRows;
  const long long TT = (nk + kKeys - 1) / kKeys;
  g.keys_per_split = (int)TT * kKeys;
  // the (row block, key tile) units spread evenly over one CTA per SM (a multiple of the
  // SM count when a CTA would otherwise hold more than kMaxChunk keys of H_j)
  const long long U = (long long)g.row_blocks * TT;
  const long long sms = device_sm_count(), per = kMaxChunk / kKeys;
  long long G = sms * ((U + sms * per - 1) / (sms * per));
  if (G > U) G = U;
  g.ctas = (int)G;
  // partial slots: a bound on the CTAs one row block's TT units are spread over (the first
  // and the last may hold one unit each, those between at least floor(U / G))
  const long long lmin = U / G;
  long long splits = TT < 2 ? 1 : 2 + (TT - 2) / lmin;
  if (splits > G) splits = G;
  g.splits = (int)splits;
  return g;
}

cudaError_t launch_umma_sweep(const void* opq, const float* nq2, int nq, const void* opk, const float* nk2, int nk,
                              int dim, const float* l2w, const float* pot, const double* shift, double s,
                              const int* maxbits, float* part, const SweepGeom& g, int* status, cudaStream_t st) {
  const __half* q = static_cast<const __half*>(opq);
  const __half* k = static_cast<const __half*>(opk);
  switch (umma_dim16(dim) / 16) {
    case 2: return run_umma<2>(q, nq2, nq, k, nk2, nk, l2w, pot, shift, s, maxbits, part, g, status, st);
    case 3: return run_umma<3>(q, nq2, nq, k, nk2, nk, l2w, pot, shift, s, maxbits, part, g, status, st);
    default: return run_umma<4>(q, nq2, nq, k, nk2, nk, l2w, pot, shift, s, maxbits, part, g, status, st);
  }
}

}  // namespace uot
