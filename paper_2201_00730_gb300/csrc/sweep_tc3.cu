// Half-step sweep of the solver for point clouds in Morton order, dim <= 3,
// p = 2, with the exponent of every cost entry formed on the tensor cores
// (tcgen05, kind::tf32, accumulators in TMEM) and the half-step epilogue fused.
//
// Keys come in tiles T of 128 consecutive (spatially compact) points with a
// local origin o_T (the tile's bounding-box centre).  For query i and key j of
// tile T the softmin exponent (log2 units, key shift left to the epilogue) is
//     t_ij = H_j + q'_i . Y_j + R_i,   q' = q - o_T,  Y_j = 2 s (k_j - o_T),
//     H_j = log2 w_j + s pot_j - s |k_j - o_T|^2,   R_i = -s |q'_i|^2,
// and the sweep needs sum_j 2^(t_ij - m_i) for a per-row reference m_i.  The
// product A_i . B_j of two 16-value tf32 rows gives
//     v_ij = (H_j - Hbar_T) + q'_i . Y_j + c_iT,
// with Hbar_T the largest live H of the tile (kept per tile in global memory)
// and c_iT = R_i (running-max mode: v = t - Hbar_T) or R_i + Hbar_T - m_i
// (fixed-reference mode: v = t - m_i).  Every term that is large where an entry
// matters is split exactly into tf32 parts:
//     A_i = [qh0 ql0 qh0 qh1 | ql1 qh1 qh2 ql2 | qh2 ch cm cl | 1 1 1 0]
//     B_j = [Yh0 Yh0 Yl0 Yh1 | Yh1 Yl1 Yh2 Yh2 | Yl2 1 1 1 | Hh Hm Hl 0]
// (q' and Y as hi + lo, 22 significant bits, the dropped lo.lo below 2^-22 of
// |q'||Y|; c and H - Hbar as three parts, exact for FP32 values), two MMAs of
// K = 8 per 128 x 128 tile.  The CUDA cores then only take ex2 and add.
//
// The key operand B of each side lives in global memory in the canonical
// K-major layout, 8 KB per tile, and is bulk-copied into shared memory.  Its
// coordinate parts are built once per solve (k_tc3_keys); its H part is
// rewritten by the epilogue of every half-step that produces that side's
// potential (the half-step's query rows are the next sweep's keys, and a row
// block of 128 rows is exactly one key tile), so no CTA ever recomputes keys.
//
// Warp roles (one CTA per SM, all 512 TMEM columns = four accumulators):
//  - warps 0..7, consumers: warp w reads TMEM lanes 32 (w % 4) .. + 31 (its
//    rows) and columns 64 (w / 4) .. + 63 of each tile, two 32-column loads
//    (the second in flight while the first is summed), then ex2 and sums; at
//    the end of the CTA's part of a row block the two column halves of a row
//    make one partial (max or reference, sum);
//  - warps 8..11, row builders: thread p builds row p of A for each tile;
//  - warp 12, lane 0: bulk copies of B and the MMAs;
//  - warps 13..16, epilogue: the CTA that completes a row block (the last of
//    its CTAs to write a partial) hands it to these warps, which merge the
//    partials, run the half-step (epi_device.cuh), write the new key constants
//    of the rows and take part in the grid-level reduction, while the other
//    roles go on with the CTA's next tiles.
// Work units are (row block, key tile) pairs in row-block order; CTA c of G
// takes units [c U / G, (c + 1) U / G), so every SM gets the same number of
// cost entries.
//
// Sums are compensated: each tile's 64-entry partial sums go into the row's
// running sum by Neumaier's two-sum.  Every mbarrier wait is bounded; a wait
// that gives up stops every role, lets the copies and MMAs in flight land,
// frees the TMEM and reports kStatusTimeout.
#include <cuda_runtime.h>

#include <mutex>

#include "epi_device.cuh"
#include "sweep_common.cuh"
#include "tc_ptx.cuh"
#include "uot_internal.cuh"

namespace uot {
namespace {

using namespace simd;

constexpr int kRows = 128;              // rows of a block = TMEM lanes = MMA M
constexpr int kKeys = 128;              // keys of a tile = MMA N = kTileKeys
constexpr int kK = 16;                  // tf32 values per operand row (two MMAs of K = 8)
constexpr int kSbo = (kK / 4) * 128;    // bytes between 8-row core-matrix groups
constexpr int kOpBytes = kKeys * kK * 4;       // operand part of a key tile
constexpr int kTileBytes = kOpBytes + 128;     // + header {o_T.x, o_T.y, o_T.z, Hbar_T}, padding
constexpr int kTileFloats = kTileBytes / 4;
constexpr int kStages = 4;              // TMEM accumulators
constexpr int kAStages = 8;             // row-operand stages (the builders run up to 8 tiles ahead)
constexpr int kBStages = 12;            // key-tile stages
constexpr int kLag = 4;                 // a key stage is refilled kLag units after its MMAs were issued
static_assert(kLag < kAStages && kLag < kBStages, "refill lag");
constexpr int kCols = kStages * kKeys;  // all 512 TMEM columns
constexpr int kConsWarps = 8;
constexpr int kBuildWarps = 4;
constexpr int kEpiWarps = 4;
constexpr int kBuildBase = 32 * kConsWarps;
constexpr int kIssueWarp = kConsWarps + kBuildWarps;
constexpr int kEpiBase = 32 * (kIssueWarp + 1);
constexpr int kThreads = kEpiBase + 32 * kEpiWarps;
constexpr int kQueue = 8;               // row blocks handed to the epilogue warps, in flight
constexpr int kBarCons = 1, kBarEpi = 2;
constexpr uint32_t kIdesc = tc::idesc_tf32(kRows, kKeys);
constexpr long long kSpin = kWaitPolls;  // drain, hand-off and epilogue waits: polls before giving up
constexpr size_t kSmemBytes = 184 * 1024;  // more than half the SM: one CTA per SM
static_assert(kTileKeys == kKeys, "the key tiles of the ordering step are the MMA tiles");

struct Smem {
  float A[kAStages][kRows * kK];
  float B[kBStages][kTileFloats];
  float2 half[kRows];             // column half 1 of each row -> half 0
  float2 halfc[kRows];            // its compensation (reference mode) / unused
  uint64_t a_full[kAStages];      // the builders wrote A of the stage
  uint64_t a_free[kAStages];      // the MMAs that read A of the stage (and every earlier MMA) completed
  uint64_t b_full[kBStages];      // the key tile of the stage landed
  uint64_t m_done[kStages];       // the MMAs of the stage completed
  uint64_t acc_empty[kStages];    // the consumers read the accumulator
  uint64_t q_full[kQueue];        // a row block was handed to the epilogue warps
  uint64_t q_empty[kQueue];       // the epilogue warps finished with a queue entry
  int queue[kQueue];
  uint32_t tmem;
  int err;
  int nbad;
  int bad[kRows];
  float2 bad_res[kRows];
  float hmax[kEpiWarps];
};
static_assert(sizeof(Smem) <= kSmemBytes, "shared memory layout");

__device__ __forceinline__ void put4(float* tile, int r, int k, float a, float b, float c, float d) {
  *reinterpret_cast<float4*>(reinterpret_cast<char*>(tile) + tc::kmajor_offset(r, k, kSbo)) = make_float4(a, b, c, d);
}

// Three tf32 parts of an FP32 value (their sum is the value exactly).
__device__ __forceinline__ void split3(float v, float& h, float& m, float& l) {
  h = tc::to_tf32(v);
  const float r = v - h;
  m = tc::to_tf32(r);
  l = tc::to_tf32(r - m);
}

// First CTA whose unit range [c U / G, (c + 1) U / G) holds unit x.
__host__ __device__ __forceinline__ long long cta_of_unit(long long x, long long U, long long G) {
  return ((x + 1) * G + U - 1) / U - 1;
}

// ex2 of four packed pairs summed into acc (two independent chains).
__device__ __forceinline__ void ex2_sum8(const float* v, u64& a0, u64& a1) {
  a0 = add2(a0, pk(ex2f(v[0]), ex2f(v[1])));
  a1 = add2(a1, pk(ex2f(v[2]), ex2f(v[3])));
  a0 = add2(a0, pk(ex2f(v[4]), ex2f(v[5])));
  a1 = add2(a1, pk(ex2f(v[6]), ex2f(v[7])));
}

// Neumaier's compensated addition of x into (s, c).
__device__ __forceinline__ void two_add(float& s, float& c, float x) {
  const float t = s + x;
  c += (fabsf(s) >= fabsf(x)) ? ((s - t) + x) : ((x - t) + s);
  s = t;
}

// 32 TMEM columns of this thread's lane into r, without waiting (the caller
// waits with wait_ld32 before reading r).
__device__ __forceinline__ void ld32_async(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr)
      : "memory");
}
// Waits for this thread's TMEM loads; r is tied in so that no read of it moves above the wait.
__device__ __forceinline__ void wait_ld32(uint32_t (&r)[32]) {
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]), "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]), "+r"(r[15]), "+r"(r[16]), "+r"(r[17]), "+r"(r[18]), "+r"(r[19]), "+r"(r[20]), "+r"(r[21]), "+r"(r[22]), "+r"(r[23]), "+r"(r[24]), "+r"(r[25]), "+r"(r[26]), "+r"(r[27]), "+r"(r[28]), "+r"(r[29]), "+r"(r[30]), "+r"(r[31])
               :
               : "memory");
}

// Largest v over the threads of a group of whole warps (each thread one value).
__device__ __forceinline__ float group_max(float v, const epi::Grp& g, float* sh) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, off));
  if ((g.tid & 31) == 0) sh[g.tid >> 5] = v;
  g.sync();
  float m = sh[0];
  for (int w = 1; w < (g.n >> 5); ++w) m = fmaxf(m, sh[w]);
  g.sync();
  return m;
}

// The H part of the operand rows of key tile T (one thread per key p of the
// tile, the whole group): Hbar_T = the largest live H (0 if none), the row
// gets H - Hbar_T in three tf32 parts (dead and padding keys: kZeroW, so that
// their entries vanish), and Hbar_T goes into the tile's header (for the row
// builders) and into hb[T] (for the consumers).
__device__ __forceinline__ void write_key_h(float* __restrict__ Bop, float* __restrict__ hb, int T, int p, bool live,
                                            float H, const epi::Grp& g, float* sh) {
  float hm = group_max(live ? H : -INFINITY, g, sh);
  if (!(hm > -INFINITY)) hm = 0.f;
  float h0 = kZeroW, h1 = 0.f, h2 = 0.f;
  if (live) split3(H - hm, h0, h1, h2);
  float* tile = Bop + (size_t)T * kTileFloats;
  put4(tile, p, 12, h0, h1, h2, 0.f);
  if (g.tid == 0) {
    tile[kOpBytes / 4 + 3] = hm;
    hb[T] = hm;
  }
}

// Key operand of one side, one CTA (128 threads) per tile: with `full` the
// coordinate parts [Yh0 Yh0 Yl0 Yh1 | Yh1 Yl1 Yh2 Yh2 | Yl2 1 1 1 | . . . .]
// of Y_j = 2 s (k_j - o_T) and the header's o_T, always the H part from pot
// (null: 0) and the header's Hbar_T.
template <int D>
__global__ void __launch_bounds__(kKeys)
k_tc3_keys(const float* __restrict__ pts, int n, const float4* __restrict__ cen, const float* __restrict__ l2w,
           const float* __restrict__ pot, double s, float* __restrict__ Bop, float* __restrict__ hb, int full) {
  __shared__ float sh[kKeys / 32];
  const int T = blockIdx.x, p = threadIdx.x, j = T * kKeys + p;
  const float sf = (float)s, s2 = (float)(2.0 * s);
  const float4 o = cen[T];
  const float oc[3] = {o.x, o.y, o.z};
  float Y[3] = {0.f, 0.f, 0.f};
  float r2 = 0.f;
  const bool in = j < n;
  if (in) {
#pragma unroll
    for (int d = 0; d < D; ++d) {
      const float yl = pts[(size_t)j * D + d] - oc[d];
      Y[d] = s2 * yl;
      r2 = fmaf(yl, yl, r2);
    }
  }
  float* tile = Bop + (size_t)T * kTileFloats;
  if (full) {
    if (p < 3) tile[kOpBytes / 4 + p] = oc[p];
    float yh[3], yl[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      yh[d] = tc::to_tf32(Y[d]);
      yl[d] = tc::to_tf32(Y[d] - yh[d]);
    }
    put4(tile, p, 0, yh[0], yh[0], yl[0], yh[1]);
    put4(tile, p, 4, yh[1], yl[1], yh[2], yh[2]);
    put4(tile, p, 8, yl[2], 1.f, 1.f, 1.f);
  }
  const float lw = in ? l2w[j] : kZeroW;
  const bool live = in && lw > 0.5f * kZeroW;
  // H_j = log2 w_j + s pot_j - s |k'_j|^2 in FP32, as the CUDA-core tiled sweep forms it
  const float H = live ? fmaf(-sf, r2, fmaf(sf, pot ? pot[j] : 0.f, lw)) : kZeroW;
  write_key_h(Bop, hb, T, p, live, H, epi::whole_block(), sh);
}

// Parameters of one launch (the query side's rows, the key side's operand).
struct Tc3Args {
  const float* q;       // query points, Morton order [nq x D]
  const float* kp;      // key points, Morton order [nk x D] (exact recompute of missed rows)
  const float4* kcen;   // key tile centres
  const float* kl2w;    // key log2 weights (exact recompute)
  const float* kpot;    // key potential (exact recompute)
  const float* Bk;      // key tiles: [TT][128 x 16 tf32, canonical K-major | header]
  const float* hbk;     // Hbar of each key tile (also in the headers)
  float* part;          // partials [slots][2][nq]
  int nq, nk, TT;
  double s;
  long long spin;       // polls of a main-loop wait before it gives up
};

template <int D>
__global__ void __launch_bounds__(kThreads, 1) k_sweep_tc3(Tc3Args a, EpiParams e) {
  static_assert(D >= 1 && D <= 3, "the tensor-core tiled sweep covers dim 1..3");
  // Programmatic dependent launch: wait for the previous kernel of the stream
  // (its results and its TMEM) before anything else, then let the next one be
  // scheduled.
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  extern __shared__ __align__(1024) unsigned char smraw[];
  Smem& sm = *reinterpret_cast<Smem*>(smraw);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nq = a.nq, TT = a.TT;
  const int RB = (nq + kRows - 1) / kRows;
  const long long U = (long long)RB * TT, G = gridDim.x;
  const long long u0 = (long long)blockIdx.x * U / G, u1 = ((long long)blockIdx.x + 1) * U / G;
  const int L = (int)(u1 - u0);
  const int rb0 = (int)(u0 / TT), T0 = (int)(u0 % TT);  // the range's first unit (units advance tile-major)
  const float sf = (float)a.s;
  const bool use_ref = e.lse_buf != nullptr && e.state->lse_ok[e.out_is_f] != 0;

  if (warp == 0) tc::tmem_alloc(&sm.tmem, kCols);
  if (tid == 32 * kIssueWarp) {
    for (int b = 0; b < kAStages; ++b) {
      tc::mbar_init(&sm.a_full[b], kBuildWarps);
      tc::mbar_init(&sm.a_free[b], 1);
    }
    for (int b = 0; b < kStages; ++b) {
      tc::mbar_init(&sm.m_done[b], 1);
      tc::mbar_init(&sm.acc_empty[b], kConsWarps / 2);  // the group that takes the unit
    }
    for (int b = 0; b < kBStages; ++b) tc::mbar_init(&sm.b_full[b], 1);
    for (int k = 0; k < kQueue; ++k) {
      tc::mbar_init(&sm.q_full[k], 1);
      tc::mbar_init(&sm.q_empty[k], 1);
    }
    tc::fence_mbar_init();
    sm.err = 0;
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = sm.tmem;
  volatile int* err = &sm.err;

  if (warp == kIssueWarp) {
    // ------------------------------------------------------------------ copies and MMAs
    // Key tile of unit t in stage t % kBStages, refilled with unit t + kBStages once the MMAs
    // of unit t completed (the builders read its header before those MMAs).
    if (lane == 0) {
      int armed[kBStages] = {}, used[kBStages] = {};
      int committed = -1, freed = -1;  // units committed; a_free seen for units <= freed
      int Tc = T0;                     // key tile of the next unit to copy (copies go in unit order)
      auto copy_b = [&](int t) {
        const int sb = t % kBStages;
        const int T = Tc;
        if (++Tc == TT) Tc = 0;
        tc::mbar_arrive_expect_tx(&sm.b_full[sb], (uint32_t)kTileBytes);
        tc::bulk_g2s(sm.B[sb], a.Bk + (size_t)T * kTileFloats, (uint32_t)kTileBytes, &sm.b_full[sb]);
        ++armed[sb];
      };
      for (int t = 0; t < L && t < kBStages; ++t) copy_b(t);
      for (int t = 0; t < L && !*err; ++t) {
        const int st = t % kStages, sa = t % kAStages, sb = t % kBStages;
        bool ok = tc::mbar_wait(&sm.a_full[sa], (uint32_t)((t / kAStages) & 1), a.spin);
        ok = ok && tc::mbar_wait(&sm.b_full[sb], (uint32_t)((t / kBStages) & 1), a.spin);
        if (ok) ++used[sb];
        // accumulator st was last read for unit t - kStages
        ok = ok && (t < kStages ||
                    tc::mbar_wait(&sm.acc_empty[st], (uint32_t)(((t - kStages) / kStages) & 1), a.spin));
        if (!ok) { *err = 1; break; }
        tc::fence_after_sync();
        const uint32_t d = tmem + (uint32_t)(st * kKeys);
        const uint64_t da = tc::smem_desc(tc::smem_addr(sm.A[sa]), 128, kSbo);
        const uint64_t db = tc::smem_desc(tc::smem_addr(sm.B[sb]), 128, kSbo);
        tc::mma_tf32(d, da, db, kIdesc, false);
        tc::mma_tf32(d, da + (256 >> 4), db + (256 >> 4), kIdesc, true);  // K values 8..15
        tc::commit(&sm.m_done[st]);
        tc::commit(&sm.a_free[sa]);
        committed = t;
        // the key stage of unit t - kLag takes unit t - kLag + kBStages once the MMAs of that unit
        // completed (kLag units back, so that this wait does not hold up the next MMAs: a commit's
        // arrival trails the MMAs by hundreds of cycles)
        if (t >= kLag && t - kLag + kBStages < L) {
          if (!tc::mbar_wait(&sm.a_free[(t - kLag) % kAStages], (uint32_t)(((t - kLag) / kAStages) & 1), a.spin)) {
            *err = 1;
            break;
          }
          freed = t - kLag;
          copy_b(t - kLag + kBStages);
        }
      }
      // every copy armed lands and every MMA commit arrives before the CTA ends (bounded)
      if (*err) {
        for (int sb = 0; sb < kBStages; ++sb)
          for (; used[sb] < armed[sb]; ++used[sb])
            (void)tc::mbar_wait(&sm.b_full[sb], (uint32_t)(used[sb] & 1), kSpin);
      }
      for (int t = freed + 1; t <= committed; ++t) {
        if (t + kAStages <= committed) continue;  // only the latest commit of each row stage
        (void)tc::mbar_wait(&sm.a_free[t % kAStages], (uint32_t)((t / kAStages) & 1), kSpin);
      }
      for (int t = committed - kStages + 1; t <= committed; ++t)
        if (t >= 0) (void)tc::mbar_wait(&sm.m_done[t % kStages], (uint32_t)((t / kStages) & 1), kSpin);
    }
    __syncwarp();
  } else if (warp >= kConsWarps && warp < kIssueWarp) {
    // ------------------------------------------------------------------ row builders
    const int p = tid - kBuildBase;
    int rb = rb0, T = T0;
    bool live = false;
    float xq[3] = {0.f, 0.f, 0.f}, mref = 0.f;
    for (int t = 0; t < L; ++t) {
      if (t > 0 && ++T == TT) { T = 0; ++rb; }
      if (t == 0 || T == 0) {
        const int i = rb * kRows + p;
        live = i < nq;
#pragma unroll
        for (int d = 0; d < 3; ++d) xq[d] = (live && d < D) ? a.q[(size_t)i * D + d] : 0.f;
        mref = (live && use_ref) ? e.lse_buf[i] : 0.f;
      }
      const int sa = t % kAStages, sb = t % kBStages;
      // the tile's header arrives with its copy; the row stage is free once the MMAs that read it completed
      bool ok = !*err && tc::mbar_wait(&sm.b_full[sb], (uint32_t)((t / kBStages) & 1), a.spin);
      if (ok && t >= kAStages) ok = tc::mbar_wait(&sm.a_free[sa], (uint32_t)(((t - kAStages) / kAStages) & 1), a.spin);
      ok = __all_sync(0xffffffffu, ok);
      if (!ok) {
        if (lane == 0) *err = 1;
        break;
      }
      const float4 hd = *reinterpret_cast<const float4*>(sm.B[sb] + kOpBytes / 4);  // {o_T, Hbar_T}
      const float x0 = xq[0] - hd.x, x1 = (D > 1) ? xq[1] - hd.y : 0.f, x2 = (D > 2) ? xq[2] - hd.z : 0.f;
      float q2 = x0 * x0;
      if (D > 1) q2 = fmaf(x1, x1, q2);
      if (D > 2) q2 = fmaf(x2, x2, q2);
      const float R = -sf * q2;
      const float c = live ? (use_ref ? R + (hd.w - mref) : R) : 0.f;
      const float h0 = tc::to_tf32(x0), h1 = tc::to_tf32(x1), h2 = tc::to_tf32(x2);
      const float l0 = tc::to_tf32(x0 - h0), l1 = tc::to_tf32(x1 - h1), l2 = tc::to_tf32(x2 - h2);
      float ch, cm, cl;
      split3(c, ch, cm, cl);
      float* A = sm.A[sa];
      put4(A, p, 0, h0, l0, h0, h1);
      put4(A, p, 4, l1, h1, h2, l2);
      put4(A, p, 8, h2, ch, cm, cl);
      put4(A, p, 12, 1.f, 1.f, 1.f, 0.f);
      tc::fence_proxy_async();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&sm.a_full[sa]);
    }
  } else if (warp < kConsWarps) {
    // ------------------------------------------------------------------ consumers
    // Two groups of four warps take alternate units (group pg the units t with
    // t % 2 == pg), so that one group reads its accumulator while the other is on
    // the MUFU; warp w reads TMEM lanes 32 (w % 4) .. + 31, all 128 columns.
    const int lq = warp & 3, pg = warp >> 2;
    const int row = 32 * lq + lane;
    const uint32_t tl = tmem + ((uint32_t)(32 * lq) << 16);
    float M = kInitMax, S = 0.f, Cc = 0.f;  // running (max, sum, compensation) of the row
    bool dead = false;
    int qpost = 0;  // row blocks handed to the epilogue warps (thread 0 of the consumers)
    auto post = [&](int rbp) -> bool {
      const int k = qpost % kQueue;
      if (qpost >= kQueue &&
          !tc::mbar_wait(&sm.q_empty[k], (uint32_t)(((qpost / kQueue) - 1) & 1), kSpin))
        return false;
      sm.queue[k] = rbp;
      tc::mbar_arrive(&sm.q_full[k]);
      ++qpost;
      return true;
    };
    // 64 exponents of v (log2 units) summed into (S, Cc), with the running max in running-max mode
    auto consume = [&](const uint32_t (&r0)[32], const uint32_t (&r1)[32], float hbar) {
      float v[64];
#pragma unroll
      for (int k = 0; k < 32; ++k) { v[k] = __uint_as_float(r0[k]); v[32 + k] = __uint_as_float(r1[k]); }
      u64 s0 = pk(0.f, 0.f), s1 = pk(0.f, 0.f);
      if (use_ref) {
        // v = t - m: the sum needs no max
#pragma unroll
        for (int k = 0; k < 64; k += 8) ex2_sum8(v + k, s0, s1);
        float x0, x1;
        upk(add2(s0, s1), x0, x1);
        two_add(S, Cc, x0 + x1);
      } else {
        // v = t - Hbar_T: the max and sum of these 64, merged into the running pair
        float cm = fmaxf(v[0], v[1]);
#pragma unroll
        for (int k = 2; k < 64; k += 2) cm = max3f(cm, v[k], v[k + 1]);
        const u64 nm = pk(-cm, -cm);
#pragma unroll
        for (int k = 0; k < 64; k += 8) {
          float w[8];
#pragma unroll
          for (int h = 0; h < 8; h += 2) upk(add2(pk(v[k + h], v[k + h + 1]), nm), w[h], w[h + 1]);
          ex2_sum8(w, s0, s1);
        }
        float x0, x1;
        upk(add2(s0, s1), x0, x1);
        const float mT = cm + hbar;
        const float Mn = fmaxf(M, mT);
        const float f0 = ex2f(M - Mn);
        S *= f0;
        Cc *= f0;
        two_add(S, Cc, (x0 + x1) * ex2f(mT - Mn));
        M = Mn;
      }
    };
    int rb = rb0, T = T0;
    for (int t = 0; t < L; ++t) {
      if (t > 0 && ++T == TT) { T = 0; ++rb; }
      const int st = t % kStages;
      if ((t & 1) == pg && !dead) {
        const float hbar = use_ref ? 0.f : __ldg(a.hbk + T);
        bool ok = !*err && tc::mbar_wait(&sm.m_done[st], (uint32_t)((t / kStages) & 1), a.spin);
        ok = __all_sync(0xffffffffu, ok);  // tcgen05.ld is warp-wide
        if (!ok) {
          if (lane == 0) *err = 1;
          dead = true;
        } else {
          tc::fence_after_sync();
          uint32_t r0[32], r1[32];
          const uint32_t ta = tl + (uint32_t)(st * kKeys);
          ld32_async(ta, r0);
          ld32_async(ta + 32, r1);
          wait_ld32(r0);
          wait_ld32(r1);
          consume(r0, r1, hbar);
          ld32_async(ta + 64, r0);
          ld32_async(ta + 96, r1);
          wait_ld32(r0);
          wait_ld32(r1);
          tc::fence_before_sync();
          __syncwarp();
          if (lane == 0) tc::mbar_arrive(&sm.acc_empty[st]);
          consume(r0, r1, hbar);
        }
      }
      if (T == TT - 1 || t == L - 1) {
        // the end of this CTA's part of row block rb: the two groups' sums of a row make one partial
        const int i = rb * kRows + row;
        if (pg == 1) {
          sm.half[row] = make_float2(M, S);
          sm.halfc[row] = make_float2(Cc, 0.f);
        }
        asm volatile("bar.sync %0, %1;" ::"n"(kBarCons), "n"(32 * kConsWarps) : "memory");
        if (pg == 0 && i < nq) {
          const float2 h1 = sm.half[row];
          const float c1 = sm.halfc[row].x;
          float Mo, So;
          if (use_ref) {
            two_add(S, Cc, h1.y);
            Mo = e.lse_buf[i];
            So = S + (Cc + c1);
          } else {
            const float Mn = fmaxf(M, h1.x);
            const float f0 = ex2f(M - Mn), f1 = ex2f(h1.x - Mn);
            float Sx = S * f0, Cx = Cc * f0;
            two_add(Sx, Cx, h1.y * f1);
            Mo = Mn;
            So = Sx + (Cx + c1 * f1);
          }
          const int slot = (int)((long long)blockIdx.x - cta_of_unit((long long)rb * TT, U, G));
          const bool bad = *err != 0;
          float* base = a.part + (size_t)slot * 2 * nq;
          base[i] = bad ? __int_as_float(0x7fc00000) : Mo;
          base[(size_t)nq + i] = bad ? __int_as_float(0x7fc00000) : So;
        }
        // publish the partials; the CTA that writes the last one of the row block hands it on
        asm volatile("bar.sync %0, %1;" ::"n"(kBarCons), "n"(32 * kConsWarps) : "memory");
        if (tid == 0) {
          __threadfence();
          const long long c0 = cta_of_unit((long long)rb * TT, U, G);
          const long long c1 = cta_of_unit((long long)rb * TT + TT - 1, U, G);
          const unsigned int n = (unsigned int)(c1 - c0 + 1);
          if (atomicAdd(&e.rb_counter[rb], 1u) == n - 1) {
            __threadfence();
            e.rb_counter[rb] = 0;
            if (!post(rb)) *err = 1;
          }
        }
        M = kInitMax;
        S = 0.f;
        Cc = 0.f;
      }
    }
    if (tid == 0) (void)post(-1);  // no more row blocks
  } else {
    // ------------------------------------------------------------------ epilogue warps
    const epi::Grp g{tid - kEpiBase, 32 * kEpiWarps, kBarEpi};
    const int ew = g.tid >> 5;
    for (int k = 0;; ++k) {
      const int qs = k % kQueue;
      bool ok = tc::mbar_wait(&sm.q_full[qs], (uint32_t)((k / kQueue) & 1), kSpin);
      if (tc::bar_or(kBarEpi, g.n, !ok)) {
        if (g.tid == 0) *err = 1;
        break;
      }
      const int rb = sm.queue[qs];
      if (rb < 0) break;
      const int i = rb * kRows + g.tid;
      const int idx = i < nq ? i : -1;
      const int nslot = (int)(cta_of_unit((long long)rb * TT + TT - 1, U, G) - cta_of_unit((long long)rb * TT, U, G)) + 1;
      const epi::Pre pre = epi::prefetch(e, idx);
      int one[1] = {idx};
      float Mg[1], Lg[1];
      if (use_ref) {
        const float ref[1] = {idx >= 0 ? e.lse_buf[idx] : 0.f};
        epi::merge_rows_ref<1>(a.part, 2, nq, nslot, one, ref, Mg, Lg);
        // rows whose log-sum-exp left the window around the reference: recomputed exactly, a warp each
        if (g.tid == 0) sm.nbad = 0;
        g.sync();
        int mine = -1;
        if (idx >= 0 && !(fabsf((Mg[0] + Lg[0]) - ref[0]) <= (float)kLseWindow)) {
          mine = atomicAdd(&sm.nbad, 1);
          sm.bad[mine] = idx;
        }
        g.sync();
        const int nbad = sm.nbad;
        if (nbad > 0) {
          for (int b = ew; b < nbad; b += kEpiWarps) {
            float Mx, Sx;
            exact_row<D>(a.q + (size_t)sm.bad[b] * D, a.kp, a.nk, a.kl2w, a.kpot, sf, lane, Mx, Sx);
            if (lane == 0) sm.bad_res[b] = make_float2(Mx, Sx);
          }
          if (g.tid == 0) atomicAdd(&e.state->lse_miss, (unsigned)nbad);
          g.sync();
          if (mine >= 0) {
            Mg[0] = sm.bad_res[mine].x;
            Lg[0] = log2f(sm.bad_res[mine].y);
          }
        }
      } else {
        epi::merge_rows<1>(a.part, 2, nq, nslot, one, Mg, Lg);
      }
      const epi::Consts& c = epi::block_consts(e, g);
      epi::RowAcc ea = epi::rowacc_empty();
      float vo = 0.f;
      if (idx >= 0) vo = epi::row_ff(e, c, idx, Mg[0], Lg[0], pre, ea);
      if (e.tc_b_out) {
        // these rows are the keys of the next sweep over this side: their new H parts
        const float lw = idx >= 0 ? e.l2w_o[idx] : kZeroW;
        const bool live = idx >= 0 && lw > 0.5f * kZeroW;
        float H = kZeroW;
        if (live) {
          const float4 o = e.tc_cen_out[rb];
          const float oc[3] = {o.x, o.y, o.z};
          float r2 = 0.f;
#pragma unroll
          for (int d = 0; d < D; ++d) {
            const float yl = e.tc_pts_out[(size_t)idx * D + d] - oc[d];
            r2 = fmaf(yl, yl, r2);
          }
          H = fmaf(-sf, r2, fmaf(sf, vo, lw));
        }
        write_key_h(e.tc_b_out, e.tc_hb_out, rb, g.tid, live, H, g, sm.hmax);
      }
      epi::block_finish(e, ea, rb, RB, g);
      g.sync();
      if (g.tid == 0) tc::mbar_arrive(&sm.q_empty[qs]);
    }
  }

  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, kCols);
  if (tid == 0 && sm.err) atomicOr(&e.state->status, kStatusTimeout);
}

template <int D>
cudaError_t set_attributes() {
  static cudaError_t done = cudaErrorNotReady;
  static std::mutex mu;
  std::lock_guard<std::mutex> lk(mu);
  if (done != cudaSuccess) {
    done = cudaFuncSetAttribute(k_sweep_tc3<D>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes);
  }
  return done;
}

}  // namespace

bool tc3_fits(int nq, int nk) {
  return nq > 0 && nk > 0 && (nq + kRows - 1) / kRows <= kMaxBlocks && (nk + kKeys - 1) / kKeys <= kMaxBlocks;
}

size_t tc3_operand_floats(int n) { return (size_t)((n + kKeys - 1) / kKeys) * kTileFloats; }

// One CTA per SM over the (row block, key tile) units; slots = the most CTAs
// that one row block's units are spread over.
SweepGeom tc3_geom(int nq, int nk) {
  SweepGeom g{};
  g.threads = kThreads;
  g.rows = 1;
  g.row_blocks = (nq + kRows - 1) / kRows;
  const long long TT = (nk + kKeys - 1) / kKeys;
  g.keys_per_split = (int)TT * kKeys;
  const long long U = (long long)g.row_blocks * TT;
  long long G = device_sm_count();
  if (G > U) G = U;
  g.ctas = (int)G;
  long long slots = 1;
  for (long long rb = 0; rb < g.row_blocks; ++rb) {
    const long long n = cta_of_unit(rb * TT + TT - 1, U, G) - cta_of_unit(rb * TT, U, G) + 1;
    if (n > slots) slots = n;
  }
  g.splits = (int)slots;
  return g;
}

cudaError_t launch_tc3_keys(const float* pts, int n, int dim, const float4* cen, const float* l2w, const float* pot,
                            double s, float* Bop, float* hb, bool full, cudaStream_t st) {
  const int tiles = (n + kKeys - 1) / kKeys;
  switch (dim) {
    case 1: k_tc3_keys<1><<<tiles, kKeys, 0, st>>>(pts, n, cen, l2w, pot, s, Bop, hb, full ? 1 : 0); break;
    case 2: k_tc3_keys<2><<<tiles, kKeys, 0, st>>>(pts, n, cen, l2w, pot, s, Bop, hb, full ? 1 : 0); break;
    default: k_tc3_keys<3><<<tiles, kKeys, 0, st>>>(pts, n, cen, l2w, pot, s, Bop, hb, full ? 1 : 0);
  }
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_tc3_sweep(const SideDesc& q, const SideDesc& k, const float4* centers_k, int dim,
                             const float* pot_k, const float* Bk, const float* hbk, double s, float* part,
                             const SweepGeom& g, const EpiParams& epi, cudaStream_t st) {
  EpiParams e = epi;
  epi_finish_params(e);
  Tc3Args a{q.pts, k.pts, centers_k, k.l2w, pot_k, Bk, hbk, part, q.n, k.n, (k.n + kKeys - 1) / kKeys, s,
            wait_limit()};
  cudaLaunchConfig_t cfg{};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.gridDim = dim3(g.ctas);
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = kSmemBytes;
  cfg.stream = st;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaError_t err;
  switch (dim) {
    case 1:
      if ((err = set_attributes<1>()) != cudaSuccess) return err;
      err = cudaLaunchKernelEx(&cfg, k_sweep_tc3<1>, a, e);
      break;
    case 2:
      if ((err = set_attributes<2>()) != cudaSuccess) return err;
      err = cudaLaunchKernelEx(&cfg, k_sweep_tc3<2>, a, e);
      break;
    default:
      if ((err = set_attributes<3>()) != cudaSuccess) return err;
      err = cudaLaunchKernelEx(&cfg, k_sweep_tc3<3>, a, e);
  }
  if (err != cudaSuccess) return err;
  note_launch();
  return cudaGetLastError();
}

}  // namespace uot
