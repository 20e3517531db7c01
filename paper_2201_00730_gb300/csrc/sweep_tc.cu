// Tensor-core fused softmin sweep for point clouds in Morton order, dim <= 3,
// p = 2, with the half-step epilogue.
//
// A block of 128 query rows (one TMEM lane each) meets the keys in tiles of
// 128, each taken in the frame of its own centre o_t and shifted by a tile
// constant mu_t (s times the potential of the tile's first key).  For query i
// and key j the exponent of the softmin relative to the row's reference m_i
// (log2 units) is
//     t_ij - m_i = X_i . Y_j + H_j + c_i,
//     X_i = q_i - o_t,   Y_j = 2 s (k_j - o_t),
//     H_j = log2 w_j + s pot_j - mu_t - s |k_j - o_t|^2,   c_i = -s |q_i - o_t|^2 + mu_t - m_i,
// every term of which is small wherever the entry matters.  The whole sum is
// one K = 16 product on the tensor cores in the 4xTF32 split (x = x_hi + x_lo
// with tf32 parts; the constants carried as two tf32 parts each):
//     row [Xh, Xh, Xl, Xl, 1, 1, c_hi, c_lo] . key [Yh, Yl, Yh, Yl, H_hi, H_lo, 1, 1]
// (two tcgen05.mma of K = 8 per tile into TMEM); the warps only read the
// exponents back, take ex2 and sum: one FP32 add per entry, so the MUFU ex2
// rate bounds the kernel.
//
// Warp roles (one CTA per SM, all 512 TMEM columns = four accumulators),
// linked only by mbarriers:
//  - 4 row warps and 4 key warps stage the operands of a tile (row p, key p)
//    into one of four shared-memory slots once empty[slot] allows, and arrive
//    on staged[slot]; the key warps keep the raw data of the next two tiles
//    in flight;
//  - one issuer lane waits on staged[slot], issues the MMAs into the matching
//    accumulator and commits them to full[slot];
//  - 8 consumer warps: warps w and w + 4 share the TMEM lanes 32 (w % 4) .. and
//    take alternate tiles (so one reads TMEM while the other is on the MUFU);
//    a consumer waits on full[slot], reads the tile's 128 columns, releases the
//    slot through empty[slot] and sums the ex2; at the end of a work unit the
//    two partial sums of each row make one partial, and the CTA that completes
//    a row block runs its half-step epilogue on the consumer warps' named
//    barrier while the producers already stage the next unit.
// Work units (row block, chunk of key tiles) are walked in row-block order by
// a persistent grid.
//
// The sweep needs the references m_i: the solver runs it from the second
// sweep of each side on (e.lse_buf holds the previous iteration's row
// log-sum-exps).  When the previous change was small (e.state->lse_ok) the
// consumers sum 2^(t - m) directly; otherwise they keep a running max of the
// shifted exponents.  Rows whose result leaves +-kLseWindow of the reference
// are recomputed exactly in the epilogue.  Every mbarrier wait is bounded; a
// timeout sets kStatusTimeout and both roles stop at their next barrier.
#include <cuda_runtime.h>

#include <mutex>

#include "epi_device.cuh"
#include "sweep_common.cuh"
#include "tc_ptx.cuh"
#include "uot_internal.cuh"

namespace uot {
namespace {

using namespace simd;

constexpr int kRowWarps = 4;             // stage the row operand (thread p: row p)
constexpr int kKeyWarps = 4;             // stage the key operand (thread p: key p)
constexpr int kStageWarps = kRowWarps + kKeyWarps;
constexpr int kIssueWarp = kStageWarps;  // one lane issues the MMAs
constexpr int kConsWarps = 8;
constexpr int kConsBase = 32 * (kStageWarps + 1);
constexpr int kCons = 32 * kConsWarps;   // two consumer threads per row (alternate tiles)
constexpr int kThreads = kConsBase + kCons;
constexpr int kStages = 4;              // operand slots = TMEM accumulators
constexpr int kRows = 128;              // rows of a block = TMEM lanes = MMA M
constexpr int kKeys = 128;              // keys of a tile = MMA N
constexpr int kK = 16;                  // tf32 values per operand row (two MMAs of K = 8)
constexpr int kSbo = (kK / 4) * 128;    // bytes between 8-row core-matrix groups
constexpr int kCols = kStages * kKeys;  // all 512 TMEM columns
constexpr int kBarCons = 1;
constexpr uint32_t kIdesc = tc::idesc_tf32(kRows, kKeys);
constexpr long long kSpin = 1LL << 24;      // mbarrier polls before giving up
constexpr size_t kSmemBytes = 120 * 1024;   // more than half the SM: one CTA per SM

struct Smem {
  float A[kStages][kRows * kK];
  float B[kStages][kKeys * kK];
  float2 half[kRows];
  uint64_t staged[kStages];  // the 8 staging warps wrote the slot
  uint64_t full[kStages];    // the MMAs of the slot completed
  uint64_t empty[kStages];   // the 4 consumer warps of the slot's tile read it
  uint32_t tmem;
  int err;
  int nbad;
  int bad[kRows];
};
static_assert(sizeof(Smem) <= kSmemBytes, "shared memory layout");
static_assert(32 * kRowWarps == kRows && 32 * kKeyWarps == kKeys, "one row or key per staging thread");

// Chunk of key tiles of work unit u (row block rb): rotated by the row block,
// so that the CTA that finishes a row block last (and runs its epilogue)
// changes from one row block to the next.
__device__ __forceinline__ int chunk_of(int u, int rb, int nchunks) { return (u - rb * nchunks + rb) % nchunks; }

__device__ __forceinline__ void put4(float* tile, int r, int k, float a, float b, float c, float d) {
  *reinterpret_cast<float4*>(reinterpret_cast<char*>(tile) + tc::kmajor_offset(r, k, kSbo)) = make_float4(a, b, c, d);
}

template <int D>
__global__ void __launch_bounds__(kThreads, 1)
k_sweep_tc(const float* __restrict__ q, int nq, const float* __restrict__ kp, int nk,
           const float4* __restrict__ kcen, const float* __restrict__ l2w, const float* __restrict__ pot, double s,
           int tpc, int nchunks, float* __restrict__ part, EpiParams e) {
  static_assert(D >= 1 && D <= 3, "tensor-core sweep covers dim 1..3");
  extern __shared__ __align__(128) unsigned char smraw[];
  Smem& sm = *reinterpret_cast<Smem*>(smraw);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const float sf = (float)s;
  const float s2 = (float)(2.0 * s);
  const bool use_ref = e.lse_buf != nullptr && e.state->lse_ok[e.out_is_f] != 0;
  const int nrb = (nq + kRows - 1) / kRows;
  const int ntiles = (nk + kKeys - 1) / kKeys;
  const int nunits = nrb * nchunks;

  if (warp == 0) tc::tmem_alloc(&sm.tmem, kCols);
  if (tid == 0) {
    for (int b = 0; b < kStages; ++b) {
      tc::mbar_init(&sm.staged[b], kStageWarps);
      tc::mbar_init(&sm.full[b], 1);
      tc::mbar_init(&sm.empty[b], kConsWarps / 2);  // the four warps that take the tile
    }
    tc::fence_mbar_init();
    sm.err = 0;
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = sm.tmem;

  if (warp < kStageWarps) {
    // ---------------------------------------------------------------- staging warps
    const bool rowside = warp < kRowWarps;
    const int p = tid & 127;
    int g = 0;  // tiles staged so far: slot g % kStages, use g / kStages
    bool stop = false;
    for (int u = blockIdx.x; u < nunits && !stop; u += gridDim.x) {
      const int rb = u / nchunks;
      const int ta = chunk_of(u, rb, nchunks) * tpc;
      const int tb = min(ntiles, ta + tpc);
      // row side: the row's point and reference; key side: raw key data of a tile
      const int i = rb * kRows + p;
      const bool live = rowside && i < nq;
      float xq[3] = {0.f, 0.f, 0.f};
      if (live) {
#pragma unroll
        for (int d = 0; d < D; ++d) xq[d] = q[(size_t)i * D + d];
      }
      const float mref = live ? e.lse_buf[i] : 0.f;
      struct KeyData {
        float k[3], lw, pj, p0;
        float4 o;
      };
      auto load = [&](int t, KeyData& v) {
        v.k[0] = v.k[1] = v.k[2] = 0.f;
        v.lw = kZeroW;
        v.pj = 0.f;
        if (!rowside) {
          const int j = t * kKeys + p;
          if (j < nk) {
#pragma unroll
            for (int d = 0; d < D; ++d) v.k[d] = kp[(size_t)j * D + d];
            v.lw = l2w[j];
            v.pj = pot ? pot[j] : 0.f;
          }
        }
        v.p0 = pot ? pot[(size_t)t * kKeys] : 0.f;
        v.o = kcen[t];
      };
      // one tile into slot g % kStages; loads tile t + 2 into the same registers
      // (the loop is unrolled by two, so the loads land in place)
      auto step = [&](int t, KeyData& kd) -> bool {
        const int b = g % kStages;
        const int n = g / kStages;
        const float k0 = kd.k[0], k1 = kd.k[1], k2 = kd.k[2], lw = kd.lw, pj = kd.pj;
        const float mu = sf * kd.p0;
        const float4 o = kd.o;
        if (t + 2 < tb) load(t + 2, kd);
        if (n > 0 && !tc::mbar_wait(&sm.empty[b], (uint32_t)((n - 1) & 1), kSpin)) {
          sm.err = 1;
          return false;
        }
        if (rowside) {
          // row p: [Xh, Xh, Xl, Xl, 1, 1, c_hi, c_lo]
          const float x0 = xq[0] - o.x, x1 = (D > 1) ? xq[1] - o.y : 0.f, x2 = (D > 2) ? xq[2] - o.z : 0.f;
          float q2 = x0 * x0;
          if (D > 1) q2 = fmaf(x1, x1, q2);
          if (D > 2) q2 = fmaf(x2, x2, q2);
          const float cc = live ? fmaf(-sf, q2, mu - mref) : kZeroW;
          const float h0 = tc::to_tf32(x0), h1 = tc::to_tf32(x1), h2 = tc::to_tf32(x2);
          const float l0 = tc::to_tf32(x0 - h0), l1 = tc::to_tf32(x1 - h1), l2 = tc::to_tf32(x2 - h2);
          const float ch_ = tc::to_tf32(cc), cl_ = tc::to_tf32(cc - ch_);
          put4(sm.A[b], p, 0, h0, h1, h2, h0);
          put4(sm.A[b], p, 4, h1, h2, l0, l1);
          put4(sm.A[b], p, 8, l2, l0, l1, l2);
          put4(sm.A[b], p, 12, 1.f, 1.f, ch_, cl_);
        } else {
          // key p: [Yh, Yl, Yh, Yl, H_hi, H_lo, 1, 1]
          const float y0 = k0 - o.x, y1 = (D > 1) ? k1 - o.y : 0.f, y2 = (D > 2) ? k2 - o.z : 0.f;
          float r2 = y0 * y0;
          if (D > 1) r2 = fmaf(y1, y1, r2);
          if (D > 2) r2 = fmaf(y2, y2, r2);
          const float Y0 = s2 * y0, Y1 = s2 * y1, Y2 = s2 * y2;
          const float h0 = tc::to_tf32(Y0), h1 = tc::to_tf32(Y1), h2 = tc::to_tf32(Y2);
          const float l0 = tc::to_tf32(Y0 - h0), l1 = tc::to_tf32(Y1 - h1), l2 = tc::to_tf32(Y2 - h2);
          // H_j in FP32 (a constant shift of pot is applied exactly in the epilogue)
          const float H = (lw > 0.5f * kZeroW) ? fmaf(-sf, r2, fmaf(sf, pj, lw) - mu) : kZeroW;
          const float Hh = tc::to_tf32(H), Hl = tc::to_tf32(H - Hh);
          put4(sm.B[b], p, 0, h0, h1, h2, l0);
          put4(sm.B[b], p, 4, l1, l2, h0, h1);
          put4(sm.B[b], p, 8, h2, l0, l1, l2);
          put4(sm.B[b], p, 12, Hh, Hl, 1.f, 1.f);
        }
        tc::fence_proxy_async();
        __syncwarp();
        if (lane == 0) tc::mbar_arrive(&sm.staged[b]);
        ++g;
        return true;
      };
      KeyData ka, kb;
      load(ta, ka);
      if (ta + 1 < tb) load(ta + 1, kb);
      for (int t = ta; t < tb && !stop; t += 2) {
        if (!step(t, ka)) { stop = true; break; }
        if (t + 1 < tb && !step(t + 1, kb)) { stop = true; break; }
      }
    }
  } else if (warp == kIssueWarp) {
    // ---------------------------------------------------------------- MMA issuer
    if (lane == 0) {
      int g = 0;
      bool stop = false;
      for (int u = blockIdx.x; u < nunits && !stop; u += gridDim.x) {
        const int rb = u / nchunks;
        const int ta = chunk_of(u, rb, nchunks) * tpc;
        const int tb = min(ntiles, ta + tpc);
        for (int t = ta; t < tb; ++t, ++g) {
          const int b = g % kStages;
          const int n = g / kStages;
          if (!tc::mbar_wait(&sm.staged[b], (uint32_t)(n & 1), kSpin)) {
            sm.err = 1;
            stop = true;
            break;
          }
          tc::fence_after_sync();
          const uint32_t d = tmem + (uint32_t)(b * kKeys);
          const uint64_t da = tc::smem_desc(tc::smem_addr(sm.A[b]), 128, kSbo);
          const uint64_t db = tc::smem_desc(tc::smem_addr(sm.B[b]), 128, kSbo);
          tc::mma_tf32(d, da, db, kIdesc, false);
          tc::mma_tf32(d, da + (256 >> 4), db + (256 >> 4), kIdesc, true);  // K values 8..15
          tc::commit(&sm.full[b]);
        }
      }
    }
    __syncwarp();
  } else {
    // ---------------------------------------------------------------- consumers
    const epi::Grp grp{tid - kConsBase, kCons, kBarCons};
    const int cw = grp.tid >> 5;   // consumer warp 0..7
    const int lq = warp & 3;       // TMEM lane quarter of this warp
    const int colh = cw >> 2;      // parity of the tiles this warp takes
    const int row = lq * 32 + lane;
    const uint32_t tl = tmem + ((uint32_t)(lq * 32) << 16);
    int g = 0;
    for (int u = blockIdx.x; u < nunits; u += gridDim.x) {
      const int rb = u / nchunks;
      const int ch = chunk_of(u, rb, nchunks);
      const int ta = ch * tpc;
      const int tb = min(ntiles, ta + tpc);
      const int i = rb * kRows + row;
      const bool live = i < nq;
      const float mref = live ? e.lse_buf[i] : 0.f;
      float accM = use_ref ? 0.f : kInitMax;  // max of the shifted exponents t - m (0 in reference mode)
      float accS = 0.f;
      u64 acc2[4] = {pk(0.f, 0.f), pk(0.f, 0.f), pk(0.f, 0.f), pk(0.f, 0.f)};
      bool err = false;
      auto sum32 = [&](const float (&v)[32]) {
        if (use_ref) {
#pragma unroll
          for (int j = 0; j < 32; j += 2)
            acc2[(j >> 1) & 3] = add2(acc2[(j >> 1) & 3], pk(ex2f(v[j]), ex2f(v[j + 1])));
        } else {
          float cm = v[0];
#pragma unroll
          for (int j = 1; j < 31; j += 2) cm = max3f(cm, v[j], v[j + 1]);
          cm = fmaxf(cm, v[31]);
          const float mn = fmaxf(accM, cm);
          const u64 nm = pk(-mn, -mn);
          u64 a2[4] = {pk(0.f, 0.f), pk(0.f, 0.f), pk(0.f, 0.f), pk(0.f, 0.f)};
#pragma unroll
          for (int j = 0; j < 32; j += 2) {
            float w0, w1;
            upk(add2(pk(v[j], v[j + 1]), nm), w0, w1);
            a2[(j >> 1) & 3] = add2(a2[(j >> 1) & 3], pk(ex2f(w0), ex2f(w1)));
          }
          float a0, a1;
          upk(add2(add2(a2[0], a2[1]), add2(a2[2], a2[3])), a0, a1);
          accS = accS * ex2f(accM - mn) + (a0 + a1);
          accM = mn;
        }
      };
      for (int t = ta; t < tb; ++t, ++g) {
        if ((g & 1) != colh) continue;  // the other warp of the lane quarter takes this tile
        const int b = g % kStages;
        const int n = g / kStages;
        const bool ok = !err && tc::mbar_wait(&sm.full[b], (uint32_t)(n & 1), kSpin);
        err = err || !ok;
        tc::fence_after_sync();
        float v[32];
        if (ok) {
#pragma unroll 1
          for (int c = 0; c < kKeys - 32; c += 32) {
            tc::ld32(tl + (uint32_t)(b * kKeys + c), v);
            sum32(v);
          }
          tc::ld32(tl + (uint32_t)(b * kKeys + kKeys - 32), v);
        }
        tc::fence_before_sync();
        __syncwarp();
        if (lane == 0) tc::mbar_arrive(&sm.empty[b]);
        if (ok) sum32(v);
      }
      if (use_ref) {
        float a0, a1;
        upk(add2(add2(acc2[0], acc2[1]), add2(acc2[2], acc2[3])), a0, a1);
        accS = a0 + a1;
      }
      // the two halves of each row (even and odd tiles) -> one partial (m + max of the shifted exponents, sum)
      if (colh == 1) sm.half[row] = make_float2(accM, accS);
      if (tc::bar_or(kBarCons, kCons, err || sm.err != 0)) {
        if (grp.tid == 0) sm.err = 1;
        break;
      }
      if (colh == 0 && live) {
        const float2 h = sm.half[row];
        const float M = fmaxf(accM, h.x);
        const float S = accS * ex2f(accM - M) + h.y * ex2f(h.x - M);
        float* base = part + (size_t)ch * 2 * nq;
        base[i] = mref + M;
        base[(size_t)nq + i] = S;
      }

      // the CTA that completes the last chunk of a row block runs its half-step
      if (!epi::arrive_last(&e.rb_counter[rb], nchunks, grp)) continue;
      if (grp.tid == 0) e.rb_counter[rb] = 0;
      const int idx = (colh == 0 && live) ? i : -1;
      const epi::Pre pre = epi::prefetch(e, idx);
      int one[1] = {idx};
      float Mg[1], Lg[1];
      epi::merge_rows<1>(part, 2, nq, nchunks, one, Mg, Lg);
      if (use_ref) {
        if (grp.tid == 0) sm.nbad = 0;
        grp.sync();
        bool redo = false;
        if (idx >= 0 && !(fabsf((Mg[0] + Lg[0]) - mref) <= (float)kLseWindow)) {
          redo = true;
          sm.bad[atomicAdd(&sm.nbad, 1)] = idx;
        }
        grp.sync();
        const int nbad = sm.nbad;
        if (nbad > 0) {
          for (int k = cw; k < nbad; k += kConsWarps) {
            const int ib = sm.bad[k];
            float Mx, Sx;
            exact_row<D>(q + (size_t)ib * D, kp, nk, l2w, pot, sf, lane, Mx, Sx);
            for (int sp = lane; sp < nchunks; sp += 32) {
              float* base = part + (size_t)sp * 2 * nq;
              base[ib] = sp == 0 ? Mx : kInitMax;
              base[(size_t)nq + ib] = sp == 0 ? Sx : 0.f;
            }
          }
          if (grp.tid == 0) atomicAdd(&e.state->lse_miss, (unsigned)nbad);
          grp.sync();
          if (redo) epi::merge_rows<1>(part, 2, nq, nchunks, one, Mg, Lg);
        }
      }
      const epi::Consts& c = epi::block_consts(e, grp);
      epi::RowAcc ea = epi::rowacc_empty();
      if (idx >= 0) epi::row_ff(e, c, idx, Mg[0], Lg[0], pre, ea);
      epi::block_finish(e, ea, rb, nrb, grp);
    }
  }

  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, kCols);
  if (tid == 0 && sm.err) atomicOr(&e.state->status, kStatusTimeout);
}

template <int D>
void set_attributes() {
  static bool done = false;
  static std::mutex mu;
  std::lock_guard<std::mutex> lk(mu);
  if (!done) {
    cudaFuncSetAttribute(k_sweep_tc<D>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes);
    cudaFuncSetAttribute(k_sweep_tc<D>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    done = true;
  }
}

}  // namespace

bool tc_sweep_fits(int nq) { return nq > 0 && (nq + kRows - 1) / kRows <= kMaxBlocks; }

// Work units = (row block, chunk of key tiles); about eight units per CTA (one
// per SM) balance the persistent grid, chunks of at least four tiles keep the
// four-slot pipeline busy.
SweepGeom tc_geom(int nq, int nk, int dim) {
  (void)dim;
  SweepGeom g{};
  g.threads = kThreads;
  g.rows = 1;
  g.row_blocks = (nq + kRows - 1) / kRows;
  const int ntiles = (nk + kKeys - 1) / kKeys;
  const long long slots = (long long)device_sm_count();
  long long chunks = (8 * slots + g.row_blocks - 1) / g.row_blocks;
  const long long cap = ntiles / 4 > 1 ? ntiles / 4 : 1;
  if (chunks > cap) chunks = cap;
  if (chunks > 64) chunks = 64;
  if (chunks < 1) chunks = 1;
  const int tpc = (int)((ntiles + chunks - 1) / chunks);
  g.splits = (ntiles + tpc - 1) / tpc;
  g.keys_per_split = tpc * kKeys;
  return g;
}

cudaError_t launch_tc_sweep(const SideDesc& q, const SideDesc& k, const float4* centers_k, int dim,
                            const float* pot_k, double s, float* part, const SweepGeom& g, const EpiParams& epi,
                            cudaStream_t st) {
  EpiParams e = epi;
  epi_finish_params(e);
  const int tpc = g.keys_per_split / kKeys;
  const long long units = (long long)g.row_blocks * g.splits;
  long long grid = device_sm_count();
  if (grid > units) grid = units;
  switch (dim) {
    case 1:
      set_attributes<1>();
      k_sweep_tc<1><<<(int)grid, kThreads, kSmemBytes, st>>>(q.pts, q.n, k.pts, k.n, centers_k, k.l2w, pot_k, s, tpc,
                                                               g.splits, part, e);
      break;
    case 2:
      set_attributes<2>();
      k_sweep_tc<2><<<(int)grid, kThreads, kSmemBytes, st>>>(q.pts, q.n, k.pts, k.n, centers_k, k.l2w, pot_k, s, tpc,
                                                               g.splits, part, e);
      break;
    default:
      set_attributes<3>();
      k_sweep_tc<3><<<(int)grid, kThreads, kSmemBytes, st>>>(q.pts, q.n, k.pts, k.n, centers_k, k.l2w, pot_k, s, tpc,
                                                               g.splits, part, e);
  }
  note_launch();
  return cudaGetLastError();
}

}  // namespace uot
