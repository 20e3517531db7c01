// Resident solver for small point-cloud problems (dim <= 3, p = 2, both clouds
// in shared memory): the whole plain or TI Sinkhorn loop of uot_sinkhorn /
// uot_ti_sinkhorn in one launch of one thread-block cluster, so that an
// iteration costs no kernel launch and no global-memory round trip.
//
// Same iteration, epilogue and stopping rule as the multi-launch solver: the
// g half-step of iteration t + 1 (which also gives the residual of iterate t),
// the stopping test, then the f half-step.  Every CTA of the cluster holds
// both clouds in shared memory as (negated coordinates, key bias h = log2 w +
// s pot_hat) in a pair-major layout that feeds packed f32x2 arithmetic, and
// owns a contiguous slice of the query rows of each half-step.  A row's
// log-sum-exp over all keys takes one pass against the row's log-sum-exp of
// the previous half-step on its side as reference (two rows per group of G
// lanes share each key load; a sum outside [2^-60, 2^60] is redone), or two
// passes (maximum, then the sum of 2^(t - max)) the first time; the rows
// then go, one per thread, through the float-pair epilogue of the large
// sweeps (epi_device.cuh).  The new key
// bias of each row is pushed into every CTA's copy of its side, and the CTA
// partials of the epilogue (mass, residual, flags) into every CTA's partial
// table, through distributed shared memory; after one cluster barrier every
// CTA reduces the same table in the same order and finalises its own copy of
// the iteration state, so all copies agree bit for bit and no second barrier
// is needed.  The finalisation of a half-step (table reduction, scalars,
// stopping test, the next half-step's constants) runs on warp 0 while the
// other warps take the next half-step's log-sum-exps, which need only the key
// biases.  The scalar pending shift of the TI key potential stays with the
// epilogue, as in the fused tiled sweeps.
//
// Races: the values pushed in half-step h are read as keys in half-step h + 1;
// a CTA pushes into a side only after the cluster barrier that follows every
// CTA's last read of that side as keys (half-step h - 1), and the partial
// table is double-buffered by half-step parity.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include "epi_device.cuh"
#include "sweep_common.cuh"
#include "uot_internal.cuh"

namespace uot {
namespace {

namespace cg = cooperative_groups;
using namespace simd;

constexpr int kThreads = 1024;
constexpr int kLseThreads = kThreads - 32;
constexpr int kMaxCluster = 16;
constexpr size_t kSmemLimit = 200 * 1024;

// 64-bit words per pair of points: (x pair, h pair) in 1-D, else (x, y, z | pad, h)
__host__ __device__ constexpr int pair_words(int dim) { return dim == 1 ? 2 : 4; }

__host__ __device__ constexpr size_t small_smem_bytes(int n, int m, int dim) {
  // both clouds (pair-major), f_hat, g by parity, log2 weights as float pairs, row references,
  // row log-sum-exps, the miss list
  return 8 * (size_t)pair_words(dim) * (size_t)(((n + 1) / 2) + ((m + 1) / 2)) + 16 * (size_t)n + 20 * (size_t)m +
         12 * (size_t)(n > m ? n : m);
}

struct SmallArgs {
  const float* x;   // N x dim
  const float* y;   // M x dim
  int n, m, ti, max_iter, check_every;
  double tol;
  float sf;         // s = log2(e) / eps in float
  float* fst;       // f_hat (in: initial, out: final)
  float* gb0;       // g buffers by iteration parity (out: the final g in gb[iters & 1])
  float* gb1;
};

// One side in shared memory.
struct Side {
  float* pk;     // pair-major points: pair p holds points 2p, 2p + 1
  float* l2h;    // log2 w (float pair hi, lo)
  float* l2l;
  float* ref;    // each row's log-sum-exp of the side's previous half-step (this CTA's rows)
  int n;
};

template <int D>
__device__ __forceinline__ int coord_at(int i, int d) {
  return (i >> 1) * (2 * pair_words(D)) + 2 * d + (i & 1);
}
template <int D>
__device__ __forceinline__ int bias_at(int i) {
  return (i >> 1) * (2 * pair_words(D)) + 2 * D + (i & 1);
}

__device__ __forceinline__ float key_bias(float lw, float sf, float pot) {
  return (lw > 0.5f * kZeroW) ? fmaf(sf, pot, lw) : kZeroW;
}

// t = h - s |q - k|^2 for the two keys of a pair (coordinates stored negated).
template <int D>
__device__ __forceinline__ u64 pair_t(const u64* __restrict__ k, const u64 (&q2)[3], u64 nsf2) {
  const u64 d0 = add2(q2[0], k[0]);
  u64 r2 = mul2(d0, d0);
  if (D > 1) { const u64 d1 = add2(q2[1], k[1]); r2 = fma2(d1, d1, r2); }
  if (D > 2) { const u64 d2 = add2(q2[2], k[2]); r2 = fma2(d2, d2, r2); }
  return fma2(nsf2, r2, k[D]);
}

// Lanes of this lane's group of G (groups of a warp may branch apart).
template <int G>
__device__ __forceinline__ unsigned group_mask() {
  return G == 32 ? 0xffffffffu : ((1u << G) - 1u) << ((threadIdx.x & 31) & ~(G - 1));
}

// log2 sum_k 2^(t_qk) = M + L over all keys of one row: lanes sub, sub + G,
// ... of a group of G lanes take every G-th pair; first the maximum, then the
// sum of 2^(t - M).  np = 0 skips the work (the group still joins the shuffles).
template <int D, int G>
__device__ __forceinline__ void group_lse(const u64* __restrict__ keys, int np, const float (&q)[3], float sf, int sub,
                                          float& Mo, float& Lo) {
  constexpr int W = pair_words(D);
  const unsigned mask = group_mask<G>();
  u64 q2[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) q2[d] = pk(q[d], q[d]);
  const u64 nsf2 = pk(-sf, -sf);
  float M0 = kInitMax, M1 = kInitMax;
  int p = sub;
  for (; p + G < np; p += 2 * G) {
    float a, b, c, e;
    upk(pair_t<D>(keys + (size_t)p * W, q2, nsf2), a, b);
    upk(pair_t<D>(keys + (size_t)(p + G) * W, q2, nsf2), c, e);
    M0 = max3f(M0, a, b);
    M1 = max3f(M1, c, e);
  }
  if (p < np) {
    float a, b;
    upk(pair_t<D>(keys + (size_t)p * W, q2, nsf2), a, b);
    M0 = max3f(M0, a, b);
  }
  float M = fmaxf(M0, M1);
#pragma unroll
  for (int off = 1; off < G; off <<= 1) M = fmaxf(M, __shfl_xor_sync(mask, M, off));
  const u64 nM2 = pk(-M, -M);
  u64 S0 = pk(0.f, 0.f), S1 = S0;
  p = sub;
  for (; p + G < np; p += 2 * G) {
    float a, b, c, e;
    upk(add2(pair_t<D>(keys + (size_t)p * W, q2, nsf2), nM2), a, b);
    upk(add2(pair_t<D>(keys + (size_t)(p + G) * W, q2, nsf2), nM2), c, e);
    S0 = add2(S0, pk(ex2f(a), ex2f(b)));
    S1 = add2(S1, pk(ex2f(c), ex2f(e)));
  }
  if (p < np) {
    float a, b;
    upk(add2(pair_t<D>(keys + (size_t)p * W, q2, nsf2), nM2), a, b);
    S0 = add2(S0, pk(ex2f(a), ex2f(b)));
  }
  float s0, s1, s2, s3;
  upk(S0, s0, s1);
  upk(S1, s2, s3);
  float S = (s0 + s1) + (s2 + s3);
#pragma unroll
  for (int off = 1; off < G; off <<= 1) S += __shfl_xor_sync(mask, S, off);
  Mo = M;
  Lo = log2f(S);
}

// One pass for R rows at once against a fixed reference per row (the row's
// log-sum-exp of the previous half-step on this side): S_r = sum_k 2^(t_rk -
// ref_r), each key pair read once for all R rows.
template <int D, int G, int R>
__device__ __forceinline__ void group_sum_ref(const u64* __restrict__ keys, int np, const float (&q)[R][3],
                                              const float (&ref)[R], float sf, int sub, float (&S)[R]) {
  constexpr int W = pair_words(D);
  const unsigned mask = group_mask<G>();
  u64 q2[R][3], nr2[R], acc[R];
#pragma unroll
  for (int r = 0; r < R; ++r) {
#pragma unroll
    for (int d = 0; d < 3; ++d) q2[r][d] = pk(q[r][d], q[r][d]);
    nr2[r] = pk(-ref[r], -ref[r]);
    acc[r] = pk(0.f, 0.f);
  }
  const u64 nsf2 = pk(-sf, -sf);
  for (int p = sub; p < np; p += G) {
    u64 k[4];
#pragma unroll
    for (int w = 0; w <= D; ++w) k[w] = keys[(size_t)p * W + w];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      float a, b;
      upk(add2(pair_t<D>(k, q2[r], nsf2), nr2[r]), a, b);
      acc[r] = add2(acc[r], pk(ex2f(a), ex2f(b)));
    }
  }
#pragma unroll
  for (int r = 0; r < R; ++r) {
    float a, b;
    upk(acc[r], a, b);
    float v = a + b;
#pragma unroll
    for (int off = 1; off < G; off <<= 1) v += __shfl_xor_sync(mask, v, off);
    S[r] = v;
  }
}

constexpr int kRows = 2;  // rows per group in the fixed-reference pass

// Named barrier of the log-sum-exp warps (1..).
__device__ __forceinline__ void lse_sync() { asm volatile("bar.sync 1, %0;" ::"n"(kLseThreads) : "memory"); }

// Exact two-pass log-sum-exps of the rows lo + idx[k] (idx = null: lo + k),
// k < cnt, a group of G lanes per row; lane 0 of the group stores M, L and
// the row's new reference.
template <int D, int G>
__device__ void lse_rows_exact(const Side& Qs, const Side& Ks, int lo, int cnt, const int* idx, float sf, float* sM,
                               float* sL) {
  const int tid = threadIdx.x - 32;  // warps 1.. (warp 0 finalises the previous half-step meanwhile)
  const int sub = tid % G, grp = tid / G;
  const int np = (Ks.n + 1) >> 1;
  for (int k0 = 0; k0 < cnt; k0 += kLseThreads / G) {  // the same trip count on every lane (shuffles)
    const int k = k0 + grp;
    const bool valid = k < cnt;
    const int i = valid ? lo + (idx ? idx[k] : k) : lo;
    float q[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) q[d] = (valid && d < D) ? -Qs.pk[coord_at<D>(i, d)] : 0.f;
    float M, L;
    group_lse<D, G>(reinterpret_cast<const u64*>(Ks.pk), valid ? np : 0, q, sf, sub, M, L);
    if (valid && sub == 0) {
      sM[i - lo] = M;
      sL[i - lo] = L;
      Qs.ref[i] = M + L;
    }
  }
}

// Single pass of kRows rows per group of G lanes against the stored
// references; a row whose sum leaves [2^-60, 2^60] (or whose reference is not
// finite) goes to the list `fail` (count *nfail) for the exact form.
template <int D, int G>
__device__ void lse_rows_ref(const Side& Qs, const Side& Ks, int lo, int hi, float sf, float* sM, float* sL,
                             int* fail, int* nfail) {
  const int tid = threadIdx.x - 32;
  const int sub = tid % G, grp = tid / G;
  const int np = (Ks.n + 1) >> 1;
  for (int r0 = lo; r0 < hi; r0 += (kLseThreads / G) * kRows) {  // the same trip count on every lane
    float q[kRows][3], ref[kRows];
    bool any = false;
#pragma unroll
    for (int r = 0; r < kRows; ++r) {
      const int i = r0 + grp * kRows + r;
      const bool valid = i < hi;
      any |= valid;
#pragma unroll
      for (int d = 0; d < 3; ++d) q[r][d] = (valid && d < D) ? -Qs.pk[coord_at<D>(i, d)] : 0.f;
      ref[r] = valid ? Qs.ref[i] : 0.f;
    }
    float S[kRows];
    group_sum_ref<D, G, kRows>(reinterpret_cast<const u64*>(Ks.pk), any ? np : 0, q, ref, sf, sub, S);
    if (sub == 0) {
#pragma unroll
      for (int r = 0; r < kRows; ++r) {
        const int i = r0 + grp * kRows + r;
        if (i >= hi) continue;
        if (ref[r] > 0.25f * kZeroW && S[r] >= 0x1p-60f && S[r] <= 0x1p60f) {
          const float L = log2f(S[r]);
          sM[i - lo] = ref[r];
          sL[i - lo] = L;
          Qs.ref[i] = ref[r] + L;
        } else {
          fail[atomicAdd(nfail, 1)] = i - lo;
        }
      }
    }
  }
}

// Per-iteration fields of the two half-steps of iteration t + 1.
__device__ __forceinline__ void g_fields(EpiParams& e, int t, int ti, float* g0, float* g1, DevState* st) {
  const int so = (t + 1) & 1, si = t & 1;
  e.old_out = (t >= 1) ? (si ? g1 : g0) : nullptr;
  e.out = so ? g1 : g0;
  e.hist_index = t;
  e.slot_in = si;
  e.slot_out = so;
  e.key_shift = ti ? &st->slot[si].cf : nullptr;
}
__device__ __forceinline__ void f_fields(EpiParams& e, int t, int ti, DevState* st) {
  const int so = (t + 1) & 1;
  e.slot_in = so;
  e.slot_out = so;
  e.key_shift = ti ? &st->slot[so].cg : nullptr;
}

struct Shared {
  DevState st;                        // this CTA's copy of the iteration state
  EpiParams e[2];                     // [0] g half-step, [1] f half-step
  epi::Consts c[2];
  ffl::Exp2Table tab;                 // exp2 table of the float-pair epilogue
  epi::Part wp[kThreads / 32];        // warp partials
  epi::Part table[2][kMaxCluster];    // CTA partials by half-step parity
  int stop;
  int nfail;                          // entries of the miss list
  unsigned misses;                    // rows redone in the exact form (this CTA)
};

// Rows [lo, hi) of the query side owned by this CTA.
__device__ __forceinline__ void my_rows(int nq, int rank, int csize, int& lo, int& hi) {
  lo = (int)((long long)nq * rank / csize);
  hi = (int)((long long)nq * (rank + 1) / csize);
}

// Log-sum-exps of this CTA's rows of a half-step on warps 1.. (G lanes per row).
// Group size for cnt groups on the log-sum-exp warps: the largest (<= 32
// lanes) with which all groups run in one pass.
#define UOT_LSE_DISPATCH(cnt, CALL)                        \
  do {                                                     \
    if ((cnt) * 2 > kLseThreads) { constexpr int G = 1; CALL; }       \
    else if ((cnt) * 4 > kLseThreads) { constexpr int G = 2; CALL; }  \
    else if ((cnt) * 8 > kLseThreads) { constexpr int G = 4; CALL; }  \
    else if ((cnt) * 16 > kLseThreads) { constexpr int G = 8; CALL; } \
    else if ((cnt) * 32 > kLseThreads) { constexpr int G = 16; CALL; } \
    else { constexpr int G = 32; CALL; }                   \
  } while (0)

template <int D>
__device__ void lse_phase(const Side& Qs, const Side& Ks, float sf, bool use_ref, int rank, int csize, float* sM,
                          float* sL, int* fail, int* nfail, unsigned* misses) {
  int lo, hi;
  my_rows(Qs.n, rank, csize, lo, hi);
  const int nr = hi - lo;
  if (!use_ref) {
    UOT_LSE_DISPATCH(nr, (lse_rows_exact<D, G>(Qs, Ks, lo, nr, nullptr, sf, sM, sL)));
    return;
  }
  UOT_LSE_DISPATCH((nr + kRows - 1) / kRows, (lse_rows_ref<D, G>(Qs, Ks, lo, hi, sf, sM, sL, fail, nfail)));
  lse_sync();
  const int nf = *(volatile int*)nfail;
  if (nf > 0) UOT_LSE_DISPATCH(nf, (lse_rows_exact<D, G>(Qs, Ks, lo, nf, fail, sf, sM, sL)));
  lse_sync();
  if (threadIdx.x == 32) {
    *nfail = 0;
    *misses += (unsigned)nf;
  }
}

// Epilogue of this CTA's rows (one per thread): outputs, new key biases pushed
// to every CTA's copy of Qs, the CTA partial pushed to every CTA's table.
// The caller's cluster barrier then publishes both.
template <int D>
__device__ void epilogue_phase(const EpiParams& e, const epi::Consts& c, const Side& Qs, float sf, Shared& sh,
                               int par, int rank, int csize, const float* sM, const float* sL) {
  cg::cluster_group cl = cg::this_cluster();
  int lo, hi;
  my_rows(Qs.n, rank, csize, lo, hi);
  const int nr = hi - lo;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // warps holding rows (at least one: a CTA without rows still contributes an empty partial)
  const int nw = nr > 0 ? ((nr < kThreads ? nr : kThreads) + 31) >> 5 : 1;
  if (warp < nw) {
    epi::RowAcc acc = epi::rowacc_empty();
    for (int k = threadIdx.x; k < nr; k += kThreads) {
      const int i = lo + k;
      const epi::Pre pre = epi::prefetch(e, i);
      epi::row_ff(e, c, i, sM[k], sL[k], pre, acc);
      const float h = key_bias(Qs.l2h[i], sf, e.out[i]);
      float* dst = Qs.pk + bias_at<D>(i);
      for (int r = 0; r < csize; ++r) *cl.map_shared_rank(dst, r) = h;
    }
    const epi::Part p = epi::warp_reduce(epi::Part{acc.ref, acc.bad, acc.sum.hi, acc.sum.lo, acc.r, acc.gap});
    if (nw > 1 && lane == 0) sh.wp[warp] = p;
    if (nw == 1 && lane < csize) *cl.map_shared_rank(&sh.table[par][rank], lane) = p;
  }
  if (nw > 1) {
    __syncthreads();
    if (warp == 0) {
      const epi::Part q = epi::warp_reduce((lane < nw) ? sh.wp[lane] : epi::Part{INT_MIN, 0, 0.f, 0.f, 0.f, 0.f});
      if (lane < csize) *cl.map_shared_rank(&sh.table[par][rank], lane) = q;
    }
  }
}

template <int D>
__global__ void __launch_bounds__(kThreads, 1) k_small_solve(SmallArgs a, EpiParams eg0, EpiParams ef0) {
  extern __shared__ __align__(16) float smem[];
  __shared__ Shared sh;
  cg::cluster_group cl = cg::this_cluster();
  const int csize = (int)cl.num_blocks(), rank = (int)cl.block_rank();
  const int n = a.n, m = a.m;
  const float sf = a.sf;
  constexpr int W = pair_words(D);
  float* Px = smem;
  float* Py = Px + 2 * W * ((n + 1) / 2);
  float* fs = Py + 2 * W * ((m + 1) / 2);
  float* g0 = fs + n;
  float* g1 = g0 + m;
  float* lah = g1 + m;
  float* lal = lah + n;
  float* lbh = lal + n;
  float* lbl = lbh + m;
  float* sM = lbl + m;                 // per-row log-sum-exp (max, log2 of the sum)
  float* sL = sM + (n > m ? n : m);
  float* rfx = sL + (n > m ? n : m);   // per-row references of each side
  float* rfy = rfx + n;
  int* fail = reinterpret_cast<int*>(rfy + m);  // rows whose reference missed
  DevState* gst = eg0.state;

  // both clouds, negated, pair-major; odd counts end with a zero-weight key
  for (int i = threadIdx.x; i < 2 * ((n + 1) / 2); i += kThreads) {
    const bool in = i < n;
    const float lw = in ? ef0.l2w_o[i] : kZeroW;
    if (in) {
      lah[i] = lw;
      lal[i] = ef0.l2lo_o ? ef0.l2lo_o[i] : 0.f;
      fs[i] = a.fst[i];
    }
#pragma unroll
    for (int d = 0; d < W - 1; ++d) Px[coord_at<D>(i, d)] = (in && d < D) ? -a.x[(size_t)i * D + d] : 0.f;
    Px[bias_at<D>(i)] = in ? key_bias(lw, sf, fs[i]) : kZeroW;
  }
  for (int j = threadIdx.x; j < 2 * ((m + 1) / 2); j += kThreads) {
    const bool in = j < m;
    if (in) {
      lbh[j] = eg0.l2w_o[j];
      lbl[j] = eg0.l2lo_o ? eg0.l2lo_o[j] : 0.f;
    }
#pragma unroll
    for (int d = 0; d < W - 1; ++d) Py[coord_at<D>(j, d)] = (in && d < D) ? -a.y[(size_t)j * D + d] : 0.f;
    Py[bias_at<D>(j)] = kZeroW;
  }
  // the two half-steps' parameters live in shared memory (thread 0 updates the
  // per-iteration fields before a barrier); a per-thread copy would sit in
  // local memory, whose lines the cluster barriers' acquire drops from L1
  EpiParams& eg = sh.e[0];
  EpiParams& ef = sh.e[1];
  for (int k = threadIdx.x; k < 65; k += kThreads) {
    sh.tab.hi[k] = ffl::kExp2Tab.hi[k];
    sh.tab.lo[k] = ffl::kExp2Tab.lo[k];
  }
  if (threadIdx.x == 0) {
    eg = eg0;
    ef = ef0;
    eg.state = &sh.st; eg.l2w_o = lbh; eg.l2lo_o = lbl;
    ef.state = &sh.st; ef.l2w_o = lah; ef.l2lo_o = lal; ef.out = fs; ef.old_out = nullptr;
    eg.ff_only = ef.ff_only = 1;
    if (rank != 0) eg.resid_hist = nullptr;
    sh.st = *gst;
    g_fields(eg, 0, a.ti, g0, g1, &sh.st);
    sh.c[0] = epi::make_consts(eg);
    sh.c[0].tab = &sh.tab;
  }
  if (threadIdx.x == 0) {
    sh.stop = 0;
    sh.nfail = 0;
    sh.misses = 0;
  }
  cl.sync();  // every copy complete before the first push
  const Side X{Px, lah, lal, rfx, n}, Y{Py, lbh, lbl, rfy, m};
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // half-steps h = 0, 1, ...: even h the g half-step of iteration t + 1 = h / 2 + 1
  // (rows y, keys x with fb_t = f_hat + cf), odd h its f half-step (rows x, keys
  // y with gb_{t+1} = g_hat + cg).  While warps 1.. take the log-sum-exps of
  // half-step h, warp 0 reduces the partial table of h - 1, finalises it, runs
  // the stopping test after a g half-step and makes the constants of h; a stop
  // discards the log-sum-exps just taken.
  int h = 0;
  for (;;) {
    const int par = h & 1;
    if (warp == 0) {
      if (h > 0) {
        const epi::Part q = epi::warp_reduce((lane < csize) ? sh.table[par ^ 1][lane]
                                                            : epi::Part{INT_MIN, 0, 0.f, 0.f, 0.f, 0.f});
        if (lane == 0) {
          epi::finalize(sh.e[par ^ 1], q, sh.tab);
          const int t = h >> 1;  // iteration index of the pair (h - 1, h) or (h, h + 1)
          bool stop = false;
          if (par == 1) {  // h - 1 was the g half-step of iteration t + 1
            const bool last = (t == a.max_iter);
            if (t >= 1 && (last || (a.tol > 0.0 && t % a.check_every == 0))) {
              const float r = sh.st.resid;
              stop = sh.st.status != 0 || isnan(r) || last || (double)r <= a.tol;
            }
          }
          sh.stop = stop;
          if (!stop) {
            if (par == 1) f_fields(ef, t, a.ti, &sh.st);
            else g_fields(eg, t, a.ti, g0, g1, &sh.st);
            sh.c[par] = epi::make_consts(sh.e[par]);
            sh.c[par].tab = &sh.tab;
          }
        }
      }
    } else if (par == 0) {
      lse_phase<D>(Y, X, sf, h >= 2, rank, csize, sM, sL, fail, &sh.nfail, &sh.misses);
    } else {
      lse_phase<D>(X, Y, sf, h >= 2, rank, csize, sM, sL, fail, &sh.nfail, &sh.misses);
    }
    __syncthreads();
    if (sh.stop) break;  // the same decision in every CTA (identical state copies)
    if (par == 0) epilogue_phase<D>(eg, sh.c[0], Y, sf, sh, 0, rank, csize, sM, sL);
    else epilogue_phase<D>(ef, sh.c[1], X, sf, sh, 1, rank, csize, sM, sL);
    cl.sync();
    ++h;
  }
  const int t = h >> 1;
  // this CTA's rows of the final iterate; rank 0 writes the state
  const float* gl = (t & 1) ? g1 : g0;
  float* gout = (t & 1) ? a.gb1 : a.gb0;
  const int flo = (int)((long long)n * rank / csize), fhi = (int)((long long)n * (rank + 1) / csize);
  const int glo = (int)((long long)m * rank / csize), ghi = (int)((long long)m * (rank + 1) / csize);
  for (int i = flo + threadIdx.x; i < fhi; i += kThreads) a.fst[i] = fs[i];
  for (int j = glo + threadIdx.x; j < ghi; j += kThreads) gout[j] = gl[j];
  if (rank == 0 && threadIdx.x == 0) {
    if (a.ti) {
      epi::slot_doubles(sh.st.slot[0]);
      epi::slot_doubles(sh.st.slot[1]);
    }
    sh.st.iters = t;
    *gst = sh.st;
  }
  cl.sync();  // no CTA leaves while another may still address its shared memory
  if (threadIdx.x == 0 && sh.misses) atomicAdd(&gst->lse_miss, sh.misses);
}

template <int D>
cudaError_t launch_dim(const SmallArgs& a, const EpiParams& eg, const EpiParams& ef, size_t smem, cudaStream_t st) {
  auto kern = k_small_solve<D>;
  cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err == cudaSuccess) err = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  if (err != cudaSuccess) return err;
  // largest cluster (<= 16, no more CTAs than ~32 query rows each) that the device can place
  const int rows = a.n > a.m ? a.n : a.m;
  int want = kMaxCluster;
  while (want > 1 && rows < 32 * want) want >>= 1;
  cudaLaunchConfig_t cfg{};
  cudaLaunchAttribute attr[1];
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  attr[0].id = cudaLaunchAttributeClusterDimension;
  for (int c = want; c >= 1; c >>= 1) {
    cfg.gridDim = dim3(c);
    attr[0].val.clusterDim.x = c;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    int nclusters = 0;
    if (cudaOccupancyMaxActiveClusters(&nclusters, kern, &cfg) != cudaSuccess) {
      (void)cudaGetLastError();
      nclusters = 0;
    }
    if (nclusters >= 1 || c == 1) return cudaLaunchKernelEx(&cfg, kern, a, eg, ef);
  }
  return cudaErrorInvalidConfiguration;
}

}  // namespace

bool small_path(const uot_problem& p) {
  return p.cost_kind == UOT_COST_POINTS && p.dim >= 1 && p.dim <= 3 && p.p == 2.0f &&
         (double)p.n * (double)p.m <= 1048576.0 && small_smem_bytes(p.n, p.m, p.dim) <= kSmemLimit;
}

cudaError_t launch_small_solve(const float* x, const float* y, const float* l2a, const float* l2b, int n, int m,
                               int dim, int ti, int max_iter, int check_every, double tol, double s, float* fst,
                               float* gb0, float* gb1, const EpiParams& eg0, const EpiParams& ef0, cudaStream_t st) {
  (void)l2a;
  (void)l2b;  // carried in eg0 / ef0 (l2w_o)
  SmallArgs a{x, y, n, m, ti, max_iter, check_every, tol, (float)s, fst, gb0, gb1};
  EpiParams eg = eg0, ef = ef0;
  epi_finish_params(eg);
  epi_finish_params(ef);
  const size_t smem = small_smem_bytes(n, m, dim);
  cudaError_t err;
  switch (dim) {
    case 1: err = launch_dim<1>(a, eg, ef, smem, st); break;
    case 2: err = launch_dim<2>(a, eg, ef, smem, st); break;
    default: err = launch_dim<3>(a, eg, ef, smem, st);
  }
  if (err != cudaSuccess) return err;
  note_launch();
  return cudaGetLastError();
}

}  // namespace uot
