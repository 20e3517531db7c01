// Device-side half-step epilogue shared by the standalone combine kernel and
// the sweeps that finish their own rows (last CTA of a row block).
//
// Per query row i: merge the key-chunk partials into the softmin
// S_i = -(max + log2 sum)/s, then apply the half-step of the mode:
//   softmin : out_i = S_i
//   plain   : out_i = rho_o/(rho_o+eps) S_i                          (aprox for rho KL, Sec. 3)
//   TI      : out_i = rho_o/(rho_o+eps) S_i - eps/(eps+rho_o) rho_o/(rho_o+rho_i) X_in
//             with the mass sum_i w_i e^{-out_i/rho_o}                      (proof of Prop. 4, App. B)
// and the residual against the previous vector.  The per-row arithmetic runs
// on float pairs (ffloat.cuh: FP64 is slow here), the mass terms through a
// table-driven exp2, summed per block against an integer power-of-two
// reference; blocks combine in FP64.  Grid-level results are reduced by the
// last block to arrive (no block ever waits on another).
//
// With e.lse_buf the raw log-sum-exp of every row (log2 units, before the key
// shift) is kept between launches of the same side, and the largest change
// since the previous launch decides whether the next launch of that side may
// take the stored value as its fixed exponent reference (see the tiled sweep).
#pragma once

#include <cuda_runtime.h>
#include <math.h>

#include <climits>

#include "ffloat.cuh"
#include "sweep_common.cuh"
#include "uot_internal.cuh"

namespace uot {
namespace epi {

__device__ __forceinline__ float ex2f(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Merge of the key-chunk partials of R query rows at once (all loads of a group
// of 8 chunks issued before any use): per row the pair (M, log2 S) with
// log-sum-exp = M + log2 S in log2 units.  The chunk sums are added with
// Neumaier's compensation (the compensation rescaled with the sum).
template <int R>
__device__ __forceinline__ void merge_rows(const float* part, int CH, int nq, int splits, const int (&idx)[R],
                                           float (&Mo)[R], float (&Lo)[R]) {
  const size_t stride = (size_t)CH * nq;
  float M[R], S[R], C[R];
#pragma unroll
  for (int r = 0; r < R; ++r) { M[r] = kInitMax; S[r] = 0.f; C[r] = 0.f; }
  for (int k0 = 0; k0 < splits; k0 += 8) {
    float mv[R][8], sv[R][8];
#pragma unroll
    for (int r = 0; r < R; ++r) {
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int k = k0 + u;
        if (k < splits && idx[r] >= 0) {
          const float* b = part + (size_t)k * stride;
          mv[r][u] = __ldcg(b + idx[r]);
          sv[r][u] = __ldcg(b + (size_t)nq + idx[r]);
        } else {
          mv[r][u] = kInitMax;
          sv[r][u] = 0.f;
        }
      }
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
      float cm = M[r];
#pragma unroll
      for (int u = 0; u < 8; ++u) cm = fmaxf(cm, mv[r][u]);
      const float so = ex2f(M[r] - cm);
      float a = S[r] * so, c = C[r] * so;
#pragma unroll
      for (int u = 0; u < 8; ++u) simd::neu_add(a, c, sv[r][u] * ex2f(mv[r][u] - cm));
      S[r] = a;
      C[r] = c;
      M[r] = cm;
    }
  }
#pragma unroll
  for (int r = 0; r < R; ++r) { Mo[r] = M[r]; Lo[r] = log2f(S[r] + C[r]); }
}

// The same when every chunk's partial was taken against the same reference
// ref[r] (fixed-reference sweeps): the maxima are ref and the merge is a plain
// sum of the chunks' sums, in the same order and with the same result as
// merge_rows, without the maxima's loads and the rescaling exponentials.
// G chunks' loads are issued together (one round trip per G chunks).
template <int R, int G = 8>
__device__ __forceinline__ void merge_rows_ref(const float* part, int CH, int nq, int splits, const int (&idx)[R],
                                               const float (&ref)[R], float (&Mo)[R], float (&Lo)[R]) {
  const size_t stride = (size_t)CH * nq;
  float S[R], C[R];
#pragma unroll
  for (int r = 0; r < R; ++r) { S[r] = 0.f; C[r] = 0.f; }
  for (int k0 = 0; k0 < splits; k0 += G) {
    float sv[R][G];
#pragma unroll
    for (int r = 0; r < R; ++r) {
#pragma unroll
      for (int u = 0; u < G; ++u) {
        const int k = k0 + u;
        sv[r][u] = (k < splits && idx[r] >= 0) ? __ldcg(part + (size_t)k * stride + (size_t)nq + idx[r]) : 0.f;
      }
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
#pragma unroll
      for (int u = 0; u < G; ++u) simd::neu_add(S[r], C[r], sv[r][u]);
    }
  }
#pragma unroll
  for (int r = 0; r < R; ++r) { Mo[r] = ref[r]; Lo[r] = log2f(S[r] + C[r]); }
}

// Per-launch constants of the half-step as float pairs, made once per block
// (thread 0, FP32 only: the FP64 parts come precomputed from the host and the
// state's float-pair copies) and read from shared memory by the rows.
struct Consts {
  ffl::ff U;    // 1/s = eps ln 2 (log2 units -> cost units)
  ffl::ff KS;   // constant shift of the key potential left out by the sweep
  ffl::ff CS;   // aprox factor rho_o/(rho_o+eps)
  ffl::ff CXX;  // TI: eps/(eps+rho_o) rho_o/(rho_o+rho_i) * key-side Smin scalar
  ffl::ff K1;   // TI residual: stored hat + shift - (the part of the next step fixed by the other side)
  ffl::ff RL;   // log2(e)/rho_o (mass exponent)
  int lse_ready;
  const ffl::Exp2Table* tab;  // exp2 table (global, or a shared-memory copy)
};

__device__ __forceinline__ ffl::ff pair(const float (&v)[2]) { return ffl::ff{v[0], v[1]}; }

__device__ inline Consts make_consts(const EpiParams& e) {
  using namespace ffl;
  const Slot& si = e.state->slot[e.slot_in];
  const ff Xin = pair(e.out_is_f ? si.Bf : si.Af);    // key-side Smin^rho scalar
  const ff base_old = pair(e.out_is_f ? si.cff : si.cgf);  // stored hat + shift = bar
  const ff own = pair(e.out_is_f ? si.Af : si.Bf);
  Consts c;
  c.U = pair(e.U2);
  const ff shift = pair(e.out_is_f ? si.cgf : si.cff);  // the key side's pending shift
  c.KS = e.key_shift ? shift : ff{0.f, 0.f};            // null: the sweep applied it
  c.CS = pair(e.CS2);
  // G-Sinkhorn: the output moves with the key shift (v = aprox(S) + shift)
  c.CXX = e.mode == EPI_G ? neg(shift) : mul(pair(e.CX2), Xin);
  c.K1 = add(base_old, neg(mul(pair(e.CR2), own)));
  c.RL = pair(e.RL2);
  c.lse_ready = e.lse_buf ? e.state->lse_ready[e.out_is_f] : 0;
  c.tab = &kExp2Tab;
  return c;
}

// The threads that run an epilogue together: the whole block (barrier 0), or
// a group of whole warps that synchronises on its own named barrier (the
// consumer warps of a warp-specialised sweep).  tid is the thread's index in
// the group, n the group's size (a multiple of 32).
struct Grp {
  int tid, n, bar;
  __device__ __forceinline__ void sync() const {
    if (bar == 0) __syncthreads();
    else asm volatile("bar.sync %0, %1;" ::"r"(bar), "r"(n) : "memory");
  }
};

__device__ __forceinline__ Grp whole_block() { return Grp{(int)threadIdx.x, (int)blockDim.x, 0}; }

// Group-wide constants: the group's thread 0 computes, everyone reads (one barrier).
__device__ __forceinline__ const Consts& block_consts(const EpiParams& e, const Grp& g) {
  __shared__ Consts sc;
  if (g.tid == 0) sc = make_consts(e);
  g.sync();
  return sc;
}
__device__ __forceinline__ const Consts& block_consts(const EpiParams& e) { return block_consts(e, whole_block()); }

// Row inputs read ahead of the merge.
struct Pre {
  float lwh, lwl;  // log2 w of the output side as a float pair (TI mass term)
  float old;       // previous output (residual)
  float prev;      // previous log-sum-exp of the row (fixed-reference bookkeeping)
};

__device__ __forceinline__ Pre prefetch(const EpiParams& e, int i) {
  Pre p;
  const bool ti = (e.mode == EPI_TI || e.mode == EPI_G) && i >= 0;
  p.lwh = ti ? e.l2w_o[i] : 0.f;
  p.lwl = ti ? e.l2lo_o[i] : 0.f;
  p.old = (e.old_out && i >= 0) ? e.old_out[i] : 0.f;
  p.prev = (e.lse_buf && i >= 0) ? e.lse_buf[i] : 0.f;
  return p;
}

// Thread-level accumulator of the rows: TI mass sum_i 2^(y_i) kept as
// 2^ref * (sum.hi + sum.lo) with an integer ref (rescaling is exact).
struct RowAcc {
  int ref;       // INT_MIN: no term yet
  ffl::ff sum;
  float r;       // residual max
  float gap;     // max |lse - previous lse|
  int bad;
};

__device__ __forceinline__ RowAcc rowacc_empty() { return RowAcc{INT_MIN, ffl::ff{0.f, 0.f}, 0.f, 0.f, 0}; }

// a * 2^-k for k >= 0; below 2^-100 of the reference a term no longer matters
// (every sum holds a term of at least half its reference).
__device__ __forceinline__ ffl::ff scale2(ffl::ff a, int k) {
  if (k > 100) return ffl::ff{0.f, 0.f};
  const float sc = ffl::pow2f(-k);
  return ffl::ff{a.hi * sc, a.lo * sc};
}

// Adds the mass term 2^y (y a float pair, |y| < 1e9) to the accumulator: the sum
// is kept against the integer reference ceil(y) of its largest term, so every
// rescaling is by an exact power of two.
__device__ __forceinline__ void mass_add(RowAcc& a, const ffl::ff& y, const ffl::Exp2Table& tab) {
  const int yr = (int)ceilf(y.hi);
  if (a.ref == INT_MIN) a.ref = yr;
  else if (yr > a.ref) { a.sum = scale2(a.sum, yr - a.ref); a.ref = yr; }
  a.sum = ffl::add(a.sum, ffl::exp2(ffl::add(y, (float)(-a.ref)), tab));
}

// Half-step of one query row from its merged log-sum-exp M + L (log2 units);
// returns the value stored in the output vector.
__device__ __forceinline__ float row_ff(const EpiParams& e, const Consts& c, int i, float M, float L, const Pre& p,
                                        RowAcc& a) {
  using namespace ffl;
  const ff lse = two_sum(M, L);
  if (!(lse.hi > 0.25f * kZeroW)) a.bad = 1;  // every key had zero weight (or NaN)
  if (e.lse_buf) {
    const float d = fabsf(lse.hi - p.prev);
    if (!c.lse_ready || !(d <= 1e30f) || !(lse.hi > 0.25f * kZeroW)) a.gap = INFINITY;
    else a.gap = fmaxf(a.gap, d);
    e.lse_buf[i] = lse.hi;
  }
  // Smin in cost units; a shift tau of the key potential moves it by -tau exactly
  const ff S = neg(add(mul(lse, c.U), c.KS));
  ff v = S;
  if (e.mode != EPI_SOFTMIN) v = mul(S, c.CS);
  if (e.mode == EPI_TI || e.mode == EPI_G) v = add(v, neg(c.CXX));
  const float vo = v.hi + v.lo;
  if (!isfinite(vo)) a.bad = 1;
  e.out[e.perm_out ? e.perm_out[i] : i] = vo;
  if (e.old_out) {
    const ff d = (e.mode == EPI_TI) ? add(add(c.K1, p.old), neg(v)) : add(neg(v), p.old);
    a.r = fmaxf(a.r, fabsf(d.hi + d.lo));
  }
  if ((e.mode == EPI_TI || e.mode == EPI_G) && p.lwh > 0.5f * kZeroW) {
    // mass term w_i e^{-v/rho_o} = 2^y, y = log2 w_i - v log2(e)/rho_o
    const ff y = add(ff{p.lwh, p.lwl}, neg(mul(v, c.RL)));
    if (!(fabsf(y.hi) < 1e9f)) {
      a.bad = 1;
      return vo;
    }
    mass_add(a, y, *c.tab);
  }
  return vo;
}

// The old per-row interface (merge + half-step), used by the combine kernel.
__device__ __forceinline__ void row(const EpiParams& e, const Consts& c, int i, RowAcc& a) {
  const Pre p = prefetch(e, i);
  int idx[1] = {i};
  float M[1], L[1];
  merge_rows<1>(e.part, 2 + e.moments, e.nq, e.splits, idx, M, L);
  row_ff(e, c, i, M[0], L[0], p, a);
}

// Last-arriver test of a group of blocks.  The group's barrier orders every
// thread's earlier writes before thread 0's fence (fences are cumulative), so
// one fence before the increment publishes the whole block's writes, and one
// after it (last arriver only) orders the other blocks' writes before what
// the group reads next.
__device__ __forceinline__ bool arrive_last(unsigned int* counter, unsigned int total, const Grp& g) {
  __shared__ bool last;
  g.sync();
  if (g.tid == 0) {
    __threadfence();
    last = (atomicAdd(counter, 1u) == total - 1);
    if (last) __threadfence();
  }
  g.sync();
  return last;
}
__device__ __forceinline__ bool arrive_last(unsigned int* counter, unsigned int total) {
  return arrive_last(counter, total, whole_block());
}

// Partial of one block (and of the grid, once reduced): the TI mass as
// 2^ref * (hi + lo), residual and lse-change maxima, non-finite flag.
struct Part {
  int ref, bad;
  float hi, lo, r, gap;
};

__device__ __forceinline__ Part part_merge(Part a, const Part& b) {
  if (b.ref != INT_MIN) {
    if (a.ref == INT_MIN) { a.ref = b.ref; a.hi = b.hi; a.lo = b.lo; }
    else if (b.ref > a.ref) {
      const ffl::ff s = ffl::add(scale2(ffl::ff{a.hi, a.lo}, b.ref - a.ref), ffl::ff{b.hi, b.lo});
      a.ref = b.ref; a.hi = s.hi; a.lo = s.lo;
    } else {
      const ffl::ff s = ffl::add(ffl::ff{a.hi, a.lo}, scale2(ffl::ff{b.hi, b.lo}, a.ref - b.ref));
      a.hi = s.hi; a.lo = s.lo;
    }
  }
  a.bad = max(a.bad, b.bad);
  a.r = fmaxf(a.r, b.r);
  a.gap = fmaxf(a.gap, b.gap);
  return a;
}

__device__ __forceinline__ Part part_shfl(const Part& p, int off) {
  Part o;
  o.ref = __shfl_xor_sync(0xffffffffu, p.ref, off);
  o.bad = __shfl_xor_sync(0xffffffffu, p.bad, off);
  o.hi = __shfl_xor_sync(0xffffffffu, p.hi, off);
  o.lo = __shfl_xor_sync(0xffffffffu, p.lo, off);
  o.r = __shfl_xor_sync(0xffffffffu, p.r, off);
  o.gap = __shfl_xor_sync(0xffffffffu, p.gap, off);
  return o;
}

// Warp-wide reduction of the partials, the result on every lane: the largest
// reference by an integer reduction, each lane's sum rescaled to it (exact
// powers of two), a butterfly of float-pair sums (commutative, so every lane
// ends with the same pair), and the maxima and flag by integer reductions
// (r and gap are >= +0, so their bit patterns order like their values).
__device__ __forceinline__ Part warp_reduce(const Part& p) {
  const int R = __reduce_max_sync(0xffffffffu, p.ref);
  ffl::ff s{0.f, 0.f};
  if (p.ref != INT_MIN) s = scale2(ffl::ff{p.hi, p.lo}, R - p.ref);
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const ffl::ff o{__shfl_xor_sync(0xffffffffu, s.hi, off), __shfl_xor_sync(0xffffffffu, s.lo, off)};
    s = ffl::add(s, o);
  }
  Part q;
  q.ref = R;
  q.hi = s.hi;
  q.lo = s.lo;
  q.bad = __reduce_or_sync(0xffffffffu, (unsigned)p.bad) ? 1 : 0;
  q.r = __uint_as_float(__reduce_max_sync(0xffffffffu, __float_as_uint(p.r)));
  q.gap = __uint_as_float(__reduce_max_sync(0xffffffffu, __float_as_uint(p.gap)));
  return q;
}

// Thread 0 of the last block: scalars of the half-step, residual, status.
// Float-pair arithmetic throughout; the FP64 copies of the slot are written
// last (skipped with e.ff_only) so that nothing waits on the FP64 pipe.
__device__ inline void finalize(const EpiParams& e, const Part& t, const ffl::Exp2Table& tab = ffl::kExp2Tab) {
  using namespace ffl;
  DevState* st = e.state;
  int status = st->status;
  if (t.bad != 0 || isnan(t.r)) status |= kStatusNonfinite;
  if (e.mode == EPI_TI) {
    // log <w, e^{-hat/rho_o}> = ref ln 2 + ln(hi + lo) (empty sum: -inf)
    const bool empty = t.ref == INT_MIN || !(t.hi > 0.f);
    const ff lse = empty ? ff{-INFINITY, 0.f} : add(mul(kLn2ff, from_int(t.ref)), log_ff(ff{t.hi, t.lo}, tab));
    const ff Xhat = mul(lse, pair(e.NR2));           // Smin_w^rho_o(hat) = -rho_o lse
    const ff c = mul(Xhat, pair(e.KK2));             // closed-form translation k/(1-k) Xhat
    const ff X = add(Xhat, c);                       // Smin(hat + c) = Smin(hat) + c
    if (!isfinite(X.hi) || !isfinite(X.lo)) status |= kStatusNonfinite;
    Slot& so = st->slot[e.slot_out];
    ff lam{0.f, 0.f};
    if (e.out_is_f) {
      so.Af[0] = X.hi; so.Af[1] = X.lo; so.cff[0] = c.hi; so.cff[1] = c.lo;
      // lambda* = tau1 Smin_b(gb) - tau2 Smin_a(fb)
      lam = add(mul(pair(e.T12), pair(so.Bf)), neg(mul(pair(e.T22), X)));
      so.lamf[0] = lam.hi; so.lamf[1] = lam.lo;
    } else {
      so.Bf[0] = X.hi; so.Bf[1] = X.lo; so.cgf[0] = c.hi; so.cgf[1] = c.lo;
    }
    if (e.old_out) {
      st->resid = t.r;
      if (e.resid_hist) e.resid_hist[e.loop_ctl ? st->loop_t : e.hist_index] = t.r;
    }
    st->status = status;
    if (!e.ff_only) {
      if (e.out_is_f) { so.A = to_double(X); so.cf = to_double(c); so.lam = to_double(lam); }
      else { so.B = to_double(X); so.cg = to_double(c); }
    }
  } else if (e.mode == EPI_G) {
    // Smin_w^rho_o of the new iterate; after the f half-step lambda_{t+1} =
    // tau1 Smin_b(gb_{t+1}) - tau2 Smin_a(fb_{t+1}) (Prop. 2), which the next
    // g half-step adds to its keys (cf) and the f half-step after it
    // subtracts (cg, set by the g half-step from the slot it read)
    const bool empty = t.ref == INT_MIN || !(t.hi > 0.f);
    const ff lse = empty ? ff{-INFINITY, 0.f} : add(mul(kLn2ff, from_int(t.ref)), log_ff(ff{t.hi, t.lo}, tab));
    const ff X = mul(lse, pair(e.NR2));
    if (!isfinite(X.hi) || !isfinite(X.lo)) status |= kStatusNonfinite;
    Slot& so = st->slot[e.slot_out];
    ff lam{0.f, 0.f}, cg{0.f, 0.f};
    if (e.out_is_f) {
      so.Af[0] = X.hi; so.Af[1] = X.lo;
      lam = add(mul(pair(e.T12), pair(so.Bf)), neg(mul(pair(e.T22), X)));
      so.lamf[0] = lam.hi; so.lamf[1] = lam.lo;
      so.cff[0] = lam.hi; so.cff[1] = lam.lo;
    } else {
      cg = neg(pair(st->slot[e.slot_in].cff));
      so.Bf[0] = X.hi; so.Bf[1] = X.lo;
      so.cgf[0] = cg.hi; so.cgf[1] = cg.lo;
    }
    if (e.old_out) {
      st->resid = t.r;
      if (e.resid_hist) e.resid_hist[e.loop_ctl ? st->loop_t : e.hist_index] = t.r;
    }
    st->status = status;
    if (!e.ff_only) {
      if (e.out_is_f) { so.A = to_double(X); so.cf = to_double(lam); so.lam = so.cf; }
      else { so.B = to_double(X); so.cg = to_double(cg); }
    }
  } else {
    if (e.old_out) {
      st->resid = t.r;
      if (e.resid_hist) e.resid_hist[e.loop_ctl ? st->loop_t : e.hist_index] = t.r;
    }
    st->status = status;
  }
  if (e.lse_buf) {
    // policy 2: always use the stored reference; 0: only after a small change
    const int side = e.out_is_f;
    st->lse_ok[side] = (e.lse_policy == 2) || (e.lse_policy == 0 && t.gap <= (float)kLseGate);
    st->lse_ready[side] = 1;
  }
  if (e.loop_ctl == 1) {
    st->loop_t += 1;
  } else if (e.loop_ctl == 2) {
    // the host driver's stopping rule at iterate loop_t, whose residual this g half-step measured:
    // tested at every check_every-th iterate and at max_iter; a non-finite state also stops
    const int it = st->loop_t;
    const bool last = it >= e.loop_max_iter;
    bool stop = false;
    if (it >= 1 && (last || (e.loop_tol > 0.0 && it % e.loop_check_every == 0)))
      stop = st->status != 0 || isnan(t.r) || last || (double)t.r <= e.loop_tol;
    st->loop_done = stop ? 1 : 0;
    if (e.cond_while) cudaGraphSetConditional(e.cond_while, stop ? 0u : 1u);
    if (e.cond_if) cudaGraphSetConditional(e.cond_if, stop ? 0u : 1u);
  }
}

// The FP64 copies of a slot from its float pairs.
__device__ inline void slot_doubles(Slot& s) {
  s.A = ffl::to_double(pair(s.Af));
  s.B = ffl::to_double(pair(s.Bf));
  s.cf = ffl::to_double(pair(s.cff));
  s.cg = ffl::to_double(pair(s.cgf));
  s.lam = ffl::to_double(pair(s.lamf));
}

// Grid-level tail: block partial -> blk[slot]; the last of `nblocks` arrivals
// reduces all partials in its first warp (exact power-of-two rescaling, no
// exponentials) and finalises.
__device__ inline void grid_tail(const EpiParams& e, const Part& mine, int slot, int nblocks, const Grp& g) {
  Part* bp = reinterpret_cast<Part*>(e.blk);
  if (g.tid == 0) bp[slot] = mine;
  if (!arrive_last(&e.state->counter, (unsigned)nblocks, g)) return;
  if (g.tid >= 32) return;
  Part t{INT_MIN, 0, 0.f, 0.f, 0.f, 0.f};
  for (int k = g.tid; k < nblocks; k += 32) {
    const Part* o = bp + k;
    Part q;
    q.ref = __ldcg(&o->ref); q.bad = __ldcg(&o->bad); q.hi = __ldcg(&o->hi); q.lo = __ldcg(&o->lo);
    q.r = __ldcg(&o->r); q.gap = __ldcg(&o->gap);
    t = part_merge(t, q);
  }
  t = warp_reduce(t);
  if (g.tid == 0) {
    finalize(e, t);
    e.state->counter = 0;
  }
}

// Block reduction of the thread accumulators, then the grid-level tail.
__device__ inline void block_finish(const EpiParams& e, const RowAcc& a, int slot, int nblocks, const Grp& g) {
  __shared__ Part sp[32];
  const int lane = g.tid & 31, warp = g.tid >> 5, nw = g.n >> 5;
  Part p{a.ref, a.bad, a.sum.hi, a.sum.lo, a.r, a.gap};
  p = warp_reduce(p);
  if (lane == 0) sp[warp] = p;
  g.sync();
  if (warp == 0) {
    Part q = (lane < nw) ? sp[lane] : Part{INT_MIN, 0, 0.f, 0.f, 0.f, 0.f};
    q = warp_reduce(q);
    if (lane == 0) sp[0] = q;
  }
  g.sync();
  grid_tail(e, sp[0], slot, nblocks, g);
}
__device__ inline void block_finish(const EpiParams& e, const RowAcc& a, int slot, int nblocks) {
  block_finish(e, a, slot, nblocks, whole_block());
}

}  // namespace epi
}  // namespace uot
