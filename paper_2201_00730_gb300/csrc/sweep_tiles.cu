// Fast fused softmin sweep for point clouds in Morton order, dim <= 3, p = 2.
//
// For query point i and key j the exponent of the softmin is (log2 units)
//     t_ij = h_j - s |q_i - k_j|^2,   h_j = log2 w_j + s (pot_j + shift),  s = log2(e)/eps.
// Keys are processed in tiles of kTileKeys consecutive (spatially compact) keys
// with a local origin o = centre of the tile's bounding box.  With q' = q - o,
// k' = k - o:
//     t_ij = H_j + R_i + q'_i . Y_j,   H_j = h_j - s |k'_j|^2,  Y_j = 2 s k'_j,  R_i = -s |q'_i|^2,
// so the per-entry work is dim FMAs (H_j and Y_j are formed once per key when
// the tile is staged; R_i once per row and tile and added when the tile's
// partial is merged, since a per-row constant leaves the log-sum-exp over the
// tile unchanged).  Because tiles and the rows near them are compact, the
// large terms stay of the size of the direct difference form and the FP32
// rounding matches it.
//
// The inner loop runs on packed f32x2 instructions over key pairs (FFMA2 /
// FADD2 / FMUL2: one issue slot for two lanes), one MUFU ex2 per entry, and a
// running max per group of 8 keys.  Each tile's sum (64 terms per lane) is
// added to the row's running sum with Neumaier's compensated addition, so the
// rounding of a chunk's sum does not grow with the number of its tiles.
// Output: per (query, key chunk) partials (max, sum of 2^(t - max)), merged by
// the epilogue (compensated as well).
//
// Fixed-reference mode (fused epilogue with a stored reference, decided per
// launch on the device): inside a Sinkhorn solve a row's log-sum-exp moves
// little between two iterations, so the previous launch's value m_i can stand
// in for the running max.  The sum of 2^(t_ij - m_i) then needs no max and no
// rescaling: per key pair one FADD2 (tile constant R_i - m_i), dim FFMA2, two
// ex2 and one FADD2.  The result is exact as long as |lse_i - m_i| stays inside
// a window far from FP32 over- and underflow; the epilogue checks every row and
// recomputes the rows outside it from scratch (warp per row, running max), so
// a poor reference costs time, never accuracy.
#include <cuda_runtime.h>

#include <mutex>

#include "epi_device.cuh"
#include "sweep_common.cuh"
#include "uot_internal.cuh"

namespace uot {
namespace {

using namespace simd;
constexpr int kThreads = 256;
constexpr int kStageKeys = 512;
constexpr int kTilesPerStage = kStageKeys / kTileKeys;
constexpr int kPairsPerStage = kStageKeys / 2;
constexpr int kPairsPerTile = kTileKeys / 2;

// R = 2 is limited to 80 registers so that 3 CTAs (24 warps) share an SM (at 64
// registers and 4 CTAs it spilled); R = 4 takes up to 128 registers, 2 CTAs.
template <int D, int R, bool EPI>
__global__ void __launch_bounds__(kThreads, (R == 2 ? 3 : 2))
k_sweep_tiles(const float* __restrict__ q, int nq, const float* __restrict__ kp, int nk,
              const float4* __restrict__ centers, const float* __restrict__ l2w, const float* __restrict__ pot,
              const double* __restrict__ shift, double s, int kps, float* __restrict__ part, EpiParams e) {
  static_assert(D >= 1 && D <= 3, "tiled sweep covers dim 1..3");
  // Programmatic dependent launch: this grid may be scheduled while the
  // previous kernel of the stream finishes; it waits here for that kernel's
  // completion (and memory) before reading anything, and lets the next grid
  // be scheduled as soon as all of its own CTAs have started.
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  __shared__ ulonglong2 sA[kPairsPerStage];  // {Y0 pair, Y1 pair}
  __shared__ ulonglong2 sB[kPairsPerStage];  // {Y2 pair, H pair}
  __shared__ float4 sC[kTilesPerStage];
  const int split = blockIdx.y;
  const int j0 = split * kps;  // kps is a multiple of kTileKeys
  const int j1 = min(nk, j0 + kps);
  const float sf = (float)s;
  const float s2 = (float)(2.0 * s);

  bool use_ref = false;
  if constexpr (EPI) use_ref = e.lse_buf != nullptr && e.state->lse_ok[e.out_is_f] != 0;

  float xq[R][3];
  float M[R], acc[R], cmp[R];  // running (max, sum, compensation); in fixed-reference mode M holds the reference
  const int ibase = blockIdx.x * (kThreads * R) + threadIdx.x;
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int i = ibase + r * kThreads;
#pragma unroll
    for (int d = 0; d < 3; ++d) xq[r][d] = (i < nq && d < D) ? q[(size_t)i * D + d] : 0.f;
    M[r] = kInitMax;
    if constexpr (EPI) {
      if (use_ref) M[r] = (i < nq) ? e.lse_buf[i] : 0.f;
    }
    acc[r] = 0.f;
    cmp[r] = 0.f;
  }

  for (int jt = j0; jt < j1; jt += kStageKeys) {
    const int cnt = min(kStageKeys, j1 - jt);
    const int tile0 = jt / kTileKeys;
    __syncthreads();
    if (threadIdx.x < kTilesPerStage)
      sC[threadIdx.x] = (threadIdx.x * kTileKeys < cnt) ? centers[tile0 + threadIdx.x] : make_float4(0.f, 0.f, 0.f, 0.f);
    {
      // one key pair per thread: keys jt + 2p and jt + 2p + 1 of tile (2p / kTileKeys)
      const int p = threadIdx.x;
      const int u0 = 2 * p;
      float Y[2][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
      float H[2] = {kZeroW, kZeroW};
      if (u0 < cnt) {
        const float4 o = centers[tile0 + u0 / kTileKeys];
        const float oc[3] = {o.x, o.y, o.z};
#pragma unroll
        for (int k = 0; k < 2; ++k) {
          const int u = u0 + k;
          if (u < cnt) {
            const int j = jt + u;
            float r2 = 0.f;
#pragma unroll
            for (int d = 0; d < D; ++d) {
              const float yl = kp[(size_t)j * D + d] - oc[d];
              Y[k][d] = s2 * yl;
              r2 = fmaf(yl, yl, r2);
            }
            const float lw = l2w[j];
            if (lw > 0.5f * kZeroW) {
              // H_j = log2 w_j + s pot_j - s |k'_j|^2 in FP32 (two roundings at the size of H);
              // a constant shift of pot is applied exactly to the row result instead.
              const float pj = pot ? pot[j] : 0.f;
              H[k] = fmaf(-sf, r2, fmaf(sf, pj, lw));
            }
          }
        }
      }
      sA[p] = make_ulonglong2(pk(Y[0][0], Y[1][0]), pk(Y[0][1], Y[1][1]));
      sB[p] = make_ulonglong2(pk(Y[0][2], Y[1][2]), pk(H[0], H[1]));
    }
    __syncthreads();
    const int ntiles = (cnt + kTileKeys - 1) / kTileKeys;
    for (int lt = 0; lt < ntiles; ++lt) {
      const float4 o = sC[lt];
      u64 X[R][3];
      float Rr[R], mu[R];
      u64 ac[R];
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const float x0 = xq[r][0] - o.x, x1 = xq[r][1] - o.y, x2 = xq[r][2] - o.z;
        X[r][0] = pk(x0, x0);
        X[r][1] = pk(x1, x1);
        X[r][2] = pk(x2, x2);
        float q2 = x0 * x0;
        if (D > 1) q2 = fmaf(x1, x1, q2);
        if (D > 2) q2 = fmaf(x2, x2, q2);
        Rr[r] = -sf * q2;
        mu[r] = kInitMax;
        ac[r] = pk(0.f, 0.f);
      }
      const ulonglong2* A = sA + lt * kPairsPerTile;
      const ulonglong2* B = sB + lt * kPairsPerTile;
      if (use_ref) {
        // exponent t_ij - m_i = H_j + q'_i . Y_j + (R_i - m_i)
        u64 cc[R];
#pragma unroll
        for (int r = 0; r < R; ++r) { const float c0 = Rr[r] - M[r]; cc[r] = pk(c0, c0); }
#pragma unroll 2
        for (int pp = 0; pp < kPairsPerTile; pp += 4) {
          ulonglong2 a[4], b[4];
#pragma unroll
          for (int k = 0; k < 4; ++k) { a[k] = A[pp + k]; b[k] = B[pp + k]; }
#pragma unroll
          for (int r = 0; r < R; ++r) {
#pragma unroll
            for (int k = 0; k < 4; ++k) {
              u64 v = add2(b[k].y, cc[r]);
              if (D > 2) v = fma2(X[r][2], b[k].x, v);
              if (D > 1) v = fma2(X[r][1], a[k].y, v);
              v = fma2(X[r][0], a[k].x, v);
              float w0, w1;
              upk(v, w0, w1);
              ac[r] = add2(ac[r], pk(ex2f(w0), ex2f(w1)));
            }
          }
        }
#pragma unroll
        for (int r = 0; r < R; ++r) {
          float a0, a1;
          upk(ac[r], a0, a1);
          neu_add(acc[r], cmp[r], a0 + a1);
        }
        continue;
      }
#pragma unroll 2
      for (int pp = 0; pp < kPairsPerTile; pp += 4) {
        ulonglong2 a[4], b[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) { a[k] = A[pp + k]; b[k] = B[pp + k]; }
#pragma unroll
        for (int r = 0; r < R; ++r) {
          u64 u[4];
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            u64 v = b[k].y;
            if (D > 2) v = fma2(X[r][2], b[k].x, v);
            if (D > 1) v = fma2(X[r][1], a[k].y, v);
            u[k] = fma2(X[r][0], a[k].x, v);
          }
          float uf[8];
#pragma unroll
          for (int k = 0; k < 4; ++k) upk(u[k], uf[2 * k], uf[2 * k + 1]);
          const float gm = max3f(max3f(uf[0], uf[1], uf[2]), max3f(uf[3], uf[4], uf[5]), fmaxf(uf[6], uf[7]));
          const float mn = fmaxf(mu[r], gm);
          const float sc = ex2f(mu[r] - mn);
          mu[r] = mn;
          const u64 nm = pk(-mn, -mn);
          u64 a2 = mul2(ac[r], pk(sc, sc));
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            float w0, w1;
            upk(add2(u[k], nm), w0, w1);
            a2 = add2(a2, pk(ex2f(w0), ex2f(w1)));
          }
          ac[r] = a2;
        }
      }
      // merge the tile's partial (in the frame shifted by R_i) into the running pair
#pragma unroll
      for (int r = 0; r < R; ++r) {
        float a0, a1;
        upk(ac[r], a0, a1);
        const float MT = mu[r] + Rr[r];
        const float Mn = fmaxf(M[r], MT);
        const float so = ex2f(M[r] - Mn);
        acc[r] *= so;
        cmp[r] *= so;
        neu_add(acc[r], cmp[r], (a0 + a1) * ex2f(MT - Mn));
        M[r] = Mn;
      }
    }
  }
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int i = ibase + r * kThreads;
    if (i < nq) {
      float* base = part + (size_t)split * 2 * nq;
      base[i] = M[r];
      base[(size_t)nq + i] = acc[r] + cmp[r];
    }
  }
  if constexpr (EPI) {
    // The last CTA of this row block to finish merges the row block's partials
    // and applies the half-step; the last row block finishes the scalars.
    if (!epi::arrive_last(&e.rb_counter[blockIdx.x], gridDim.y)) return;
    if (threadIdx.x == 0) e.rb_counter[blockIdx.x] = 0;
    const int r1 = min(nq, blockIdx.x * (kThreads * R) + kThreads * R);
    int idx[R];
    epi::Pre pre[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int i = ibase + r * kThreads;
      idx[r] = (i < r1) ? i : -1;
      pre[r] = epi::prefetch(e, idx[r]);
    }
    float Mg[R], Lg[R];
    if (use_ref) epi::merge_rows_ref<R, 16>(part, 2, nq, gridDim.y, idx, M, Mg, Lg);
    else epi::merge_rows<R>(part, 2, nq, gridDim.y, idx, Mg, Lg);
    if (use_ref) {
      // rows whose log-sum-exp left the window around the reference are listed,
      // recomputed (one warp each) into chunk 0 of their partials, and merged again
      __shared__ int s_nbad;
      int* s_bad = reinterpret_cast<int*>(sA);  // kThreads * R ints fit in sA
      static_assert(sizeof(int) * kThreads * 4 <= sizeof(ulonglong2) * kPairsPerStage, "bad-row list size");
      if (threadIdx.x == 0) s_nbad = 0;
      __syncthreads();
      bool redo[R];
#pragma unroll
      for (int r = 0; r < R; ++r) {
        redo[r] = false;
        if (idx[r] >= 0 && !(fabsf((Mg[r] + Lg[r]) - M[r]) <= (float)kLseWindow)) {
          redo[r] = true;
          s_bad[atomicAdd(&s_nbad, 1)] = idx[r];
        }
      }
      __syncthreads();
      const int nbad = s_nbad;
      if (nbad > 0) {
        const int lane = threadIdx.x & 31;
        for (int k = threadIdx.x >> 5; k < nbad; k += kThreads / 32) {
          const int i = s_bad[k];
          float Mx, Sx;
          exact_row<D>(q + (size_t)i * D, kp, nk, l2w, pot, sf, lane, Mx, Sx);
          for (int sp = lane; sp < (int)gridDim.y; sp += 32) {
            float* base = part + (size_t)sp * 2 * nq;
            base[i] = sp == 0 ? Mx : kInitMax;
            base[(size_t)nq + i] = sp == 0 ? Sx : 0.f;
          }
        }
        if (threadIdx.x == 0) atomicAdd(&e.state->lse_miss, (unsigned)nbad);
        __syncthreads();
#pragma unroll
        for (int r = 0; r < R; ++r) {
          if (redo[r]) {
            int one[1] = {idx[r]};
            float m1[1], l1[1];
            epi::merge_rows<1>(part, 2, nq, gridDim.y, one, m1, l1);
            Mg[r] = m1[0];
            Lg[r] = l1[0];
          }
        }
      }
    }
    const epi::Consts& c = epi::block_consts(e);
    epi::RowAcc ea = epi::rowacc_empty();
#pragma unroll
    for (int r = 0; r < R; ++r)
      if (idx[r] >= 0) epi::row_ff(e, c, idx[r], Mg[r], Lg[r], pre[r], ea);
    epi::block_finish(e, ea, blockIdx.x, gridDim.x);
  }
}

template <int D, int R>
int occupancy() {
  static int occ[4][5] = {};
  static std::mutex mu;
  std::lock_guard<std::mutex> lk(mu);
  if (occ[D][R] == 0) {
    int v = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, k_sweep_tiles<D, R, true>, kThreads, 0) != cudaSuccess ||
        v < 1)
      v = 2;
    occ[D][R] = v;
  }
  return occ[D][R];
}

int occupancy_for(int dim, int R) {
  switch (dim * 10 + R) {
    case 12: return occupancy<1, 2>();
    case 14: return occupancy<1, 4>();
    case 22: return occupancy<2, 2>();
    case 24: return occupancy<2, 4>();
    case 32: return occupancy<3, 2>();
    default: return occupancy<3, 4>();
  }
}

template <int D, int R>
cudaError_t run(const SideDesc& q, const SideDesc& k, const float4* centers, const float* pot, const double* shift,
                double s, float* part, const SweepGeom& g, const EpiParams* epi, cudaStream_t st) {
  dim3 grid(g.row_blocks, g.splits);
  if (epi) {
    EpiParams e = *epi;
    epi_finish_params(e);
    // launched with programmatic stream serialisation: the launch latency of
    // one half-step hides behind the previous half-step's epilogue tail
    cudaLaunchConfig_t cfg{};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.gridDim = grid;
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaError_t err = cudaLaunchKernelEx(&cfg, k_sweep_tiles<D, R, true>, q.pts, q.n, k.pts, k.n, centers, k.l2w,
                                         pot, shift, s, g.keys_per_split, part, e);
    if (err != cudaSuccess) return err;
  } else {
    EpiParams none{};
    k_sweep_tiles<D, R, false><<<grid, kThreads, 0, st>>>(q.pts, q.n, k.pts, k.n, centers, k.l2w, pot, shift, s,
                                                          g.keys_per_split, part, none);
  }
  note_launch();
  return cudaGetLastError();
}

}  // namespace

SweepGeom tile_geom(int nq, int nk, int dim, bool tuned) {
  SweepGeom g{};
  g.threads = kThreads;
  const int sms = device_sm_count();
  const long long entries = (long long)nq * nk;
  // 4 rows per thread (half the shared-memory loads per entry, 2 CTAs of 128
  // registers per SM) once there are a few row blocks; 2 rows (3 CTAs of 80
  // registers per SM) for small query sets, where more CTAs balance better
  int R = (nq >= 4096) ? 4 : 2;
  if (tuned) R = (int)tune_value("tile.rows", dim, entries, R);
  // row blocks index per-block counters and partial slots (kMaxBlocks of each)
  if ((nq + kThreads * R - 1) / (kThreads * R) > kMaxBlocks) R = 4;
  g.rows = R;
  const int rows_per_cta = kThreads * R;
  g.row_blocks = (nq + rows_per_cta - 1) / rows_per_cta;
  const double cta_cost = tuned ? 0.1 * (double)tune_value("tile.cta_cost", dim, entries, 15) : 1.5;
  // at least this many waves of CTAs when the keys allow it: with several waves
  // an SM whose resident CTA ends early takes the next one instead of idling
  const int min_waves = tuned ? (int)tune_value("tile.waves", dim, entries, 1) : 1;
  const long long target = (long long)sms * occupancy_for(dim, R);
  const int max_tiles = (nk + kTileKeys - 1) / kTileKeys;
  // Pick the number of key chunks minimising (waves of CTAs) x (tiles per CTA +
  // a fixed per-CTA cost, by default 1.5 tiles: staging, merges, partial write).
  // A chunk is a whole number of tiles.
  double best = 1e300;
  int best_k = 1;
  for (int k = 1; k <= 512 && k <= max_tiles; ++k) {
    const int tiles_per = (max_tiles + k - 1) / k;
    const int kk = (max_tiles + tiles_per - 1) / tiles_per;
    if (kk != k) continue;
    const long long ctas = (long long)g.row_blocks * kk;
    const long long waves = (ctas + target - 1) / target;
    if (waves < min_waves && tiles_per > 1) continue;
    const double est = (double)waves * (tiles_per + cta_cost);
    if (est < best * 0.999) { best = est; best_k = kk; }
  }
  const int tiles_per = (max_tiles + best_k - 1) / best_k;
  g.keys_per_split = tiles_per * kTileKeys;
  g.splits = (nk + g.keys_per_split - 1) / g.keys_per_split;
  return g;
}

cudaError_t launch_tile_sweep(const SideDesc& q, const SideDesc& k, const float4* centers_k, int dim,
                              const float* pot_k, const double* shift_k, double s, float* part, const SweepGeom& g,
                              const EpiParams* epi, cudaStream_t st) {
  switch (dim * 10 + g.rows) {
    case 12: return run<1, 2>(q, k, centers_k, pot_k, shift_k, s, part, g, epi, st);
    case 14: return run<1, 4>(q, k, centers_k, pot_k, shift_k, s, part, g, epi, st);
    case 22: return run<2, 2>(q, k, centers_k, pot_k, shift_k, s, part, g, epi, st);
    case 24: return run<2, 4>(q, k, centers_k, pot_k, shift_k, s, part, g, epi, st);
    case 32: return run<3, 2>(q, k, centers_k, pot_k, shift_k, s, part, g, epi, st);
    default: return run<3, 4>(q, k, centers_k, pot_k, shift_k, s, part, g, epi, st);
  }
}

}  // namespace uot
