// C ABI of libuot (declared in include/uot.h): argument validation, workspace
// layout, and the host-side iteration driver of plain and translation-invariant
// Sinkhorn.  All arithmetic runs in the kernels of sweep_points.cu,
// sweep_dense.cu and epilogue.cu.
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <atomic>
#include <algorithm>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "uot_internal.cuh"

namespace uot {

namespace {
thread_local std::string g_last_error;
std::atomic<uint64_t> g_launches{0};

// Per-thread sweep profile: event pairs around each sweep launch.
struct Profile {
  bool open = false;
  std::vector<cudaEvent_t> ev;  // 2 per timed launch, created lazily
  size_t used = 0;              // events recorded
  int64_t launches = 0;
};
thread_local Profile g_prof;
constexpr size_t kMaxTimed = 65536;

uot_status fail(uot_status s, const char* fmt, ...) __attribute__((format(printf, 2, 3)));
uot_status fail(uot_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return s;
}

uot_status cuda_fail(cudaError_t e, const char* where) {
  return fail(UOT_ERR_CUDA, "%s: %s", where, cudaGetErrorString(e));
}

#define UOT_CUDA(call)                                   \
  do {                                                   \
    cudaError_t e_ = (call);                             \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call);  \
  } while (0)

size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

bool finite_pos(double v) { return isfinite(v) && v > 0.0; }

uot_status validate(const uot_problem* p) {
  if (!p) return fail(UOT_ERR_INVALID_ARG, "problem is NULL");
  if (p->n < 1 || p->m < 1) return fail(UOT_ERR_INVALID_ARG, "n and m must be >= 1 (got %d, %d)", p->n, p->m);
  if (!finite_pos(p->eps) || !finite_pos(p->rho1) || !finite_pos(p->rho2))
    return fail(UOT_ERR_INVALID_ARG, "eps, rho1, rho2 must be finite and > 0");
  if (!p->a || !p->b) return fail(UOT_ERR_INVALID_ARG, "weights a and b must be device pointers");
  if (p->ordering < 0 || p->ordering > 2) return fail(UOT_ERR_INVALID_ARG, "ordering must be 0, 1 or 2");
  if (p->cost_kind == UOT_COST_POINTS) {
    if (p->dim < 1 || p->dim > 64) return fail(UOT_ERR_INVALID_ARG, "dim must be in 1..64 (got %d)", p->dim);
    if (!(p->p >= 1.0f) || !isfinite(p->p)) return fail(UOT_ERR_INVALID_ARG, "cost exponent p must be >= 1");
    if (!p->x || !p->y) return fail(UOT_ERR_INVALID_ARG, "points x and y must be device pointers");
    if ((long long)p->n * p->dim > (1ll << 31) || (long long)p->m * p->dim > (1ll << 31))
      return fail(UOT_ERR_INVALID_ARG, "point arrays larger than 2^31 elements");
  } else if (p->cost_kind == UOT_COST_DENSE) {
    if (!p->C) return fail(UOT_ERR_INVALID_ARG, "dense cost C must be a device pointer");
    if (reinterpret_cast<uintptr_t>(p->C) & 15) return fail(UOT_ERR_INVALID_ARG, "C must be 16-byte aligned");
  } else {
    return fail(UOT_ERR_INVALID_ARG, "unknown cost_kind %d", p->cost_kind);
  }
  return UOT_OK;
}

struct PartSizes { size_t rows, cols; };

PartSizes part_sizes(const uot_problem& p) {
  PartSizes ps{0, 0};
  auto upd = [](size_t& acc, size_t v) { if (v > acc) acc = v; };
  // the largest partials over every shape the tuning table allows (and the
  // built-in one), so that a workspace stays valid whatever the table holds later
  if (p.cost_kind == UOT_COST_POINTS) {
    for (long long R : tune_allowed("points.rows")) {
      for (long long res : tune_allowed("points.resident")) {
        const TuneFix fx[2] = {{"points.rows", R}, {"points.resident", res}};
        TuneScope scope(fx, 2);
        for (int mom = 0; mom < 2; ++mom) {
          const int ch = 2 + (mom ? p.dim : 0);
          upd(ps.rows, (size_t)points_geom(p.n, p.m, p.dim, mom).splits * ch * p.n);
          upd(ps.cols, (size_t)points_geom(p.m, p.n, p.dim, mom).splits * ch * p.m);
        }
      }
    }
    for (int mom = 0; mom < 2; ++mom) {
      const int ch = 2 + (mom ? p.dim : 0);
      upd(ps.rows, (size_t)points_geom(p.n, p.m, p.dim, mom, false).splits * ch * p.n);
      upd(ps.cols, (size_t)points_geom(p.m, p.n, p.dim, mom, false).splits * ch * p.m);
    }
    if (tiled_path(p)) {
      for (long long R : tune_allowed("tile.rows")) {
        for (long long cost : tune_allowed("tile.cta_cost")) {
          for (long long w : tune_allowed("tile.waves")) {
            const TuneFix fx[3] = {{"tile.rows", R}, {"tile.cta_cost", cost}, {"tile.waves", w}};
            TuneScope scope(fx, 3);
            upd(ps.rows, (size_t)tile_geom(p.n, p.m, p.dim).splits * 2 * p.n);
            upd(ps.cols, (size_t)tile_geom(p.m, p.n, p.dim).splits * 2 * p.m);
          }
        }
      }
      upd(ps.rows, (size_t)tile_geom(p.n, p.m, p.dim, false).splits * 2 * p.n);
      upd(ps.cols, (size_t)tile_geom(p.m, p.n, p.dim, false).splits * 2 * p.m);
    }
    if (mma_path(p)) {
      upd(ps.rows, (size_t)umma_geom(p.n, p.m).splits * 2 * p.n);
      upd(ps.cols, (size_t)umma_geom(p.m, p.n).splits * 2 * p.m);
      upd(ps.rows, (size_t)mom_geom(p.n, p.m).splits * (2 + p.dim) * p.n);
      upd(ps.cols, (size_t)mom_geom(p.m, p.n).splits * (2 + p.dim) * p.m);
    }
  } else {
    for (long long ch : tune_allowed("dense.row_chunk")) {
      const TuneFix fx[1] = {{"dense.row_chunk", ch}};
      TuneScope scope(fx, 1);
      upd(ps.rows, (size_t)dense_row_geom(p.n, p.m).splits * 2 * p.n);
    }
    for (long long k : tune_allowed("dense.col_ctas")) {
      const TuneFix fx[1] = {{"dense.col_ctas", k}};
      TuneScope scope(fx, 1);
      upd(ps.cols, (size_t)dense_col_geom(p.n, p.m).splits * 2 * p.m);
    }
    upd(ps.rows, (size_t)dense_row_geom(p.n, p.m, false).splits * 2 * p.n);
    upd(ps.cols, (size_t)dense_col_geom(p.n, p.m, false).splits * 2 * p.m);
  }
  return ps;
}

struct WsLayout {
  size_t state, ln_a, ln_b, l2_a, l2_b, lo_a, lo_b, g_alt, f_tmp, g_tmp, part_r, part_c, blk, rbc, center;
  size_t op_x, op_y, n2_x, n2_y, op_sc;  // tcgen05 operands of the dim >= 32 path (empty otherwise)
  size_t zt, zsc;                        // Z^T operand scratch of its moment sweeps
  // ordering of the tiled path (empty otherwise)
  size_t perm_x, perm_y, xs, ys, as, bs, fs, gs, cen_x, cen_y, blk_f, box, code_in, code_out, idx_in, sort_tmp;
  size_t sort_tmp_bytes, total;
};

WsLayout ws_layout(const uot_problem& p) {
  WsLayout L{};
  size_t off = 0;
  auto take = [&](size_t bytes) { size_t o = off; off = align256(off + bytes); return o; };
  L.state = take(sizeof(DevState));
  L.ln_a = take(sizeof(double) * p.n);
  L.ln_b = take(sizeof(double) * p.m);
  L.l2_a = take(sizeof(float) * p.n);
  L.l2_b = take(sizeof(float) * p.m);
  L.lo_a = take(sizeof(float) * p.n);
  L.lo_b = take(sizeof(float) * p.m);
  L.g_alt = take(sizeof(float) * p.m);
  L.f_tmp = take(sizeof(float) * p.n);
  L.g_tmp = take(sizeof(float) * p.m);
  const PartSizes ps = part_sizes(p);
  L.part_r = take(sizeof(float) * ps.rows);
  L.part_c = take(sizeof(float) * ps.cols);
  L.blk = take(sizeof(double) * kMaxBlocks * 10);
  L.rbc = take(sizeof(unsigned int) * kMaxBlocks);
  L.center = take(sizeof(float) * 64);
  if (mma_path(p)) {
    L.op_x = take(sizeof(float) * umma_operand_floats(p.n, p.dim));
    L.op_y = take(sizeof(float) * umma_operand_floats(p.m, p.dim));
    L.n2_x = take(sizeof(float) * p.n);
    L.n2_y = take(sizeof(float) * p.m);
    L.op_sc = take(sizeof(int));
    L.zt = take(mom_zt_bytes(p.n > p.m ? p.n : p.m, p.dim));
    L.zsc = take(sizeof(int));
  }
  if (tiled_path(p)) {
    const int nmax = p.n > p.m ? p.n : p.m;
    L.perm_x = take(sizeof(int) * p.n);
    L.perm_y = take(sizeof(int) * p.m);
    L.xs = take(sizeof(float) * p.n * p.dim);
    L.ys = take(sizeof(float) * p.m * p.dim);
    L.as = take(sizeof(float) * p.n);
    L.bs = take(sizeof(float) * p.m);
    L.fs = take(sizeof(float) * p.n);
    L.gs = take(sizeof(float) * p.m);
    L.cen_x = take(sizeof(float4) * ((p.n + kTileKeys - 1) / kTileKeys));
    L.cen_y = take(sizeof(float4) * ((p.m + kTileKeys - 1) / kTileKeys));
    L.blk_f = take(sizeof(float) * kMaxBlocks * 6);
    L.box = take(sizeof(float) * 8);
    L.code_in = take(sizeof(unsigned int) * nmax);
    L.code_out = take(sizeof(unsigned int) * nmax);
    L.idx_in = take(sizeof(int) * nmax);
    L.sort_tmp_bytes = sort_temp_bytes(nmax);
    L.sort_tmp = take(L.sort_tmp_bytes);
  }
  L.total = off;
  return L;
}

struct Ctx {
  uot_problem p;        // as given by the caller
  DevState* state;
  double *ln_a, *ln_b, *blk;
  float *l2_a, *l2_b, *lo_a, *lo_b, *g_alt, *f_tmp, *g_tmp, *part_r, *part_c;  // lo_*: log2 w - l2_*
  size_t cap_r, cap_c;  // floats in part_r, part_c
  unsigned int* rbc;  // per-row-block counters of the fused sweeps
  float* center;      // common centre of the clouds (tensor-core path)
  float *op_x, *op_y, *n2_x, *n2_y;  // tcgen05 operands and squared norms (dim >= 32)
  int* op_sc;                        // their power-of-two scale (largest |x - c|, as float bits)
  void* zt;                          // Z^T operand of the moment sweeps
  int* zsc;                          // its multiplier scale (largest |mult|, as float bits)
  cudaStream_t st;
  double s;  // log2(e) / eps
  // tiled path: clouds in Morton order (px..pb point at the sorted copies)
  bool tiled;
  const float *px, *py, *pa, *pb;
  int *perm_x, *perm_y;
  float4 *cen_x, *cen_y;
  float *xs, *ys, *as, *bs, *fs, *gs;
  OrderScratch osc;
};

// Putting the clouds in Morton order costs a few hundred microseconds per call
// (bounding box, codes, radix sort, gathers); it pays off once the sweeps it
// speeds up cover more than about 1.5e9 cost entries in total.
bool worth_ordering(const uot_problem& p, double sweeps) {
  if (!tiled_path(p) || p.ordering == 2) return false;
  if (p.ordering == 0 && small_path(p)) return false;  // the resident cluster solver needs no ordering
  return p.ordering == 1 || (double)p.n * (double)p.m * sweeps > 1.5e9;
}

uot_status make_ctx(const uot_problem* prob, void* ws, size_t ws_bytes, void* stream, Ctx* c,
                    double sweeps = 1.0) {
  uot_status v = validate(prob);
  if (v != UOT_OK) return v;
  if (!ws) return fail(UOT_ERR_WORKSPACE, "workspace is NULL");
  if (reinterpret_cast<uintptr_t>(ws) & 255) return fail(UOT_ERR_WORKSPACE, "workspace must be 256-byte aligned");
  const WsLayout L = ws_layout(*prob);
  if (ws_bytes < L.total)
    return fail(UOT_ERR_WORKSPACE, "workspace too small: %zu bytes given, %zu needed", ws_bytes, L.total);
  char* b = static_cast<char*>(ws);
  c->p = *prob;
  c->state = reinterpret_cast<DevState*>(b + L.state);
  c->ln_a = reinterpret_cast<double*>(b + L.ln_a);
  c->ln_b = reinterpret_cast<double*>(b + L.ln_b);
  c->l2_a = reinterpret_cast<float*>(b + L.l2_a);
  c->l2_b = reinterpret_cast<float*>(b + L.l2_b);
  c->lo_a = reinterpret_cast<float*>(b + L.lo_a);
  c->lo_b = reinterpret_cast<float*>(b + L.lo_b);
  c->g_alt = reinterpret_cast<float*>(b + L.g_alt);
  c->f_tmp = reinterpret_cast<float*>(b + L.f_tmp);
  c->g_tmp = reinterpret_cast<float*>(b + L.g_tmp);
  c->part_r = reinterpret_cast<float*>(b + L.part_r);
  c->part_c = reinterpret_cast<float*>(b + L.part_c);
  {
    const PartSizes ps = part_sizes(*prob);
    c->cap_r = ps.rows;
    c->cap_c = ps.cols;
  }
  c->blk = reinterpret_cast<double*>(b + L.blk);
  c->rbc = reinterpret_cast<unsigned int*>(b + L.rbc);
  c->center = reinterpret_cast<float*>(b + L.center);
  c->op_x = c->op_y = c->n2_x = c->n2_y = nullptr;
  c->op_sc = nullptr;
  c->zt = nullptr;
  c->zsc = nullptr;
  if (mma_path(*prob)) {
    c->op_x = reinterpret_cast<float*>(b + L.op_x);
    c->op_y = reinterpret_cast<float*>(b + L.op_y);
    c->n2_x = reinterpret_cast<float*>(b + L.n2_x);
    c->n2_y = reinterpret_cast<float*>(b + L.n2_y);
    c->op_sc = reinterpret_cast<int*>(b + L.op_sc);
    c->zt = b + L.zt;
    c->zsc = reinterpret_cast<int*>(b + L.zsc);
  }
  c->st = static_cast<cudaStream_t>(stream);
  c->s = kLog2e / prob->eps;
  c->tiled = worth_ordering(*prob, sweeps);
  c->px = prob->x; c->py = prob->y; c->pa = prob->a; c->pb = prob->b;
  c->perm_x = c->perm_y = nullptr;
  c->cen_x = c->cen_y = nullptr;
  c->xs = c->ys = c->as = c->bs = c->fs = c->gs = nullptr;
  if (c->tiled) {
    c->perm_x = reinterpret_cast<int*>(b + L.perm_x);
    c->perm_y = reinterpret_cast<int*>(b + L.perm_y);
    c->xs = reinterpret_cast<float*>(b + L.xs);
    c->ys = reinterpret_cast<float*>(b + L.ys);
    c->as = reinterpret_cast<float*>(b + L.as);
    c->bs = reinterpret_cast<float*>(b + L.bs);
    c->fs = reinterpret_cast<float*>(b + L.fs);
    c->gs = reinterpret_cast<float*>(b + L.gs);
    c->cen_x = reinterpret_cast<float4*>(b + L.cen_x);
    c->cen_y = reinterpret_cast<float4*>(b + L.cen_y);
    c->osc.blk_f = reinterpret_cast<float*>(b + L.blk_f);
    c->osc.box = reinterpret_cast<float*>(b + L.box);
    c->osc.counter = &c->state->counter;
    c->osc.code_in = reinterpret_cast<unsigned int*>(b + L.code_in);
    c->osc.code_out = reinterpret_cast<unsigned int*>(b + L.code_out);
    c->osc.idx_in = reinterpret_cast<int*>(b + L.idx_in);
    c->osc.temp = b + L.sort_tmp;
    c->osc.temp_bytes = L.sort_tmp_bytes;
    c->px = c->xs; c->py = c->ys; c->pa = c->as; c->pb = c->bs;
  }
  return UOT_OK;
}

// Common preamble: zero the state; on the tiled path put both clouds in Morton
// order; log weights of both sides (in the order the sweeps use).
uot_status prepare(Ctx& c) {
  UOT_CUDA(cudaMemsetAsync(c.state, 0, sizeof(DevState), c.st));
  UOT_CUDA(cudaMemsetAsync(c.rbc, 0, sizeof(unsigned int) * kMaxBlocks, c.st));
  if (c.tiled) {
    UOT_CUDA(launch_order_points(c.p.x, c.p.a, c.p.n, c.p.dim, c.osc, c.perm_x, c.xs, c.as, c.cen_x, c.st));
    UOT_CUDA(launch_order_points(c.p.y, c.p.b, c.p.m, c.p.dim, c.osc, c.perm_y, c.ys, c.bs, c.cen_y, c.st));
  }
  if (mma_path(c.p)) {
    UOT_CUDA(launch_center(c.p.x, c.p.n, c.p.y, c.p.m, c.p.dim, c.center, c.st));
    UOT_CUDA(launch_umma_scale(c.p.x, c.p.n, c.p.y, c.p.m, c.p.dim, c.center, c.op_sc, c.st));
    UOT_CUDA(launch_umma_operand(c.p.x, c.p.n, c.p.dim, c.center, c.op_sc, c.op_x, c.n2_x, c.st));
    UOT_CUDA(launch_umma_operand(c.p.y, c.p.m, c.p.dim, c.center, c.op_sc, c.op_y, c.n2_y, c.st));
  }
  UOT_CUDA(launch_log_weights(c.pa, c.p.n, c.ln_a, c.l2_a, c.lo_a, &c.state->status, c.st));
  UOT_CUDA(launch_log_weights(c.pb, c.p.m, c.ln_b, c.l2_b, c.lo_b, &c.state->status, c.st));
  return UOT_OK;
}

// A caller-order vector of side x (axis 0) or y (axis 1) in the order the sweeps use.
uot_status to_internal(Ctx& c, int side, const float* v, float* tmp, const float** out) {
  if (!c.tiled) { *out = v; return UOT_OK; }
  UOT_CUDA(launch_gather_vec(v, side == 0 ? c.perm_x : c.perm_y, side == 0 ? c.p.n : c.p.m, tmp, c.st));
  *out = tmp;
  return UOT_OK;
}

cudaEvent_t prof_event() {
  if (g_prof.used >= 2 * kMaxTimed) return nullptr;
  if (g_prof.used == g_prof.ev.size()) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    g_prof.ev.push_back(e);
  }
  return g_prof.ev[g_prof.used++];
}

uot_status sweep_inner(Ctx& c, int axis, const float* pot, const double* shift, bool moments, int* splits,
                       EpiParams* epi, bool* fused);

// One softmin sweep.  With `epi` (the half-step to apply afterwards, its nq,
// splits and part filled in here), the tiled path runs the epilogue inside the
// sweep and sets *fused; otherwise the caller launches the combine kernel.
uot_status sweep(Ctx& c, int axis, const float* pot, const double* shift, bool moments, int* splits,
                 EpiParams* epi = nullptr, bool* fused = nullptr) {
  bool fz = false;
  if (!g_prof.open) {
    uot_status v = sweep_inner(c, axis, pot, shift, moments, splits, epi, &fz);
    if (fused) *fused = fz;
    return v;
  }
  ++g_prof.launches;
  cudaEvent_t e0 = prof_event();
  cudaEvent_t e1 = e0 ? prof_event() : nullptr;
  if (e0 && !e1) --g_prof.used;
  if (e1) UOT_CUDA(cudaEventRecord(e0, c.st));
  uot_status v = sweep_inner(c, axis, pot, shift, moments, splits, epi, &fz);
  if (e1) UOT_CUDA(cudaEventRecord(e1, c.st));
  if (fused) *fused = fz;
  return v;
}

uot_status sweep_inner(Ctx& c, int axis, const float* pot, const double* shift, bool moments, int* splits,
                       EpiParams* epi, bool* fused) {
  const uot_problem& p = c.p;
  float* part = axis == 0 ? c.part_r : c.part_c;
  const size_t cap = axis == 0 ? c.cap_r : c.cap_c;
  if (p.cost_kind == UOT_COST_POINTS) {
    SideDesc X{c.px, c.l2_a, c.ln_a, p.n}, Y{c.py, c.l2_b, c.ln_b, p.m};
    const SideDesc& q = axis == 0 ? X : Y;
    const SideDesc& k = axis == 0 ? Y : X;
    if (c.tiled && !moments) {
      SweepGeom g = tile_geom(q.n, k.n, p.dim);
      if ((size_t)g.splits * 2 * q.n > cap) g = tile_geom(q.n, k.n, p.dim, false);
      *splits = g.splits;
      if (epi) {
        epi->nq = q.n; epi->splits = g.splits; epi->part = part; epi->rb_counter = c.rbc; epi->moments = 0;
        epi->key_shift = shift;
        *fused = true;
      } else if (shift) {
        return fail(UOT_ERR_UNSUPPORTED, "internal: shifted tiled sweep without epilogue");
      }
      UOT_CUDA(launch_tile_sweep(q, k, axis == 0 ? c.cen_y : c.cen_x, p.dim, pot, shift, c.s, part, g, epi,
                                 c.st));
    } else if (mma_path(p) && !moments) {
      SweepGeom g = umma_geom(q.n, k.n);
      *splits = g.splits;
      UOT_CUDA(launch_umma_sweep(axis == 0 ? c.op_x : c.op_y, axis == 0 ? c.n2_x : c.n2_y, q.n,
                                 axis == 0 ? c.op_y : c.op_x, axis == 0 ? c.n2_y : c.n2_x, k.n, p.dim, k.l2w, pot,
                                 shift, c.s, c.op_sc, part, g, &c.state->status, c.st));
    } else if (mma_path(p)) {
      // gradient sweep with moments: dC/dx = 2 (x - y)
      SweepGeom g = mom_geom(q.n, k.n);
      *splits = g.splits;
      UOT_CUDA(launch_mom_sweep(axis == 0 ? c.op_x : c.op_y, axis == 0 ? c.n2_x : c.n2_y, q.n,
                                axis == 0 ? c.op_y : c.op_x, axis == 0 ? c.n2_y : c.n2_x, k.n, q.pts, k.pts, p.dim,
                                c.center, c.op_sc, k.l2w, pot, shift, nullptr, nullptr, nullptr, c.s, 2.0f, c.zt, c.zsc,
                                part, g, &c.state->status, c.st));
    } else {
      SweepGeom g = points_geom(q.n, k.n, p.dim, moments);
      if ((size_t)g.splits * (2 + (moments ? p.dim : 0)) * q.n > cap) g = points_geom(q.n, k.n, p.dim, moments, false);
      *splits = g.splits;
      UOT_CUDA(launch_points_sweep(q, k, p.dim, p.p, pot, shift, c.s, moments, part, g, c.st));
    }
  } else {
    SweepGeom g = axis == 0 ? dense_row_geom(p.n, p.m) : dense_col_geom(p.n, p.m);
    if ((size_t)g.splits * 2 * (axis == 0 ? p.n : p.m) > cap)
      g = axis == 0 ? dense_row_geom(p.n, p.m, false) : dense_col_geom(p.n, p.m, false);
    *splits = g.splits;
    UOT_CUDA(launch_dense_sweep(axis, p.C, p.n, p.m, axis == 0 ? c.l2_b : c.l2_a, pot, shift, c.s, part, g,
                                c.st));
  }
  return UOT_OK;
}

uot_status read_flags(Ctx& c, int* status, float* resid) {
  struct { int status; float resid; } h;
  UOT_CUDA(cudaMemcpyAsync(&h, &c.state->status, sizeof(h), cudaMemcpyDeviceToHost, c.st));
  UOT_CUDA(cudaStreamSynchronize(c.st));
  *status = h.status;
  *resid = h.resid;
  return UOT_OK;
}

// ---- the Sinkhorn loop ---------------------------------------------------------
// One solve's set-up, shared by the host-driven loop (uot_sinkhorn and
// friends: the host reads the residual at every check) and the device-driven
// loop of a plan (the same launches captured in a CUDA graph, the stopping
// rule evaluated on the device).
struct Loop {
  Ctx c;
  uot_options opt;
  int variant;  // 0 plain (F-)Sinkhorn, 1 H-Sinkhorn (TI), 2 G-Sinkhorn
  bool ti;      // slots, key shifts and lambda in use
  int mode;     // epilogue mode of the half-steps
  bool small;   // the resident cluster solver runs the whole loop
  float *f, *g;           // the caller's outputs
  float* fst;             // f_hat in the sweeps' order
  float* gbuf[2];         // g_hat by iteration parity
  float *lse_f, *lse_g;   // per-row log-sum-exps kept between sweeps (tiled path)
};

// variant: 0 plain (F-)Sinkhorn, 1 H-Sinkhorn (TI), 2 G-Sinkhorn.
uot_status loop_setup(Loop& L, int variant, const uot_problem* prob, const uot_options* opt, float* f, float* g,
                      void* ws, size_t ws_bytes, void* stream) {
  uot_status v0 = validate(prob);
  if (v0 != UOT_OK) return v0;
  if (!opt) return fail(UOT_ERR_INVALID_ARG, "options is NULL");
  uot_status v = make_ctx(prob, ws, ws_bytes, stream, &L.c, 2.0 * opt->max_iter + 1.0);
  if (v != UOT_OK) return v;
  if (!f || !g) return fail(UOT_ERR_INVALID_ARG, "f and g must be device pointers");
  if (opt->max_iter < 1) return fail(UOT_ERR_INVALID_ARG, "max_iter must be >= 1");
  if (opt->check_every < 1) return fail(UOT_ERR_INVALID_ARG, "check_every must be >= 1");
  if (!(opt->tol >= 0.0) || !isfinite(opt->tol)) return fail(UOT_ERR_INVALID_ARG, "tol must be finite and >= 0");
  if (opt->lse_reference < 0 || opt->lse_reference > 2)
    return fail(UOT_ERR_INVALID_ARG, "lse_reference must be 0, 1 or 2");
  const int AK = opt->anderson_k;
  if (AK != 0) {
    if (AK < 2 || AK > 6) return fail(UOT_ERR_INVALID_ARG, "anderson_k must be 0 or 2..6");
    if (!(opt->anderson_reg >= 0.0) || !isfinite(opt->anderson_reg))
      return fail(UOT_ERR_INVALID_ARG, "anderson_reg must be finite and >= 0");
    if (!opt->anderson_buf || (reinterpret_cast<uintptr_t>(opt->anderson_buf) & 15))
      return fail(UOT_ERR_INVALID_ARG, "anderson_buf must be a 16-byte aligned device pointer");
  }
  L.opt = *opt;
  L.variant = variant;
  L.ti = variant != 0;
  L.mode = variant == 1 ? EPI_TI : variant == 2 ? EPI_G : EPI_PLAIN;
  Ctx& c = L.c;
  const uot_problem& p = c.p;
  L.small = p.ordering == 0 && small_path(p) && AK == 0;
  L.f = f;
  L.g = g;
  // tiled path: every row's log-sum-exp is kept between the sweeps of a side
  // (the temporaries, which a solve does not otherwise use), for the fixed
  // reference (lse_reference != 1)
  L.lse_g = c.tiled ? c.g_tmp : nullptr;
  L.lse_f = c.tiled ? c.f_tmp : nullptr;
  L.fst = c.tiled ? c.fs : f;
  L.gbuf[0] = c.tiled ? c.gs : g;
  L.gbuf[1] = c.g_alt;
  return UOT_OK;
}

// Everything before the first half-step: state, ordering, log weights, the
// initial iterate and its scalars, the tensor-core key operands.
uot_status loop_prologue(Loop& L) {
  Ctx& c = L.c;
  const uot_problem& p = c.p;
  uot_status v = prepare(c);
  if (v != UOT_OK) return v;
  if (!L.opt.warm_start) UOT_CUDA(cudaMemsetAsync(L.fst, 0, sizeof(float) * p.n, c.st));
  else if (c.tiled) UOT_CUDA(launch_gather_vec(L.f, c.perm_x, p.n, L.fst, c.st));
  UOT_CUDA(cudaMemsetAsync(L.gbuf[0], 0, sizeof(float) * p.m, c.st));
  if (L.ti) UOT_CUDA(launch_ti_init(L.fst, c.ln_a, p.n, p.rho1, c.state, c.blk, c.st));
  return UOT_OK;
}

// Device-driven loop control of a half-step (see EpiParams::loop_ctl).
struct LoopCtl {
  int ctl = 0;
  unsigned long long cond_while = 0, cond_if = 0;
};

// g half-step of iteration t + 1: column sweep over x with fb_t = f_hat + cf.
uot_status g_half(Loop& L, int t, const LoopCtl& lc) {
  Ctx& c = L.c;
  const uot_problem& p = c.p;
  const int so = (t + 1) & 1, si = t & 1;
  int splits = 0;
  bool fused = false;
  EpiParams e{};
  e.mode = L.mode; e.nq = p.m; e.moments = 0; e.s = c.s;
  e.eps = p.eps; e.rho_o = p.rho2; e.rho_i = p.rho1; e.out_is_f = 0; e.lnw_o = c.ln_b;
  e.l2w_o = c.l2_b; e.l2lo_o = c.lo_b;
  e.old_out = (t >= 1) ? L.gbuf[si] : nullptr; e.out = L.gbuf[so];
  e.resid_hist = L.opt.residual_history; e.hist_index = t;
  e.slot_in = si; e.slot_out = so; e.state = c.state; e.part = c.part_c; e.blk = c.blk;
  e.lse_buf = L.lse_g; e.lse_policy = L.opt.lse_reference;
  e.loop_ctl = lc.ctl;
  e.loop_max_iter = L.opt.max_iter; e.loop_check_every = L.opt.check_every; e.loop_tol = L.opt.tol;
  e.cond_while = lc.cond_while; e.cond_if = lc.cond_if;
  uot_status v = sweep(c, 1, L.fst, L.ti ? &c.state->slot[si].cf : nullptr, false, &splits, &e, &fused);
  if (v != UOT_OK) return v;
  e.splits = splits;
  if (!fused) UOT_CUDA(launch_combine(e, c.st));
  return UOT_OK;
}

// f half-step of iteration t + 1: row sweep over y with gb_{t+1} = g_hat + cg.
uot_status f_half(Loop& L, int t, const LoopCtl& lc) {
  Ctx& c = L.c;
  const uot_problem& p = c.p;
  const int so = (t + 1) & 1;
  int splits = 0;
  bool fused = false;
  EpiParams ef{};
  ef.mode = L.mode; ef.nq = p.n; ef.moments = 0; ef.s = c.s;
  ef.eps = p.eps; ef.rho_o = p.rho1; ef.rho_i = p.rho2; ef.out_is_f = 1; ef.lnw_o = c.ln_a;
  ef.l2w_o = c.l2_a; ef.l2lo_o = c.lo_a;
  ef.old_out = nullptr; ef.out = L.fst;
  ef.resid_hist = nullptr; ef.hist_index = t;
  ef.slot_in = so; ef.slot_out = so; ef.state = c.state; ef.part = c.part_r; ef.blk = c.blk;
  ef.lse_buf = L.lse_f; ef.lse_policy = L.opt.lse_reference;
  ef.loop_ctl = lc.ctl;
  uot_status v = sweep(c, 0, L.gbuf[so], L.ti ? &c.state->slot[so].cg : nullptr, false, &splits, &ef, &fused);
  if (v != UOT_OK) return v;
  ef.splits = splits;
  if (!fused) UOT_CUDA(launch_combine(ef, c.st));
  return UOT_OK;
}

// The resident cluster solver: the whole loop in one launch.
uot_status small_loop(Loop& L) {
  Ctx& c = L.c;
  const uot_problem& p = c.p;
  EpiParams eg{};
  eg.mode = L.mode; eg.nq = p.m; eg.moments = 0; eg.s = c.s;
  eg.eps = p.eps; eg.rho_o = p.rho2; eg.rho_i = p.rho1; eg.out_is_f = 0; eg.lnw_o = c.ln_b;
  eg.l2w_o = c.l2_b; eg.l2lo_o = c.lo_b;
  eg.resid_hist = L.opt.residual_history; eg.state = c.state; eg.blk = c.blk; eg.lse_policy = 1;
  EpiParams ef = eg;
  ef.nq = p.n; ef.rho_o = p.rho1; ef.rho_i = p.rho2; ef.out_is_f = 1;
  ef.lnw_o = c.ln_a; ef.old_out = nullptr; ef.out = L.fst; ef.resid_hist = nullptr;
  ef.l2w_o = c.l2_a; ef.l2lo_o = c.lo_a;
  UOT_CUDA(launch_small_solve(c.px, c.py, c.l2_a, c.l2_b, p.n, p.m, p.dim, L.ti ? 1 : 0, L.opt.max_iter,
                              L.opt.check_every, L.opt.tol, c.s, L.fst, L.gbuf[0], L.gbuf[1], eg, ef, c.st));
  return UOT_OK;
}

// Host-driven solve: the host reads the residual at every check and decides.
uot_status solve(int variant, const uot_problem* prob, const uot_options* opt, float* f, float* g,
                 uot_result* res, void* ws, size_t ws_bytes, void* stream) {
  Loop L;
  uot_status v = loop_setup(L, variant, prob, opt, f, g, ws, ws_bytes, stream);
  if (v != UOT_OK) return v;
  Ctx& c = L.c;
  const uot_problem& p = c.p;
  const int AK = opt->anderson_k;
  v = loop_prologue(L);
  if (v != UOT_OK) return v;
  const LoopCtl host{};
  int t = 0, status = 0;
  float r = NAN;
  if (L.small) {
    v = small_loop(L);
    if (v != UOT_OK) return v;
    int iters = 0;
    UOT_CUDA(cudaMemcpyAsync(&iters, &c.state->iters, sizeof(int), cudaMemcpyDeviceToHost, c.st));
    v = read_flags(c, &status, &r);
    if (v != UOT_OK) return v;
    t = iters;
  } else for (;;) {
    if (AK && t == 0) {
      UOT_CUDA(anderson_reset(opt->anderson_buf, p.n, AK, c.st));
      UOT_CUDA(launch_anderson_store(L.fst, p.n, AK, 0, variant, &c.state->slot[0], opt->anderson_buf, c.st));
    }
    v = g_half(L, t, host);
    if (v != UOT_OK) return v;
    const bool last = (t == opt->max_iter);
    if (t >= 1 && (last || (opt->tol > 0.0 && t % opt->check_every == 0))) {
      v = read_flags(c, &status, &r);
      if (v != UOT_OK) return v;
      if (status != 0 || isnan(r)) break;
      if (last || r <= opt->tol) break;
    }
    v = f_half(L, t, host);
    if (v != UOT_OK) return v;
    ++t;
    if (AK) {
      // Anderson: keep x_t; after every AK-th iteration that is neither the last nor a
      // residual check, the last AK + 1 iterates give the next one
      Slot* sl = &c.state->slot[t & 1];
      UOT_CUDA(launch_anderson_store(L.fst, p.n, AK, t % (AK + 1), variant, sl, opt->anderson_buf, c.st));
      if (t % AK == 0 && t < opt->max_iter && !(opt->tol > 0.0 && t % opt->check_every == 0)) {
        const int p0 = (t - AK) % (AK + 1);
        UOT_CUDA(launch_anderson_extrapolate(L.fst, p.n, AK, p0, opt->anderson_reg, opt->anderson_buf,
                                             variant == 2 ? sl : nullptr, &c.state->status, c.st));
        // H: the new fb is held in full (cf = 0); its Smin_a^rho1 for the next g half-step
        if (variant == 1) UOT_CUDA(launch_ti_init(L.fst, c.ln_a, p.n, p.rho1, c.state, c.blk, c.st, t & 1));
      }
    }
  }
  UOT_CUDA(launch_finalize(variant, L.fst, L.gbuf[t & 1], f, g, p.n, p.m, c.state, t & 1, c.perm_x, c.perm_y,
                           c.st));
  Slot slot{};
  unsigned int misses = 0;
  UOT_CUDA(cudaMemcpyAsync(&slot, &c.state->slot[t & 1], sizeof(Slot), cudaMemcpyDeviceToHost, c.st));
  UOT_CUDA(cudaMemcpyAsync(&misses, &c.state->lse_miss, sizeof(misses), cudaMemcpyDeviceToHost, c.st));
  UOT_CUDA(cudaStreamSynchronize(c.st));
  uot_status out = UOT_OK;
  const bool converged = !isnan(r) && r <= opt->tol;
  if (status & kStatusTimeout) out = fail(UOT_ERR_TIMEOUT, "a bounded device-side wait gave up (tensor-core sweep)");
  else if (status & kStatusBadWeights) out = fail(UOT_ERR_NONFINITE, "negative, NaN or infinite weights");
  else if (status != 0 || isnan(r)) out = fail(UOT_ERR_NONFINITE, "non-finite value met during the iteration");
  else if (opt->tol > 0.0 && !converged) out = UOT_NOT_CONVERGED;
  if (res) {
    res->iters = t;
    res->converged = converged ? 1 : 0;
    res->status = out;
    res->lse_misses = (int32_t)(misses > 0x7fffffffu ? 0x7fffffffu : misses);
    res->residual = r;
    res->lambda = L.ti ? slot.lam : 0.0;
  }
  return out;
}

// ---- unrolled backward -------------------------------------------------------
// Extra workspace of uot_grad_unrolled after the regular layout of the problem.
// uot_sinkhorn_phi: the solver workspace, then fb, gb, the softmin S (sweep
// order), the lambda* state and its block partials.
struct PhiLayout {
  size_t fb, gb, S, lam, lblk, total;
};

PhiLayout phi_layout(const uot_problem& p) {
  PhiLayout L{};
  size_t off = align256(ws_layout(p).total);
  auto take = [&](size_t bytes) { size_t o = off; off = align256(off + bytes); return o; };
  L.fb = take(sizeof(float) * p.n);
  L.gb = take(sizeof(float) * p.m);
  L.S = take(sizeof(float) * (p.n > p.m ? p.n : p.m));
  L.lam = take(sizeof(LamState));
  L.lblk = take(sizeof(double) * 2 * kMaxBlocks);
  L.total = off;
  return L;
}

struct URLayout {
  size_t base, ck_f, ck_slot, fbar, gbarn, Sp, Gp, ghat, S, G, fhat, rec, fst, g0, fbb, gbb, Sb, Spb, ffin, gfin,
      fbT, gbT, ga, gb, gx, gy, val, mom, adj, sums, total;
  int nck, K;
};

URLayout ur_layout(const uot_problem& p, int T, int K) {
  URLayout L{};
  L.K = K;
  L.nck = (T + K - 1) / K;
  size_t off = align256(ws_layout(p).total);
  L.base = off;
  auto take = [&](size_t bytes) { size_t o = off; off = align256(off + bytes); return o; };
  const size_t N = p.n, M = p.m, D = p.dim;
  L.ck_f = take(sizeof(float) * N * L.nck);
  L.ck_slot = take(sizeof(Slot) * 2 * L.nck);
  L.fbar = take(sizeof(float) * N * K);
  L.gbarn = take(sizeof(float) * M * K);
  L.Sp = take(sizeof(float) * M * K);
  L.Gp = take(sizeof(float) * M * D * K);
  L.ghat = take(sizeof(float) * M * K);
  L.S = take(sizeof(float) * N * K);
  L.G = take(sizeof(float) * N * D * K);
  L.fhat = take(sizeof(float) * N * K);
  L.rec = take(sizeof(double) * 8 * K);
  L.fst = take(sizeof(float) * N);
  L.g0 = take(sizeof(float) * M);
  L.fbb = take(sizeof(float) * N);
  L.gbb = take(sizeof(float) * M);
  L.Sb = take(sizeof(float) * N);
  L.Spb = take(sizeof(float) * M);
  L.ffin = take(sizeof(float) * N);
  L.gfin = take(sizeof(float) * M);
  L.fbT = take(sizeof(float) * N);
  L.gbT = take(sizeof(float) * M);
  L.ga = take(sizeof(float) * N);
  L.gb = take(sizeof(float) * M);
  L.gx = take(sizeof(float) * N * D);
  L.gy = take(sizeof(float) * M * D);
  const size_t Q = N > M ? N : M;
  L.val = take(sizeof(double) * Q);
  L.mom = take(sizeof(double) * Q * D);
  const SweepGeom a1 = adjoint_geom(p.m, p.n), a2 = adjoint_geom(p.n, p.m);
  size_t ap = (size_t)a1.splits * (2 + D) * M;
  if ((size_t)a2.splits * (2 + D) * N > ap) ap = (size_t)a2.splits * (2 + D) * N;
  if (mma_path(p)) {
    const SweepGeom b1 = mom_geom(p.m, p.n), b2 = mom_geom(p.n, p.m);
    if ((size_t)b1.splits * (2 + D) * M > ap) ap = (size_t)b1.splits * (2 + D) * M;
    if ((size_t)b2.splits * (2 + D) * N > ap) ap = (size_t)b2.splits * (2 + D) * N;
  }
  L.adj = take(sizeof(float) * ap);
  L.sums = take(sizeof(double) * 8);
  L.total = off;
  return L;
}

uot_status ur_check(const uot_problem* prob, int T, int K) {
  uot_status v = validate(prob);
  if (v != UOT_OK) return v;
  if (prob->cost_kind != UOT_COST_POINTS || prob->p != 2.0f)
    return fail(UOT_ERR_UNSUPPORTED, "the unrolled backward covers the points cost with p = 2");
  if (T < 1 || K < 1) return fail(UOT_ERR_INVALID_ARG, "need T >= 1 and ckpt_every >= 1");
  return UOT_OK;
}

// One TI iteration t -> t+1 on the direct kernels.  With rec != nullptr the
// iteration is recorded for the backward pass at segment index j.
uot_status ur_iteration(Ctx& c, const URLayout& L, char* b, int t, float* fst, float* gbuf[2], bool rec, int j) {
  const uot_problem& p = c.p;
  const int si = t & 1, so = (t + 1) & 1;
  const size_t N = p.n, M = p.m, D = p.dim;
  const int mom = rec ? p.dim : 0;
  const double gscale = (p.dim <= 3) ? 2.0 / sqrt(c.s) : 1.0;  // moment convention of the sweep kernels
  float* fbar = reinterpret_cast<float*>(b + L.fbar) + N * j;
  float* gbarn = reinterpret_cast<float*>(b + L.gbarn) + M * j;
  float* Sp = reinterpret_cast<float*>(b + L.Sp) + M * j;
  float* Gp = reinterpret_cast<float*>(b + L.Gp) + M * D * j;
  float* ghat = reinterpret_cast<float*>(b + L.ghat) + M * j;
  float* S = reinterpret_cast<float*>(b + L.S) + N * j;
  float* G = reinterpret_cast<float*>(b + L.G) + N * D * j;
  float* fhat = reinterpret_cast<float*>(b + L.fhat) + N * j;
  double* recd = reinterpret_cast<double*>(b + L.rec) + 8 * j;
  if (rec) UOT_CUDA(launch_add_scalar(fst, &c.state->slot[si].cf, p.n, fbar, c.st));
  // g half-step
  int splits = 0;
  uot_status v = sweep(c, 1, fst, &c.state->slot[si].cf, rec, &splits);
  if (v != UOT_OK) return v;
  EpiParams e{};
  e.nq = p.m; e.splits = splits; e.moments = mom; e.s = c.s; e.eps = p.eps; e.rho_o = p.rho2; e.rho_i = p.rho1;
  e.out_is_f = 0; e.lnw_o = c.ln_b; e.slot_in = si; e.slot_out = so; e.state = c.state; e.part = c.part_c;
  e.l2w_o = c.l2_b; e.l2lo_o = c.lo_b;
  e.blk = c.blk;
  if (rec) {
    EpiParams es = e;
    es.mode = EPI_SOFTMIN; es.out = Sp;
    UOT_CUDA(launch_combine(es, c.st));
    UOT_CUDA(launch_moments(c.part_c, p.m, p.dim, splits, gscale, Gp, c.st));
  }
  e.mode = EPI_TI; e.out = gbuf[so];
  UOT_CUDA(launch_combine(e, c.st));
  if (rec) {
    UOT_CUDA(cudaMemcpyAsync(ghat, gbuf[so], sizeof(float) * M, cudaMemcpyDeviceToDevice, c.st));
    UOT_CUDA(launch_add_scalar(gbuf[so], &c.state->slot[so].cg, p.m, gbarn, c.st));
  }
  // f half-step
  v = sweep(c, 0, gbuf[so], &c.state->slot[so].cg, rec, &splits);
  if (v != UOT_OK) return v;
  EpiParams ef = e;
  ef.nq = p.n; ef.splits = splits; ef.rho_o = p.rho1; ef.rho_i = p.rho2; ef.out_is_f = 1; ef.lnw_o = c.ln_a;
  ef.l2w_o = c.l2_a; ef.l2lo_o = c.lo_a;
  ef.slot_in = so; ef.slot_out = so; ef.part = c.part_r;
  if (rec) {
    EpiParams es = ef;
    es.mode = EPI_SOFTMIN; es.out = S;
    UOT_CUDA(launch_combine(es, c.st));
    UOT_CUDA(launch_moments(c.part_r, p.n, p.dim, splits, gscale, G, c.st));
  }
  ef.mode = EPI_TI; ef.out = fst;
  UOT_CUDA(launch_combine(ef, c.st));
  if (rec) {
    UOT_CUDA(cudaMemcpyAsync(fhat, fst, sizeof(float) * N, cudaMemcpyDeviceToDevice, c.st));
    UOT_CUDA(launch_record_scalars(c.state, si, so, recd, c.st));
  }
  return UOT_OK;
}

uot_status grad_unrolled(const uot_problem* prob, int T, int K, double* value, float* grad_a, float* grad_b,
                         float* grad_x, float* grad_y, void* ws, size_t ws_bytes, void* stream) {
  uot_status v = ur_check(prob, T, K);
  if (v != UOT_OK) return v;
  uot_problem pd = *prob;
  pd.ordering = 2;  // natural order and the direct kernels
  const URLayout L = ur_layout(pd, T, K);
  if (!ws) return fail(UOT_ERR_WORKSPACE, "workspace is NULL");
  if (ws_bytes < L.total) return fail(UOT_ERR_WORKSPACE, "workspace too small: %zu given, %zu needed", ws_bytes, L.total);
  if (!value) return fail(UOT_ERR_INVALID_ARG, "value must be a device pointer");
  Ctx c;
  v = make_ctx(&pd, ws, ws_bytes, stream, &c);
  if (v != UOT_OK) return v;
  v = prepare(c);
  if (v != UOT_OK) return v;
  char* b = static_cast<char*>(ws);
  const uot_problem& p = c.p;
  const size_t N = p.n, M = p.m, D = p.dim;
  float* fst = reinterpret_cast<float*>(b + L.fst);
  float* gbuf[2] = {reinterpret_cast<float*>(b + L.g0), c.g_alt};
  float* ck_f = reinterpret_cast<float*>(b + L.ck_f);
  Slot* ck_slot = reinterpret_cast<Slot*>(b + L.ck_slot);
  double* sums = reinterpret_cast<double*>(b + L.sums);
  float *fbb = reinterpret_cast<float*>(b + L.fbb), *gbb = reinterpret_cast<float*>(b + L.gbb);
  float *Sb = reinterpret_cast<float*>(b + L.Sb), *Spb = reinterpret_cast<float*>(b + L.Spb);
  float *ffin = reinterpret_cast<float*>(b + L.ffin), *gfin = reinterpret_cast<float*>(b + L.gfin);
  float *fbT = reinterpret_cast<float*>(b + L.fbT), *gbT = reinterpret_cast<float*>(b + L.gbT);
  float *ga = reinterpret_cast<float*>(b + L.ga), *gb = reinterpret_cast<float*>(b + L.gb);
  float *gx = reinterpret_cast<float*>(b + L.gx), *gy = reinterpret_cast<float*>(b + L.gy);
  double *val = reinterpret_cast<double*>(b + L.val), *mom = reinterpret_cast<double*>(b + L.mom);
  float* adj = reinterpret_cast<float*>(b + L.adj);
  unsigned int* ctr = &c.state->counter;

  // forward with checkpoints of (f_hat, scalar slots) every K iterations
  UOT_CUDA(cudaMemsetAsync(fst, 0, sizeof(float) * N, c.st));
  UOT_CUDA(cudaMemsetAsync(gbuf[0], 0, sizeof(float) * M, c.st));
  UOT_CUDA(launch_ti_init(fst, c.ln_a, p.n, p.rho1, c.state, c.blk, c.st));
  for (int t = 0; t < T; ++t) {
    if (t % K == 0) {
      UOT_CUDA(cudaMemcpyAsync(ck_f + N * (t / K), fst, sizeof(float) * N, cudaMemcpyDeviceToDevice, c.st));
      UOT_CUDA(cudaMemcpyAsync(ck_slot + 2 * (t / K), c.state->slot, sizeof(Slot) * 2, cudaMemcpyDeviceToDevice,
                               c.st));
    }
    v = ur_iteration(c, L, b, t, fst, gbuf, false, 0);
    if (v != UOT_OK) return v;
  }
  // output pair, value and the direct partials of F_eps
  const int sT = T & 1;
  UOT_CUDA(launch_finalize(1, fst, gbuf[sT], ffin, gfin, p.n, p.m, c.state, sT, nullptr, nullptr, c.st));
  UOT_CUDA(launch_add_scalar(fst, &c.state->slot[sT].cf, p.n, fbT, c.st));
  UOT_CUDA(launch_add_scalar(gbuf[sT], &c.state->slot[sT].cg, p.m, gbT, c.st));
  int sr = 0, sc = 0;
  v = sweep(c, 0, gfin, nullptr, false, &sr);
  if (v != UOT_OK) return v;
  DualParams d{};
  d.n = p.n; d.m = p.m; d.splits_r = sr; d.splits_c = 0; d.s = c.s; d.eps = p.eps; d.rho1 = p.rho1;
  d.rho2 = p.rho2; d.f = ffin; d.g = gfin; d.a = c.pa; d.b = c.pb; d.ln_a = c.ln_a; d.ln_b = c.ln_b;
  d.part_r = c.part_r; d.part_c = nullptr; d.blk = c.blk; d.state = c.state; d.out = value; d.want_primal = 0;
  UOT_CUDA(launch_dual(d, c.st));
  const double tau1 = p.rho1 / (p.rho1 + p.rho2), tau2 = p.rho2 / (p.rho1 + p.rho2);
  for (int side = 0; side < 2; ++side) {
    v = sweep(c, side, side == 0 ? gfin : ffin, nullptr, true, side == 0 ? &sr : &sc);
    if (v != UOT_OK) return v;
    UOT_CUDA(launch_mass(side == 0 ? p.b : p.a, side == 0 ? p.m : p.n, c.blk, c.state, 0, c.st));
    GradParams gp{};
    gp.nq = side == 0 ? p.n : p.m; gp.splits = side == 0 ? sr : sc; gp.dim = p.dim; gp.moments = p.dim;
    gp.s = c.s; gp.eps = p.eps; gp.rho_o = side == 0 ? p.rho1 : p.rho2; gp.p = p.p;
    gp.pot_o = side == 0 ? ffin : gfin; gp.part = side == 0 ? c.part_r : c.part_c;
    gp.grad_w = side == 0 ? ga : gb; gp.grad_pts = side == 0 ? gx : gy; gp.lnw_o = side == 0 ? c.ln_a : c.ln_b;
    gp.perm = nullptr; gp.state = c.state;
    UOT_CUDA(launch_grad_epilogue(gp, c.st));
    UOT_CUDA(launch_final_side(side == 0 ? c.part_r : c.part_c, 2 + p.dim, gp.nq, gp.splits, c.s, p.eps, gp.rho_o,
                               gp.pot_o, gp.lnw_o, side == 0 ? fbb : gbb, c.blk, ctr, sums + side, c.st));
  }
  // lambda = tau1 B(gb_T) - tau2 A(fb_T):  Abar_T = -tau2 lambda_bar,  Bbar_T = tau1 lambda_bar
  UOT_CUDA(launch_final_lambda(p.n, fbT, c.ln_a, &c.state->slot[sT].A, p.rho1, -tau2, sums, sums + 1, fbb, ga, c.blk,
                               ctr, sums + 2, c.st));
  UOT_CUDA(launch_final_lambda(p.m, gbT, c.ln_b, &c.state->slot[sT].B, p.rho2, tau1, sums, sums + 1, gbb, gb, c.blk,
                               ctr, nullptr, c.st));
  // reverse sweep over segments, recomputing each from its checkpoint
  const double eps = p.eps, r1 = p.rho1, r2 = p.rho2;
  const double a1 = r1 / (r1 + eps), b1 = eps / (eps + r1) * r1 / (r1 + r2);
  const double a2 = r2 / (r2 + eps), b2 = eps / (eps + r2) * r2 / (r1 + r2);
  const float* ctr_c = mma_path(c.p) ? c.center : nullptr;  // tensor-core adjoint sweeps for dim >= 32
  const double kf0 = eps / (eps + r1) * r2 / (r1 + r2), kg0 = eps / (eps + r2) * r1 / (r1 + r2);
  const double kf = kf0 / (1.0 - kf0), kg = kg0 / (1.0 - kg0);
  for (int sgi = L.nck - 1; sgi >= 0; --sgi) {
    const int t0 = sgi * K, t1 = std::min(T, t0 + K);
    UOT_CUDA(cudaMemcpyAsync(fst, ck_f + N * sgi, sizeof(float) * N, cudaMemcpyDeviceToDevice, c.st));
    UOT_CUDA(cudaMemcpyAsync(c.state->slot, ck_slot + 2 * sgi, sizeof(Slot) * 2, cudaMemcpyDeviceToDevice, c.st));
    for (int t = t0; t < t1; ++t) {
      v = ur_iteration(c, L, b, t, fst, gbuf, true, t - t0);
      if (v != UOT_OK) return v;
    }
    for (int t = t1 - 1; t >= t0; --t) {
      const int j = t - t0;
      const float* fbar = reinterpret_cast<float*>(b + L.fbar) + N * j;
      const float* gbarn = reinterpret_cast<float*>(b + L.gbarn) + M * j;
      const float* Sp = reinterpret_cast<float*>(b + L.Sp) + M * j;
      const float* Gp = reinterpret_cast<float*>(b + L.Gp) + M * D * j;
      const float* ghat = reinterpret_cast<float*>(b + L.ghat) + M * j;
      const float* S = reinterpret_cast<float*>(b + L.S) + N * j;
      const float* G = reinterpret_cast<float*>(b + L.G) + N * D * j;
      const float* fhat = reinterpret_cast<float*>(b + L.fhat) + N * j;
      const double* rec = reinterpret_cast<double*>(b + L.rec) + 8 * j;
      // f half-step of iteration t+1
      UOT_CUDA(launch_bw_f1(p.n, p.dim, fbb, fhat, c.ln_a, rec + 3, sums + 2, kf, r1, a1, G, ga, gx, Sb, c.blk, ctr,
                            sums + 3, c.st));
      UOT_CUDA(launch_bw_smin_init(p.m, gbarn, c.ln_b, rec + 2, r2, -b1, sums + 3, gbb, gb, c.st));
      UOT_CUDA(launch_adjoint(p.y, p.m, p.x, p.n, p.dim, gbarn, S, Sb, c.s, adj, val, mom, ctr_c, c.op_sc,
                              MomOperands{c.op_y, c.n2_y, c.op_x, c.n2_x, c.zt, c.zsc, &c.state->status}, c.st));
      UOT_CUDA(launch_bw_adj(p.m, p.dim, val, mom, c.ln_b, eps, gbb, gb, gy, c.blk, ctr, sums + 4, c.st));
      // g half-step of iteration t+1
      UOT_CUDA(launch_bw_g1(p.m, p.dim, gbb, ghat, c.ln_b, rec + 1, sums + 4, kg, r2, a2, Gp, gb, gy, Spb, c.blk, ctr,
                            sums + 5, c.st));
      UOT_CUDA(launch_bw_fset(p.n, fbar, c.ln_a, rec + 0, r1, -b2, sums + 5, fbb, ga, c.st));
      UOT_CUDA(launch_adjoint(p.x, p.n, p.y, p.m, p.dim, fbar, Sp, Spb, c.s, adj, val, mom, ctr_c, c.op_sc,
                              MomOperands{c.op_x, c.n2_x, c.op_y, c.n2_y, c.zt, c.zsc, &c.state->status}, c.st));
      UOT_CUDA(launch_bw_adj(p.n, p.dim, val, mom, c.ln_a, eps, fbb, ga, gx, c.blk, ctr, sums + 2, c.st));
    }
  }
  if (grad_a) UOT_CUDA(cudaMemcpyAsync(grad_a, ga, sizeof(float) * N, cudaMemcpyDeviceToDevice, c.st));
  if (grad_b) UOT_CUDA(cudaMemcpyAsync(grad_b, gb, sizeof(float) * M, cudaMemcpyDeviceToDevice, c.st));
  if (grad_x) UOT_CUDA(cudaMemcpyAsync(grad_x, gx, sizeof(float) * N * D, cudaMemcpyDeviceToDevice, c.st));
  if (grad_y) UOT_CUDA(cudaMemcpyAsync(grad_y, gy, sizeof(float) * M * D, cudaMemcpyDeviceToDevice, c.st));
  int status = 0;
  UOT_CUDA(cudaMemcpyAsync(&status, &c.state->status, sizeof(int), cudaMemcpyDeviceToHost, c.st));
  UOT_CUDA(cudaStreamSynchronize(c.st));
  if (status != 0) return fail(UOT_ERR_NONFINITE, "non-finite value met in the unrolled pass");
  return UOT_OK;
}

// ---- device-driven solve (plans) ---------------------------------------------
// The whole solve as stream work with no host synchronisation: the set-up and
// the first g half-step, then a conditional while node whose body runs two
// iterations (the second inside a conditional if node, so that each captured
// iteration keeps a fixed buffer parity), each g half-step's grid tail
// evaluating the stopping rule and writing both conditions, then the output
// map Phi and the device-side uot_result.  `s` must be capturing; `b1` and
// `b2` are idle streams the two bodies are captured on.
uot_status emit_solve(Loop& L, cudaStream_t s, cudaStream_t b1, cudaStream_t b2, uot_result* res) {
  Ctx& c = L.c;
  const uot_problem& p = c.p;
  const bool prof = g_prof.open;  // event records cannot enter conditional bodies
  g_prof.open = false;
  struct Restore {
    bool v;
    ~Restore() { g_prof.open = v; }
  } restore{prof};
  c.st = s;
  uot_status v = loop_prologue(L);
  if (v != UOT_OK) return v;
  if (L.small) {
    v = small_loop(L);
    if (v != UOT_OK) return v;
    UOT_CUDA(launch_finalize_loop(L.variant, L.fst, L.gbuf[0], L.gbuf[1], L.f, L.g, p.n, p.m, c.state, c.perm_x,
                                  c.perm_y, 1, s));
    UOT_CUDA(launch_write_result(c.state, L.ti ? 1 : 0, 1, L.opt.tol, res, s));
    return UOT_OK;
  }
  const LoopCtl host{};
  v = g_half(L, 0, host);
  if (v != UOT_OK) return v;
  // the while node, after what the stream has captured so far
  cudaStreamCaptureStatus cs;
  cudaGraph_t graph = nullptr;
  const cudaGraphNode_t* deps = nullptr;
  size_t ndeps = 0;
  UOT_CUDA(cudaStreamGetCaptureInfo(s, &cs, nullptr, &graph, &deps, nullptr, &ndeps));
  if (cs != cudaStreamCaptureStatusActive) return fail(UOT_ERR_CUDA, "internal: the solve stream is not capturing");
  cudaGraphConditionalHandle hw = 0, hi = 0;
  UOT_CUDA(cudaGraphConditionalHandleCreate(&hw, graph, 1, cudaGraphCondAssignDefault));
  cudaGraphNodeParams wp{};
  wp.type = cudaGraphNodeTypeConditional;
  wp.conditional.handle = hw;
  wp.conditional.type = cudaGraphCondTypeWhile;
  wp.conditional.size = 1;
  cudaGraphNode_t wnode = nullptr;
  UOT_CUDA(cudaGraphAddNode(&wnode, graph, deps, nullptr, ndeps, &wp));
  cudaGraph_t body = wp.conditional.phGraph_out[0];
  UOT_CUDA(cudaGraphConditionalHandleCreate(&hi, body, 0, 0));
  // body: iteration t = 1, 3, 5, ... (f half-step of iteration t, g half-step of iteration t + 1)
  UOT_CUDA(cudaStreamBeginCaptureToGraph(b1, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
  c.st = b1;
  LoopCtl fc;
  fc.ctl = 1;
  LoopCtl gc;
  gc.ctl = 2;
  gc.cond_while = hw;
  gc.cond_if = hi;
  v = f_half(L, 0, fc);
  if (v == UOT_OK) v = g_half(L, 1, gc);
  cudaGraphNode_t inode = nullptr;
  cudaGraphNodeParams ip{};
  if (v == UOT_OK) {
    const cudaGraphNode_t* bdeps = nullptr;
    size_t nbdeps = 0;
    cudaError_t e = cudaStreamGetCaptureInfo(b1, &cs, nullptr, nullptr, &bdeps, nullptr, &nbdeps);
    ip.type = cudaGraphNodeTypeConditional;
    ip.conditional.handle = hi;
    ip.conditional.type = cudaGraphCondTypeIf;
    ip.conditional.size = 1;
    if (e == cudaSuccess) e = cudaGraphAddNode(&inode, body, bdeps, nullptr, nbdeps, &ip);
    if (e != cudaSuccess) v = cuda_fail(e, "adding the conditional if node");
  }
  if (v == UOT_OK) {
    // iteration t + 1 = 2, 4, ... in the if body, then back to the while condition
    cudaError_t e = cudaStreamBeginCaptureToGraph(b2, ip.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                                  cudaStreamCaptureModeRelaxed);
    if (e != cudaSuccess) v = cuda_fail(e, "capturing the second iteration");
    else {
      c.st = b2;
      LoopCtl gc2 = gc;
      v = f_half(L, 1, fc);
      if (v == UOT_OK) v = g_half(L, 2, gc2);
      cudaGraph_t tmp = nullptr;
      e = cudaStreamEndCapture(b2, &tmp);
      if (v == UOT_OK && e != cudaSuccess) v = cuda_fail(e, "ending the second iteration's capture");
    }
    if (v == UOT_OK) {
      e = cudaStreamUpdateCaptureDependencies(b1, &inode, nullptr, 1, cudaStreamSetCaptureDependencies);
      if (e != cudaSuccess) v = cuda_fail(e, "ordering the if node");
    }
  }
  cudaGraph_t tmp = nullptr;
  const cudaError_t e1 = cudaStreamEndCapture(b1, &tmp);
  c.st = s;
  if (v != UOT_OK) return v;
  if (e1 != cudaSuccess) return cuda_fail(e1, "ending the loop body's capture");
  UOT_CUDA(cudaStreamUpdateCaptureDependencies(s, &wnode, nullptr, 1, cudaStreamSetCaptureDependencies));
  UOT_CUDA(launch_finalize_loop(L.variant, L.fst, L.gbuf[0], L.gbuf[1], L.f, L.g, p.n, p.m, c.state, c.perm_x,
                                c.perm_y, 0, s));
  UOT_CUDA(launch_write_result(c.state, L.ti ? 1 : 0, 0, L.opt.tol, res, s));
  return UOT_OK;
}

}  // namespace

void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

namespace {
std::atomic<long long> g_wait_limit{0};  // 0: kWaitPolls; < 0: no polls
}  // namespace

long long wait_limit() {
  const long long v = g_wait_limit.load(std::memory_order_relaxed);
  return v > 0 ? v : (v < 0 ? 0 : kWaitPolls);
}

void set_wait_limit(long long polls) { g_wait_limit.store(polls, std::memory_order_relaxed); }

void set_last_error(const char* msg) { g_last_error = msg; }

int device_sm_count() {
  static std::mutex mu;
  static int cache[64] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 148;
  std::lock_guard<std::mutex> lk(mu);
  if (cache[dev] == 0) {
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) v = 148;
    cache[dev] = v;
  }
  return cache[dev];
}

}  // namespace uot

using namespace uot;

// A problem with its options and variant, prepared once: host-side state of
// uot_plan_solve (private streams for capturing, executable graphs per set of
// buffers).
struct uot_plan {
  uot_problem prob;
  uot_options opt;
  int variant;
  int device;
  cudaStream_t cap = nullptr, b1 = nullptr, b2 = nullptr;
  std::mutex mu;
  struct Exec {
    float* f;
    float* g;
    uot_result* res;
    void* ws;
    size_t ws_bytes;
    cudaGraphExec_t exec;
  };
  std::vector<Exec> cache;  // most recent last
};

namespace {
constexpr size_t kPlanCache = 4;

void plan_release(uot_plan* P) {
  if (!P) return;
  for (auto& x : P->cache) cudaGraphExecDestroy(x.exec);
  if (P->cap) cudaStreamDestroy(P->cap);
  if (P->b1) cudaStreamDestroy(P->b1);
  if (P->b2) cudaStreamDestroy(P->b2);
  delete P;
}
}  // namespace


extern "C" {

size_t uot_workspace_size(const uot_problem* prob) {
  if (validate(prob) != UOT_OK) return 0;
  return ws_layout(*prob).total;
}

uot_status uot_softmin(const uot_problem* prob, int32_t axis, const float* pot, float* out, void* ws,
                       size_t ws_bytes, void* stream) {
  Ctx c;
  uot_status v = make_ctx(prob, ws, ws_bytes, stream, &c);
  if (v != UOT_OK) return v;
  if (axis != 0 && axis != 1) return fail(UOT_ERR_INVALID_ARG, "axis must be 0 or 1");
  if (!pot || !out) return fail(UOT_ERR_INVALID_ARG, "pot and out must be device pointers");
  v = prepare(c);
  if (v != UOT_OK) return v;
  const float* pot_i = nullptr;  // the key side's potential in the sweeps' order
  v = to_internal(c, 1 - axis, pot, axis == 0 ? c.g_tmp : c.f_tmp, &pot_i);
  if (v != UOT_OK) return v;
  int splits = 0;
  bool fused = false;
  EpiParams e{};
  e.perm_out = axis == 0 ? c.perm_x : c.perm_y;
  e.mode = EPI_SOFTMIN; e.nq = axis == 0 ? c.p.n : c.p.m; e.s = c.s;
  e.eps = c.p.eps; e.rho_o = axis == 0 ? c.p.rho1 : c.p.rho2; e.rho_i = axis == 0 ? c.p.rho2 : c.p.rho1;
  e.out_is_f = axis == 0; e.lnw_o = axis == 0 ? c.ln_a : c.ln_b; e.out = out; e.state = c.state;
  e.l2w_o = axis == 0 ? c.l2_a : c.l2_b; e.l2lo_o = axis == 0 ? c.lo_a : c.lo_b;
  e.part = axis == 0 ? c.part_r : c.part_c; e.blk = c.blk;
  v = sweep(c, axis, pot_i, nullptr, false, &splits, &e, &fused);
  if (v != UOT_OK) return v;
  e.splits = splits;
  if (!fused) UOT_CUDA(launch_combine(e, c.st));
  return UOT_OK;
}

uot_status uot_sinkhorn(const uot_problem* prob, const uot_options* opt, float* f, float* g,
                        uot_result* result, void* ws, size_t ws_bytes, void* stream) {
  return solve(0, prob, opt, f, g, result, ws, ws_bytes, stream);
}

uot_status uot_ti_sinkhorn(const uot_problem* prob, const uot_options* opt, float* f, float* g,
                           uot_result* result, void* ws, size_t ws_bytes, void* stream) {
  return solve(1, prob, opt, f, g, result, ws, ws_bytes, stream);
}

uot_status uot_g_sinkhorn(const uot_problem* prob, const uot_options* opt, float* f, float* g,
                          uot_result* result, void* ws, size_t ws_bytes, void* stream) {
  return solve(2, prob, opt, f, g, result, ws, ws_bytes, stream);
}

size_t uot_sinkhorn_phi_workspace_size(const uot_problem* prob) {
  if (validate(prob) != UOT_OK) return 0;
  return phi_layout(*prob).total;
}

uot_status uot_sinkhorn_phi(const uot_problem* prob, const uot_options* opt, int32_t variant, int32_t phi1,
                            int32_t phi2, float* f, float* g, uot_result* result, void* ws, size_t ws_bytes,
                            void* stream) {
  if (!opt) return fail(UOT_ERR_INVALID_ARG, "options is NULL");
  if (variant != 0 && variant != 2) return fail(UOT_ERR_INVALID_ARG, "variant must be 0 (F) or 2 (G)");
  if ((phi1 != UOT_PHI_KL && phi1 != UOT_PHI_BERG) || (phi2 != UOT_PHI_KL && phi2 != UOT_PHI_BERG))
    return fail(UOT_ERR_INVALID_ARG, "phi1, phi2 must be UOT_PHI_KL or UOT_PHI_BERG");
  if (opt->max_iter < 1 || opt->check_every < 1) return fail(UOT_ERR_INVALID_ARG, "need max_iter, check_every >= 1");
  if (!(opt->tol >= 0.0) || !isfinite(opt->tol)) return fail(UOT_ERR_INVALID_ARG, "tol must be finite and >= 0");
  if (!f || !g) return fail(UOT_ERR_INVALID_ARG, "f and g must be device pointers");
  uot_status v = validate(prob);
  if (v != UOT_OK) return v;
  const PhiLayout PL = phi_layout(*prob);
  if (ws_bytes < PL.total)
    return fail(UOT_ERR_WORKSPACE, "workspace too small: %zu bytes given, %zu needed", ws_bytes, PL.total);
  Ctx c;
  v = make_ctx(prob, ws, ws_bytes, stream, &c, 2.0 * opt->max_iter);
  if (v != UOT_OK) return v;
  v = prepare(c);
  if (v != UOT_OK) return v;
  const uot_problem& p = c.p;
  char* b = static_cast<char*>(ws);
  float* fb = reinterpret_cast<float*>(b + PL.fb);
  float* gb = reinterpret_cast<float*>(b + PL.gb);
  float* S = reinterpret_cast<float*>(b + PL.S);
  LamState* ls = reinterpret_cast<LamState*>(b + PL.lam);
  double* lblk = reinterpret_cast<double*>(b + PL.lblk);
  const bool G = variant == 2;
  if (opt->warm_start) {
    if (c.tiled) UOT_CUDA(launch_gather_vec(f, c.perm_x, p.n, fb, c.st));
    else UOT_CUDA(cudaMemcpyAsync(fb, f, sizeof(float) * p.n, cudaMemcpyDeviceToDevice, c.st));
  } else {
    UOT_CUDA(cudaMemsetAsync(fb, 0, sizeof(float) * p.n, c.st));
  }
  UOT_CUDA(cudaMemsetAsync(gb, 0, sizeof(float) * p.m, c.st));
  UOT_CUDA(cudaMemsetAsync(ls, 0, sizeof(LamState), c.st));
  Slot* sl = &c.state->slot[0];
  // one softmin half-step into S (the key potential in the sweeps' order, its shift exact)
  auto softmin_into_S = [&](int axis, const float* pot, const double* shift) -> uot_status {
    EpiParams e{};
    e.mode = EPI_SOFTMIN; e.nq = axis == 0 ? p.n : p.m; e.s = c.s;
    e.eps = p.eps; e.rho_o = axis == 0 ? p.rho1 : p.rho2; e.rho_i = axis == 0 ? p.rho2 : p.rho1;
    e.out_is_f = axis == 0; e.lnw_o = axis == 0 ? c.ln_a : c.ln_b; e.out = S; e.state = c.state;
    e.l2w_o = axis == 0 ? c.l2_a : c.l2_b; e.l2lo_o = axis == 0 ? c.lo_a : c.lo_b;
    e.part = axis == 0 ? c.part_r : c.part_c; e.blk = c.blk; e.slot_in = 0; e.slot_out = 0;
    int splits = 0;
    bool fused = false;
    uot_status w = sweep(c, axis, pot, shift, false, &splits, &e, &fused);
    if (w != UOT_OK) return w;
    e.splits = splits;
    if (!fused) UOT_CUDA(launch_combine(e, c.st));
    return UOT_OK;
  };
  int t = 0, status = 0;
  float r = NAN;
  while (t < opt->max_iter) {
    ++t;
    UOT_CUDA(cudaMemsetAsync(&c.state->resid, 0, sizeof(float), c.st));
    // g half-step: keys f (plus lambda for G)
    v = softmin_into_S(1, fb, G ? &sl->cf : nullptr);
    if (v != UOT_OK) return v;
    UOT_CUDA(launch_phi_half(S, gb, p.m, phi2, p.rho2, p.eps, G ? &ls->lam : nullptr, 1.0, &c.state->resid,
                             &c.state->status, c.st));
    // f half-step: keys g (minus lambda for G)
    v = softmin_into_S(0, gb, G ? &sl->cg : nullptr);
    if (v != UOT_OK) return v;
    UOT_CUDA(launch_phi_half(S, fb, p.n, phi1, p.rho1, p.eps, G ? &ls->lam : nullptr, -1.0, nullptr,
                             &c.state->status, c.st));
    if (G)
      UOT_CUDA(launch_lambda_star(fb, gb, c.pa, c.pb, p.n, p.m, phi1, phi2, p.rho1, p.rho2, ls, lblk, c.state, 0,
                                  48, c.st));
    if (t == opt->max_iter || (opt->tol > 0.0 && t % opt->check_every == 0)) {
      v = read_flags(c, &status, &r);
      if (v != UOT_OK) return v;
      if (status != 0 || isnan(r)) break;
      if (opt->tol > 0.0 && r <= opt->tol) break;
    }
  }
  UOT_CUDA(launch_phi_out(fb, gb, c.perm_x, c.perm_y, f, g, p.n, p.m, &ls->lam, G ? 1 : 0, c.st));
  double lam = 0.0;
  UOT_CUDA(cudaMemcpyAsync(&lam, &ls->lam, sizeof(double), cudaMemcpyDeviceToHost, c.st));
  UOT_CUDA(cudaStreamSynchronize(c.st));
  uot_status out = UOT_OK;
  const bool converged = !isnan(r) && r <= opt->tol;
  if (status & kStatusBadWeights) out = fail(UOT_ERR_NONFINITE, "negative, NaN or infinite weights");
  else if (status & kStatusTimeout) out = fail(UOT_ERR_TIMEOUT, "a bounded device-side wait gave up (tensor-core sweep)");
  else if (status != 0 || isnan(r)) out = fail(UOT_ERR_NONFINITE, "non-finite value met during the iteration");
  else if (opt->tol > 0.0 && !converged) out = UOT_NOT_CONVERGED;
  if (result) {
    result->iters = t;
    result->converged = converged ? 1 : 0;
    result->status = out;
    result->lse_misses = 0;
    result->residual = r;
    result->lambda = G ? lam : 0.0;
  }
  return out;
}

uot_status uot_dual_value(const uot_problem* prob, const float* f, const float* g, double* out,
                          int32_t want_primal, void* ws, size_t ws_bytes, void* stream) {
  Ctx c;
  uot_status v = make_ctx(prob, ws, ws_bytes, stream, &c, want_primal ? 2.0 : 1.0);
  if (v != UOT_OK) return v;
  if (!f || !g || !out) return fail(UOT_ERR_INVALID_ARG, "f, g and out must be device pointers");
  v = prepare(c);
  if (v != UOT_OK) return v;
  const float *fi = nullptr, *gi = nullptr;
  v = to_internal(c, 0, f, c.f_tmp, &fi);
  if (v != UOT_OK) return v;
  v = to_internal(c, 1, g, c.g_tmp, &gi);
  if (v != UOT_OK) return v;
  int sr = 0, sc = 0;
  v = sweep(c, 0, gi, nullptr, false, &sr);
  if (v != UOT_OK) return v;
  if (want_primal) {
    v = sweep(c, 1, fi, nullptr, false, &sc);
    if (v != UOT_OK) return v;
  }
  DualParams d{};
  d.n = c.p.n; d.m = c.p.m; d.splits_r = sr; d.splits_c = sc; d.s = c.s; d.eps = c.p.eps;
  d.rho1 = c.p.rho1; d.rho2 = c.p.rho2; d.f = fi; d.g = gi; d.a = c.pa; d.b = c.pb;
  d.ln_a = c.ln_a; d.ln_b = c.ln_b; d.part_r = c.part_r; d.part_c = want_primal ? c.part_c : nullptr;
  d.blk = c.blk; d.state = c.state; d.out = out; d.want_primal = want_primal;
  UOT_CUDA(launch_dual(d, c.st));
  return UOT_OK;
}

uot_status uot_grad(const uot_problem* prob, const float* f, const float* g, float* grad_a, float* grad_b,
                    float* grad_x, float* grad_y, void* ws, size_t ws_bytes, void* stream) {
  Ctx c;
  uot_status v = make_ctx(prob, ws, ws_bytes, stream, &c, 2.0);
  if (v != UOT_OK) return v;
  if (!f || !g) return fail(UOT_ERR_INVALID_ARG, "f and g must be device pointers");
  if ((grad_x || grad_y) && c.p.cost_kind != UOT_COST_POINTS)
    return fail(UOT_ERR_INVALID_ARG, "point gradients need the points cost");
  v = prepare(c);
  if (v != UOT_OK) return v;
  const uot_problem& p = c.p;
  const float *fi = nullptr, *gi = nullptr;
  v = to_internal(c, 0, f, c.f_tmp, &fi);
  if (v != UOT_OK) return v;
  v = to_internal(c, 1, g, c.g_tmp, &gi);
  if (v != UOT_OK) return v;
  for (int side = 0; side < 2; ++side) {
    float* gw = side == 0 ? grad_a : grad_b;
    float* gpts = side == 0 ? grad_x : grad_y;
    if (!gw && !gpts) continue;
    const bool mom = gpts != nullptr;
    int splits = 0;
    // side 0: rows (x side) against y with pot g; side 1: columns against x with pot f
    v = sweep(c, side, side == 0 ? gi : fi, nullptr, mom, &splits);
    if (v != UOT_OK) return v;
    UOT_CUDA(launch_mass(side == 0 ? p.b : p.a, side == 0 ? p.m : p.n, c.blk, c.state, 0, c.st));
    GradParams gp{};
    gp.nq = side == 0 ? p.n : p.m; gp.splits = splits; gp.dim = p.dim; gp.moments = mom ? p.dim : 0;
    gp.s = c.s; gp.eps = p.eps; gp.rho_o = side == 0 ? p.rho1 : p.rho2; gp.p = p.p;
    gp.pot_o = side == 0 ? fi : gi; gp.part = side == 0 ? c.part_r : c.part_c;
    gp.grad_w = gw; gp.grad_pts = gpts; gp.lnw_o = side == 0 ? c.ln_a : c.ln_b; gp.state = c.state;
    gp.perm = side == 0 ? c.perm_x : c.perm_y;
    UOT_CUDA(launch_grad_epilogue(gp, c.st));
  }
  return UOT_OK;
}

size_t uot_unrolled_workspace_size(const uot_problem* prob, int32_t T, int32_t ckpt_every) {
  if (ur_check(prob, T, ckpt_every) != UOT_OK) return 0;
  uot_problem pd = *prob;
  pd.ordering = 2;
  return ur_layout(pd, T, ckpt_every).total;
}

uot_status uot_grad_unrolled(const uot_problem* prob, int32_t T, int32_t ckpt_every, double* value, float* grad_a,
                             float* grad_b, float* grad_x, float* grad_y, void* ws, size_t ws_bytes, void* stream) {
  return grad_unrolled(prob, T, ckpt_every, value, grad_a, grad_b, grad_x, grad_y, ws, ws_bytes, stream);
}

uint64_t uot_kernel_launches(void) { return g_launches.load(); }

uot_status uot_profile_begin(void) {
  g_prof.open = true;
  g_prof.used = 0;
  g_prof.launches = 0;
  return UOT_OK;
}

uot_status uot_profile_end(double* sweep_ms, int64_t* timed_launches, int64_t* launches) {
  if (!g_prof.open) return fail(UOT_ERR_INVALID_ARG, "no profile open on this thread");
  g_prof.open = false;
  double total = 0.0;
  for (size_t k = 0; k + 1 < g_prof.used; k += 2) {
    if (cudaEventSynchronize(g_prof.ev[k + 1]) != cudaSuccess) return cuda_fail(cudaGetLastError(), "event sync");
    float ms = 0.f;
    cudaError_t e = cudaEventElapsedTime(&ms, g_prof.ev[k], g_prof.ev[k + 1]);
    if (e != cudaSuccess) return cuda_fail(e, "cudaEventElapsedTime");
    total += ms;
  }
  if (sweep_ms) *sweep_ms = total;
  if (timed_launches) *timed_launches = (int64_t)(g_prof.used / 2);
  if (launches) *launches = g_prof.launches;
  for (cudaEvent_t e : g_prof.ev) cudaEventDestroy(e);
  g_prof.ev.clear();
  g_prof.used = 0;
  return UOT_OK;
}

uot_status uot_plan_create(const uot_problem* prob, const uot_options* opt, int32_t variant, uot_plan** out) {
  if (!out) return fail(UOT_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  tune_autoload();
  uot_status v = validate(prob);
  if (v != UOT_OK) return v;
  if (!opt) return fail(UOT_ERR_INVALID_ARG, "options is NULL");
  if (variant < 0 || variant > 2) return fail(UOT_ERR_INVALID_ARG, "variant must be 0 (plain), 1 (TI) or 2 (G)");
  if (opt->max_iter < 1 || opt->check_every < 1) return fail(UOT_ERR_INVALID_ARG, "need max_iter, check_every >= 1");
  if (!(opt->tol >= 0.0) || !isfinite(opt->tol)) return fail(UOT_ERR_INVALID_ARG, "tol must be finite and >= 0");
  if (opt->lse_reference < 0 || opt->lse_reference > 2)
    return fail(UOT_ERR_INVALID_ARG, "lse_reference must be 0, 1 or 2");
  if (opt->anderson_k != 0)
    return fail(UOT_ERR_UNSUPPORTED, "Anderson extrapolation is host-driven: use uot_sinkhorn / uot_ti_sinkhorn / "
                                     "uot_g_sinkhorn for it");
  uot_plan* P = new (std::nothrow) uot_plan();
  if (!P) return fail(UOT_ERR_INVALID_ARG, "out of host memory");
  P->prob = *prob;
  P->opt = *opt;
  P->variant = variant;
  cudaError_t e = cudaGetDevice(&P->device);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&P->cap, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&P->b1, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&P->b2, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    plan_release(P);
    return cuda_fail(e, "uot_plan_create");
  }
  // launch geometry (occupancy queries) is settled here, outside any capture
  (void)ws_layout(*prob);
  *out = P;
  return UOT_OK;
}

void uot_plan_destroy(uot_plan* plan) { plan_release(plan); }

size_t uot_plan_workspace_size(const uot_plan* plan) {
  if (!plan) {
    fail(UOT_ERR_INVALID_ARG, "plan is NULL");
    return 0;
  }
  return ws_layout(plan->prob).total;
}

uot_status uot_plan_solve(uot_plan* plan, float* f, float* g, uot_result* res_dev, void* ws, size_t ws_bytes,
                          void* stream) {
  if (!plan) return fail(UOT_ERR_INVALID_ARG, "plan is NULL");
  if (!res_dev) return fail(UOT_ERR_INVALID_ARG, "res_dev must be a device pointer");
  int dev = -1;
  UOT_CUDA(cudaGetDevice(&dev));
  if (dev != plan->device) return fail(UOT_ERR_INVALID_ARG, "the plan was created on another device");
  std::lock_guard<std::mutex> lk(plan->mu);
  Loop L;
  uot_status v = loop_setup(L, plan->variant, &plan->prob, &plan->opt, f, g, ws, ws_bytes, stream);
  if (v != UOT_OK) return v;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  UOT_CUDA(cudaStreamIsCapturing(st, &cs));
  if (cs == cudaStreamCaptureStatusActive) return emit_solve(L, st, plan->b1, plan->b2, res_dev);
  if (cs != cudaStreamCaptureStatusNone) return fail(UOT_ERR_CUDA, "the stream's capture was invalidated");
  cudaGraphExec_t exec = nullptr;
  for (size_t k = 0; k < plan->cache.size(); ++k) {
    const uot_plan::Exec& x = plan->cache[k];
    if (x.f == f && x.g == g && x.res == res_dev && x.ws == ws && x.ws_bytes == ws_bytes) {
      exec = x.exec;
      uot_plan::Exec keep = x;
      plan->cache.erase(plan->cache.begin() + (long)k);
      plan->cache.push_back(keep);
      break;
    }
  }
  if (!exec) {
    UOT_CUDA(cudaStreamBeginCapture(plan->cap, cudaStreamCaptureModeThreadLocal));
    v = emit_solve(L, plan->cap, plan->b1, plan->b2, res_dev);
    cudaGraph_t graph = nullptr;
    const cudaError_t ee = cudaStreamEndCapture(plan->cap, &graph);
    if (v != UOT_OK || ee != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      return v != UOT_OK ? v : cuda_fail(ee, "capturing the solve");
    }
    const cudaError_t ie = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ie != cudaSuccess) return cuda_fail(ie, "instantiating the solve graph");
    if (plan->cache.size() >= kPlanCache) {
      cudaGraphExecDestroy(plan->cache.front().exec);
      plan->cache.erase(plan->cache.begin());
    }
    plan->cache.push_back(uot_plan::Exec{f, g, res_dev, ws, ws_bytes, exec});
  }
  UOT_CUDA(cudaGraphLaunch(exec, st));
  return UOT_OK;
}

void uot_test_set_wait_limit(int64_t polls) { set_wait_limit((long long)polls); }

const char* uot_last_error(void) { return g_last_error.c_str(); }

const char* uot_version(void) { return "uot 0.1.0 (sm_103a)"; }

}  // extern "C"
