// Host driver of the batched solver (uot_sinkhorn_batched): validation,
// workspace layout, longest-first work queues and the iteration loop, with
// chunks of iterations captured as a CUDA graph.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>

#include <algorithm>
#include <string>
#include <vector>

#include "batched.cuh"
#include "uot_internal.cuh"

namespace uot {
namespace {

size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

struct BLayout {
  size_t probs, st, units, queue_f, queue_g, upart, ctr, l2a, l2b, lna, lnb, g1, total;
  long long na, nb;   // lengths of the packed weight arrays
  int units_f, units_g;
};

uot_status bfail(uot_status s, const char* msg) {
  set_last_error(msg);
  return s;
}

uot_status validate_batch(const uot_batch* b, BLayout* L) {
  if (!b) return bfail(UOT_ERR_INVALID_ARG, "batch is NULL");
  if (b->count < 1) return bfail(UOT_ERR_INVALID_ARG, "batch count must be >= 1");
  if (!b->n || !b->m || !b->dim || !b->eps || !b->rho1 || !b->rho2 || !b->x_off || !b->y_off || !b->a_off ||
      !b->b_off)
    return bfail(UOT_ERR_INVALID_ARG, "batch host arrays must not be NULL");
  if (!b->x || !b->y || !b->a || !b->b) return bfail(UOT_ERR_INVALID_ARG, "batch device arrays must not be NULL");
  const int rpu = batch_rows_per_unit();
  long long na = 0, nb = 0, uf = 0, ug = 0;
  for (int k = 0; k < b->count; ++k) {
    if (b->n[k] < 1 || b->m[k] < 1) return bfail(UOT_ERR_INVALID_ARG, "every problem needs n, m >= 1");
    if (b->dim[k] < 1 || b->dim[k] > 3) return bfail(UOT_ERR_UNSUPPORTED, "batched problems need dim 1..3");
    if (!(b->eps[k] > 0) || !(b->rho1[k] > 0) || !(b->rho2[k] > 0) || !isfinite(b->eps[k]) ||
        !isfinite(b->rho1[k]) || !isfinite(b->rho2[k]))
      return bfail(UOT_ERR_INVALID_ARG, "every problem needs finite eps, rho1, rho2 > 0");
    if (b->x_off[k] < 0 || b->y_off[k] < 0 || b->a_off[k] < 0 || b->b_off[k] < 0)
      return bfail(UOT_ERR_INVALID_ARG, "offsets must be >= 0");
    na = std::max(na, (long long)(b->a_off[k] + b->n[k]));
    nb = std::max(nb, (long long)(b->b_off[k] + b->m[k]));
    uf += (b->n[k] + rpu - 1) / rpu;
    ug += (b->m[k] + rpu - 1) / rpu;
  }
  if (uf + ug > (1ll << 30)) return bfail(UOT_ERR_INVALID_ARG, "batch too large");
  size_t off = 0;
  auto take = [&](size_t bytes) { size_t o = off; off = align256(off + bytes); return o; };
  L->probs = take(sizeof(BProb) * b->count);
  L->st = take(sizeof(BState) * b->count);
  L->units = take(sizeof(int2) * (uf + ug));
  L->queue_f = take(sizeof(int) * uf);
  L->queue_g = take(sizeof(int) * ug);
  L->upart = take(sizeof(double) * 4 * (uf + ug));
  L->ctr = take(sizeof(unsigned int) * 8);
  L->l2a = take(sizeof(float) * na);
  L->l2b = take(sizeof(float) * nb);
  L->lna = take(sizeof(double) * na);
  L->lnb = take(sizeof(double) * nb);
  L->g1 = take(sizeof(float) * nb);
  L->total = off;
  L->na = na;
  L->nb = nb;
  L->units_f = (int)uf;
  L->units_g = (int)ug;
  return UOT_OK;
}

#define BCUDA(call)                                                    \
  do {                                                                 \
    cudaError_t e_ = (call);                                           \
    if (e_ != cudaSuccess) {                                           \
      std::string m_ = std::string(#call) + ": " + cudaGetErrorString(e_); \
      return bfail(UOT_ERR_CUDA, m_.c_str());                          \
    }                                                                  \
  } while (0)

}  // namespace
}  // namespace uot

using namespace uot;

extern "C" {

size_t uot_batch_workspace_size(const uot_batch* batch) {
  BLayout L;
  if (validate_batch(batch, &L) != UOT_OK) return 0;
  return L.total;
}

uot_status uot_sinkhorn_batched(const uot_batch* b, const uot_options* opt, int32_t ti, float* f, float* g,
                                uot_result* results, void* ws, size_t ws_bytes, void* stream) {
  BLayout L;
  uot_status v = validate_batch(b, &L);
  if (v != UOT_OK) return v;
  if (!opt) return bfail(UOT_ERR_INVALID_ARG, "options is NULL");
  if (opt->max_iter < 1 || opt->check_every < 1 || !(opt->tol >= 0.0))
    return bfail(UOT_ERR_INVALID_ARG, "need max_iter >= 1, check_every >= 1, tol >= 0");
  if (opt->warm_start || opt->residual_history || opt->anderson_k)
    return bfail(UOT_ERR_UNSUPPORTED, "batched solves take no warm start, residual history or Anderson extrapolation");
  if (!f || !g || !results) return bfail(UOT_ERR_INVALID_ARG, "f, g and results must not be NULL");
  if (!ws) return bfail(UOT_ERR_WORKSPACE, "workspace is NULL");
  if (reinterpret_cast<uintptr_t>(ws) & 255) return bfail(UOT_ERR_WORKSPACE, "workspace must be 256-byte aligned");
  if (ws_bytes < L.total) return bfail(UOT_ERR_WORKSPACE, "workspace too small for the batch");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  char* base = static_cast<char*>(ws);
  BProb* d_probs = reinterpret_cast<BProb*>(base + L.probs);
  BState* d_st = reinterpret_cast<BState*>(base + L.st);
  int2* d_units = reinterpret_cast<int2*>(base + L.units);
  int* d_qf = reinterpret_cast<int*>(base + L.queue_f);
  int* d_qg = reinterpret_cast<int*>(base + L.queue_g);
  double* d_upart = reinterpret_cast<double*>(base + L.upart);
  unsigned int* d_ctr = reinterpret_cast<unsigned int*>(base + L.ctr);
  float* d_l2a = reinterpret_cast<float*>(base + L.l2a);
  float* d_l2b = reinterpret_cast<float*>(base + L.l2b);
  double* d_lna = reinterpret_cast<double*>(base + L.lna);
  double* d_lnb = reinterpret_cast<double*>(base + L.lnb);
  float* d_g1 = reinterpret_cast<float*>(base + L.g1);

  // host tables: problems, units (problem-contiguous), longest-first queues
  const int count = b->count, rpu = batch_rows_per_unit();
  std::vector<BProb> probs(count);
  std::vector<int2> units;
  units.reserve(L.units_f + L.units_g);
  for (int k = 0; k < count; ++k) {
    BProb& p = probs[k];
    p.n = b->n[k]; p.m = b->m[k]; p.dim = b->dim[k];
    p.units_f = (p.n + rpu - 1) / rpu; p.units_g = (p.m + rpu - 1) / rpu;
    p.x_off = b->x_off[k]; p.y_off = b->y_off[k]; p.a_off = b->a_off[k]; p.b_off = b->b_off[k];
    p.eps = b->eps[k]; p.rho1 = b->rho1[k]; p.rho2 = b->rho2[k]; p.s = kLog2e / p.eps;
    p.pad = 0;
  }
  for (int k = 0; k < count; ++k) {
    probs[k].ubase_f = (int)units.size();
    for (int r = 0; r < probs[k].units_f; ++r) units.push_back(make_int2(k, r * rpu));
  }
  for (int k = 0; k < count; ++k) {
    probs[k].ubase_g = (int)units.size();
    for (int r = 0; r < probs[k].units_g; ++r) units.push_back(make_int2(k, r * rpu));
  }
  // cost of a unit ~ rows x keys x (dim + 4)
  auto cost = [&](int u, bool fside) {
    const BProb& p = probs[units[u].x];
    const int rows = std::min(rpu, (fside ? p.n : p.m) - units[u].y);
    return (double)rows * (fside ? p.m : p.n) * (p.dim + 4);
  };
  std::vector<int> qf(L.units_f), qg(L.units_g);
  for (int i = 0; i < L.units_f; ++i) qf[i] = i;
  for (int i = 0; i < L.units_g; ++i) qg[i] = L.units_f + i;
  std::stable_sort(qf.begin(), qf.end(), [&](int a, int c) { return cost(a, true) > cost(c, true); });
  std::stable_sort(qg.begin(), qg.end(), [&](int a, int c) { return cost(a, false) > cost(c, false); });

  BCUDA(cudaMemcpyAsync(d_probs, probs.data(), sizeof(BProb) * count, cudaMemcpyHostToDevice, st));
  BCUDA(cudaMemcpyAsync(d_units, units.data(), sizeof(int2) * units.size(), cudaMemcpyHostToDevice, st));
  BCUDA(cudaMemcpyAsync(d_qf, qf.data(), sizeof(int) * qf.size(), cudaMemcpyHostToDevice, st));
  BCUDA(cudaMemcpyAsync(d_qg, qg.data(), sizeof(int) * qg.size(), cudaMemcpyHostToDevice, st));
  // counters: [0] next, [1] finished, [2] active, [3] iteration index, [4] weight flags
  const unsigned int ctr0[8] = {0u, 0u, (unsigned int)count, 0u, 0u, 0u, 0u, 0u};
  BCUDA(cudaMemcpyAsync(d_ctr, ctr0, sizeof(ctr0), cudaMemcpyHostToDevice, st));
  BCUDA(cudaMemsetAsync(f, 0, sizeof(float) * L.na, st));
  BCUDA(cudaMemsetAsync(g, 0, sizeof(float) * L.nb, st));
  BCUDA(cudaMemsetAsync(d_g1, 0, sizeof(float) * L.nb, st));
  int* d_flags = reinterpret_cast<int*>(d_ctr + 4);
  BCUDA(launch_log_weights(b->a, (int)L.na, d_lna, d_l2a, nullptr, d_flags, st));
  BCUDA(launch_log_weights(b->b, (int)L.nb, d_lnb, d_l2b, nullptr, d_flags, st));
  BCUDA(launch_batch_init(d_probs, d_st, b->a, count, ti ? 1 : 0, d_ctr + 2, st));

  BHalf h{};
  h.probs = d_probs; h.st = d_st; h.units = d_units; h.ti = ti ? 1 : 0;
  h.max_iter = opt->max_iter; h.check_every = opt->check_every; h.tol = opt->tol;
  h.next = d_ctr; h.finished = d_ctr + 1; h.active = d_ctr + 2; h.iter = reinterpret_cast<int*>(d_ctr + 3);
  h.x = b->x; h.y = b->y; h.l2a = d_l2a; h.l2b = d_l2b; h.lna = d_lna; h.lnb = d_lnb;
  h.f = f; h.g0 = g; h.g1 = d_g1; h.upart = d_upart;
  BHalf hf = h, hg = h;
  hf.side = 0; hf.queue = d_qf; hf.nunits = L.units_f;
  hg.side = 1; hg.queue = d_qg; hg.nunits = L.units_g;
  const int grid = batch_grid();

  // G(1); then chunks of check_every x (F, G) until no problem is running
  BCUDA(launch_batch_half(hg, grid, st));
  const int K = opt->check_every;
  cudaGraphExec_t exec = nullptr;
  if (st) {
    cudaGraph_t graph = nullptr;
    BCUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    cudaError_t ce = cudaSuccess;
    for (int q = 0; q < K && ce == cudaSuccess; ++q) {
      ce = launch_batch_half(hf, grid, st);
      if (ce == cudaSuccess) ce = launch_batch_half(hg, grid, st);
    }
    cudaError_t ee = cudaStreamEndCapture(st, &graph);
    if (ce != cudaSuccess || ee != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      return bfail(UOT_ERR_CUDA, "capturing the batched iteration chunk failed");
    }
    cudaError_t ie = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ie != cudaSuccess) return bfail(UOT_ERR_CUDA, "instantiating the batched iteration graph failed");
  }
  long long done_iters = 0;
  unsigned int active = (unsigned int)count;
  uot_status out = UOT_OK;
  while (true) {
    if (exec) {
      if (cudaGraphLaunch(exec, st) != cudaSuccess) { out = bfail(UOT_ERR_CUDA, "graph launch failed"); break; }
    } else {
      for (int q = 0; q < K; ++q) {
        if (launch_batch_half(hf, grid, st) != cudaSuccess || launch_batch_half(hg, grid, st) != cudaSuccess) {
          out = bfail(UOT_ERR_CUDA, "batched half-step launch failed");
          break;
        }
      }
      if (out != UOT_OK) break;
    }
    done_iters += K;
    if (cudaMemcpyAsync(&active, d_ctr + 2, sizeof(unsigned int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
      out = bfail(UOT_ERR_CUDA, "reading the active-problem count failed");
      break;
    }
    if (active == 0) break;
    if (done_iters > (long long)opt->max_iter + K) {  // every problem stops at max_iter by itself
      out = bfail(UOT_ERR_CUDA, "batched solve did not terminate");
      break;
    }
  }
  if (exec) cudaGraphExecDestroy(exec);
  if (out != UOT_OK) return out;
  BCUDA(launch_batch_phi(d_probs, d_st, f, g, d_g1, count, ti ? 1 : 0, st));
  std::vector<BState> hst(count);
  int flags = 0;
  BCUDA(cudaMemcpyAsync(hst.data(), d_st, sizeof(BState) * count, cudaMemcpyDeviceToHost, st));
  BCUDA(cudaMemcpyAsync(&flags, d_flags, sizeof(int), cudaMemcpyDeviceToHost, st));
  BCUDA(cudaStreamSynchronize(st));
  if (flags & kStatusBadWeights) return bfail(UOT_ERR_NONFINITE, "negative, NaN or infinite weights in the batch");
  bool all_conv = true, bad = false;
  for (int k = 0; k < count; ++k) {
    const BState& s = hst[k];
    uot_result& r = results[k];
    r.iters = s.conv_iter;
    r.converged = s.status == 1;
    r.status = s.status == 1 ? UOT_OK : (s.status == 3 ? UOT_NOT_CONVERGED : UOT_ERR_NONFINITE);
    r.lse_misses = 0;
    r.residual = s.resid;
    r.lambda = ti ? s.slot[s.conv_iter & 1].lam : 0.0;
    if (s.status != 1) all_conv = false;
    if (s.status == 2) bad = true;
  }
  if (bad) return bfail(UOT_ERR_NONFINITE, "some problems met non-finite values or invalid weights");
  return all_conv ? UOT_OK : UOT_NOT_CONVERGED;
}

}  // extern "C"
