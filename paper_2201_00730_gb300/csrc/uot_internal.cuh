// Internal declarations shared by the libuot translation units (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "../../include/uot.h"

namespace uot {

constexpr double kLog2e = 1.4426950408889634074;  // log2(e)
constexpr double kLn2 = 0.69314718055994530942;   // ln(2)
// Log2-weight sentinel of a zero weight: finite so that (t - max) never forms inf - inf.
constexpr float kZeroW = -1.0e30f;
constexpr float kInitMax = -2.0e30f;

// Scalars of one half-step of the iteration, FP64 (Prop. 2 / App. B quantities),
// with float-pair copies (hi, lo) that the half-step epilogues read and write:
// FP64 arithmetic is slow on this GPU and sits on every launch's critical path.
struct Slot {
  double A;    // Smin_a^rho1(fb) of the current fb
  double B;    // Smin_b^rho2(gb) of the current gb
  double cf;   // fb = f_hat + cf (the stored f vector is f_hat)
  double cg;   // gb = g_hat + cg
  double lam;  // lambda*(fb, gb) = tau1 B - tau2 A
  double pad;
  float Af[2], Bf[2], cff[2], cgf[2], lamf[2];  // float pairs of A, B, cf, cg, lam
  float padf[2];
};

// Device-resident iteration state, at the start of the workspace.
struct DevState {
  Slot slot[2];          // ring indexed by iteration parity
  unsigned int counter;  // last-block-done counter (reset by the last block)
  int status;            // bit flags, see kStatus*
  float resid;           // residual of the latest finished g half-step
  float pad0;
  double dual[4];        // uot_dual_value scratch results
  double pad[4];
  // fixed-reference log-sum-exp (tiled sweeps of a solve), indexed by out_is_f
  int lse_ready[2];      // the side's buffer holds the previous launch's row values
  int lse_ok[2];         // the next launch of the side takes them as exponent reference
  unsigned int lse_miss; // rows recomputed because the reference was too far off
  int iters;             // iterations done by the resident small-problem solver
  // device-driven iteration (uot_plan_solve): index t of the latest f half-step's
  // iterate, and whether the latest check stopped the loop
  int loop_t;
  int loop_done;
};

// Resident solver for small point problems (dim <= 3, p = 2, N M <= 2^20, both
// clouds in one SM's shared memory): the plain / TI loop of the solver in one
// launch of a thread-block cluster, eg and ef the g- and f-half-step templates
// (per-iteration fields are set on the device); writes the iteration count to
// state->iters.
bool small_path(const uot_problem& p);
struct EpiParams;
cudaError_t launch_small_solve(const float* x, const float* y, const float* l2a, const float* l2b, int n, int m,
                               int dim, int ti, int max_iter, int check_every, double tol, double s, float* fst,
                               float* gb0, float* gb1, const EpiParams& eg, const EpiParams& ef, cudaStream_t st);

// Largest change of a row's log-sum-exp (log2 units) between two launches of a
// side after which the next launch uses the stored values as reference, and
// the window |lse2 - reference| within which the fixed-reference sum is kept.
constexpr double kLseGate = 24.0;
constexpr double kLseWindow = 60.0;

constexpr int kStatusNonfinite = 1;
constexpr int kStatusBadWeights = 2;
constexpr int kStatusTimeout = 4;  // a bounded device-side wait gave up

// ---- launch geometry -----------------------------------------------------

struct SweepGeom {
  int threads;      // CTA size
  int rows;         // rows per thread (R)
  int row_blocks;   // grid.x
  int splits;       // grid.y (key chunks); partial slots per query
  int keys_per_split;
  int ctas;         // persistent unit-range grids: CTAs in the grid (0 elsewhere)
};

int device_sm_count();
// Polls allowed to a main-loop mbarrier wait of the tensor-core sweeps before it
// gives up (default kWaitPolls; lowered only by the test hook uot_test_set_wait_limit).
constexpr long long kWaitPolls = 1LL << 24;
long long wait_limit();
// Counts one kernel launch (process-wide counter read by uot_kernel_launches).
void note_launch();
// Sets the calling thread's message returned by uot_last_error().
void set_last_error(const char* msg);
// Test hook behind uot_test_set_wait_limit (0 restores kWaitPolls).
void set_wait_limit(long long polls);
// tuned = false: the built-in shape, whatever the tuning table holds.
SweepGeom points_geom(int nq, int nk, int dim, bool moments, bool tuned = true);
SweepGeom dense_row_geom(int nrows, int ncols, bool tuned = true);
SweepGeom dense_col_geom(int nrows, int ncols, bool tuned = true);
int max_splits_for(const uot_problem& p);
// General phi^* (general_phi.cu).  State of the lambda* search: the current
// lambda, the bracket [lo, hi] of the root of F', the last-block counter.
struct LamState {
  double lam, lo, hi;
  unsigned int counter;
  int done;
};
// out = -aprox_{phi^*}(-S) + sign * *shift (shift nullable), elementwise over n;
// resid (nullable) gets max |out_new - out_old| by an atomic max.
cudaError_t launch_phi_half(const float* S, float* out, int n, int phi, double rho, double eps, const double* shift,
                            double sign, float* resid, int* status, cudaStream_t st);
// lambda*(fb, gb): one bracketing launch and `steps` Newton launches (each a no-op
// once converged); the result goes to ls->lam and to the shifts of st->slot[slot].
cudaError_t launch_lambda_star(const float* fb, const float* gb, const float* a, const float* b, int n, int m,
                               int phi1, int phi2, double rho1, double rho2, LamState* ls, double* blk, DevState* st,
                               int slot, int steps, cudaStream_t s);
// f = fb + lambda, g = gb - lambda (g_mode; else plain copies) in the caller's order.
cudaError_t launch_phi_out(const float* fb, const float* gb, const int* pf, const int* pg, float* f, float* g, int n,
                           int m, const double* lam, int g_mode, cudaStream_t st);

// Launch-shape tuning (tune.cu): the value of a knob for a sweep of `entries`
// cost entries in dimension dim (-1: none), dflt when the table has none;
// floor(log2(entries)); the one-time load of UOT_TUNE_FILE.
long long tune_value(const char* knob, int dim, long long entries, long long dflt);
int tune_bucket(long long entries);
void tune_autoload();
// While a TuneScope lives, tune_value returns its values for its knobs on this
// thread (workspace sizing takes the largest partials over every allowed shape,
// so that a workspace stays valid whatever the table holds later).
struct TuneFix {
  const char* knob;
  long long value;
};
class TuneScope {
 public:
  TuneScope(const TuneFix* f, int n);
  ~TuneScope();
  TuneScope(const TuneScope&) = delete;
  TuneScope& operator=(const TuneScope&) = delete;

 private:
  int n_;
};
std::vector<long long> tune_allowed(const char* knob);

constexpr int kMaxBlocks = 4096;
constexpr int kTileKeys = 128;  // keys per local-frame tile of the tiled sweep

// True when the tensor-core sweep (split-FP16 cross term) serves this problem.
inline bool mma_path(const uot_problem& p) {
  return p.cost_kind == UOT_COST_POINTS && p.dim >= 32 && p.p == 2.0f;
}
cudaError_t launch_center(const float* x, int n, const float* y, int m, int dim, float* center, cudaStream_t st);

// True when the tiled (Morton-ordered, local-frame) sweep serves this problem.
inline bool tiled_path(const uot_problem& p) {
  return p.cost_kind == UOT_COST_POINTS && p.dim <= 3 && p.p == 2.0f;
}

// Scratch of the ordering step (bounding box, Morton codes, radix sort).
struct OrderScratch {
  float* blk_f;           // [kMaxBlocks * 6]
  float* box;             // [6]
  unsigned int* counter;  // last-block counter (zero between launches)
  unsigned int* code_in;  // [max(n, m)]
  unsigned int* code_out; // [max(n, m)]
  int* idx_in;            // [max(n, m)]
  void* temp;             // radix-sort temporary storage
  size_t temp_bytes;
};
size_t sort_temp_bytes(int n);
// Morton-order pts (n x dim) and w: perm[i] = source index of sorted point i;
// pts_s / w_s = gathered copies; centers = bounding-box centre of every tile.
cudaError_t launch_order_points(const float* pts, const float* w, int n, int dim, OrderScratch sc, int* perm,
                                float* pts_s, float* w_s, float4* centers, cudaStream_t st);
cudaError_t launch_gather_vec(const float* v, const int* perm, int n, float* out, cudaStream_t st);
cudaError_t launch_scatter_rows(const float* v, const int* perm, int n, int dim, float* out, cudaStream_t st);

// ---- kernels (launchers) --------------------------------------------------

struct EpiParams;

// Side description: the "query" side owns the output vector, the "key" side is
// summed over.
struct SideDesc {
  const float* pts;     // points (points cost) [n x dim]
  const float* l2w;     // log2 weights (kZeroW for 0)
  const double* lnw;    // natural log weights
  int n;
};

// Softmin partials: for each query row, (max, sum) of 2^{t} over each key chunk,
// t = log2 w_j + s (pot_j + shift) - s C_ij.  Moments (optional) accumulate
// sum 2^{t - max} (q_i - k_j)_d * (dC/dq factor) for gradient sweeps.
cudaError_t launch_points_sweep(const SideDesc& q, const SideDesc& k, int dim, float p,
                                const float* pot_k, const double* shift_k, double s,
                                bool moments, float* part, const SweepGeom& g, cudaStream_t st);
// Tiled sweep (sorted clouds, dim <= 3, p = 2); centers_k = tile centres of the key side.
SweepGeom tile_geom(int nq, int nk, int dim, bool tuned = true);
// With epi != nullptr the last CTA of each row block also runs the half-step
// epilogue for its rows (no separate combine launch); epi->part must be `part`.
// The sweep itself ignores shift_k: it is handed to the epilogue (epi->key_shift),
// which applies it exactly, so a shift needs epi != nullptr.
cudaError_t launch_tile_sweep(const SideDesc& q, const SideDesc& k, const float4* centers_k, int dim,
                              const float* pot_k, const double* shift_k, double s, float* part, const SweepGeom& g,
                              const struct EpiParams* epi, cudaStream_t st);
// Moment / adjoint sweep on tcgen05 (dim >= 32, p = 2; sweep_umma_mom.cu):
// partials [splits][2 + dim][nq] (max, sum of mult_j 2^(t - max), momscale *
// the moments of (x_i - y_j)).  Forward gradient sweep: l2w, pot, shift of the
// keys, zrow = hk = mk = null, momscale = 2.  Adjoint sweep: zrow = the query
// potential, hk = the keys' h, mk = the keys' signed cotangents, momscale = 1.
// opq / nq2 and opk / nk2: the plain tcgen05 sweep's operands and squared norms
// of the query and key clouds; zt (mom_zt_bytes of the key cloud) and multbits
// (one int) are scratch for the Z^T operand.
struct MomOperands {
  const void* opq;
  const float* nq2;
  const void* opk;
  const float* nk2;
  void* zt;
  int* multbits;
  int* status;
};
size_t mom_zt_bytes(int n, int dim);
SweepGeom mom_geom(int nq, int nk);
cudaError_t launch_mom_sweep(const void* opq, const float* nq2, int nq, const void* opk, const float* nk2, int nk,
                             const float* q, const float* kp, int dim, const float* center, const int* maxbits,
                             const float* l2w, const float* pot, const double* shift, const float* zrow,
                             const float* hk, const float* mk, double s, float momscale, void* zt, int* multbits,
                             float* part, const SweepGeom& g, int* status, cudaStream_t st);
// tcgen05 sweep (dim >= 32, p = 2): the operand matrices of both clouds (split
// FP16 coordinates relative to the common centre, scaled by a power of two
// from the largest |x - c| in *maxbits, canonical K-major layout, rows padded
// to 128) and their squared norms, built once per call.
int umma_dim16(int dim);
size_t umma_operand_floats(int n, int dim);
cudaError_t launch_umma_scale(const float* x, int n, const float* y, int m, int dim, const float* center,
                              int* maxbits, cudaStream_t st);
cudaError_t launch_umma_operand(const float* pts, int n, int dim, const float* center, const int* maxbits,
                                void* op, float* norm2, cudaStream_t st);
SweepGeom umma_geom(int nq, int nk);
// A main-loop wait that gives up (bounded, wait_limit()) sets kStatusTimeout in
// *status (nullable) and NaN partials; copies and MMAs in flight land first.
cudaError_t launch_umma_sweep(const void* opq, const float* nq2, int nq, const void* opk, const float* nk2, int nk,
                              int dim, const float* l2w, const float* pot, const double* shift, double s,
                              const int* maxbits, float* part, const SweepGeom& g, int* status, cudaStream_t st);
// Dense cost: axis 0 = rows of C are queries, axis 1 = columns of C are queries.
cudaError_t launch_dense_sweep(int axis, const float* C, int n, int m, const float* l2w_k,
                               const float* pot_k, const double* shift_k, double s, float* part,
                               const SweepGeom& g, cudaStream_t st);

// Epilogue modes of the combine kernel.
enum EpiMode {
  EPI_SOFTMIN = 0,   // out = S (cost units)
  EPI_PLAIN = 1,     // out = rho_o/(rho_o+eps) S; residual vs old (if given)
  EPI_TI = 2,        // out = g_hat / f_hat; FP64 mass reduction; finalize scalars
  EPI_G = 3,         // G-Sinkhorn: out = aprox(S) +- lambda_t; mass reduction; lambda_{t+1} after the f half-step
};

struct EpiParams {
  int mode;
  int nq;
  int splits;
  int moments;          // number of moment channels in the partials (0 or dim)
  double s;             // log2(e)/eps
  double eps, rho_o, rho_i;   // rho of the output side and of the key side
  int out_is_f;         // 1: output side is (f, a, rho1); 0: (g, b, rho2)
  const double* lnw_o;  // natural log weights of the output side
  const float* old_out; // previous value of the output vector (residual), nullable
  float* out;           // output vector
  const int* perm_out;  // nullable: out[perm_out[i]] receives row i (scatter to caller order)
  float* resid_hist;    // residual history (device), nullable
  int hist_index;
  int slot_in;          // slot read (key-side scalars, residual baseline)
  int slot_out;         // slot written
  DevState* state;
  const float* part;
  double* blk;
  unsigned int* rb_counter;  // per-row-block arrival counters (fused sweeps), zero between launches
  // nullable: the key side's pending shift in slot_in (cf for a g half-step, cg
  // for an f half-step), which the sweep left out and the epilogue applies
  const double* key_shift;
  // host-computed float pairs (hi, lo), see epi_finish_params
  float U2[2];    // 1/s = eps ln 2
  float CS2[2];   // rho_o/(rho_o+eps)
  float CX2[2];   // eps/(eps+rho_o) rho_o/(rho_o+rho_i)
  float CR2[2];   // eps/(eps+rho_o) rho_i/(rho_o+rho_i)
  float RL2[2];   // log2(e)/rho_o
  float NR2[2];   // -rho_o
  float KK2[2];   // TI translation k/(1-k), k = CR
  float T12[2];   // lambda* weights tau1 = rho_o/(rho_o+rho_i), tau2 = rho_i/(rho_o+rho_i)
  float T22[2];
  int ff_only;    // 1: the finalisation writes only the float pairs of the slot (resident solver)
  float* lse_buf;       // nullable: per-row log-sum-exp kept between launches of this side (tiled sweeps)
  int lse_policy;       // 0: reference after a small change, 2: whenever one is stored
  const float* l2w_o;   // TI: log2 weights of the output side as float pairs (hi, lo)
  const float* l2lo_o;
  // device-driven iteration (a solve captured in a CUDA graph, the loop a
  // conditional while node): 1 = this f half-step advances state->loop_t; 2 =
  // this g half-step evaluates the stopping rule of the host driver at iterate
  // loop_t and writes "go on" into the conditional handles (0 = not set)
  int loop_ctl;
  int loop_max_iter, loop_check_every;
  double loop_tol;
  unsigned long long cond_while, cond_if;
};
// Fills the constants of an EpiParams that depend only on s, eps and the rhos
// (call after setting s, eps, rho_o, rho_i).
void epi_finish_params(EpiParams& e);
cudaError_t launch_combine(const EpiParams& e, cudaStream_t st);

// Initial TI scalars: slot 0 = {A = Smin_a^rho1(f0), B = 0, cf = cg = 0}.
// only >= 0: refresh slot `only`'s A for a new fb held in full (cf <- 0), keep the rest.
cudaError_t launch_ti_init(const float* f0, const double* ln_a, int n, double rho1, DevState* st_dev,
                           double* blk, cudaStream_t st, int only = -1);

// ---- Anderson extrapolation (uot_options.anderson_*) ----------------------
// Scratch: a ring of K + 1 iterates (n floats each), their lambdas, the weights.
size_t anderson_bytes(int n, int K);
// Zeroes the scratch's block counter (before the first extrapolation of a solve).
cudaError_t anderson_reset(void* buf, int n, int K, cudaStream_t st);
// Stores iterate x into ring position pos: x = f (mode 0), f + slot->cf (mode 1,
// the TI fb = f_hat + cf), or f with slot->lam kept alongside (mode 2, G).
cudaError_t launch_anderson_store(const float* f, int n, int K, int pos, int mode, const Slot* slot, void* buf,
                                  cudaStream_t st);
// Replaces f by sum_{k<K} c_k x_{p0+k} (ring positions mod K + 1) and writes it to
// ring position (p0 + K) mod (K + 1); with slot_g (G) also lambda (slot cf and lam).
cudaError_t launch_anderson_extrapolate(float* f, int n, int K, int p0, double r, void* buf, Slot* slot_g,
                                        int* status, cudaStream_t st);
// Output map Phi (TI) or copy (plain) of iterate in slot `slot`; perm_f / perm_g
// (nullable) scatter sorted rows back to the caller's order.
cudaError_t launch_finalize(int ti, const float* f_hat, const float* g_hat, float* f, float* g, int n,
                            int m, const DevState* st_dev, int slot, const int* perm_f, const int* perm_g,
                            cudaStream_t st);
// The same for a device-driven loop: the iterate index and slot come from
// state->loop_t (small: state->iters), its g from g0 or g1 by parity.
cudaError_t launch_finalize_loop(int ti, const float* f_hat, const float* g0, const float* g1, float* f, float* g,
                                 int n, int m, const DevState* s, const int* perm_f, const int* perm_g, int small,
                                 cudaStream_t st);
// uot_result of a finished solve from the device state, written to device memory
// (small = the resident solver ran the loop).
cudaError_t launch_write_result(const DevState* s, int ti, int small, double tol, uot_result* out, cudaStream_t st);
// log weights (natural FP64, log2 FP32 and, if l2lo is not null, the FP32
// remainder log2 w - l2w); negative / non-finite weights set kStatusBadWeights
// in *flags (nullable).
cudaError_t launch_log_weights(const float* w, int n, double* lnw, float* l2w, float* l2lo, int* flags,
                               cudaStream_t st);

// Dual value / primal value reductions from the row (and column) sweep partials.
struct DualParams {
  int n, m, splits_r, splits_c;
  double s, eps, rho1, rho2;
  const float* f; const float* g;
  const float* a; const float* b;
  const double* ln_a; const double* ln_b;
  const float* part_r;   // row sweep partials (S_i)
  const float* part_c;   // column sweep partials (S'_j), nullable
  double* blk;
  DevState* state;
  double* out;           // device
  int want_primal;
};
cudaError_t launch_dual(const DualParams& d, cudaStream_t st);

// Envelope gradient epilogue for one side from its sweep partials (with moments).
struct GradParams {
  int nq, splits, dim, moments;
  double s, eps, rho_o;   // m(other side) is read from state->dual[0]
  float p;
  const float* pot_o;    // f (rows) or g (cols)
  const float* part;
  float* grad_w;         // d/d weights of this side, nullable
  float* grad_pts;       // d/d points of this side [nq x dim], nullable
  const double* lnw_o;   // natural log weights of this side
  const int* perm;       // nullable: outputs of row i go to caller row perm[i]
  DevState* state;
};
cudaError_t launch_grad_epilogue(const GradParams& gp, cudaStream_t st);

// ---- unrolled backward (adjoint.cu, unrolled.cu) -----------------------------
SweepGeom adjoint_geom(int nq, int nk);
// center != null (dim >= 32): the sweep runs on the tensor cores (tcgen05 moment sweep).
cudaError_t launch_adjoint(const float* q, int nq, const float* kp, int nk, int dim, const float* pot_q,
                           const float* h_k, const float* c_k, double s, float* part, double* val, double* mom,
                           const float* center, const int* maxbits, const struct MomOperands& mo, cudaStream_t st);
cudaError_t launch_add_scalar(const float* u, const double* c, int n, float* v, cudaStream_t st);
cudaError_t launch_moments(const float* part, int nq, int dim, int splits, double scale, float* G, cudaStream_t st);
cudaError_t launch_final_side(const float* part, int CH, int nq, int splits, double s, double eps, double rho,
                              const float* pot, const double* lnw, float* cot, double* blk, unsigned int* ctr,
                              double* sum, cudaStream_t st);
cudaError_t launch_final_lambda(int n, const float* u, const double* lnw, const double* X, double rho, double coef,
                                const double* sum_f, const double* sum_g, float* cot, float* gw, double* blk,
                                unsigned int* ctr, double* sum, cudaStream_t st);
cudaError_t launch_bw_f1(int n, int dim, const float* fbb, const float* fhat, const double* lna, const double* Ahat,
                         const double* sum_fbb, double kf, double rho1, double a1, const float* G, float* ga,
                         float* gx, float* Sb, double* blk, unsigned int* ctr, double* sum_out, cudaStream_t st);
cudaError_t launch_bw_smin_init(int n, const float* u, const double* lnw, const double* X, double rho, double coef,
                                const double* sum_in, float* cot, float* gw, cudaStream_t st);
cudaError_t launch_bw_adj(int n, int dim, const double* val, const double* mom, const double* lnw, double eps,
                          float* cot, float* gw, float* gpts, double* blk, unsigned int* ctr, double* sum,
                          cudaStream_t st);
cudaError_t launch_bw_g1(int m, int dim, float* gbb, const float* ghat, const double* lnb, const double* Bhat,
                         const double* sum_gbb, double kg, double rho2, double a2, const float* Gp, float* gb,
                         float* gy, float* Spb, double* blk, unsigned int* ctr, double* sum_out, cudaStream_t st);
cudaError_t launch_bw_fset(int n, const float* fb, const double* lna, const double* A, double rho1, double coef,
                           const double* sum_in, float* fbb, float* ga, cudaStream_t st);
cudaError_t launch_record_scalars(const DevState* s, int slot_t, int slot_t1, double* rec, cudaStream_t st);

// Sum of weights in FP64 into state->dual[slot_idx].
cudaError_t launch_mass(const float* w, int n, double* blk, DevState* st_dev, int idx, cudaStream_t st);

}  // namespace uot
