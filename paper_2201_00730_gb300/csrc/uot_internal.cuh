// Internal declarations shared by the libuot translation units (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/uot.h"

namespace uot {

constexpr double kLog2e = 1.4426950408889634074;  // log2(e)
constexpr double kLn2 = 0.69314718055994530942;   // ln(2)
// Log2-weight sentinel of a zero weight: finite so that (t - max) never forms inf - inf.
constexpr float kZeroW = -1.0e30f;
constexpr float kInitMax = -2.0e30f;

// Scalars of one half-step of the iteration, FP64 (Prop. 2 / App. B quantities).
struct Slot {
  double A;    // Smin_a^rho1(fb) of the current fb
  double B;    // Smin_b^rho2(gb) of the current gb
  double cf;   // fb = f_hat + cf (the stored f vector is f_hat)
  double cg;   // gb = g_hat + cg
  double lam;  // lambda*(fb, gb) = tau1 B - tau2 A
  double pad[3];
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
};

constexpr int kStatusNonfinite = 1;
constexpr int kStatusBadWeights = 2;

// ---- launch geometry -----------------------------------------------------

struct SweepGeom {
  int threads;      // CTA size
  int rows;         // rows per thread (R)
  int row_blocks;   // grid.x
  int splits;       // grid.y (key chunks)
  int keys_per_split;
};

int device_sm_count();
// Counts one kernel launch (process-wide counter read by uot_kernel_launches).
void note_launch();
// Sets the calling thread's message returned by uot_last_error().
void set_last_error(const char* msg);
SweepGeom points_geom(int nq, int nk, int dim, bool moments);
SweepGeom dense_row_geom(int nrows, int ncols);
SweepGeom dense_col_geom(int nrows, int ncols);
int max_splits_for(const uot_problem& p);

constexpr int kMaxBlocks = 4096;

// ---- kernels (launchers) --------------------------------------------------

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
// Dense cost: axis 0 = rows of C are queries, axis 1 = columns of C are queries.
cudaError_t launch_dense_sweep(int axis, const float* C, int n, int m, const float* l2w_k,
                               const float* pot_k, const double* shift_k, double s, float* part,
                               const SweepGeom& g, cudaStream_t st);

// Epilogue modes of the combine kernel.
enum EpiMode {
  EPI_SOFTMIN = 0,   // out = S (cost units)
  EPI_PLAIN = 1,     // out = rho_o/(rho_o+eps) S; residual vs old (if given)
  EPI_TI = 2,        // out = g_hat / f_hat; FP64 mass reduction; finalize scalars
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
  float* resid_hist;    // residual history (device), nullable
  int hist_index;
  int slot_in;          // slot read (key-side scalars, residual baseline)
  int slot_out;         // slot written
  DevState* state;
  const float* part;
  double* blk;
};
cudaError_t launch_combine(const EpiParams& e, cudaStream_t st);

// Initial TI scalars: slot 0 = {A = Smin_a^rho1(f0), B = 0, cf = cg = 0}.
cudaError_t launch_ti_init(const float* f0, const double* ln_a, int n, double rho1, DevState* st_dev,
                           double* blk, cudaStream_t st);
// Output map Phi (TI) or copy (plain) of iterate in slot `slot`.
cudaError_t launch_finalize(int ti, const float* f_hat, const float* g_hat, float* f, float* g, int n,
                            int m, const DevState* st_dev, int slot, cudaStream_t st);
// log weights (natural FP64 and log2 FP32) and validity flags.
cudaError_t launch_log_weights(const float* w, int n, double* lnw, float* l2w, DevState* st_dev,
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
  DevState* state;
};
cudaError_t launch_grad_epilogue(const GradParams& gp, cudaStream_t st);

// Sum of weights in FP64 into state->dual[slot_idx].
cudaError_t launch_mass(const float* w, int n, double* blk, DevState* st_dev, int idx, cudaStream_t st);

}  // namespace uot
