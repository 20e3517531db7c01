// Internal types of the batched ragged solver (batched.cu).
#pragma once

#include <cuda_runtime.h>

#include "uot_internal.cuh"

namespace uot {

// Constant description of problem k of a batch.
struct BProb {
  int n, m, dim;
  int units_f, units_g;       // work units (row blocks) of the f and g half-steps
  int ubase_f, ubase_g;       // first partial slot of this problem's units
  int pad;
  long long x_off, y_off;     // float offsets of the first coordinate in x / y
  long long a_off, b_off;     // offsets of the first weight in a / b (and f / g)
  double eps, rho1, rho2, s;  // s = log2(e) / eps
};

// Mutable per-problem state.
struct BState {
  Slot slot[2];          // TI scalars by iteration parity
  unsigned int cnt;      // unit arrivals in the current half-step
  int status;            // 0 running, 1 converged, 2 non-finite / invalid, 3 stopped at max_iter
  int conv_iter;         // index of the returned iterate
  float resid;           // residual of the latest tested iterate
};

// Parameters of one half-step launch over the whole batch.
struct BHalf {
  const BProb* probs;
  BState* st;
  const int2* units;     // slot -> (problem, first row)
  const int* queue;      // launch order of the slots (longest first)
  int nunits;
  int side;              // 0: f half-step (queries x, keys y); 1: g half-step
  int ti;
  int max_iter, check_every;
  double tol;
  unsigned int* next;    // queue head
  unsigned int* finished;
  unsigned int* active;  // problems still running
  int* iter;             // t: the half-step belongs to iteration t + 1
  const float *x, *y;
  const float *l2a, *l2b;
  const double *lna, *lnb;
  float* f;              // f_hat (caller's f)
  float* g0;             // g_hat of even iterations (caller's g)
  float* g1;             // g_hat of odd iterations (workspace)
  double* upart;         // [slots][4] unit partials
};

int batch_rows_per_unit();
int batch_grid();
cudaError_t launch_batch_half(const BHalf& h, int grid, cudaStream_t st);
cudaError_t launch_batch_init(const BProb* probs, BState* st, const float* a, int count, int ti,
                              unsigned int* active, cudaStream_t s);
cudaError_t launch_batch_phi(const BProb* probs, const BState* st, float* f, float* g0, const float* g1, int count,
                             int ti, cudaStream_t s);

}  // namespace uot
