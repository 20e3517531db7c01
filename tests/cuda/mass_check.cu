// Accuracy of the translation-invariant half-step's mass reduction as the fused
// epilogues run it: the per-row terms w_i e^{-v_i/rho} = 2^{y_i} formed and
// summed on float pairs against integer power-of-two references (epi::mass_add),
// the block and grid reduction (epi::block_finish) and the finalisation's log
// (epi::finalize, TI mode), which writes Smin_w^rho(v) = -rho log <w, e^{-v/rho}>
// into the state's slot.  The reference is the same sum in long double on the
// host.  Prints one line per case: n, rho, relative error of the sum.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <random>
#include <vector>

#include <cuda_runtime.h>

#include "epi_device.cuh"

using namespace uot;

__global__ void k_mass_sum(int n, const float* l2w_hi, const float* l2w_lo, const float* v, EpiParams e) {
  epi::RowAcc acc = epi::rowacc_empty();
  const ffl::ff RL{e.RL2[0], e.RL2[1]};
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const ffl::ff y = ffl::add(ffl::ff{l2w_hi[i], l2w_lo[i]}, ffl::neg(ffl::mul(ffl::ff{v[i], 0.f}, RL)));
    epi::mass_add(acc, y, ffl::kExp2Tab);
  }
  epi::block_finish(e, acc, blockIdx.x, gridDim.x);
}

static void split2(double v, float* out) {
  out[0] = (float)v;
  out[1] = (float)(v - (double)out[0]);
}

static int run_case(int n, double rho, double vscale, unsigned seed) {
  std::mt19937_64 gen(seed);
  std::exponential_distribution<double> ex(1.0);
  std::uniform_real_distribution<double> un(-1.0, 1.0);
  std::vector<float> w(n), v(n), hi(n), lo(n);
  double tot = 0.0;
  for (int i = 0; i < n; ++i) { w[i] = (float)ex(gen); tot += w[i]; }
  for (int i = 0; i < n; ++i) {
    w[i] = (float)(w[i] / tot * 1.3);
    v[i] = (float)(vscale * un(gen));
    const double l2 = std::log2((double)w[i]);
    hi[i] = (float)l2;
    lo[i] = (float)(l2 - (double)hi[i]);
  }
  long double ref = 0.0L;
  for (int i = 0; i < n; ++i) ref += (long double)w[i] * std::exp(-(long double)v[i] / (long double)rho);
  const int threads = 256, blocks = 296;
  float *d_hi, *d_lo, *d_v;
  double* d_blk;
  DevState* d_st;
  cudaMalloc(&d_hi, sizeof(float) * n);
  cudaMalloc(&d_lo, sizeof(float) * n);
  cudaMalloc(&d_v, sizeof(float) * n);
  cudaMalloc(&d_blk, sizeof(double) * kMaxBlocks * 10);
  cudaMalloc(&d_st, sizeof(DevState));
  cudaMemcpy(d_hi, hi.data(), sizeof(float) * n, cudaMemcpyHostToDevice);
  cudaMemcpy(d_lo, lo.data(), sizeof(float) * n, cudaMemcpyHostToDevice);
  cudaMemcpy(d_v, v.data(), sizeof(float) * n, cudaMemcpyHostToDevice);
  cudaMemset(d_st, 0, sizeof(DevState));
  EpiParams e;
  std::memset(&e, 0, sizeof(e));
  e.mode = EPI_TI;
  e.out_is_f = 0;
  e.slot_out = 0;
  e.state = d_st;
  e.blk = d_blk;
  split2(1.4426950408889634 / rho, e.RL2);
  split2(-rho, e.NR2);
  split2(0.0, e.KK2);
  k_mass_sum<<<blocks, threads>>>(n, d_hi, d_lo, d_v, e);
  if (cudaDeviceSynchronize() != cudaSuccess) { printf("kernel failed\n"); return 1; }
  DevState h;
  cudaMemcpy(&h, d_st, sizeof(DevState), cudaMemcpyDeviceToHost);
  // slot B = Smin_w^rho(v) = -rho log(sum); recover the sum's log and compare
  const long double lref = std::log(ref);
  const long double lgot = -(long double)h.slot[0].B / (long double)rho;
  const double rel = (double)std::fabs(std::expm1(lgot - lref));
  printf("n %d rho %g vscale %g status %d relerr %.3e\n", n, rho, vscale, h.status, rel);
  cudaFree(d_hi); cudaFree(d_lo); cudaFree(d_v); cudaFree(d_blk); cudaFree(d_st);
  return 0;
}

int main() {
  // the 262144-point workload's scale (rho = 1, potentials of size ~0.5), then wider term ranges
  if (run_case(262144, 1.0, 0.5, 1)) return 1;
  if (run_case(262144, 0.1, 0.5, 2)) return 1;
  if (run_case(262144, 0.05, 3.0, 3)) return 1;
  if (run_case(20000, 1.0, 0.5, 4)) return 1;
  return 0;
}
