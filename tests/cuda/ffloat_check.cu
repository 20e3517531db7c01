// Accuracy check of the float-pair helpers used by the half-step epilogues:
// the table-driven exp2 against CUDA's double exp2, the product / sum against
// FP64, and the pair log against CUDA's double log (absolute error, the
// finalisation's use).  Prints one line: max errors.
#include <cstdio>
#include <cstdlib>
#include <vector>
#include <cuda_runtime.h>

#include "ffloat.cuh"

using namespace uot;

__global__ void k_check(int n, unsigned seed, double* err) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  // deterministic pseudo-random inputs (xorshift on the index)
  unsigned s = seed ^ (2654435761u * (unsigned)(t + 1));
  auto nxt = [&s]() { s ^= s << 13; s ^= s >> 17; s ^= s << 5; return (double)s / 4294967296.0; };
  // the epilogues sum terms 2^y relative to their largest (y <= 0); terms below
  // 2^-60 of it do not matter, and near 2^-126 the low float of a pair underflows
  const double y = -60.0 + 124.0 * nxt();
  const ffl::ff yf = ffl::from_double(y);
  const ffl::ff e = ffl::exp2(yf);
  const double ref = exp2(ffl::to_double(yf));
  err[4 * t + 0] = fabs(ffl::to_double(e) - ref) / ref;
  const double a = (nxt() - 0.5) * 1e3, b = (nxt() - 0.5) * 1e-2;
  const ffl::ff fa = ffl::from_double(a), fb = ffl::from_double(b);
  const ffl::ff p = ffl::mul(fa, fb);
  const double pr = ffl::to_double(fa) * ffl::to_double(fb);
  err[4 * t + 1] = fabs(ffl::to_double(p) - pr) / fabs(pr);
  const ffl::ff q = ffl::add(fa, ffl::neg(ffl::from_double(a * (1.0 + 1e-6))));
  const double qr = ffl::to_double(fa) - ffl::to_double(ffl::from_double(a * (1.0 + 1e-6)));
  err[4 * t + 2] = fabs(ffl::to_double(q) - qr) / fabs(qr);
  // log of a mass sum hi + lo in [2^-30, 2^30] (the finalisation's range after rescaling)
  const double u = exp2(-30.0 + 60.0 * nxt());
  const ffl::ff fu = ffl::from_double(u);
  err[4 * t + 3] = fabs(ffl::to_double(ffl::log_ff(fu)) - log(ffl::to_double(fu)));
}

int main() {
  const int n = 1 << 20;
  double* d = nullptr;
  if (cudaMalloc(&d, sizeof(double) * 4 * n) != cudaSuccess) { printf("alloc failed\n"); return 1; }
  k_check<<<(n + 255) / 256, 256>>>(n, 12345u, d);
  if (cudaDeviceSynchronize() != cudaSuccess) { printf("kernel failed\n"); return 1; }
  std::vector<double> h(4 * (size_t)n);
  cudaMemcpy(h.data(), d, sizeof(double) * 4 * n, cudaMemcpyDeviceToHost);
  double m[4] = {0, 0, 0, 0};
  for (int t = 0; t < n; ++t)
    for (int k = 0; k < 4; ++k) m[k] = h[4 * t + k] > m[k] ? h[4 * t + k] : m[k];
  printf("exp2 %.3e mul %.3e add %.3e log %.3e\n", m[0], m[1], m[2], m[3]);
  cudaFree(d);
  return 0;
}
