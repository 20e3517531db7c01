// Common centre of the two point clouds for the dim >= 32 tensor-core sweeps:
// coordinates are taken relative to it so that |x - c| and |y - c| stay small
// next to the |x - y| the cost needs.
#include <cuda_runtime.h>

#include "uot_internal.cuh"

namespace uot {
namespace {

// centre = mean of the two clouds, one block per coordinate: keeps |x - c|, |y - c| small in the expansion
__global__ void k_center(const float* x, int n, const float* y, int m, int dim, float* center) {
  __shared__ double sh[256];
  const int d = blockIdx.x;
  double acc = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) acc += x[(size_t)i * dim + d];
  for (int j = threadIdx.x; j < m; j += blockDim.x) acc += y[(size_t)j * dim + d];
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int off = blockDim.x / 2; off > 0; off >>= 1) {
    if (threadIdx.x < off) sh[threadIdx.x] += sh[threadIdx.x + off];
    __syncthreads();
  }
  if (threadIdx.x == 0) center[d] = (float)(sh[0] / (double)(n + m));
}

}  // namespace

cudaError_t launch_center(const float* x, int n, const float* y, int m, int dim, float* center, cudaStream_t st) {
  k_center<<<dim, 256, 0, st>>>(x, n, y, m, dim, center);
  note_launch();
  return cudaGetLastError();
}

}  // namespace uot
