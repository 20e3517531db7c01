// Spatial ordering of point clouds for the tiled sweep.
//
// The fast points sweep evaluates |q - k|^2 as |q'|^2 + |k'|^2 - 2 q'.k' in a
// local frame centred on each 128-key tile (see sweep_tiles.cu).  That form
// keeps FP32 rounding at the level of the direct difference only when every
// tile is spatially compact, so both clouds are put in Morton (Z-curve) order
// once per call: bounding box -> 30-bit interleaved codes -> radix sort of
// (code, index) -> gather of points and weights.  Results are scattered back to
// the caller's order at the end of each entry point.
#include <cub/device/device_radix_sort.cuh>
#include <cuda_runtime.h>

#include "uot_internal.cuh"

namespace uot {
namespace {

constexpr int kBlk = 256;

__device__ __forceinline__ bool last_block_done(unsigned int* counter) {
  __shared__ bool am_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) am_last = (atomicAdd(counter, 1u) == gridDim.x - 1);
  __syncthreads();
  if (am_last) __threadfence();
  return am_last;
}

// Bounding box of pts [n x dim] (dim <= 3) -> box[0..2] = lo, box[3..5] = hi.
__global__ void __launch_bounds__(kBlk) k_bbox(const float* pts, int n, int dim, float* blk, float* box,
                                               unsigned int* counter) {
  __shared__ float sh[6][kBlk];
  float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    for (int d = 0; d < dim; ++d) {
      const float v = pts[(size_t)i * dim + d];
      lo[d] = fminf(lo[d], v);
      hi[d] = fmaxf(hi[d], v);
    }
  for (int d = 0; d < 3; ++d) { sh[d][threadIdx.x] = lo[d]; sh[3 + d][threadIdx.x] = hi[d]; }
  __syncthreads();
  for (int off = blockDim.x / 2; off > 0; off >>= 1) {
    if (threadIdx.x < off)
      for (int d = 0; d < 3; ++d) {
        sh[d][threadIdx.x] = fminf(sh[d][threadIdx.x], sh[d][threadIdx.x + off]);
        sh[3 + d][threadIdx.x] = fmaxf(sh[3 + d][threadIdx.x], sh[3 + d][threadIdx.x + off]);
      }
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int d = 0; d < 6; ++d) blk[6 * blockIdx.x + d] = sh[d][0];
  if (!last_block_done(counter)) return;
  if (threadIdx.x == 0) {
    float r[6] = {INFINITY, INFINITY, INFINITY, -INFINITY, -INFINITY, -INFINITY};
    for (int k = 0; k < (int)gridDim.x; ++k)
      for (int d = 0; d < 3; ++d) {
        r[d] = fminf(r[d], __ldcg(blk + 6 * k + d));
        r[3 + d] = fmaxf(r[3 + d], __ldcg(blk + 6 * k + 3 + d));
      }
    for (int d = 0; d < 6; ++d) box[d] = r[d];
    *counter = 0;
  }
}

__device__ __forceinline__ unsigned int spread3(unsigned int v) {  // 10 bits -> every third bit
  v &= 0x3ffu;
  v = (v | (v << 16)) & 0x030000ffu;
  v = (v | (v << 8)) & 0x0300f00fu;
  v = (v | (v << 4)) & 0x030c30c3u;
  v = (v | (v << 2)) & 0x09249249u;
  return v;
}

__device__ __forceinline__ unsigned int spread2(unsigned int v) {  // 15 bits -> every second bit
  v &= 0x7fffu;
  v = (v | (v << 8)) & 0x00ff00ffu;
  v = (v | (v << 4)) & 0x0f0f0f0fu;
  v = (v | (v << 2)) & 0x33333333u;
  v = (v | (v << 1)) & 0x55555555u;
  return v;
}

__global__ void k_morton(const float* pts, int n, int dim, const float* box, unsigned int* code, int* idx) {
  const int bits = dim == 1 ? 30 : (dim == 2 ? 15 : 10);
  const float cells = (float)((1u << bits) - 1u);
  float lo[3], sc[3];
  for (int d = 0; d < dim; ++d) {
    lo[d] = box[d];
    const float ext = box[3 + d] - box[d];
    sc[d] = ext > 0.f ? cells / ext : 0.f;
  }
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    unsigned int q[3] = {0u, 0u, 0u};
    for (int d = 0; d < dim; ++d) {
      float c = (pts[(size_t)i * dim + d] - lo[d]) * sc[d];
      c = fminf(fmaxf(c, 0.f), cells);
      q[d] = (unsigned int)c;
    }
    unsigned int key;
    if (dim == 1) key = q[0];
    else if (dim == 2) key = spread2(q[0]) | (spread2(q[1]) << 1);
    else key = spread3(q[0]) | (spread3(q[1]) << 1) | (spread3(q[2]) << 2);
    code[i] = key;
    idx[i] = i;
  }
}

__global__ void k_gather_pts(const float* pts, const float* w, const int* perm, int n, int dim, float* pts_s,
                             float* w_s) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int src = perm[i];
    for (int d = 0; d < dim; ++d) pts_s[(size_t)i * dim + d] = pts[(size_t)src * dim + d];
    w_s[i] = w[src];
  }
}

__global__ void k_gather_vec(const float* v, const int* perm, int n, float* out) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) out[i] = v[perm[i]];
}

__global__ void k_scatter_rows(const float* v, const int* perm, int n, int dim, float* out) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    for (int d = 0; d < dim; ++d) out[(size_t)perm[i] * dim + d] = v[(size_t)i * dim + d];
}

// Centre of the bounding box of every tile of kTileKeys consecutive points.
__global__ void k_tile_centers(const float* pts, int n, int dim, float4* centers) {
  const int ntiles = (n + kTileKeys - 1) / kTileKeys;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  for (int t = warp; t < ntiles; t += nwarps) {
    float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    const int j0 = t * kTileKeys, j1 = min(n, j0 + kTileKeys);
    for (int j = j0 + lane; j < j1; j += 32)
      for (int d = 0; d < dim; ++d) {
        const float v = pts[(size_t)j * dim + d];
        lo[d] = fminf(lo[d], v);
        hi[d] = fmaxf(hi[d], v);
      }
    for (int off = 16; off > 0; off >>= 1)
      for (int d = 0; d < 3; ++d) {
        lo[d] = fminf(lo[d], __shfl_xor_sync(0xffffffffu, lo[d], off));
        hi[d] = fmaxf(hi[d], __shfl_xor_sync(0xffffffffu, hi[d], off));
      }
    if (lane == 0) {
      float c[3] = {0.f, 0.f, 0.f};
      for (int d = 0; d < dim; ++d) c[d] = 0.5f * (lo[d] + hi[d]);
      centers[t] = make_float4(c[0], c[1], c[2], 0.f);
    }
  }
}

int grid_for(int n) {
  int g = (n + kBlk - 1) / kBlk;
  return g < 1 ? 1 : (g > 1024 ? 1024 : g);
}

}  // namespace

size_t sort_temp_bytes(int n) {
  size_t bytes = 0;
  cub::DeviceRadixSort::SortPairs<unsigned int, int>(nullptr, bytes, (const unsigned int*)nullptr,
                                                     (unsigned int*)nullptr, (const int*)nullptr, (int*)nullptr,
                                                     n, 0, 30);
  return bytes;
}

cudaError_t launch_order_points(const float* pts, const float* w, int n, int dim, OrderScratch sc, int* perm,
                                float* pts_s, float* w_s, float4* centers, cudaStream_t st) {
  k_bbox<<<grid_for(n), kBlk, 0, st>>>(pts, n, dim, sc.blk_f, sc.box, sc.counter);
  note_launch();
  k_morton<<<grid_for(n), kBlk, 0, st>>>(pts, n, dim, sc.box, sc.code_in, sc.idx_in);
  note_launch();
  cudaError_t e = cub::DeviceRadixSort::SortPairs<unsigned int, int>(sc.temp, sc.temp_bytes, sc.code_in, sc.code_out,
                                                                     sc.idx_in, perm, n, 0, 30, st);
  if (e != cudaSuccess) return e;
  k_gather_pts<<<grid_for(n), kBlk, 0, st>>>(pts, w, perm, n, dim, pts_s, w_s);
  note_launch();
  const int ntiles = (n + kTileKeys - 1) / kTileKeys;
  k_tile_centers<<<(ntiles + 7) / 8, kBlk, 0, st>>>(pts_s, n, dim, centers);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_gather_vec(const float* v, const int* perm, int n, float* out, cudaStream_t st) {
  k_gather_vec<<<grid_for(n), kBlk, 0, st>>>(v, perm, n, out);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_scatter_rows(const float* v, const int* perm, int n, int dim, float* out, cudaStream_t st) {
  k_scatter_rows<<<grid_for(n), kBlk, 0, st>>>(v, perm, n, dim, out);
  note_launch();
  return cudaGetLastError();
}

}  // namespace uot
