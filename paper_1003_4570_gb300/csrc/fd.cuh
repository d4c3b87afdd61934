// The 7-point finite-difference operator of the Poisson equation and the deterministic grid
// reductions of the cooperative CG kernels (paper Section III-A item 3: finite-difference
// Poisson solver).  -div(grad) on the interior unknowns, periodic x and y, phi = 0 on the z = 0
// and z = Lz planes; unknown index ((k-1)*ny + j)*nx + i.
#pragma once

#include <cuda_runtime.h>

constexpr double kEps0 = 8.8541878128e-12;  // F/m

struct PGrid {
  int nx, ny, nzi;           // nzi = nz - 1 interior planes
  double cx, cy, cz;         // 1/h^2 (1/m^2)
  long long n;
};

__device__ __forceinline__ double stencil(const double* __restrict__ v, const PGrid& g, long long idx) {
  const int i = (int)(idx % g.nx);
  const int j = (int)((idx / g.nx) % g.ny);
  const int k = (int)(idx / ((long long)g.nx * g.ny));
  const long long plane = (long long)g.nx * g.ny;
  const double c = v[idx];
  const int ip = (i + 1 == g.nx) ? 0 : i + 1, im = (i == 0) ? g.nx - 1 : i - 1;
  const int jp = (j + 1 == g.ny) ? 0 : j + 1, jm = (j == 0) ? g.ny - 1 : j - 1;
  const long long row = idx - i - (long long)j * g.nx;
  double s = g.cx * (2.0 * c - v[row + (long long)j * g.nx + ip] - v[row + (long long)j * g.nx + im]);
  s += g.cy * (2.0 * c - v[row + (long long)jp * g.nx + i] - v[row + (long long)jm * g.nx + i]);
  const double up = (k + 1 < g.nzi) ? v[idx + plane] : 0.0;
  const double dn = (k > 0) ? v[idx - plane] : 0.0;
  s += g.cz * (2.0 * c - up - dn);
  return s;
}

// The same stencil with the cell coordinates given (no divisions per element).
__device__ __forceinline__ double stencil_at(const double* __restrict__ v, const PGrid& g, int i, int j, int k,
                                            long long idx) {
  const long long plane = (long long)g.nx * g.ny;
  const double c = v[idx];
  const int ip = (i + 1 == g.nx) ? 0 : i + 1, im = (i == 0) ? g.nx - 1 : i - 1;
  const int jp = (j + 1 == g.ny) ? 0 : j + 1, jm = (j == 0) ? g.ny - 1 : j - 1;
  const long long row = idx - i;
  double s = g.cx * (2.0 * c - v[row + ip] - v[row + im]);
  s += g.cy * (2.0 * c - v[row + (long long)(jp - j) * g.nx + i] - v[row + (long long)(jm - j) * g.nx + i]);
  const double up = (k + 1 < g.nzi) ? v[idx + plane] : 0.0;
  const double dn = (k > 0) ? v[idx - plane] : 0.0;
  s += g.cz * (2.0 * c - up - dn);
  return s;
}

__device__ __forceinline__ double block_sum(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[w] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += sh[i];
  return t;  // valid in thread 0
}

// The sum of a float per thread over the block: warp sums in FP32, then FP64 across warps
// (valid in thread 0).  For the FP32 passes, whose per-thread sums are FP32 already; it keeps
// the reduction off GB300's narrow FP64 pipe.
__device__ __forceinline__ double block_sum_f(float v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[w] = (double)v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += sh[i];
  return t;  // valid in thread 0
}

// Every block sums the partials of all blocks in the same fixed order (the same result
// everywhere): warp 0 adds them and broadcasts the total through shared memory, so the FP64
// additions are one warp's, not the whole block's.
__device__ __forceinline__ double grid_total(const double* __restrict__ part, double* sh) {
  __syncthreads();
  if (threadIdx.x < 32) {
    double t = 0.0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += 32) t += part[b];
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (threadIdx.x == 0) sh[0] = t;
  }
  __syncthreads();
  const double s = sh[0];
  __syncthreads();
  return s;
}

