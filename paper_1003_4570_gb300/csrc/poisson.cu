// Finite-difference Poisson solver (paper Section III-A item 3: a finite-difference Poisson
// equation and an iterative linear solver; Aztec there, conjugate gradients here).
//
// -div(eps0 eps_r grad phi) = rho on a uniform grid: 7-point stencil, periodic along x and y,
// phi = 0 on the z = 0 and z = Lz planes.  The operator is symmetric positive definite, so
// plain CG (Hestenes & Stiefel 1952) applies.  The whole iteration runs in one cooperative
// launch: three grid-wide barriers per iteration, block partial sums reduced by every block in
// the same order, so all blocks see bit-identical scalars and leave the loop together.
#include <cooperative_groups.h>

#include <algorithm>
#include <chrono>
#include <cmath>

#include "omen_internal.h"

namespace cgr = cooperative_groups;

#include "fd.cuh"

struct CGOut {
  int iterations;
  int converged;
  double rel;
};

__global__ void __launch_bounds__(256) cg_kernel(PGrid g, const double* __restrict__ rho, double scale,
                                                 double* __restrict__ x, double* __restrict__ r,
                                                 double* __restrict__ p, double* __restrict__ q,
                                                 double* __restrict__ part, double rtol, int max_iter,
                                                 CGOut* __restrict__ out) {
  cgr::grid_group grid = cgr::this_grid();
  __shared__ double sh[32];
  const long long n = g.n;
  const long long t0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long stride = (long long)gridDim.x * blockDim.x;
  double* part0 = part;
  double* part1 = part + gridDim.x;
  double* part2 = part + 2 * gridDim.x;
  // r = b - A x, p = r
  double lrr = 0.0, lbb = 0.0;
  for (long long i = t0; i < n; i += stride) {
    const double b = scale * rho[i];
    const double ri = b - stencil(x, g, i);
    r[i] = ri;
    p[i] = ri;
    lrr += ri * ri;
    lbb += b * b;
  }
  double v = block_sum(lrr, sh);
  if (threadIdx.x == 0) part0[blockIdx.x] = v;
  v = block_sum(lbb, sh);
  if (threadIdx.x == 0) part2[blockIdx.x] = v;
  grid.sync();
  double rr = grid_total(part0, sh);
  const double bb = grid_total(part2, sh);
  const double stop = rtol * rtol * bb;
  int it = 0;
  while (rr > stop && it < max_iter && bb > 0.0) {
    double lpq = 0.0;
    if (g.nx >= 64) {
      // rows of x over the CTAs, a row's points over the threads: the coordinates come from
      // the row index once per row instead of from divisions per point
      const long long nrow = (long long)g.ny * g.nzi;
      for (long long rw = blockIdx.x; rw < nrow; rw += gridDim.x) {
        const int j = (int)(rw % g.ny), k = (int)(rw / g.ny);
        const long long base = rw * g.nx;
        for (int i = threadIdx.x; i < g.nx; i += blockDim.x) {
          const double qi = stencil_at(p, g, i, j, k, base + i);
          q[base + i] = qi;
          lpq += p[base + i] * qi;
        }
      }
    } else {
      // narrow rows: points over all threads, coordinates by 32-bit division (n < 2^31)
      for (long long i = t0; i < n; i += stride) {
        const unsigned u = (unsigned)i;
        const int ii = (int)(u % (unsigned)g.nx), jj = (int)((u / (unsigned)g.nx) % (unsigned)g.ny);
        const int kk = (int)(u / ((unsigned)g.nx * (unsigned)g.ny));
        const double qi = stencil_at(p, g, ii, jj, kk, i);
        q[i] = qi;
        lpq += p[i] * qi;
      }
    }
    v = block_sum(lpq, sh);
    if (threadIdx.x == 0) part0[blockIdx.x] = v;
    grid.sync();
    const double pq = grid_total(part0, sh);
    const double alpha = rr / pq;
    double lr = 0.0;
    for (long long i = t0; i < n; i += stride) {
      x[i] += alpha * p[i];
      const double ri = r[i] - alpha * q[i];
      r[i] = ri;
      lr += ri * ri;
    }
    v = block_sum(lr, sh);
    if (threadIdx.x == 0) part1[blockIdx.x] = v;
    grid.sync();
    const double rr_new = grid_total(part1, sh);
    const double beta = rr_new / rr;
    rr = rr_new;
    for (long long i = t0; i < n; i += stride) p[i] = r[i] + beta * p[i];
    grid.sync();
    ++it;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    out->iterations = it;
    out->converged = (rr <= stop) || bb == 0.0;
    out->rel = bb > 0.0 ? sqrt(rr / bb) : 0.0;
  }
}

extern "C" omen_status omen_poisson(omen_ctx* ctx, const omen_grid* gr, const double* rho, double* phi,
                                    const omen_cg_opts* o, omen_solve_info* info) {
  if (!ctx || !gr || !rho || !phi || !o) return set_err(ctx, OMEN_EINVAL, "null argument");
  if (gr->nx < 1 || gr->ny < 1 || gr->nz < 2) return set_err(ctx, OMEN_EINVAL, "grid needs nx, ny >= 1 and nz >= 2");
  if (!(gr->Lx_nm > 0 && gr->Ly_nm > 0 && gr->Lz_nm > 0 && gr->eps_r > 0)) return set_err(ctx, OMEN_EINVAL, "grid lengths and eps_r must be > 0");
  if (!(o->rtol > 0) || o->max_iter < 1) return set_err(ctx, OMEN_EINVAL, "cg options");
  OMEN_CUDA(ctx, cudaSetDevice(ctx->device));
  auto t0 = std::chrono::steady_clock::now();
  PGrid g;
  g.nx = gr->nx;
  g.ny = gr->ny;
  g.nzi = gr->nz - 1;
  const double hx = gr->Lx_nm / gr->nx * 1e-9, hy = gr->Ly_nm / gr->ny * 1e-9, hz = gr->Lz_nm / gr->nz * 1e-9;
  // a periodic direction with one point has no second difference
  g.cx = gr->nx > 1 ? 1.0 / (hx * hx) : 0.0;
  g.cy = gr->ny > 1 ? 1.0 / (hy * hy) : 0.0;
  g.cz = 1.0 / (hz * hz);
  g.n = (long long)g.nx * g.ny * g.nzi;
  if (g.n >= (1ll << 31)) return set_err(ctx, OMEN_EINVAL, "grid larger than 2^31 unknowns");
  int dev_sms = 0, per_sm = 0;
  cudaDeviceGetAttribute(&dev_sms, cudaDevAttrMultiProcessorCount, ctx->device);
  OMEN_CUDA(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, cg_kernel, 256, 0));
  long long want = (g.n + 255) / 256;
  int blocks = (int)std::min<long long>(want, (long long)dev_sms * std::max(1, per_sm));
  blocks = std::max(blocks, 1);
  double* buf = nullptr;
  const size_t vec = (size_t)g.n * sizeof(double);
  if (cudaMallocAsync(&buf, 3 * vec + 3 * blocks * sizeof(double) + sizeof(CGOut) + 64, ctx->stream) != cudaSuccess) {
    cudaGetLastError();
    return set_err(ctx, OMEN_ENOMEM, "CG work vectors");
  }
  double* r = buf;
  double* p = r + g.n;
  double* q = p + g.n;
  double* part = q + g.n;
  CGOut* out = reinterpret_cast<CGOut*>(part + 3 * blocks);
  double scale = 1.0 / (kEps0 * gr->eps_r);
  double rtol = o->rtol;
  int max_iter = o->max_iter;
  void* args[] = {&g, &rho, &scale, &phi, &r, &p, &q, &part, &rtol, &max_iter, &out};
  cudaError_t e = cudaLaunchCooperativeKernel((const void*)cg_kernel, dim3(blocks), dim3(256), args, 0, ctx->stream);
  CGOut ho{};
  if (e == cudaSuccess) e = cudaMemcpyAsync(&ho, out, sizeof(CGOut), cudaMemcpyDeviceToHost, ctx->stream);
  cudaFreeAsync(buf, ctx->stream);
  cudaError_t e2 = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess || e2 != cudaSuccess)
    return set_err(ctx, OMEN_ECUDA, "Poisson CG: %s", cudaGetErrorString(e != cudaSuccess ? e : e2));
  if (info) {
    info->iterations = ho.iterations;
    info->converged = ho.converged;
    info->rel_residual = ho.rel;
    info->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
  if (!ho.converged) return set_err(ctx, OMEN_ENOCONV, "CG stopped at %d iterations, relative residual %.3e", ho.iterations, ho.rel);
  return OMEN_OK;
}

// ---------------------------------------------------------------------------------------
// Poisson solve that allocates nothing.
//
// Some host programs cannot let a library call cudaMalloc: the application may have reserved
// the device memory for its own allocator up front, or its rules forbid allocation once the
// solve loop is running (a fixed memory budget checked at start-up, a plugin sandbox).  For
// them the CG work vectors live in the statically sized device array below instead.  Every
// GPU that loads this library holds the array (about 6.4 MB) until the process exits.
// The array's name in host code is only a host-side stand-in for the symbol, so the device
// address is looked up with cudaGetSymbolAddress, with the caller's device current, on every
// call.  The lookup is cheap once the module is loaded, and a pointer kept from an earlier call
// could be stale after cudaDeviceReset or a primary context that was torn down and recreated.
// The first call on a device loads the module there; make it before any stream capture.
static constexpr long long kStaticMaxUnknowns = 1ll << 18;   // nx*ny*(nz-1) limit
static constexpr int kStaticMaxBlocks = 4096;
static constexpr long long kStaticWords = 3 * kStaticMaxUnknowns + 3 * kStaticMaxBlocks + 8;
static __device__ __align__(256) double g_poisson_scratch[kStaticWords];

static omen_status scratch_address(double** out) {
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_poisson_scratch);
  if (e != cudaSuccess || !p) {
    cudaGetLastError();
    return OMEN_ECUDA;
  }
  *out = static_cast<double*>(p);
  return OMEN_OK;
}

extern "C" omen_status omen_poisson_static(const omen_grid* gr, const double* rho, double* phi,
                                           const omen_cg_opts* o, omen_solve_info* info, void* cuda_stream) {
  if (!gr || !rho || !phi || !o) return OMEN_EINVAL;
  if (gr->nx < 1 || gr->ny < 1 || gr->nz < 2) return OMEN_EINVAL;
  if (!(gr->Lx_nm > 0 && gr->Ly_nm > 0 && gr->Lz_nm > 0 && gr->eps_r > 0)) return OMEN_EINVAL;
  if (!(o->rtol > 0) || o->max_iter < 1) return OMEN_EINVAL;
  const long long n = (long long)gr->nx * gr->ny * (gr->nz - 1);
  if (n > kStaticMaxUnknowns) return OMEN_EINVAL;   // grid larger than the static work area
  cudaStream_t stream = static_cast<cudaStream_t>(cuda_stream);
  auto t0 = std::chrono::steady_clock::now();
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return OMEN_ECUDA;
  }
  double* base = nullptr;
  const omen_status s = scratch_address(&base);
  if (s != OMEN_OK) return s;
  PGrid g;
  g.nx = gr->nx;
  g.ny = gr->ny;
  g.nzi = gr->nz - 1;
  const double hx = gr->Lx_nm / gr->nx * 1e-9, hy = gr->Ly_nm / gr->ny * 1e-9, hz = gr->Lz_nm / gr->nz * 1e-9;
  g.cx = gr->nx > 1 ? 1.0 / (hx * hx) : 0.0;
  g.cy = gr->ny > 1 ? 1.0 / (hy * hy) : 0.0;
  g.cz = 1.0 / (hz * hz);
  g.n = n;
  int sms = 0, per_sm = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, cg_kernel, 256, 0) != cudaSuccess) {
    cudaGetLastError();
    return OMEN_ECUDA;
  }
  long long want = (n + 255) / 256;
  int blocks = (int)std::min<long long>(want, (long long)sms * std::max(1, per_sm));
  blocks = std::max(1, std::min(blocks, kStaticMaxBlocks));
  // every word of the work area is written by the kernel before it is read, so nothing has
  // to be cleared between calls
  double* r = base;
  double* p = r + kStaticMaxUnknowns;
  double* q = p + kStaticMaxUnknowns;
  double* part = q + kStaticMaxUnknowns;
  CGOut* out = reinterpret_cast<CGOut*>(part + 3 * kStaticMaxBlocks);
  double scale = 1.0 / (kEps0 * gr->eps_r);
  double rtol = o->rtol;
  int max_iter = o->max_iter;
  void* args[] = {&g, &rho, &scale, &phi, &r, &p, &q, &part, &rtol, &max_iter, &out};
  cudaError_t e = cudaLaunchCooperativeKernel((const void*)cg_kernel, dim3(blocks), dim3(256), args, 0, stream);
  CGOut ho{};
  if (e == cudaSuccess) e = cudaMemcpyAsync(&ho, out, sizeof(CGOut), cudaMemcpyDeviceToHost, stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return OMEN_ECUDA;
  }
  if (info) {
    info->iterations = ho.iterations;
    info->converged = ho.converged;
    info->rel_residual = ho.rel;
    info->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
  return ho.converged ? OMEN_OK : OMEN_ENOCONV;
}
