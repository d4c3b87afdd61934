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
  if (bb == 0.0)   // b = 0: the solution is x = 0 whatever the initial guess
    for (long long i = t0; i < n; i += stride) x[i] = 0.0;
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

// ---------------------------------------------------------------------------------------
// Mixed-precision CG: the iterations in FP32, the residual replaced by the true FP64
// residual b - A x whenever the FP32 recurrence residual has fallen by a factor kDelta since
// the last replacement ("reliable updates", van der Vorst & Ye, SIAM J. Sci. Comput. 22, 1716
// (2000)).  The search direction is kept across a replacement, so the Krylov recurrence goes
// on and the iteration count stays near the FP64 one, while each iteration moves FP32 words
// on the FP32 pipe.  The FP32 system is scaled to unit size: A^ = A / c_max and
// r^ = r * s with s = 1 / rms(r), so the FP32 sums of squares stay far from overflow for any
// grid spacing; the correction d^ it accumulates maps back as d = d^ / (c_max s).  The
// solution x and the stopping test ||b - A x|| <= rtol ||b|| stay in FP64.  The FP32
// recurrence loses the superlinear end of FP64 CG: to 1e-8 on a 256^3 grid it takes 1.15x the
// FP64 iterations, on the 11 x 11 x 217 grid of a delta layer about 1.4x, and to 1e-13 there
// 1.9x.
struct PGrid32 {
  int nx, ny, nzi;
  float cx, cy, cz;          // 1/h^2 divided by the largest of the three
};

__device__ __forceinline__ float stencil32_at(const float* __restrict__ v, const PGrid32& g, int i, int j, int k,
                                              long long idx) {
  const long long plane = (long long)g.nx * g.ny;
  const float c = v[idx];
  const int ip = (i + 1 == g.nx) ? 0 : i + 1, im = (i == 0) ? g.nx - 1 : i - 1;
  const long long row = idx - i;
  const long long rn = (j + 1 == g.ny) ? row - (long long)(g.ny - 1) * g.nx : row + g.nx;
  const long long rs = (j == 0) ? row + (long long)(g.ny - 1) * g.nx : row - g.nx;
  float s = g.cx * (2.f * c - v[row + ip] - v[row + im]);
  s += g.cy * (2.f * c - v[rn + i] - v[rs + i]);
  const float up = (k + 1 < g.nzi) ? v[idx + plane] : 0.f;
  const float dn = (k > 0) ? v[idx - plane] : 0.f;
  s += g.cz * (2.f * c - up - dn);
  return s;
}

// The 7-point stencil of r + beta p_old (the same values as stencil32_at of the stored p)
__device__ __forceinline__ float stencil32_dir_at(const float* __restrict__ r, const float* __restrict__ po, float beta,
                                                  const PGrid32& g, int i, int j, int k, long long idx) {
  const long long plane = (long long)g.nx * g.ny;
  auto val = [&](long long q) { return r[q] + beta * po[q]; };
  const float c = val(idx);
  const int ip = (i + 1 == g.nx) ? 0 : i + 1, im = (i == 0) ? g.nx - 1 : i - 1;
  const long long row = idx - i;
  const long long rn = (j + 1 == g.ny) ? row - (long long)(g.ny - 1) * g.nx : row + g.nx;
  const long long rs = (j == 0) ? row + (long long)(g.ny - 1) * g.nx : row - g.nx;
  float s = g.cx * (2.f * c - val(row + ip) - val(row + im));
  s += g.cy * (2.f * c - val(rn + i) - val(rs + i));
  const float up = (k + 1 < g.nzi) ? val(idx + plane) : 0.f;
  const float dn = (k > 0) ? val(idx - plane) : 0.f;
  s += g.cz * (2.f * c - up - dn);
  return s;
}

// Visit every interior unknown with its coordinates: rows of x over the CTAs and a row's
// points over the threads when rows are wide, otherwise points over all threads with the
// coordinates by 32-bit division (n < 2^31).
template <class F>
__device__ __forceinline__ void for_each_point(const PGrid& g, F&& f) {
  if (g.nx >= 64) {
    const long long nrow = (long long)g.ny * g.nzi;
    for (long long rw = blockIdx.x; rw < nrow; rw += gridDim.x) {
      const int j = (int)(rw % g.ny), k = (int)(rw / g.ny);
      const long long base = rw * g.nx;
      for (int i = threadIdx.x; i < g.nx; i += blockDim.x) f(i, j, k, base + i);
    }
  } else {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < g.n; idx += stride) {
      const unsigned u = (unsigned)idx;
      const int i = (int)(u % (unsigned)g.nx), j = (int)((u / (unsigned)g.nx) % (unsigned)g.ny);
      const int k = (int)(u / ((unsigned)g.nx * (unsigned)g.ny));
      f(i, j, k, idx);
    }
  }
}

static constexpr double kReliableDelta = 0.1;   // replace the residual after a 10x drop

// The FP32 passes on grids with rows of 32 points or more: a warp takes a row (its
// coordinates once), 32 consecutive points per chunk, and issues the loads of kChunks chunks
// before their arithmetic, so each thread keeps several independent loads in flight.
static constexpr int kChunks = 2;
static constexpr int kDirChunks = 1;   // the direction pass loads r and p_old: as many loads

struct Nb7 {
  float c, xp, xm, yp, ym, zp, zm;
};

// Row base pointers of one row of the grid (32-bit offsets within a row: n < 2^31).
template <typename P>
struct RowPtr {
  P c, n, s, u, d;   // this row; the rows at j+1 and j-1 (periodic); at k+1 and k-1 (or null)
};

template <typename P>
__device__ __forceinline__ RowPtr<P> row_ptr(P v, const PGrid32& g, int rw) {
  RowPtr<P> r;
  const int j = rw % g.ny, k = rw / g.ny;
  const int plane = g.nx * g.ny;
  r.c = v + (long long)rw * g.nx;
  r.n = (j + 1 == g.ny) ? r.c - (g.ny - 1) * g.nx : r.c + g.nx;
  r.s = (j == 0) ? r.c + (g.ny - 1) * g.nx : r.c - g.nx;
  r.u = (k + 1 < g.nzi) ? r.c + plane : nullptr;
  r.d = (k > 0) ? r.c - plane : nullptr;
  return r;
}

__device__ __forceinline__ void load_nb(const RowPtr<const float*>& rp, const PGrid32& g, int i, bool ok, Nb7& o) {
  o = Nb7{0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  if (ok) {
    const int ip = (i + 1 == g.nx) ? 0 : i + 1, im = (i == 0) ? g.nx - 1 : i - 1;
    o.c = rp.c[i];
    o.xp = rp.c[ip];
    o.xm = rp.c[im];
    o.yp = rp.n[i];
    o.ym = rp.s[i];
    if (rp.u) o.zp = rp.u[i];
    if (rp.d) o.zm = rp.d[i];
  }
}

__device__ __forceinline__ float apply_nb(const PGrid32& g, const Nb7& o) {
  float s = g.cx * (2.f * o.c - o.xp - o.xm);
  s += g.cy * (2.f * o.c - o.yp - o.ym);
  s += g.cz * (2.f * o.c - o.zp - o.zm);
  return s;
}

// The new direction p = r + beta p_old at a point and at its six neighbours
__device__ __forceinline__ void combine_nb(const Nb7& r, const Nb7& po, float beta, Nb7& o) {
  o.c = r.c + beta * po.c;
  o.xp = r.xp + beta * po.xp;
  o.xm = r.xm + beta * po.xm;
  o.yp = r.yp + beta * po.yp;
  o.ym = r.ym + beta * po.ym;
  o.zp = r.zp + beta * po.zp;
  o.zm = r.zm + beta * po.zm;
}

// p = r + beta p_old into pn (each point written by its own thread; the neighbours' values are
// formed again from r and p_old, so no barrier is needed between the update and the product),
// and <p, A^ p> over this thread's points (rows of 32 points or more)
__device__ __forceinline__ float pass_dir_pq_rows(const PGrid32& g, const float* __restrict__ r,
                                                  const float* __restrict__ po, float* __restrict__ pn,
                                                  float beta) {
  const int lane = threadIdx.x & 31;
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  const int nrow = g.ny * g.nzi;
  const int nch = (g.nx + 31) >> 5;
  float acc = 0.f;
  for (int rw = gw; rw < nrow; rw += nw) {
    const RowPtr<const float*> rr = row_ptr(r, g, rw);
    const RowPtr<const float*> rp = row_ptr(po, g, rw);
    float* __restrict__ pr = pn + (long long)rw * g.nx;
    for (int c0 = 0; c0 < nch; c0 += kDirChunks) {
      Nb7 nr[kDirChunks], np[kDirChunks];
#pragma unroll
      for (int u = 0; u < kDirChunks; ++u) {
        const int i = (c0 + u) * 32 + lane;
        load_nb(rr, g, i, i < g.nx, nr[u]);
        load_nb(rp, g, i, i < g.nx, np[u]);
      }
#pragma unroll
      for (int u = 0; u < kDirChunks; ++u) {
        const int i = (c0 + u) * 32 + lane;
        Nb7 nb;
        combine_nb(nr[u], np[u], beta, nb);
        if (i < g.nx) pr[i] = nb.c;
        acc += nb.c * apply_nb(g, nb);
      }
    }
  }
  return acc;
}

// d += alpha p, r -= alpha A^ p; returns the sum of the new r^2 over this thread's points
__device__ __forceinline__ float pass_update_rows(const PGrid32& g, const float* __restrict__ p,
                                                  float* __restrict__ d, float* __restrict__ r, float alpha) {
  const int lane = threadIdx.x & 31;
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  const int nrow = g.ny * g.nzi;
  const int nch = (g.nx + 31) >> 5;
  float acc = 0.f;
  for (int rw = gw; rw < nrow; rw += nw) {
    const RowPtr<const float*> rp = row_ptr(p, g, rw);
    float* __restrict__ dr = d + (long long)rw * g.nx;
    float* __restrict__ rr = r + (long long)rw * g.nx;
    for (int c0 = 0; c0 < nch; c0 += kChunks) {
      Nb7 nb[kChunks];
      float dv[kChunks], rv[kChunks];
#pragma unroll
      for (int u = 0; u < kChunks; ++u) {
        const int i = (c0 + u) * 32 + lane;
        const bool ok = i < g.nx;
        load_nb(rp, g, i, ok, nb[u]);
        dv[u] = ok ? dr[i] : 0.f;
        rv[u] = ok ? rr[i] : 0.f;
      }
#pragma unroll
      for (int u = 0; u < kChunks; ++u) {
        const int i = (c0 + u) * 32 + lane;
        if (i < g.nx) {
          dr[i] = dv[u] + alpha * nb[u].c;
          const float ri = rv[u] - alpha * apply_nb(g, nb[u]);
          rr[i] = ri;
          acc += ri * ri;
        }
      }
    }
  }
  return acc;
}

__global__ void __launch_bounds__(256, 4) cg_mixed_kernel(PGrid g, PGrid32 g32, double cmax,
                                                       const double* __restrict__ rho, double scale,
                                                       double* __restrict__ x, float* __restrict__ r,
                                                       float* p, float* q, float* __restrict__ d,
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
  // true residual in FP64 (and ||b||^2 on the first call)
  auto true_residual = [&](bool with_b, double* bb_out) -> double {
    double lrr = 0.0, lbb = 0.0;
    for_each_point(g, [&](int i, int j, int k, long long idx) {
      const double b = scale * rho[idx];
      const double ri = b - stencil_at(x, g, i, j, k, idx);
      lrr += ri * ri;
      lbb += b * b;
    });
    double v = block_sum(lrr, sh);
    if (threadIdx.x == 0) part0[blockIdx.x] = v;
    if (with_b) {
      v = block_sum(lbb, sh);
      if (threadIdx.x == 0) part2[blockIdx.x] = v;
    }
    grid.sync();
    if (with_b) *bb_out = grid_total(part2, sh);
    return grid_total(part0, sh);
  };
  // r^ = (b - A x) * s in FP32; returns ||r^||^2 (grid-wide)
  auto load_residual = [&](double s, bool init) -> double {
    float lr = 0.f;
    for_each_point(g, [&](int i, int j, int k, long long idx) {
      const double ri = scale * rho[idx] - stencil_at(x, g, i, j, k, idx);
      const float rs = (float)(ri * s);
      r[idx] = rs;
      if (init) {
        p[idx] = 0.f;   // the first direction is r itself (beta = 0 below)
        d[idx] = 0.f;
      }
      lr += rs * rs;
    });
    const double v = block_sum_f(lr, sh);
    if (threadIdx.x == 0) part1[blockIdx.x] = v;
    grid.sync();
    return grid_total(part1, sh);
  };
  double bb = 0.0;
  double rr64 = true_residual(true, &bb);
  const double stop = rtol * rtol * bb;
  int it = 0;
  bool conv = !(rr64 > stop);
  if (bb == 0.0) {
    // b = 0: the solution is x = 0 whatever the initial guess
    for (long long i = t0; i < n; i += stride) x[i] = 0.0;
    rr64 = 0.0;
    conv = true;
  }
  if (!conv && it < max_iter) {
    double s = 1.0 / sqrt(rr64 / (double)n);
    double rr = load_residual(s, true);
    double rmax = rr;
    const double delta2 = kReliableDelta * kReliableDelta;
    // the direction lives in two buffers: each iteration forms p = r + beta p_old from the old
    // one into the other, so the update needs no barrier of its own
    float* po = p;
    float* pn = q;
    float beta = 0.f;
    for (;;) {
      // p = r + beta p_old, <p, A^ p>
      float lpq = 0.f;
      if (g.nx >= 32) {
        lpq = pass_dir_pq_rows(g32, r, po, pn, beta);
      } else {
        for_each_point(g, [&](int i, int j, int k, long long idx) {
          const float pc = r[idx] + beta * po[idx];
          pn[idx] = pc;
          lpq += pc * stencil32_dir_at(r, po, beta, g32, i, j, k, idx);
        });
      }
      const float* pd = pn;   // this iteration's direction
      double v = block_sum_f(lpq, sh);
      if (threadIdx.x == 0) part0[blockIdx.x] = v;
      grid.sync();
      const float alpha = (float)(rr / grid_total(part0, sh));
      // d += alpha p, r -= alpha A^ p (the product recomputed rather than stored)
      float lr = 0.f;
      if (g.nx >= 32) {
        lr = pass_update_rows(g32, pd, d, r, alpha);
      } else {
        for_each_point(g, [&](int i, int j, int k, long long idx) {
          const float pi = pd[idx];
          const float qi = stencil32_at(pd, g32, i, j, k, idx);
          d[idx] += alpha * pi;
          const float ri = r[idx] - alpha * qi;
          r[idx] = ri;
          lr += ri * ri;
        });
      }
      v = block_sum_f(lr, sh);
      if (threadIdx.x == 0) part1[blockIdx.x] = v;
      grid.sync();
      double rn = grid_total(part1, sh);
      ++it;
      double beta_scale = 1.0;
      if (rn < delta2 * rmax || rn <= stop * s * s || it >= max_iter) {
        // fold the FP32 correction into x and replace the residual by the FP64 one
        const double back = 1.0 / (cmax * s);
        for (long long i = t0; i < n; i += stride) {
          x[i] += back * (double)d[i];
          d[i] = 0.f;
        }
        grid.sync();
        rr64 = true_residual(false, nullptr);
        if (!(rr64 > stop)) {
          conv = true;
          break;
        }
        if (it >= max_iter) break;
        const double s_new = 1.0 / sqrt(rr64 / (double)n);
        const double ratio = s_new / s;
        rn = load_residual(s_new, false);
        // p is still in the old units: rescale it inside the update below, and the old
        // <r, r> with it
        rr *= ratio * ratio;
        beta_scale = ratio;
        s = s_new;
        rmax = rn;
      }
      beta = (float)(rn / rr * beta_scale);
      rr = rn;
      float* t = po;
      po = pn;
      pn = t;
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    out->iterations = it;
    out->converged = conv;
    out->rel = bb > 0.0 ? sqrt(rr64 / bb) : 0.0;
  }
}

extern "C" omen_status omen_poisson(omen_ctx* ctx, const omen_grid* gr, const double* rho, double* phi,
                                    const omen_cg_opts* o, omen_solve_info* info) {
  if (!ctx || !gr || !rho || !phi || !o) return set_err(ctx, OMEN_EINVAL, "null argument");
  if (gr->nx < 1 || gr->ny < 1 || gr->nz < 2) return set_err(ctx, OMEN_EINVAL, "grid needs nx, ny >= 1 and nz >= 2");
  if (!(gr->Lx_nm > 0 && gr->Ly_nm > 0 && gr->Lz_nm > 0 && gr->eps_r > 0)) return set_err(ctx, OMEN_EINVAL, "grid lengths and eps_r must be > 0");
  if (!(o->rtol > 0) || o->max_iter < 1) return set_err(ctx, OMEN_EINVAL, "cg options");
  if (o->precision != OMEN_F64 && o->precision != OMEN_F32_REFINE64)
    return set_err(ctx, OMEN_EINVAL, "cg precision must be OMEN_F64 or OMEN_F32_REFINE64");
  const bool mixed = o->precision == OMEN_F32_REFINE64;
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
  const void* kern = mixed ? (const void*)cg_mixed_kernel : (const void*)cg_kernel;
  const int threads = 256;
  OMEN_CUDA(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, 0));
  if (per_sm < 1) return set_err(ctx, OMEN_ECUDA, "Poisson CG kernel does not fit on an SM");
  long long want = (g.n + threads - 1) / threads;
  int blocks = (int)std::min<long long>(want, (long long)dev_sms * per_sm);
  blocks = std::max(blocks, 1);
  // work vectors (three FP64, or four FP32 for the mixed form), three partial-sum rows, the result
  const size_t elem = mixed ? sizeof(float) : sizeof(double);
  const int nvec = mixed ? 4 : 3;
  const size_t vec = ((size_t)g.n * elem + 255) / 256 * 256;
  char* buf = nullptr;
  if (cudaMallocAsync(&buf, nvec * vec + 3 * blocks * sizeof(double) + sizeof(CGOut) + 64, ctx->stream) != cudaSuccess) {
    cudaGetLastError();
    return set_err(ctx, OMEN_ENOMEM, "CG work vectors");
  }
  double* part = reinterpret_cast<double*>(buf + nvec * vec);
  CGOut* out = reinterpret_cast<CGOut*>(part + 3 * blocks);
  double scale = 1.0 / (kEps0 * gr->eps_r);
  double rtol = o->rtol;
  int max_iter = o->max_iter;
  cudaError_t e;
  if (mixed) {
    const double cmax = std::max(g.cx, std::max(g.cy, g.cz));
    PGrid32 g32{g.nx, g.ny, g.nzi, (float)(g.cx / cmax), (float)(g.cy / cmax), (float)(g.cz / cmax)};
    float* r = reinterpret_cast<float*>(buf);
    float* p = reinterpret_cast<float*>(buf + vec);
    float* q = reinterpret_cast<float*>(buf + 2 * vec);
    float* d = reinterpret_cast<float*>(buf + 3 * vec);
    void* args[] = {&g, &g32, (void*)&cmax, &rho, &scale, &phi, &r, &p, &q, &d, &part, &rtol, &max_iter, &out};
    e = cudaLaunchCooperativeKernel(kern, dim3(blocks), dim3(threads), args, 0, ctx->stream);
  } else {
    double* r = reinterpret_cast<double*>(buf);
    double* p = reinterpret_cast<double*>(buf + vec);
    double* q = reinterpret_cast<double*>(buf + 2 * vec);
    void* args[] = {&g, &rho, &scale, &phi, &r, &p, &q, &part, &rtol, &max_iter, &out};
    e = cudaLaunchCooperativeKernel(kern, dim3(blocks), dim3(256), args, 0, ctx->stream);
  }
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
  if (!(o->rtol > 0) || o->max_iter < 1 || o->precision != OMEN_F64) return OMEN_EINVAL;
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
