// Single-band effective-mass Hamiltonian (paper Section III-A item 1: the Schrödinger solver
// takes either the tight-binding or an effective-mass Hamiltonian).  Constant diagonal mass
// tensor, second-order central differences on a uniform nx x ny x nz grid:
//   (H psi)_i = (E_c + U_i + 2 sum_d t_d) psi_i - sum_d t_d (psi_{i+e_d} + psi_{i-e_d}),
//   t_d = hbar^2 / (2 m0 m_d h_d^2).
// Per axis: hard wall (the coupling past the first and last point is dropped), periodic, or
// Bloch-periodic: a neighbour reached across the high (low) face is the image shifted by +L_d
// (-L_d) and its amplitude is multiplied by exp(+i k_d L_d) (resp. the conjugate).
//
// The product is a 7-point stencil and moves no matrix: per point and vector it reads x once
// and writes y once (the six neighbour reads hit L1/L2: a z-neighbour is one plane away, well
// inside the L2 cache), plus one potential value per point shared by all vectors.  It is
// HBM-bound.  One thread per point in a grid-stride loop; the point's (ix, iy, iz) is divided
// out once and then advanced by the stride's own (sx, sy, sz) with carries, so the loop has no
// integer division.  The six neighbour indices and a mask of the ones reached across a face are
// formed once per point and reused for every vector; the hopping energies and phases are
// kernel parameters, and only an amplitude that crosses a face is multiplied by its phase.
// Overflow: N < 2^30 and three strides stay far below 2^31.
#include <algorithm>
#include <cmath>

#include "omen_internal.h"
#include "vec.cuh"

namespace {

// hbar^2 / (2 m0) in eV nm^2 from the CODATA 2018 values of hbar, m0 and e
constexpr double kHbar = 1.054571817e-34;
constexpr double kM0 = 9.1093837015e-31;
constexpr double kQe = 1.602176634e-19;
constexpr double kHbar2Over2M0 = kHbar * kHbar / (2.0 * kM0) / kQe * 1e18;

constexpr long long kMaxPoints = 1LL << 30;

struct EmGeo {
  int nx, ny, nz, N;
  int per[3];
};

__device__ __forceinline__ void mac(double& a, double c, double x) { a = fma(c, x, a); }
__device__ __forceinline__ void mac(float& a, float c, float x) { a = fmaf(c, x, a); }
__device__ __forceinline__ void mac(double2& a, double c, double2 x) {
  a.x = fma(c, x.x, a.x);
  a.y = fma(c, x.y, a.y);
}
__device__ __forceinline__ void mac(float2& a, float c, float2 x) {
  a.x = fmaf(c, x.x, a.x);
  a.y = fmaf(c, x.y, a.y);
}
__device__ __forceinline__ double scale(double d, double x) { return d * x; }
__device__ __forceinline__ float scale(float d, float x) { return d * x; }
__device__ __forceinline__ double2 scale(double d, double2 x) { return make_double2(d * x.x, d * x.y); }
__device__ __forceinline__ float2 scale(float d, float2 x) { return make_float2(d * x.x, d * x.y); }

template <typename T>
struct EmParams {
  EmGeo g;
  T t[3];        // hopping energies t_d
  T d0;          // E_c + 2 sum_d t_d - sigma
  double2 ph[3]; // exp(i k_d L_d) (1 on axes that are not Bloch-periodic)
};

// amplitude of a neighbour reached across a face: times exp(+i k L) across the high face,
// the conjugate across the low face (identity for real vectors, whose axes carry no phase)
template <typename T, bool C, bool LOW>
__device__ __forceinline__ typename Elem<T, C>::V across(typename Elem<T, C>::V a, double2 ph) {
  if constexpr (C) {
    const T c = (T)ph.x, s = LOW ? (T)-ph.y : (T)ph.y;
    typename Elem<T, C>::V r;
    r.x = c * a.x - s * a.y;
    r.y = c * a.y + s * a.x;
    return r;
  } else {
    (void)ph;
    return a;
  }
}

// Neighbours q = 2d (low side) and 2d+1 (high side) of axis d of point i at (ix, iy, iz): the
// index, or -1 past a hard wall; bit q of `wrap` marks a neighbour reached across a face.
__device__ __forceinline__ void neighbours(const EmGeo& g, int plane, int i, int ix, int iy, int iz, int (&j)[6],
                                           unsigned& wrap) {
  const int c[3] = {ix, iy, iz};
  const int n[3] = {g.nx, g.ny, g.nz};
  const int step[3] = {1, g.nx, plane};
  wrap = 0;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const int span = (n[d] - 1) * step[d];
    if (c[d] > 0) j[2 * d] = i - step[d];
    else if (g.per[d]) { j[2 * d] = i + span; wrap |= 1u << (2 * d); }
    else j[2 * d] = -1;
    if (c[d] < n[d] - 1) j[2 * d + 1] = i + step[d];
    else if (g.per[d]) { j[2 * d + 1] = i - span; wrap |= 2u << (2 * d); }
    else j[2 * d + 1] = -1;
  }
}

// (dg x_i - sum_q t_q x_j(q)) for one point; WRAP: apply the face phases marked in `wrap`
template <typename T, bool C, bool WRAP>
__device__ __forceinline__ typename Elem<T, C>::V stencil(const EmParams<T>& p, const typename Elem<T, C>::V* __restrict__ xv,
                                                          int i, const int (&j)[6], unsigned wrap, T dg) {
  using V = typename Elem<T, C>::V;
  V acc = scale(dg, xv[i]);
#pragma unroll
  for (int q = 0; q < 6; ++q) {
    if (j[q] < 0) continue;
    V a = xv[j[q]];
    if constexpr (WRAP) {
      if (wrap & (1u << q)) a = (q & 1) ? across<T, C, false>(a, p.ph[q / 2]) : across<T, C, true>(a, p.ph[q / 2]);
    } else {
      (void)wrap;
    }
    mac(acc, -p.t[q / 2], a);
  }
  return acc;
}

// PAIR: each thread takes two points per pass, i and i + S (S = the grid's thread count), and
// issues the loads of both before either sum: twice the bytes in flight per thread; complex
// vectors take the phase path only in the passes that touch a face, so the interior carries no
// complex rotation.  Without PAIR (real FP64, which GB300's FP64 pipe bounds and the pair only
// slows) one point per pass.
template <typename T, bool C, bool PAIR>
__global__ void __launch_bounds__(256) effmass_hx_kernel(EmParams<T> p, const T* __restrict__ U,
                                                         const typename Elem<T, C>::V* __restrict__ x,
                                                         typename Elem<T, C>::V* __restrict__ y, int nvec) {
  using V = typename Elem<T, C>::V;
  const EmGeo& g = p.g;
  const int N = g.N;
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const int S = gridDim.x * blockDim.x;
  const int plane = g.nx * g.ny;
  int iz = i / plane, r = i - iz * plane;
  int iy = r / g.nx, ix = r - iy * g.nx;
  const int sz = S / plane, rs = S - sz * plane;
  const int sy = rs / g.nx, sx = rs - sy * g.nx;
  if constexpr (!PAIR) {
    for (; i < N;) {
      int ja[6];
      unsigned wa;
      neighbours(g, plane, i, ix, iy, iz, ja, wa);
      const T dga = p.d0 + U[i];
      const V* xv = x;
      V* yv = y;
      for (int v = 0; v < nvec; ++v, xv += N, yv += N) yv[i] = stencil<T, C, true>(p, xv, i, ja, wa, dga);
      i += S;
      ix += sx;
      iy += sy;
      iz += sz;
      if (ix >= g.nx) { ix -= g.nx; ++iy; }
      if (iy >= g.ny) { iy -= g.ny; ++iz; }
    }
  } else {
    for (; i < N;) {
      // the second point, one stride on
      int ib = i + S, bx = ix + sx, by = iy + sy, bz = iz + sz;
      if (bx >= g.nx) { bx -= g.nx; ++by; }
      if (by >= g.ny) { by -= g.ny; ++bz; }
      const bool has_b = ib < N;
      int ja[6], jb[6];
      unsigned wa, wb;
      neighbours(g, plane, i, ix, iy, iz, ja, wa);
      if (has_b) {
        neighbours(g, plane, ib, bx, by, bz, jb, wb);
      } else {
        // no second point: a stand-in with no neighbours at a valid index, never stored
#pragma unroll
        for (int q = 0; q < 6; ++q) jb[q] = -1;
        wb = 0;
      }
      const int ibs = has_b ? ib : i;
      const T dga = p.d0 + U[i], dgb = p.d0 + U[ibs];
      const bool faces = C && (wa | wb) != 0;
      const V* xv = x;
      V* yv = y;
      for (int v = 0; v < nvec; ++v, xv += N, yv += N) {
        V ra, rb;
        if (faces) {
          ra = stencil<T, C, true>(p, xv, i, ja, wa, dga);
          rb = stencil<T, C, true>(p, xv, ibs, jb, wb, dgb);
        } else {
          ra = stencil<T, C, false>(p, xv, i, ja, 0u, dga);
          rb = stencil<T, C, false>(p, xv, ibs, jb, 0u, dgb);
        }
        yv[i] = ra;
        if (has_b) yv[ib] = rb;
      }
      // on to the next pair: two strides from i is one stride from the second point
      i = ib + S;
      ix = bx + sx;
      iy = by + sy;
      iz = bz + sz;
      if (ix >= g.nx) { ix -= g.nx; ++iy; }
      if (iy >= g.ny) { iy -= g.ny; ++iz; }
    }
  }
}

__global__ void to_float_kernel(const double* __restrict__ a, float* __restrict__ b, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) b[i] = (float)a[i];
}

template <typename T, bool C>
cudaError_t launch_em(const omen_ham* h, const T* U, const void* x, void* y, int nvec, double sigma, cudaStream_t st) {
  using V = typename Elem<T, C>::V;
  constexpr bool kPair = !(sizeof(T) == 8 && !C);
  EmParams<T> p;
  p.g = EmGeo{h->gdim[0], h->gdim[1], h->gdim[2], (int)h->nrows, {h->gper[0], h->gper[1], h->gper[2]}};
  for (int d = 0; d < 3; ++d) {
    p.t[d] = (T)h->t_hop[d];
    p.ph[d] = h->phase[d];
  }
  p.d0 = (T)(h->ec + 2.0 * (h->t_hop[0] + h->t_hop[1] + h->t_hop[2]) - sigma);
  // One wave of resident blocks: the grid-stride sweep then advances through the grid as one
  // front, and the plane below and above the points in flight are still in L2 when read.  (A
  // second wave would start after the first finished its whole sweep and re-read from DRAM
  // the planes next to every window the first wave left.)
  static int resident = 0, sms = 0;
  if (!resident) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&resident, effmass_hx_kernel<T, C, kPair>, 256, 0) != cudaSuccess ||
        resident < 1 || sms < 1) {
      cudaGetLastError();
      resident = 1;
      sms = 152;
    }
  }
  const int blocks = (int)std::min<long long>((h->nrows + 255) / 256, (long long)sms * resident);
  effmass_hx_kernel<T, C, kPair><<<blocks, 256, 0, st>>>(p, U, static_cast<const V*>(x), static_cast<V*>(y), nvec);
  return cudaGetLastError();
}

}  // namespace

omen_status launch_hx_effmass(omen_ctx* ctx, const omen_ham* h, const void* x, void* y, int nvec, double sigma,
                              int vec_precision, cudaStream_t st) {
  if (nvec < 1 || nvec > 65535) return set_err(ctx, OMEN_EINVAL, "nvec must be 1..65535");
  cudaError_t e;
  if (vec_precision == OMEN_F64) {
    e = h->is_complex ? launch_em<double, true>(h, h->d_U, x, y, nvec, sigma, st)
                      : launch_em<double, false>(h, h->d_U, x, y, nvec, sigma, st);
  } else if (vec_precision == OMEN_F32) {
    if (!h->d_U32) return set_err(ctx, OMEN_EINVAL, "Hamiltonian has no FP32 potential");
    e = h->is_complex ? launch_em<float, true>(h, h->d_U32, x, y, nvec, sigma, st)
                      : launch_em<float, false>(h, h->d_U32, x, y, nvec, sigma, st);
  } else {
    return set_err(ctx, OMEN_EUNSUPPORTED, "effective-mass products run on FP64 or FP32 vectors");
  }
  if (e != cudaSuccess) return set_err(ctx, OMEN_ECUDA, "effective-mass H·X launch failed: %s", cudaGetErrorString(e));
  return OMEN_OK;
}

omen_status effmass_set_potential(omen_ctx* ctx, omen_ham* h, const double* U) {
  const size_t n = (size_t)h->nrows;
  if (U) OMEN_CUDA(ctx, cudaMemcpyAsync(h->d_U, U, sizeof(double) * n, cudaMemcpyDeviceToDevice, ctx->stream));
  else OMEN_CUDA(ctx, cudaMemsetAsync(h->d_U, 0, sizeof(double) * n, ctx->stream));
  if (h->d_U32) {
    const int blocks = (int)std::min<long long>(((long long)n + 255) / 256, 152LL * 8);
    to_float_kernel<<<blocks, 256, 0, ctx->stream>>>(h->d_U, h->d_U32, (int)n);
    OMEN_CHECK_LAUNCH(ctx);
  }
  return OMEN_OK;
}

extern "C" omen_status omen_assemble_effmass(omen_ctx* ctx, const omen_effmass_desc* d, const double* U_dev,
                                             omen_ham** out) {
  if (!ctx || !d || !out) return set_err(ctx, OMEN_EINVAL, "null argument");
  *out = nullptr;
  const int n[3] = {d->nx, d->ny, d->nz};
  long long N = 1;
  for (int a = 0; a < 3; ++a) {
    if (n[a] < 1) return set_err(ctx, OMEN_EINVAL, "grid sizes must be >= 1");
    if (!(d->h_nm[a] > 0) || !std::isfinite(d->h_nm[a])) return set_err(ctx, OMEN_EINVAL, "spacings must be finite and > 0");
    if (!(d->m_rel[a] > 0) || !std::isfinite(d->m_rel[a])) return set_err(ctx, OMEN_EINVAL, "masses must be finite and > 0");
    if (d->periodic[a] != OMEN_HARD_WALL && d->periodic[a] != OMEN_PERIODIC && d->periodic[a] != OMEN_BLOCH)
      return set_err(ctx, OMEN_EINVAL, "periodic flags must be HARD_WALL, PERIODIC or BLOCH");
    N *= n[a];
    if (N >= kMaxPoints) return set_err(ctx, OMEN_EINVAL, "grid must have fewer than 2^30 points");
  }
  if (!std::isfinite(d->ec_eV) || !std::isfinite(d->k[0]) || !std::isfinite(d->k[1]) || !std::isfinite(d->k[2]))
    return set_err(ctx, OMEN_EINVAL, "band edge and wave vector must be finite");
  if (d->precision == OMEN_F64_DF) return set_err(ctx, OMEN_EUNSUPPORTED, "effective-mass Hamiltonians are FP64 or FP32");
  if (d->precision != OMEN_F64 && d->precision != OMEN_F32 && d->precision != OMEN_F32_REFINE64)
    return set_err(ctx, OMEN_EINVAL, "unknown precision %d", d->precision);
  OMEN_CUDA(ctx, cudaSetDevice(ctx->device));
  omen_ham* h = new omen_ham();
  h->effmass = 1;
  h->norb = 1;
  h->nspin = 1;
  h->nb = 1;
  h->nrows = N;
  h->precision = d->precision;
  h->ec = d->ec_eV;
  for (int a = 0; a < 3; ++a) {
    h->gdim[a] = n[a];
    h->gper[a] = d->periodic[a] != OMEN_HARD_WALL;
    h->t_hop[a] = kHbar2Over2M0 / (d->m_rel[a] * d->h_nm[a] * d->h_nm[a]);
    h->phase[a] = make_double2(1.0, 0.0);
    if (d->periodic[a] == OMEN_BLOCH) {
      h->is_complex = 1;
      const double kl = d->k[a] * n[a] * d->h_nm[a];
      h->phase[a] = make_double2(std::cos(kl), std::sin(kl));
    }
  }
  if (cudaMalloc(&h->d_U, sizeof(double) * N) != cudaSuccess ||
      (d->precision != OMEN_F64 && cudaMalloc(&h->d_U32, sizeof(float) * N) != cudaSuccess)) {
    cudaGetLastError();
    omen_free_ham(h);
    return set_err(ctx, OMEN_ENOMEM, "potential of %lld points", N);
  }
  omen_status s = effmass_set_potential(ctx, h, U_dev);
  if (s != OMEN_OK) {
    cudaStreamSynchronize(ctx->stream);
    omen_free_ham(h);
    return s;
  }
  *out = h;
  return OMEN_OK;
}
