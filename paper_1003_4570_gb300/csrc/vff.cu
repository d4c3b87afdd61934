// Valence-force-field strain relaxation on the device (paper Section II-B: the atom positions of
// a structure are relaxed by minimising an atomistic VFF strain energy before the electronic
// structure is computed; Fig. 4 benchmarks that step).  The paper prints no form; this is
// Keating's (Phys. Rev. 145, 637 (1966)), per bond and per bond angle:
//
//   E = sum_bonds 3 alpha_b / (8 d_b^2) (r_b.r_b - d_b^2)^2
//     + sum_atoms sum_{bond pairs p<q at the atom} 3 beta_pq / (8 d_p d_q) (r_p.r_q + d_p d_q / 3)^2
//
// r_p leaves the vertex atom along bond p; d_b is the natural bond length of the pair (mean of
// sqrt(3)/4 a of the two species), alpha_b the mean stretching constant, beta_b the mean bending
// constant of the bond's species and beta_pq the mean over the two bonds.  Positions are
// x = F x0 + u with F a fixed homogeneous deformation of the box and u the displacements; the
// ideal A->B bond vector of direction k is dir_k a/4, so r = +-F dir_k a/4 + u_n - u_i needs no
// stored positions and no neighbour list (neighbours come from the cell index, as in H·X).
//
// Kernels: per-atom gradient by gathering every term that touches the atom (own bonds, own bond
// angles, and the angles at each neighbour that use the bond back to it), so no atomics and a
// bit-reproducible result; per-atom energy; and, for the line search of the nonlinear conjugate-
// gradient relaxation, the coefficients of the energy along a search direction.  Every term is
// the square of a quadratic polynomial in the step t (r is affine in t), so E(u + t p) is a
// quartic whose derivative c1 + 2 c2 t + 3 c3 t^2 + 4 c4 t^3 is minimised exactly; c1 = g.p is
// accumulated term by term, so no energy difference (and no cancellation) enters the step.
#include <algorithm>
#include <chrono>
#include <cmath>

#include "omen_internal.h"
#include "sk_device.cuh"

namespace {

constexpr int kThreads = 256;

struct VffArgs {
  Geo g;
  NeighbourTables nt;
  const uint8_t* species;
  double fd[4][3];            // F dir_k a/4: deformed ideal A->B vector of direction k (nm)
  double dnat[4];             // natural bond length sqrt(3)/4 a per species (nm)
  double alpha[4], beta[4];   // eV/nm^2
};

// The (up to four) bonds of one atom as vectors leaving it.
struct Bonds4 {
  int nb[4];                  // neighbour atom, -1 where the bond leaves a hard wall
  double r[4][3];
  double d[4], al[4], be[4];  // natural length, stretching and bending constant of each bond
};

__device__ __forceinline__ void atom_cell(const Geo& g, int atom, int& b, int& cell, int& ix, int& iy, int& iz) {
  b = atom / g.ncells;
  cell = atom - b * g.ncells;
  ix = cell % g.nx;
  const int t = cell / g.nx;
  iy = t % g.ny;
  iz = t / g.ny;
}

// Neighbour of `atom` along direction k (-1 if the bond leaves a hard wall).
__device__ __forceinline__ int neighbour(const VffArgs& a, int atom, int k) {
  int b, cell, ix, iy, iz;
  atom_cell(a.g, atom, b, cell, ix, iy, iz);
  int ox, oy, oz, site2;
  if (b < 4) {
    ox = a.nt.a_to_b_off[b][k][0]; oy = a.nt.a_to_b_off[b][k][1]; oz = a.nt.a_to_b_off[b][k][2];
    site2 = a.nt.a_to_b_site[b][k];
  } else {
    const int s = b - 4;
    ox = a.nt.b_to_a_off[s][k][0]; oy = a.nt.b_to_a_off[s][k][1]; oz = a.nt.b_to_a_off[s][k][2];
    site2 = a.nt.b_to_a_site[s][k];
  }
  int cell2, wrap[3];
  if (!shift_cell(a.g, ix, iy, iz, ox, oy, oz, cell2, wrap)) return -1;
  return site2 * a.g.ncells + cell2;
}

__device__ __forceinline__ void load3(const double* __restrict__ v, long long n, int i, double out[3]) {
  out[0] = v[i];
  out[1] = v[n + i];
  out[2] = v[2 * n + i];
}

__device__ __forceinline__ double dot3(const double x[3], const double y[3]) {
  return x[0] * y[0] + x[1] * y[1] + x[2] * y[2];
}

// Bonds of `atom` at displacements u ([3][natoms]).
__device__ __forceinline__ void bonds_of(const VffArgs& a, const double* __restrict__ u, int atom, Bonds4& B) {
  const long long N = a.g.natoms;
  const double sg = atom < 4 * a.g.ncells ? 1.0 : -1.0;   // A atoms sit at the tail of dir_k
  const int sp = a.species[atom];
  double ui[3];
  load3(u, N, atom, ui);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int n = neighbour(a, atom, k);
    B.nb[k] = n;
    if (n < 0) continue;
    double un[3];
    load3(u, N, n, un);
#pragma unroll
    for (int c = 0; c < 3; ++c) B.r[k][c] = sg * a.fd[k][c] + un[c] - ui[c];
    const int sn = a.species[n];
    B.d[k] = 0.5 * (a.dnat[sp] + a.dnat[sn]);
    B.al[k] = 0.5 * (a.alpha[sp] + a.alpha[sn]);
    B.be[k] = 0.5 * (a.beta[sp] + a.beta[sn]);
  }
}

// Deterministic block sum of NV values per thread into partial[v * nblocks + block]; with
// MAX_LAST the last value is reduced by max instead of sum.
template <int NV, bool MAX_LAST>
__device__ __forceinline__ void block_reduce(double (&v)[NV], double* __restrict__ partial) {
  __shared__ double sm[NV][kThreads / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < NV; ++q) {
    double x = v[q];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double y = __shfl_down_sync(0xffffffffu, x, o);
      x = (MAX_LAST && q == NV - 1) ? fmax(x, y) : x + y;
    }
    if (lane == 0) sm[q][w] = x;
  }
  __syncthreads();
  if (threadIdx.x < NV) {
    const int q = threadIdx.x;
    double x = sm[q][0];
    for (int i = 1; i < kThreads / 32; ++i) x = (MAX_LAST && q == NV - 1) ? fmax(x, sm[q][i]) : x + sm[q][i];
    partial[(size_t)q * gridDim.x + blockIdx.x] = x;
  }
}

// dE/du for every atom; partials: [0] g.g, [1] g.g_prev (0 if g_prev is null), [2] max |g_c|.
__global__ void __launch_bounds__(kThreads) vff_grad_kernel(VffArgs a, const double* __restrict__ u,
                                                            double* __restrict__ g, const double* __restrict__ g_prev,
                                                            double* __restrict__ partial) {
  const long long N = a.g.natoms;
  double acc[3] = {0.0, 0.0, 0.0};
  for (int atom = blockIdx.x * blockDim.x + threadIdx.x; atom < N; atom += gridDim.x * blockDim.x) {
    Bonds4 B;
    bonds_of(a, u, atom, B);
    double gi[3] = {0.0, 0.0, 0.0};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      if (B.nb[k] < 0) continue;
      // bond stretch: dE/dr = 3 alpha / (2 d^2) (r.r - d^2) r, and r = x_n - x_i
      const double d2 = B.d[k] * B.d[k];
      const double cst = 1.5 * B.al[k] / d2 * (dot3(B.r[k], B.r[k]) - d2);
#pragma unroll
      for (int c = 0; c < 3; ++c) gi[c] -= cst * B.r[k][c];
    }
    // bond angles with this atom at the vertex: d(r_p.r_q)/dx_i = -(r_p + r_q)
#pragma unroll
    for (int p = 0; p < 4; ++p)
#pragma unroll
      for (int q = p + 1; q < 4; ++q) {
        if (B.nb[p] < 0 || B.nb[q] < 0) continue;
        const double dd = B.d[p] * B.d[q];
        const double w = 0.75 * 0.5 * (B.be[p] + B.be[q]) / dd * (dot3(B.r[p], B.r[q]) + dd / 3.0);
#pragma unroll
        for (int c = 0; c < 3; ++c) gi[c] -= w * (B.r[p][c] + B.r[q][c]);
      }
    // bond angles at each neighbour j that use the bond j -> i: d(r_ji.r_jm)/dx_i = r_jm
#pragma unroll 1
    for (int k = 0; k < 4; ++k) {
      const int j = B.nb[k];
      if (j < 0) continue;
      const double sj = j < 4 * a.g.ncells ? 1.0 : -1.0;
      const int spj = a.species[j];
      double uj[3], rji[3];
      load3(u, N, j, uj);
#pragma unroll
      for (int c = 0; c < 3; ++c) rji[c] = -B.r[k][c];
#pragma unroll 1
      for (int k2 = 0; k2 < 4; ++k2) {
        if (k2 == k) continue;                       // j's bond along k leads back to this atom
        const int m = neighbour(a, j, k2);
        if (m < 0) continue;
        double um[3], rjm[3];
        load3(u, N, m, um);
#pragma unroll
        for (int c = 0; c < 3; ++c) rjm[c] = sj * a.fd[k2][c] + um[c] - uj[c];
        const int spm = a.species[m];
        const double djm = 0.5 * (a.dnat[spj] + a.dnat[spm]);
        const double bjm = 0.5 * (a.beta[spj] + a.beta[spm]);
        const double dd = B.d[k] * djm;
        const double w = 0.75 * 0.5 * (B.be[k] + bjm) / dd * (dot3(rji, rjm) + dd / 3.0);
#pragma unroll
        for (int c = 0; c < 3; ++c) gi[c] += w * rjm[c];
      }
    }
    double gp[3] = {0.0, 0.0, 0.0};
    if (g_prev) load3(g_prev, N, atom, gp);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      g[c * N + atom] = gi[c];
      acc[0] += gi[c] * gi[c];
      acc[1] += gi[c] * gp[c];
      acc[2] = fmax(acc[2], fabs(gi[c]));
    }
  }
  block_reduce<3, true>(acc, partial);
}

// Energy: each bond counted at its A atom, each angle at its vertex.
__global__ void __launch_bounds__(kThreads) vff_energy_kernel(VffArgs a, const double* __restrict__ u,
                                                              double* __restrict__ partial) {
  const long long N = a.g.natoms;
  double acc[1] = {0.0};
  for (int atom = blockIdx.x * blockDim.x + threadIdx.x; atom < N; atom += gridDim.x * blockDim.x) {
    Bonds4 B;
    bonds_of(a, u, atom, B);
    const bool is_a = atom < 4 * a.g.ncells;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      if (B.nb[k] < 0 || !is_a) continue;
      const double d2 = B.d[k] * B.d[k];
      const double q = dot3(B.r[k], B.r[k]) - d2;
      acc[0] += 0.375 * B.al[k] / d2 * q * q;
    }
#pragma unroll
    for (int p = 0; p < 4; ++p)
#pragma unroll
      for (int q = p + 1; q < 4; ++q) {
        if (B.nb[p] < 0 || B.nb[q] < 0) continue;
        const double dd = B.d[p] * B.d[q];
        const double c = dot3(B.r[p], B.r[q]) + dd / 3.0;
        acc[0] += 0.375 * 0.5 * (B.be[p] + B.be[q]) / dd * c * c;
      }
  }
  block_reduce<1, false>(acc, partial);
}

// Coefficients c1..c4 of E(u + t p) - E(u) = c1 t + c2 t^2 + c3 t^3 + c4 t^4.  A term
// K (q0 + q1 t + q2 t^2)^2 contributes 2K q0 q1, K (q1^2 + 2 q0 q2), 2K q1 q2, K q2^2.
__global__ void __launch_bounds__(kThreads) vff_line_kernel(VffArgs a, const double* __restrict__ u,
                                                            const double* __restrict__ p, double* __restrict__ partial) {
  const long long N = a.g.natoms;
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  for (int atom = blockIdx.x * blockDim.x + threadIdx.x; atom < N; atom += gridDim.x * blockDim.x) {
    Bonds4 B;
    bonds_of(a, u, atom, B);
    double s[4][3];                                  // change of each bond vector per unit step
    double pi[3];
    load3(p, N, atom, pi);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      if (B.nb[k] < 0) continue;
      double pn[3];
      load3(p, N, B.nb[k], pn);
#pragma unroll
      for (int c = 0; c < 3; ++c) s[k][c] = pn[c] - pi[c];
    }
    const bool is_a = atom < 4 * a.g.ncells;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      if (B.nb[k] < 0 || !is_a) continue;
      const double d2 = B.d[k] * B.d[k];
      const double K = 0.375 * B.al[k] / d2;
      const double q0 = dot3(B.r[k], B.r[k]) - d2, q1 = 2.0 * dot3(B.r[k], s[k]), q2 = dot3(s[k], s[k]);
      acc[0] += 2.0 * K * q0 * q1;
      acc[1] += K * (q1 * q1 + 2.0 * q0 * q2);
      acc[2] += 2.0 * K * q1 * q2;
      acc[3] += K * q2 * q2;
    }
#pragma unroll
    for (int pp = 0; pp < 4; ++pp)
#pragma unroll
      for (int q = pp + 1; q < 4; ++q) {
        if (B.nb[pp] < 0 || B.nb[q] < 0) continue;
        const double dd = B.d[pp] * B.d[q];
        const double K = 0.375 * 0.5 * (B.be[pp] + B.be[q]) / dd;
        const double q0 = dot3(B.r[pp], B.r[q]) + dd / 3.0;
        const double q1 = dot3(B.r[pp], s[q]) + dot3(s[pp], B.r[q]);
        const double q2 = dot3(s[pp], s[q]);
        acc[0] += 2.0 * K * q0 * q1;
        acc[1] += K * (q1 * q1 + 2.0 * q0 * q2);
        acc[2] += 2.0 * K * q1 * q2;
        acc[3] += K * q2 * q2;
      }
  }
  block_reduce<4, false>(acc, partial);
}

// Relaxation state on the device (one small record).
struct VffState {
  double t;          // last step length
  double c1;         // last directional derivative g.p
  double gg[2];      // g.g of the current gradient, by iteration parity
  double gmax;       // max |g_c| of the current gradient
  int restart;       // the last direction was not a descent direction: next direction is -g
  int pad;
};

// Sum of `nb` partials of row q, in a fixed order (every block computes the same value).
__device__ double sum_partials(const double* __restrict__ part, int q, int nb, double* sm) {
  double x = 0.0;
  for (int i = threadIdx.x; i < nb; i += blockDim.x) x += part[(size_t)q * nb + i];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = x;
  __syncthreads();
  double s = 0.0;
  for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += sm[i];
  __syncthreads();
  return s;
}

__device__ double max_partials(const double* __restrict__ part, int q, int nb, double* sm) {
  double x = 0.0;
  for (int i = threadIdx.x; i < nb; i += blockDim.x) x = fmax(x, part[(size_t)q * nb + i]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x = fmax(x, __shfl_down_sync(0xffffffffu, x, o));
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = x;
  __syncthreads();
  double s = 0.0;
  for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s = fmax(s, sm[i]);
  __syncthreads();
  return s;
}

// Step length minimising the quartic along the line: the first sign change of its derivative
// c1 + 2 c2 t + 3 c3 t^2 + 4 c4 t^3 (c1 < 0) bracketed by doubling, then bisected to rounding.
__device__ double quartic_step(double c1, double c2, double c3, double c4) {
  if (!(c1 < 0.0)) return 0.0;
  auto dE = [&](double t) { return c1 + t * (2.0 * c2 + t * (3.0 * c3 + t * 4.0 * c4)); };
  double hi = c2 > 0.0 ? -c1 / (2.0 * c2) : 1e-6;
  int n = 0;
  while (!(dE(hi) > 0.0) && n < 400) {
    hi *= 2.0;
    ++n;
  }
  if (!(dE(hi) > 0.0)) return 0.0;                 // no minimum along the line: restart
  double lo = 0.0;
  for (int i = 0; i < 200 && hi - lo > 1e-16 * hi; ++i) {
    const double m = 0.5 * (lo + hi);
    if (dE(m) > 0.0) hi = m; else lo = m;
  }
  return 0.5 * (lo + hi);
}

// u += t p with t from the line coefficients (every block solves the same cubic).
__global__ void __launch_bounds__(kThreads) vff_step_kernel(double* __restrict__ u, const double* __restrict__ p,
                                                            long long n3, const double* __restrict__ line_part, int nb,
                                                            VffState* st) {
  __shared__ double sm[kThreads / 32];
  __shared__ double t_sh;
  const double c1 = sum_partials(line_part, 0, nb, sm);
  const double c2 = sum_partials(line_part, 1, nb, sm);
  const double c3 = sum_partials(line_part, 2, nb, sm);
  const double c4 = sum_partials(line_part, 3, nb, sm);
  if (threadIdx.x == 0) t_sh = quartic_step(c1, c2, c3, c4);
  __syncthreads();
  const double t = t_sh;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    st->t = t;
    st->c1 = c1;
    st->restart = t > 0.0 ? 0 : 1;
  }
  if (t == 0.0) return;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n3; i += (long long)gridDim.x * blockDim.x)
    u[i] += t * p[i];
}

// New direction p = -g + beta p (Polak–Ribière, clipped at 0; beta = 0 on the first iteration or
// after a restart).  Parity selects which gg slot holds the previous g.g.
__global__ void __launch_bounds__(kThreads) vff_dir_kernel(const double* __restrict__ g, double* __restrict__ p,
                                                           long long n3, const double* __restrict__ grad_part, int nb,
                                                           VffState* st, int first, int parity) {
  __shared__ double sm[kThreads / 32];
  const double gg = sum_partials(grad_part, 0, nb, sm);
  const double gprev = sum_partials(grad_part, 1, nb, sm);
  const double gmax = max_partials(grad_part, 2, nb, sm);
  const double gg_old = st->gg[parity];
  double beta = 0.0;
  if (!first && !st->restart && gg_old > 0.0) beta = fmax(0.0, (gg - gprev) / gg_old);
  __syncthreads();                                   // every block has read the state
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n3; i += (long long)gridDim.x * blockDim.x)
    p[i] = -g[i] + beta * p[i];
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    st->gg[parity ^ 1] = gg;
    st->gmax = gmax;
  }
}

__global__ void vff_strain_kernel(VffArgs a, const double* __restrict__ u, double* __restrict__ strain) {
  const long long nslots = 16ll * a.g.ncells;
  const long long N = a.g.natoms;
  for (long long sl = blockIdx.x * (long long)blockDim.x + threadIdx.x; sl < nslots; sl += (long long)gridDim.x * blockDim.x) {
    const int ks = (int)(sl / a.g.ncells);
    const int cell = (int)(sl - (long long)ks * a.g.ncells);
    const int k = ks >> 2, s = ks & 3;
    const int atom = s * a.g.ncells + cell;
    const int n = neighbour(a, atom, k);
    if (n < 0) {
      strain[sl] = 0.0;
      continue;
    }
    double ui[3], un[3], r[3];
    load3(u, N, atom, ui);
    load3(u, N, n, un);
#pragma unroll
    for (int c = 0; c < 3; ++c) r[c] = a.fd[k][c] + un[c] - ui[c];
    const double d = 0.5 * (a.dnat[a.species[atom]] + a.dnat[a.species[n]]);
    strain[sl] = sqrt(dot3(r, r)) / d - 1.0;
  }
}

__global__ void vff_negate_kernel(double* __restrict__ v, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    v[i] = -v[i];
}

omen_status make_args(omen_ctx* ctx, const omen_lattice* L, const omen_vff_params* vp, const double* F, VffArgs& a) {
  if (!vp) return set_err(ctx, OMEN_EINVAL, "null VFF parameters");
  if (vp->nspecies < 1 || vp->nspecies > 4) return set_err(ctx, OMEN_EINVAL, "nspecies must be 1..4");
  for (int s = 0; s < vp->nspecies; ++s)
    if (!(vp->a_nm[s] > 0) || !(vp->alpha[s] >= 0) || !(vp->beta[s] >= 0))
      return set_err(ctx, OMEN_EINVAL, "species %d: a_nm must be > 0 and alpha, beta >= 0", s);
  a.g.nx = L->nx; a.g.ny = L->ny; a.g.nz = L->nz;
  a.g.ncells = L->ncells; a.g.natoms = L->natoms;
  for (int d = 0; d < 3; ++d) a.g.periodic[d] = L->periodic[d];
  a.nt = host_neighbour_tables();
  a.species = L->d_species;
  static const int dir[4][3] = {{1, 1, 1}, {1, -1, -1}, {-1, 1, -1}, {-1, -1, 1}};
  const double q4 = 0.25 * L->a_nm;
  for (int k = 0; k < 4; ++k)
    for (int r = 0; r < 3; ++r) {
      double x = 0.0;
      for (int c = 0; c < 3; ++c) x += (F ? F[r * 3 + c] : (r == c ? 1.0 : 0.0)) * dir[k][c];
      a.fd[k][r] = x * q4;
    }
  for (int s = 0; s < 4; ++s) {
    const int t = s < vp->nspecies ? s : 0;
    a.dnat[s] = 0.25 * std::sqrt(3.0) * vp->a_nm[t];
    a.alpha[s] = vp->alpha[t];
    a.beta[s] = vp->beta[t];
  }
  return OMEN_OK;
}

int reduce_blocks(omen_ctx* ctx, long long n) {
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device);
  const long long want = (n + kThreads - 1) / kThreads;
  return (int)std::max<long long>(1, std::min<long long>(want, 4ll * std::max(1, sms)));
}

// Host sum of the partials of one row, in block order.
double host_sum(const std::vector<double>& h, int q, int nb, bool take_max = false) {
  double s = 0.0;
  for (int i = 0; i < nb; ++i) s = take_max ? std::max(s, h[(size_t)q * nb + i]) : s + h[(size_t)q * nb + i];
  return s;
}

}  // namespace

extern "C" omen_status omen_vff_energy_forces(omen_ctx* ctx, const omen_lattice* L, const omen_vff_params* vp,
                                              const double* F_host, const double* u_dev, double* E_host,
                                              double* force_dev) {
  if (!ctx || !L || !u_dev) return set_err(ctx, OMEN_EINVAL, "null argument");
  VffArgs a;
  omen_status s = make_args(ctx, L, vp, F_host, a);
  if (s != OMEN_OK) return s;
  const long long N = L->natoms;
  const int nb = reduce_blocks(ctx, N);
  if ((size_t)4 * nb * sizeof(double) > ctx->work_bytes) return set_err(ctx, OMEN_EINVAL, "work area too small");
  double* part = ctx->d_work;
  std::vector<double> h((size_t)3 * nb);
  if (force_dev) {
    vff_grad_kernel<<<nb, kThreads, 0, ctx->stream>>>(a, u_dev, force_dev, nullptr, part);
    OMEN_CHECK_LAUNCH(ctx);
    // force = -dE/du
    vff_negate_kernel<<<nb, kThreads, 0, ctx->stream>>>(force_dev, 3 * N);
    OMEN_CHECK_LAUNCH(ctx);
  }
  if (E_host) {
    vff_energy_kernel<<<nb, kThreads, 0, ctx->stream>>>(a, u_dev, part);
    OMEN_CHECK_LAUNCH(ctx);
    OMEN_CUDA(ctx, cudaMemcpyAsync(h.data(), part, sizeof(double) * nb, cudaMemcpyDeviceToHost, ctx->stream));
  }
  OMEN_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  if (E_host) *E_host = host_sum(h, 0, nb);
  return OMEN_OK;
}

extern "C" omen_status omen_relax_vff(omen_ctx* ctx, const omen_lattice* L, const omen_vff_params* vp,
                                      const double* F_host, const omen_vff_opts* o, double* u_dev, double* strain_dev,
                                      omen_vff_info* info) {
  if (!ctx || !L || !o || !u_dev) return set_err(ctx, OMEN_EINVAL, "null argument");
  if (!(o->gtol > 0) || o->max_iter < 0) return set_err(ctx, OMEN_EINVAL, "gtol must be > 0 and max_iter >= 0");
  const auto t0 = std::chrono::steady_clock::now();
  VffArgs a;
  omen_status s = make_args(ctx, L, vp, F_host, a);
  if (s != OMEN_OK) return s;
  const long long N = L->natoms, n3 = 3 * N;
  const int nb = reduce_blocks(ctx, N);
  const int check = 10;                                 // iterations between host convergence checks
  // work: two gradients (ping-pong), the direction, partials of the gradient (3 rows) and of the
  // line coefficients (4 rows), and the state record
  const size_t bytes = sizeof(double) * (3 * (size_t)n3 + 7 * (size_t)nb) + sizeof(VffState);
  char* buf = nullptr;
  if (cudaMallocAsync((void**)&buf, bytes, ctx->stream) != cudaSuccess) {
    cudaGetLastError();
    return set_err(ctx, OMEN_ENOMEM, "VFF work vectors (%zu bytes)", bytes);
  }
  double* g[2] = {reinterpret_cast<double*>(buf), reinterpret_cast<double*>(buf) + n3};
  double* p = g[1] + n3;
  double* gpart = p + n3;
  double* lpart = gpart + 3 * (size_t)nb;
  VffState* st = reinterpret_cast<VffState*>(lpart + 4 * (size_t)nb);
  std::vector<double> h((size_t)nb);
  VffState hs{};
  cudaError_t e = cudaMemsetAsync(st, 0, sizeof(VffState), ctx->stream);
  double E0 = 0.0;
  if (e == cudaSuccess) {
    vff_energy_kernel<<<nb, kThreads, 0, ctx->stream>>>(a, u_dev, gpart);
    e = cudaMemcpyAsync(h.data(), gpart, sizeof(double) * nb, cudaMemcpyDeviceToHost, ctx->stream);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  if (e == cudaSuccess) E0 = host_sum(h, 0, nb);
  int cur = 0, it = 0;
  bool converged = false;
  if (e == cudaSuccess) {
    vff_grad_kernel<<<nb, kThreads, 0, ctx->stream>>>(a, u_dev, g[cur], nullptr, gpart);
    vff_dir_kernel<<<nb, kThreads, 0, ctx->stream>>>(g[cur], p, n3, gpart, nb, st, 1, 0);
    e = cudaGetLastError();
  }
  while (e == cudaSuccess) {
    if (it % check == 0 || it == o->max_iter) {
      e = cudaMemcpyAsync(&hs, st, sizeof(VffState), cudaMemcpyDeviceToHost, ctx->stream);
      if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
      if (e != cudaSuccess) break;
      if (!std::isfinite(hs.gmax)) break;
      if (hs.gmax < o->gtol) {
        converged = true;
        break;
      }
      if (it == o->max_iter) break;
    }
    vff_line_kernel<<<nb, kThreads, 0, ctx->stream>>>(a, u_dev, p, lpart);
    vff_step_kernel<<<nb, kThreads, 0, ctx->stream>>>(u_dev, p, n3, lpart, nb, st);
    vff_grad_kernel<<<nb, kThreads, 0, ctx->stream>>>(a, u_dev, g[cur ^ 1], g[cur], gpart);
    cur ^= 1;
    ++it;
    vff_dir_kernel<<<nb, kThreads, 0, ctx->stream>>>(g[cur], p, n3, gpart, nb, st, 0, it & 1);
    e = cudaGetLastError();
  }
  double E1 = 0.0;
  if (e == cudaSuccess) {
    vff_energy_kernel<<<nb, kThreads, 0, ctx->stream>>>(a, u_dev, gpart);
    e = cudaMemcpyAsync(h.data(), gpart, sizeof(double) * nb, cudaMemcpyDeviceToHost, ctx->stream);
  }
  if (e == cudaSuccess && strain_dev) {
    const long long nslots = 16ll * L->ncells;
    const int sb = (int)std::min<long long>((nslots + kThreads - 1) / kThreads, 65535);
    vff_strain_kernel<<<sb, kThreads, 0, ctx->stream>>>(a, u_dev, strain_dev);
    e = cudaGetLastError();
  }
  cudaFreeAsync(buf, ctx->stream);
  const cudaError_t e2 = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess || e2 != cudaSuccess)
    return set_err(ctx, OMEN_ECUDA, "VFF relaxation: %s", cudaGetErrorString(e != cudaSuccess ? e : e2));
  E1 = host_sum(h, 0, nb);
  if (info) {
    info->iterations = it;
    info->converged = converged ? 1 : 0;
    info->energy_start = E0;
    info->energy = E1;
    info->max_force = hs.gmax;
    info->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
  if (!std::isfinite(hs.gmax) || !std::isfinite(E1))
    return set_err(ctx, OMEN_ENUMERIC, "VFF relaxation produced a non-finite force or energy");
  if (!converged)
    return set_err(ctx, OMEN_ENOCONV, "VFF relaxation stopped at %d iterations, max force %.3e eV/nm", it, hs.gmax);
  return OMEN_OK;
}
