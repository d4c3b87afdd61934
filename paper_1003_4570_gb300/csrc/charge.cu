// Charge from eigenstates, grid deposit and gather, Fermi level (paper Section III-A item 2:
// the charge profile from filling the states at a given Fermi level, or charge and Fermi level
// together under charge neutrality).
#include <algorithm>
#include <cmath>
#include <vector>

#include "omen_internal.h"
#include "sk_device.cuh"
#include "vec.cuh"
#include "cic.cuh"

// n_atom[i] += w * sum_n occ[n] * sum_o |psi_n[o*N + i]|^2
template <bool C>
__global__ void density_kernel(const void* __restrict__ psiv, long long nrows, int natoms, int nb, int nstates,
                               const double* __restrict__ occ, double w, double* __restrict__ n_atom) {
  using E = Elem<double, C>;
  const typename E::V* psi = static_cast<const typename E::V*>(psiv);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < natoms; i += gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int s = 0; s < nstates; ++s) {
      const double f = occ[s];
      if (f == 0.0) continue;
      double a = 0.0;
      for (int o = 0; o < nb; ++o) {
        const typename E::V v = psi[(size_t)s * nrows + (size_t)o * natoms + i];
        const double re = E::re(v), im = E::im(v);
        a += re * re + im * im;
      }
      acc += f * a;
    }
    n_atom[i] += w * acc;
  }
}

__global__ void deposit_kernel(Geo g, double a_nm, GridGeo G, const double* __restrict__ q, double* __restrict__ nodes) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < g.natoms; i += gridDim.x * blockDim.x) {
    const double qi = q[i];
    if (qi == 0.0) continue;
    double p[3];
    atom_position(g, a_nm, i, p);
    long long idx[8];
    double w[8];
    cic(G, p, idx, w);
    for (int c = 0; c < 8; ++c) atomicAdd(&nodes[idx[c]], w[c] * qi);
  }
}

__global__ void interior_kernel(const double* __restrict__ nodes, long long plane, long long n, double inv_vol,
                                double* __restrict__ rho) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    rho[i] = nodes[i + plane] * inv_vol;
}

__global__ void gather_kernel(Geo g, double a_nm, GridGeo G, const double* __restrict__ phi, double* __restrict__ out) {
  const long long plane = (long long)G.nx * G.ny;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < g.natoms; i += gridDim.x * blockDim.x) {
    double p[3];
    atom_position(g, a_nm, i, p);
    long long idx[8];
    double w[8];
    cic(G, p, idx, w);
    double s = 0.0;
    for (int c = 0; c < 8; ++c) {
      const long long k = idx[c] / plane;
      if (k >= 1 && k <= G.nz - 1) s += w[c] * phi[idx[c] - plane];
    }
    out[i] = s;
  }
}

extern "C" omen_status omen_density_accum(omen_ctx* ctx, const omen_ham* h, const void* psi, int nstates,
                                          const double* occ_host, double w, double* n_atom) {
  if (!ctx || !h || !psi || !occ_host || !n_atom || nstates < 0) return set_err(ctx, OMEN_EINVAL, "null argument");
  if (nstates == 0) return OMEN_OK;
  double* d_occ = nullptr;
  if (cudaMallocAsync(&d_occ, sizeof(double) * nstates, ctx->stream) != cudaSuccess) {
    cudaGetLastError();
    return set_err(ctx, OMEN_ENOMEM, "occupations");
  }
  OMEN_CUDA(ctx, cudaMemcpyAsync(d_occ, occ_host, sizeof(double) * nstates, cudaMemcpyHostToDevice, ctx->stream));
  const int N = (int)(h->nrows / h->nb);   // atoms, or grid points of an effective-mass Hamiltonian
  const unsigned grid = (unsigned)std::min(1024, (N + 255) / 256);
  if (h->is_complex) density_kernel<true><<<grid, 256, 0, ctx->stream>>>(psi, h->nrows, N, h->nb, nstates, d_occ, w, n_atom);
  else density_kernel<false><<<grid, 256, 0, ctx->stream>>>(psi, h->nrows, N, h->nb, nstates, d_occ, w, n_atom);
  cudaError_t e = cudaGetLastError();
  cudaFreeAsync(d_occ, ctx->stream);
  if (e != cudaSuccess) return set_err(ctx, OMEN_ECUDA, "density: %s", cudaGetErrorString(e));
  return OMEN_OK;
}

static omen_status check_grid(omen_ctx* ctx, const omen_grid* gr) {
  if (!gr || gr->nx < 1 || gr->ny < 1 || gr->nz < 2 || !(gr->Lx_nm > 0) || !(gr->Ly_nm > 0) || !(gr->Lz_nm > 0))
    return set_err(ctx, OMEN_EINVAL, "invalid grid");
  return OMEN_OK;
}

extern "C" omen_status omen_deposit(omen_ctx* ctx, const omen_lattice* L, const omen_grid* gr, const double* q,
                                    double* rho) {
  if (!ctx || !L || !q || !rho) return set_err(ctx, OMEN_EINVAL, "null argument");
  omen_status s = check_grid(ctx, gr);
  if (s != OMEN_OK) return s;
  const GridGeo G = grid_geo(gr);
  const long long plane = (long long)G.nx * G.ny;
  const long long nodes_n = plane * (G.nz + 1);
  double* nodes = nullptr;
  if (cudaMallocAsync(&nodes, sizeof(double) * nodes_n, ctx->stream) != cudaSuccess) {
    cudaGetLastError();
    return set_err(ctx, OMEN_ENOMEM, "deposit nodes");
  }
  OMEN_CUDA(ctx, cudaMemsetAsync(nodes, 0, sizeof(double) * nodes_n, ctx->stream));
  const unsigned ga = (unsigned)std::min(4096, (L->natoms + 255) / 256);
  deposit_kernel<<<ga, 256, 0, ctx->stream>>>(lat_geo(L), L->a_nm, G, q, nodes);
  const long long n = plane * (G.nz - 1);
  interior_kernel<<<(unsigned)std::min<long long>(4096, (n + 255) / 256), 256, 0, ctx->stream>>>(nodes, plane, n, 1.0 / G.vol_m3, rho);
  cudaError_t e = cudaGetLastError();
  cudaFreeAsync(nodes, ctx->stream);
  if (e != cudaSuccess) return set_err(ctx, OMEN_ECUDA, "deposit: %s", cudaGetErrorString(e));
  return OMEN_OK;
}

extern "C" omen_status omen_gather(omen_ctx* ctx, const omen_lattice* L, const omen_grid* gr, const double* phi,
                                   double* out) {
  if (!ctx || !L || !phi || !out) return set_err(ctx, OMEN_EINVAL, "null argument");
  omen_status s = check_grid(ctx, gr);
  if (s != OMEN_OK) return s;
  const unsigned ga = (unsigned)std::min(4096, (L->natoms + 255) / 256);
  gather_kernel<<<ga, 256, 0, ctx->stream>>>(lat_geo(L), L->a_nm, grid_geo(gr), phi, out);
  OMEN_CHECK_LAUNCH(ctx);
  return OMEN_OK;
}

static double fermi_fn(double x) {  // 1 / (1 + exp(x)), overflow-safe
  if (x > 0) {
    const double e = exp(-x);
    return e / (1.0 + e);
  }
  return 1.0 / (1.0 + exp(x));
}

extern "C" omen_status omen_fermi_level(const double* E, const double* wgt, int n, double n_target, double kT, double* EF) {
  if (!E || !wgt || !EF || n < 1 || !(kT > 0)) return OMEN_EINVAL;
  double total = 0.0, lo = E[0], hi = E[0];
  for (int i = 0; i < n; ++i) {
    total += wgt[i];
    lo = std::min(lo, E[i]);
    hi = std::max(hi, E[i]);
  }
  if (!(n_target >= 0) || n_target > total) return OMEN_EINVAL;
  lo -= 50 * kT;
  hi += 50 * kT;
  auto count = [&](double ef) {
    double c = 0.0;
    for (int i = 0; i < n; ++i) c += wgt[i] * fermi_fn((E[i] - ef) / kT);
    return c;
  };
  for (int it = 0; it < 200 && hi - lo > 1e-13; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (count(mid) < n_target) lo = mid; else hi = mid;
  }
  *EF = 0.5 * (lo + hi);
  return OMEN_OK;
}
