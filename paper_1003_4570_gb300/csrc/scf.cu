// Self-consistent Schrödinger–Poisson loop (paper Section III-A: eigenstates -> charge ->
// Poisson -> potential back into the Hamiltonian, repeated to self-consistency).
//
// phi (grid, V) -> phi at the atoms (trilinear gather) -> onsite U = -phi (eV) -> for each k:
// the nev eigenpairs nearest sigma (folded-spectrum Lanczos) -> Fermi level from neutrality
// over the levels above e_cut -> electrons per atom -> cloud-in-cell charge + donor background
// -> Poisson CG -> dV = max|phi_out - phi|; stop when dV < tol_V, else phi += mix (phi_out - phi).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <vector>

#include "omen_internal.h"

static constexpr double kQe = 1.602176634e-19;  // C

__global__ void scale_kernel(const double* __restrict__ x, double a, double* __restrict__ y, long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = a * x[i];
}

__global__ void add_kernel(double* __restrict__ y, const double* __restrict__ x, long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] += x[i];
}

// per-block max |a - b|
__global__ void maxdiff_kernel(const double* __restrict__ a, const double* __restrict__ b, long long n,
                               double* __restrict__ part) {
  double m = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    m = fmax(m, fabs(a[i] - b[i]));
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  __shared__ double sh[32];
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t = fmax(t, sh[i]);
    part[blockIdx.x] = t;
  }
}

__global__ void mix_kernel(double* __restrict__ phi, const double* __restrict__ out, double mix, long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    phi[i] += mix * (out[i] - phi[i]);
}

// Anderson mixing (Anderson, J. ACM 12, 547 (1965)) on the grid potential.
// F = phi_out - phi.  With the differences dX_j, dF_j of the last h iterates (slots in a ring),
// gamma = argmin |F - dF gamma|, phi <- phi + beta F - sum_j gamma_j (dX_j + beta dF_j).
// part[b * (h+1)^2 + ...]: per-block partial Gram sums of the vectors (dF_0..dF_{h-1}, F).
__global__ void gram_kernel(const double* __restrict__ dF, long long ld, int h, const double* __restrict__ F, long long n,
                            double* __restrict__ part) {
  const int nv = h + 1;
  extern __shared__ double sh[];
  for (int e = threadIdx.x; e < nv * nv; e += blockDim.x) sh[e] = 0.0;
  __syncthreads();
  for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (long long)gridDim.x * blockDim.x) {
    double v[9];
    for (int a = 0; a < nv; ++a) v[a] = (a < h) ? dF[a * ld + r] : F[r];
    for (int a = 0; a < nv; ++a)
      for (int b = a; b < nv; ++b) atomicAdd(&sh[a * nv + b], v[a] * v[b]);
  }
  __syncthreads();
  for (int e = threadIdx.x; e < nv * nv; e += blockDim.x) part[(size_t)blockIdx.x * nv * nv + e] = sh[e];
}

__global__ void anderson_kernel(double* __restrict__ phi, const double* __restrict__ F, const double* __restrict__ dX,
                                const double* __restrict__ dF, long long ld, int h, const double* __restrict__ gamma,
                                double beta, long long n) {
  for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (long long)gridDim.x * blockDim.x) {
    double v = phi[r] + beta * F[r];
    for (int j = 0; j < h; ++j) v -= gamma[j] * (dX[j * ld + r] + beta * dF[j * ld + r]);
    phi[r] = v;
  }
}

__global__ void diff_kernel(const double* __restrict__ a, const double* __restrict__ b, double* __restrict__ out, long long n) {
  for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (long long)gridDim.x * blockDim.x)
    out[r] = a[r] - b[r];
}

static double fermi_occ(double x) {
  if (x > 0) {
    const double e = exp(-x);
    return e / (1.0 + e);
  }
  return 1.0 / (1.0 + exp(x));
}

struct DevVec {
  void* p = nullptr;
  ~DevVec() { if (p) cudaFree(p); }
  bool alloc(size_t bytes) {
    if (cudaMalloc(&p, bytes) != cudaSuccess) { cudaGetLastError(); p = nullptr; return false; }
    return true;
  }
  double* d() { return static_cast<double*>(p); }
};

extern "C" omen_status omen_scf(omen_ctx* ctx, const omen_scf_desc* d, double* phi, omen_scf_info* info) {
  if (!ctx || !d || !phi || !d->lat || !d->params || !d->grid || !d->k_host || !d->kw_host)
    return set_err(ctx, OMEN_EINVAL, "null argument");
  if (d->nk < 1 || d->nev < 1 || !(d->kT > 0) || !(d->mix > 0 && d->mix <= 1) || !(d->tol_V > 0) || d->max_iter < 1)
    return set_err(ctx, OMEN_EINVAL, "invalid SCF options");
  if (d->precision != OMEN_F64 && d->precision != OMEN_F32_REFINE64)
    return set_err(ctx, OMEN_EINVAL, "SCF eigen-solves need FP64 eigenvectors (F64 or F32_REFINE64)");
  OMEN_CUDA(ctx, cudaSetDevice(ctx->device));
  auto t0 = std::chrono::steady_clock::now();
  omen_scf_info loc{};
  omen_scf_info* inf = info ? info : &loc;
  *inf = omen_scf_info{};
  const omen_lattice* L = d->lat;
  const omen_grid* G = d->grid;
  const long long ng = (long long)G->nx * G->ny * (G->nz - 1);
  const int N = L->natoms;

  // one Hamiltonian per k (bond blocks with their Bloch phase), potential set per iteration
  std::vector<omen_ham*> hams(d->nk, nullptr);
  auto free_hams = [&]() {
    for (auto* h : hams) omen_free_ham(h);
  };
  for (int k = 0; k < d->nk; ++k) {
    omen_ham_opts ho{};
    ho.spin_orbit = 0;
    ho.precision = d->precision;
    ho.matrix_free = 0;
    ho.k = d->k_host + 3 * k;
    ho.U_atom_dev = nullptr;
    omen_status s = omen_assemble_H(ctx, L, d->params, &ho, &hams[k]);
    if (s != OMEN_OK) { free_hams(); return s; }
  }
  const long long nrows = hams[0]->nrows;
  const size_t elem = hams[0]->is_complex ? 16 : 8;
  DevVec phi_atom, U, n_atom, q, rho, phi_out, part, psi, v0, Fcur, Fprev, Xprev, dXh, dFh, gpart, gam, Wst, zero_rho;
  const int H = std::max(0, std::min(8, d->mix_history));
  const int nblk = 256;
  if (!phi_atom.alloc(sizeof(double) * N) || !U.alloc(sizeof(double) * N) || !n_atom.alloc(sizeof(double) * N) ||
      !q.alloc(sizeof(double) * N) || !rho.alloc(sizeof(double) * ng) || !phi_out.alloc(sizeof(double) * ng) ||
      !part.alloc(sizeof(double) * nblk) || !psi.alloc(elem * nrows * (size_t)d->nev * d->nk) ||
      !v0.alloc(elem * nrows * (size_t)std::max(1, d->eig_block)) || !Fcur.alloc(sizeof(double) * ng) ||
      !Fprev.alloc(sizeof(double) * ng) || !Xprev.alloc(sizeof(double) * ng) ||
      !dXh.alloc(sizeof(double) * ng * std::max(1, H)) || !dFh.alloc(sizeof(double) * ng * std::max(1, H)) ||
      !gpart.alloc(sizeof(double) * 81 * 256) || !gam.alloc(sizeof(double) * 8)) {
    free_hams();
    return set_err(ctx, OMEN_ENOMEM, "SCF work buffers");
  }
  if (d->poisson_newton) {
    if (!Wst.alloc(sizeof(double) * (size_t)N * d->nev * d->nk) || (!d->donor_rho_dev && !zero_rho.alloc(sizeof(double) * ng))) {
      free_hams();
      return set_err(ctx, OMEN_ENOMEM, "SCF Newton buffers");
    }
    if (!d->donor_rho_dev) OMEN_CUDA(ctx, cudaMemsetAsync(zero_rho.p, 0, sizeof(double) * ng, ctx->stream));
  }
  const unsigned ga = (unsigned)std::min(4096, (N + 255) / 256);
  const unsigned gg = (unsigned)std::min<long long>(nblk, (ng + 255) / 256);
  std::vector<double> evals((size_t)d->nev * d->nk);
  const double gs = 2.0;  // spin degeneracy (no spin-orbit in the SCF Hamiltonian)
  omen_status st = OMEN_OK;
  double EF = 0.0;
  int it = 0;
  int nhist_total = 0;
  for (it = 1; it <= d->max_iter; ++it) {
    // potential at the atoms -> onsite energies
    st = omen_gather(ctx, L, G, phi, phi_atom.d());
    if (st != OMEN_OK) break;
    scale_kernel<<<ga, 256, 0, ctx->stream>>>(phi_atom.d(), -1.0, U.d(), N);
    auto te = std::chrono::steady_clock::now();
    for (int k = 0; k < d->nk && st == OMEN_OK; ++k) {
      st = omen_ham_set_potential(ctx, hams[k], U.d());
      if (st != OMEN_OK) break;
      omen_eig_opts eo{};
      eo.nev = d->nev;
      eo.which = OMEN_NEAREST;
      eo.sigma = d->sigma;
      // early iterations need eigenpairs only to the accuracy of the current potential error
      eo.tol = (it == 1 || inf->dV_inf <= 0.0) ? std::max(d->eig_tol, 1e-6)
                                                : std::max(d->eig_tol, std::min(1e-5, 1e-4 * inf->dV_inf));
      eo.max_iter = d->eig_max_iter;
      eo.block = d->eig_block;
      eo.basis = d->eig_basis;
      eo.v0_host = nullptr;
      eo.v0_dev = nullptr;
      if (it > 1 && d->precision == OMEN_F64) {
        // warm start: the previous iteration's eigenvectors of this k span the new ones closely
        st = krylov_start_from(ctx, hams[k], OMEN_F64, static_cast<char*>(psi.p) + elem * nrows * (size_t)d->nev * k,
                               d->nev, v0.p, d->eig_block, 0x1234ull + (unsigned long long)(it * 131 + k));
        if (st != OMEN_OK) break;
        eo.v0_dev = v0.p;
      }
      omen_eig_info ei{};
      st = omen_eigs(ctx, hams[k], &eo, evals.data() + (size_t)k * d->nev,
                     static_cast<char*>(psi.p) + elem * nrows * (size_t)d->nev * k, &ei);
      inf->hx_count += ei.hx_count;
    }
    inf->eig_seconds += std::chrono::duration<double>(std::chrono::steady_clock::now() - te).count();
    if (st != OMEN_OK) break;
    // Fermi level over conduction levels (above e_cut)
    std::vector<double> E, W;
    for (int k = 0; k < d->nk; ++k)
      for (int n = 0; n < d->nev; ++n) {
        const double e = evals[(size_t)k * d->nev + n];
        if (e > d->e_cut) {
          E.push_back(e);
          W.push_back(gs * d->kw_host[k]);
        }
      }
    if (E.empty() || omen_fermi_level(E.data(), W.data(), (int)E.size(), d->n_electrons, d->kT, &EF) != OMEN_OK) {
      st = set_err(ctx, OMEN_ENUMERIC, "too few conduction states above e_cut for %.6g electrons", d->n_electrons);
      break;
    }
    for (int k = 0; k < d->nk; ++k) {
      double emax = -1e300;
      for (int n = 0; n < d->nev; ++n) emax = std::max(emax, evals[(size_t)k * d->nev + n]);
      if (fermi_occ((emax - EF) / d->kT) > 1e-12) {
        st = set_err(ctx, OMEN_ENUMERIC, "highest computed state of k %d is occupied (raise nev)", k);
        break;
      }
    }
    if (st != OMEN_OK) break;
    if (d->poisson_newton) {
      // the root of the nonlinear Poisson equation with the frozen states' predicted charge
      for (int k = 0; k < d->nk && st == OMEN_OK; ++k) {
        std::vector<double> wk(d->nev);
        for (int n = 0; n < d->nev; ++n) wk[n] = evals[(size_t)k * d->nev + n] > d->e_cut ? gs * d->kw_host[k] : 0.0;
        st = omen_state_weights(ctx, hams[k], static_cast<char*>(psi.p) + elem * nrows * (size_t)d->nev * k, d->nev,
                                wk.data(), Wst.d() + (size_t)N * d->nev * k);
      }
      if (st != OMEN_OK) break;
      OMEN_CUDA(ctx, cudaMemcpyAsync(phi_out.p, phi, sizeof(double) * ng, cudaMemcpyDeviceToDevice, ctx->stream));
      omen_frozen_states fs{d->nev * d->nk, evals.data(), Wst.d(), EF, d->kT, phi};
      omen_newton_opts no{std::min(1e-9, 0.01 * d->tol_V), 50, d->cg};
      omen_newton_info ni{};
      auto tp = std::chrono::steady_clock::now();
      st = omen_poisson_newton(ctx, L, G, &fs, d->donor_rho_dev ? d->donor_rho_dev : zero_rho.d(), phi_out.d(), &no, &ni);
      inf->poisson_seconds += std::chrono::duration<double>(std::chrono::steady_clock::now() - tp).count();
      if (st != OMEN_OK) break;
    } else {
    // electrons per atom
    OMEN_CUDA(ctx, cudaMemsetAsync(n_atom.p, 0, sizeof(double) * N, ctx->stream));
    for (int k = 0; k < d->nk && st == OMEN_OK; ++k) {
      std::vector<double> occ(d->nev);
      for (int n = 0; n < d->nev; ++n) {
        const double e = evals[(size_t)k * d->nev + n];
        occ[n] = e > d->e_cut ? fermi_occ((e - EF) / d->kT) : 0.0;
      }
      st = omen_density_accum(ctx, hams[k], static_cast<char*>(psi.p) + elem * nrows * (size_t)d->nev * k, d->nev,
                              occ.data(), gs * d->kw_host[k], n_atom.d());
    }
    if (st != OMEN_OK) break;
    // charge density: electrons (-e) deposited + donor background
    scale_kernel<<<ga, 256, 0, ctx->stream>>>(n_atom.d(), -kQe, q.d(), N);
    st = omen_deposit(ctx, L, G, q.d(), rho.d());
    if (st != OMEN_OK) break;
    if (d->donor_rho_dev) add_kernel<<<gg, 256, 0, ctx->stream>>>(rho.d(), d->donor_rho_dev, ng);
    // Poisson from the current potential as initial guess
    OMEN_CUDA(ctx, cudaMemcpyAsync(phi_out.p, phi, sizeof(double) * ng, cudaMemcpyDeviceToDevice, ctx->stream));
    auto tp = std::chrono::steady_clock::now();
    omen_solve_info si{};
    st = omen_poisson(ctx, G, rho.d(), phi_out.d(), &d->cg, &si);
    inf->poisson_seconds += std::chrono::duration<double>(std::chrono::steady_clock::now() - tp).count();
    if (st != OMEN_OK) break;
    }
    maxdiff_kernel<<<gg, 256, 0, ctx->stream>>>(phi_out.d(), phi, ng, part.d());
    std::vector<double> hp(gg);
    OMEN_CUDA(ctx, cudaMemcpyAsync(hp.data(), part.p, sizeof(double) * gg, cudaMemcpyDeviceToHost, ctx->stream));
    OMEN_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    double dV = 0.0;
    for (double v : hp) dV = std::max(dV, v);
    inf->dV_inf = dV;
    inf->E_F = EF;
    inf->iterations = it;
    if (dV < d->tol_V) {
      inf->converged = 1;
      break;
    }
    if (H == 0) {
      mix_kernel<<<gg, 256, 0, ctx->stream>>>(phi, phi_out.d(), d->mix, ng);
      continue;
    }
    // Anderson: F = phi_out - phi; history of differences in a ring of H slots
    diff_kernel<<<gg, 256, 0, ctx->stream>>>(phi_out.d(), phi, Fcur.d(), ng);
    if (nhist_total > 0) {
      const int slot = (nhist_total - 1) % H;
      diff_kernel<<<gg, 256, 0, ctx->stream>>>(Fcur.d(), Fprev.d(), dFh.d() + (size_t)slot * ng, ng);
      diff_kernel<<<gg, 256, 0, ctx->stream>>>(phi, Xprev.d(), dXh.d() + (size_t)slot * ng, ng);
    }
    OMEN_CUDA(ctx, cudaMemcpyAsync(Fprev.p, Fcur.p, sizeof(double) * ng, cudaMemcpyDeviceToDevice, ctx->stream));
    OMEN_CUDA(ctx, cudaMemcpyAsync(Xprev.p, phi, sizeof(double) * ng, cudaMemcpyDeviceToDevice, ctx->stream));
    const int h = std::min(nhist_total, H);
    ++nhist_total;
    std::vector<double> gamma(8, 0.0);
    if (h > 0) {
      const int nv = h + 1;
      const unsigned gb = (unsigned)std::min<long long>(256, (ng + 255) / 256);
      gram_kernel<<<gb, 256, sizeof(double) * nv * nv, ctx->stream>>>(dFh.d(), ng, h, Fcur.d(), ng, gpart.d());
      std::vector<double> hp((size_t)gb * nv * nv);
      OMEN_CUDA(ctx, cudaMemcpyAsync(hp.data(), gpart.p, sizeof(double) * hp.size(), cudaMemcpyDeviceToHost, ctx->stream));
      OMEN_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
      std::vector<double> G((size_t)nv * nv, 0.0);
      for (unsigned b = 0; b < gb; ++b)
        for (int e = 0; e < nv * nv; ++e) G[e] += hp[(size_t)b * nv * nv + e];
      // normal equations (dF^T dF + tiny I) gamma = dF^T F, solved by Gaussian elimination
      std::vector<double> A((size_t)h * h), rhs(h);
      double diag = 0.0;
      for (int a = 0; a < h; ++a) diag = std::max(diag, G[a * nv + a]);
      for (int a = 0; a < h; ++a) {
        for (int b2 = 0; b2 < h; ++b2) A[a * h + b2] = (a <= b2) ? G[a * nv + b2] : G[b2 * nv + a];
        A[a * h + a] += 1e-12 * diag;
        rhs[a] = G[a * nv + h];
      }
      for (int c = 0; c < h; ++c) {
        int piv = c;
        for (int r = c + 1; r < h; ++r)
          if (std::fabs(A[r * h + c]) > std::fabs(A[piv * h + c])) piv = r;
        if (piv != c) {
          for (int k2 = 0; k2 < h; ++k2) std::swap(A[c * h + k2], A[piv * h + k2]);
          std::swap(rhs[c], rhs[piv]);
        }
        const double pv = A[c * h + c];
        if (pv == 0.0) continue;
        for (int r = c + 1; r < h; ++r) {
          const double f = A[r * h + c] / pv;
          for (int k2 = c; k2 < h; ++k2) A[r * h + k2] -= f * A[c * h + k2];
          rhs[r] -= f * rhs[c];
        }
      }
      for (int c = h - 1; c >= 0; --c) {
        double v = rhs[c];
        for (int k2 = c + 1; k2 < h; ++k2) v -= A[c * h + k2] * gamma[k2];
        gamma[c] = (A[c * h + c] != 0.0) ? v / A[c * h + c] : 0.0;
      }
    }
    // ring slots hold the differences in order slot = (iteration - 1) % H; gamma is in Gram order
    // (slot order), which the update uses directly
    OMEN_CUDA(ctx, cudaMemcpyAsync(gam.p, gamma.data(), sizeof(double) * 8, cudaMemcpyHostToDevice, ctx->stream));
    anderson_kernel<<<gg, 256, 0, ctx->stream>>>(phi, Fcur.d(), dXh.d(), dFh.d(), ng, h, gam.d(), d->mix, ng);
  }
  cudaError_t e = cudaStreamSynchronize(ctx->stream);
  free_hams();
  inf->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  if (st != OMEN_OK) return st;
  if (e != cudaSuccess) return set_err(ctx, OMEN_ECUDA, "SCF: %s", cudaGetErrorString(e));
  if (!inf->converged) return set_err(ctx, OMEN_ENOCONV, "SCF not converged after %d iterations (dV %.3e V)", d->max_iter, inf->dV_inf);
  return OMEN_OK;
}
