// Newton–Raphson solution of the nonlinear Poisson equation (paper Section III-A item 3: the
// converged potential profile of the Poisson solver is obtained iteratively by Newton–Raphson).
//
// Within one outer Schrödinger–Poisson iteration the eigenstates computed in the potential
// phi_in are frozen and the electrons respond to a change of potential by a local shift of the
// levels (the predictor of Trellakis et al., J. Appl. Phys. 81, 7880 (1997)):
//
//   n_i(phi) = sum_n W_ni f((E_n - u_i - E_F) / kT),   u_i = (G phi)_i - (G phi_in)_i,
//
// W_ni the electrons state n puts on atom i when full, G the trilinear (cloud-in-cell) gather of
// the grid potential to the atoms.  The nonlinear Poisson equation on the interior unknowns,
//
//   F(phi) = L phi - (rho_D - (q / V_cell) G^T n(phi)) / eps = 0,
//
// has the symmetric positive definite Jacobian J = L + (q / (eps V_cell)) G^T diag(s) G with
// s_i = sum_n W_ni f (1 - f) / kT.  Each Newton step solves J d = -F by conjugate gradients in
// one cooperative launch; J is applied without forming it: gather the direction to the atoms,
// scale by s, and deposit back through the transposed map (node -> (atom, weight) lists built
// once per call, so every sum runs in a fixed order and the result is reproducible).
#include <cooperative_groups.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <type_traits>
#include <vector>

#include "cic.cuh"
#include "fd.cuh"
#include "omen_internal.h"

namespace cgr = cooperative_groups;

namespace {

constexpr double kQ = 1.602176634e-19;  // C

// atom -> its 8 interior unknowns (or -1 on a grounded plane) and trilinear weights
__global__ void cic_map_kernel(Geo g, double a_nm, GridGeo G, int* __restrict__ node, double* __restrict__ w) {
  const long long plane = (long long)G.nx * G.ny;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < g.natoms; i += gridDim.x * blockDim.x) {
    double p[3];
    atom_position(g, a_nm, i, p);
    long long idx[8];
    double wt[8];
    cic(G, p, idx, wt);
    for (int c = 0; c < 8; ++c) {
      const long long k = idx[c] / plane;
      const bool interior = k >= 1 && k <= G.nz - 1;
      node[(size_t)i * 8 + c] = interior ? (int)(idx[c] - plane) : -1;
      w[(size_t)i * 8 + c] = wt[c];
    }
  }
}

__device__ __forceinline__ double gather_at(const int* __restrict__ node, const double* __restrict__ w,
                                            const double* __restrict__ v, int i) {
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const int j = node[(size_t)i * 8 + c];
    if (j >= 0) s += w[(size_t)i * 8 + c] * v[j];
  }
  return s;
}

__device__ __forceinline__ double deposit_at(const int* __restrict__ col_ptr, const int* __restrict__ col_atom,
                                             const double* __restrict__ col_w, const double* __restrict__ a, long long j) {
  double s = 0.0;
  for (int e = col_ptr[j]; e < col_ptr[j + 1]; ++e) s += col_w[e] * a[col_atom[e]];
  return s;
}

__global__ void gather_map_kernel(int natoms, const int* __restrict__ node, const double* __restrict__ w,
                                  const double* __restrict__ phi, double* __restrict__ out) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < natoms; i += gridDim.x * blockDim.x)
    out[i] = gather_at(node, w, phi, i);
}

__device__ __forceinline__ double fermi(double x) {  // 1 / (1 + e^x), no overflow
  if (x > 0.0) {
    const double e = exp(-x);
    return e / (1.0 + e);
  }
  return 1.0 / (1.0 + exp(x));
}

// predicted electrons n_i and their response s_i = dn_i/du_i at the current potential
__global__ void predict_kernel(int natoms, const int* __restrict__ node, const double* __restrict__ w,
                               const double* __restrict__ phi, const double* __restrict__ u_in, int nst,
                               const double* __restrict__ E, const double* __restrict__ W, double EF, double kT,
                               double* __restrict__ n_out, double* __restrict__ s_out) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < natoms; i += gridDim.x * blockDim.x) {
    const double u = gather_at(node, w, phi, i) - u_in[i];
    double n = 0.0, s = 0.0;
    for (int st = 0; st < nst; ++st) {
      const double wi = W[(size_t)st * natoms + i];
      if (wi == 0.0) continue;
      const double f = fermi((E[st] - u - EF) / kT);
      n += wi * f;
      s += wi * f * (1.0 - f);
    }
    n_out[i] = n;
    s_out[i] = s / kT;
  }
}

struct NewtonArgs {
  PGrid g;
  int natoms;
  const int* node;
  const double* w;
  const int* col_ptr;
  const int* col_atom;
  const double* col_w;
};

// b = -F(phi) = (rho_D - (q / V) G^T n) / eps - L phi
__global__ void rhs_kernel(NewtonArgs A, const double* __restrict__ phi, const double* __restrict__ rho_d,
                           const double* __restrict__ n_atom, double q_over_vol, double inv_eps, double* __restrict__ b,
                           double* __restrict__ part) {
  double m = 0.0;
  for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < A.g.n; j += (long long)gridDim.x * blockDim.x) {
    const double rho = rho_d[j] - q_over_vol * deposit_at(A.col_ptr, A.col_atom, A.col_w, n_atom, j);
    const double v = inv_eps * rho - stencil(phi, A.g, j);
    b[j] = v;
    m = fmax(m, fabs(v));
  }
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

struct JcgOut {
  int iterations;
  int converged;
  double rel;
};

// CG on J d = b from d = 0, one cooperative launch; q = J p needs the atoms' t = s (G p) first
// (a grid barrier between the gather and the deposit), four barriers per iteration in all.
__global__ void __launch_bounds__(256) jcg_kernel(NewtonArgs A, const double* __restrict__ s_atom, double kappa,
                                                  const double* __restrict__ b, double* __restrict__ d,
                                                  double* __restrict__ r, double* __restrict__ p,
                                                  double* __restrict__ q, double* __restrict__ t,
                                                  double* __restrict__ part, double rtol, int max_iter,
                                                  JcgOut* __restrict__ out) {
  cgr::grid_group grid = cgr::this_grid();
  __shared__ double sh[32];
  const long long n = A.g.n;
  const long long t0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long stride = (long long)gridDim.x * blockDim.x;
  double* part0 = part;
  double* part1 = part + gridDim.x;
  double lrr = 0.0;
  for (long long i = t0; i < n; i += stride) {
    const double bi = b[i];
    d[i] = 0.0;
    r[i] = bi;
    p[i] = bi;
    lrr += bi * bi;
  }
  double v = block_sum(lrr, sh);
  if (threadIdx.x == 0) part0[blockIdx.x] = v;
  grid.sync();
  double rr = grid_total(part0, sh);
  const double bb = rr;
  const double stop = rtol * rtol * bb;
  int it = 0;
  while (rr > stop && it < max_iter && bb > 0.0) {
    for (long long i = t0; i < A.natoms; i += stride) t[i] = s_atom[i] * gather_at(A.node, A.w, p, (int)i);
    grid.sync();
    double lpq = 0.0;
    for (long long j = t0; j < n; j += stride) {
      const double qj = stencil(p, A.g, j) + kappa * deposit_at(A.col_ptr, A.col_atom, A.col_w, t, j);
      q[j] = qj;
      lpq += p[j] * qj;
    }
    v = block_sum(lpq, sh);
    if (threadIdx.x == 0) part0[blockIdx.x] = v;
    grid.sync();
    const double alpha = rr / grid_total(part0, sh);
    double lr = 0.0;
    for (long long j = t0; j < n; j += stride) {
      d[j] += alpha * p[j];
      const double rj = r[j] - alpha * q[j];
      r[j] = rj;
      lr += rj * rj;
    }
    v = block_sum(lr, sh);
    if (threadIdx.x == 0) part1[blockIdx.x] = v;
    grid.sync();
    const double rr_new = grid_total(part1, sh);
    const double beta = rr_new / rr;
    rr = rr_new;
    for (long long j = t0; j < n; j += stride) p[j] = r[j] + beta * p[j];
    grid.sync();
    ++it;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    out->iterations = it;
    out->converged = (rr <= stop) || bb == 0.0;
    out->rel = bb > 0.0 ? sqrt(rr / bb) : 0.0;
  }
}

__global__ void step_kernel(double* __restrict__ phi, const double* __restrict__ d, long long n,
                            double* __restrict__ part) {
  double m = 0.0;
  for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (long long)gridDim.x * blockDim.x) {
    phi[j] += d[j];
    m = fmax(m, fabs(d[j]));
  }
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

// W[n][i] = weight[n] * sum_o |psi_n(o * natoms + i)|^2
template <bool C>
__global__ void state_weight_kernel(const void* __restrict__ psiv, long long nrows, int natoms, int nb, int nst,
                                    const double* __restrict__ weight, double* __restrict__ W) {
  using V = std::conditional_t<C, double2, double>;
  const V* psi = static_cast<const V*>(psiv);
  const long long total = (long long)nst * natoms;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
    const int st = (int)(e / natoms), i = (int)(e - (long long)st * natoms);
    double a = 0.0;
    for (int o = 0; o < nb; ++o) {
      const V v = psi[(size_t)st * nrows + (size_t)o * natoms + i];
      if constexpr (C) a += v.x * v.x + v.y * v.y; else a += v * v;
    }
    W[e] = weight[st] * a;
  }
}

template <typename F>
struct Cleanup {
  F f;
  ~Cleanup() { f(); }
};
template <typename F> Cleanup<F> make_cleanup(F f) { return Cleanup<F>{f}; }

}  // namespace

extern "C" omen_status omen_state_weights(omen_ctx* ctx, const omen_ham* h, const void* psi, int nstates,
                                          const double* weight_host, double* W) {
  if (!ctx || !h || !psi || !weight_host || !W || nstates < 0) return set_err(ctx, OMEN_EINVAL, "null argument");
  if (h->effmass || !h->lat) return set_err(ctx, OMEN_EUNSUPPORTED, "state weights need a tight-binding Hamiltonian");
  if (nstates == 0) return OMEN_OK;
  double* dw = nullptr;
  if (cudaMallocAsync(&dw, sizeof(double) * nstates, ctx->stream) != cudaSuccess) {
    cudaGetLastError();
    return set_err(ctx, OMEN_ENOMEM, "state weights");
  }
  cudaError_t e = cudaMemcpyAsync(dw, weight_host, sizeof(double) * nstates, cudaMemcpyHostToDevice, ctx->stream);
  const int N = h->lat->natoms;
  const long long total = (long long)nstates * N;
  const unsigned grid = (unsigned)std::min<long long>(4096, (total + 255) / 256);
  if (e == cudaSuccess) {
    if (h->is_complex) state_weight_kernel<true><<<grid, 256, 0, ctx->stream>>>(psi, h->nrows, N, h->nb, nstates, dw, W);
    else state_weight_kernel<false><<<grid, 256, 0, ctx->stream>>>(psi, h->nrows, N, h->nb, nstates, dw, W);
    e = cudaGetLastError();
  }
  cudaFreeAsync(dw, ctx->stream);
  if (e != cudaSuccess) return set_err(ctx, OMEN_ECUDA, "state weights: %s", cudaGetErrorString(e));
  return OMEN_OK;
}

extern "C" omen_status omen_poisson_newton(omen_ctx* ctx, const omen_lattice* L, const omen_grid* gr,
                                           const omen_frozen_states* fs, const double* rho_d, double* phi,
                                           const omen_newton_opts* o, omen_newton_info* info) {
  if (!ctx || !L || !gr || !fs || !rho_d || !phi || !o) return set_err(ctx, OMEN_EINVAL, "null argument");
  if (gr->nx < 1 || gr->ny < 1 || gr->nz < 2 || !(gr->Lx_nm > 0 && gr->Ly_nm > 0 && gr->Lz_nm > 0 && gr->eps_r > 0))
    return set_err(ctx, OMEN_EINVAL, "invalid grid");
  if (fs->nstates < 0 || (fs->nstates > 0 && (!fs->E_host || !fs->W_dev)) || !fs->phi_in_dev || !(fs->kT > 0))
    return set_err(ctx, OMEN_EINVAL, "invalid frozen states");
  if (!(o->tol_V > 0) || o->max_iter < 1 || !(o->cg.rtol > 0) || o->cg.max_iter < 1)
    return set_err(ctx, OMEN_EINVAL, "invalid Newton options");
  const long long n = (long long)gr->nx * gr->ny * (gr->nz - 1);
  if (n >= (1ll << 31)) return set_err(ctx, OMEN_EINVAL, "grid larger than 2^31 unknowns");
  OMEN_CUDA(ctx, cudaSetDevice(ctx->device));
  const auto t0 = std::chrono::steady_clock::now();
  const int N = L->natoms;
  const GridGeo G = grid_geo(gr);
  cudaStream_t st = ctx->stream;

  // per-call work: maps, atom arrays, CG vectors (freed on every exit path)
  std::vector<void*> bufs;
  auto cleanup = make_cleanup([&]() {
    for (void* b : bufs)
      if (b) cudaFreeAsync(b, st);
  });
  auto alloc = [&](size_t bytes) -> void* {
    void* p = nullptr;
    if (cudaMallocAsync(&p, std::max<size_t>(bytes, 8), st) != cudaSuccess) {
      cudaGetLastError();
      p = nullptr;
    }
    bufs.push_back(p);                 // a null entry marks the failure below
    return p;
  };
  int* node = static_cast<int*>(alloc(sizeof(int) * 8 * (size_t)N));
  double* wgt = static_cast<double*>(alloc(sizeof(double) * 8 * (size_t)N));
  double* u_in = static_cast<double*>(alloc(sizeof(double) * N));
  double* n_atom = static_cast<double*>(alloc(sizeof(double) * N));
  double* s_atom = static_cast<double*>(alloc(sizeof(double) * N));
  double* t_atom = static_cast<double*>(alloc(sizeof(double) * N));
  double* vec = static_cast<double*>(alloc(sizeof(double) * 5 * (size_t)n));
  double* dE = static_cast<double*>(alloc(sizeof(double) * std::max(1, fs->nstates)));
  JcgOut* jout = static_cast<JcgOut*>(alloc(sizeof(JcgOut)));
  int* col_ptr = static_cast<int*>(alloc(sizeof(int) * (size_t)(n + 1)));
  int* col_atom = static_cast<int*>(alloc(sizeof(int) * 8 * (size_t)N));
  double* col_w = static_cast<double*>(alloc(sizeof(double) * 8 * (size_t)N));
  int dev_sms = 0, per_sm = 0;
  cudaDeviceGetAttribute(&dev_sms, cudaDevAttrMultiProcessorCount, ctx->device);
  OMEN_CUDA(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, jcg_kernel, 256, 0));
  const int blocks = (int)std::max<long long>(1, std::min<long long>(std::max<long long>((n + 255) / 256, (N + 255) / 256),
                                                                       (long long)dev_sms * std::max(1, per_sm)));
  double* part = static_cast<double*>(alloc(sizeof(double) * 2 * (size_t)std::max(blocks, 4096)));
  for (void* b : bufs)
    if (!b) return set_err(ctx, OMEN_ENOMEM, "Newton work buffers");
  double* b_vec = vec;
  double* d_vec = vec + n;
  double* r_vec = vec + 2 * n;
  double* p_vec = vec + 3 * n;
  double* q_vec = vec + 4 * n;
  if (fs->nstates > 0)
    OMEN_CUDA(ctx, cudaMemcpyAsync(dE, fs->E_host, sizeof(double) * fs->nstates, cudaMemcpyHostToDevice, st));

  // maps: atom -> nodes on the device; node -> atoms (transposed, ascending atom) on the host
  const unsigned ga = (unsigned)std::min(4096, (N + 255) / 256);
  cic_map_kernel<<<ga, 256, 0, st>>>(lat_geo(L), L->a_nm, G, node, wgt);
  OMEN_CHECK_LAUNCH(ctx);
  {
    std::vector<int> hn(8 * (size_t)N);
    std::vector<double> hw(8 * (size_t)N);
    OMEN_CUDA(ctx, cudaMemcpyAsync(hn.data(), node, sizeof(int) * hn.size(), cudaMemcpyDeviceToHost, st));
    OMEN_CUDA(ctx, cudaMemcpyAsync(hw.data(), wgt, sizeof(double) * hw.size(), cudaMemcpyDeviceToHost, st));
    OMEN_CUDA(ctx, cudaStreamSynchronize(st));
    std::vector<int> cp(n + 1, 0), ca;
    std::vector<double> cw;
    for (size_t e = 0; e < hn.size(); ++e)
      if (hn[e] >= 0) ++cp[hn[e] + 1];
    for (long long j = 0; j < n; ++j) cp[j + 1] += cp[j];
    ca.resize(cp[n]);
    cw.resize(cp[n]);
    std::vector<int> fill(cp.begin(), cp.end() - 1);
    for (size_t e = 0; e < hn.size(); ++e)
      if (hn[e] >= 0) {
        const int pos = fill[hn[e]]++;
        ca[pos] = (int)(e / 8);
        cw[pos] = hw[e];
      }
    OMEN_CUDA(ctx, cudaMemcpyAsync(col_ptr, cp.data(), sizeof(int) * cp.size(), cudaMemcpyHostToDevice, st));
    if (!ca.empty()) {
      OMEN_CUDA(ctx, cudaMemcpyAsync(col_atom, ca.data(), sizeof(int) * ca.size(), cudaMemcpyHostToDevice, st));
      OMEN_CUDA(ctx, cudaMemcpyAsync(col_w, cw.data(), sizeof(double) * cw.size(), cudaMemcpyHostToDevice, st));
    }
    OMEN_CUDA(ctx, cudaStreamSynchronize(st));   // the host vectors go out of scope here
  }
  NewtonArgs A;
  A.g.nx = gr->nx;
  A.g.ny = gr->ny;
  A.g.nzi = gr->nz - 1;
  const double hx = G.hx * 1e-9, hy = G.hy * 1e-9, hz = G.hz * 1e-9;
  A.g.cx = gr->nx > 1 ? 1.0 / (hx * hx) : 0.0;
  A.g.cy = gr->ny > 1 ? 1.0 / (hy * hy) : 0.0;
  A.g.cz = 1.0 / (hz * hz);
  A.g.n = n;
  A.natoms = N;
  A.node = node;
  A.w = wgt;
  A.col_ptr = col_ptr;
  A.col_atom = col_atom;
  A.col_w = col_w;
  const double eps = kEps0 * gr->eps_r;
  const double q_over_vol = kQ / G.vol_m3;
  double kappa = kQ / (eps * G.vol_m3);
  const double inv_eps = 1.0 / eps;

  gather_map_kernel<<<ga, 256, 0, st>>>(N, node, wgt, fs->phi_in_dev, u_in);
  OMEN_CHECK_LAUNCH(ctx);
  const unsigned gn = (unsigned)std::min<long long>(1024, (n + 255) / 256);
  std::vector<double> hp(std::max<unsigned>(gn, 1));
  int it = 0;
  bool converged = false;
  double last = 0.0;
  long long cg_total = 0;
  double rtol = o->cg.rtol;
  int cg_max = o->cg.max_iter;
  while (it < o->max_iter) {
    predict_kernel<<<ga, 256, 0, st>>>(N, node, wgt, phi, u_in, fs->nstates, dE, fs->W_dev, fs->E_F, fs->kT, n_atom,
                                       s_atom);
    rhs_kernel<<<gn, 256, 0, st>>>(A, phi, rho_d, n_atom, q_over_vol, inv_eps, b_vec, part);
    OMEN_CHECK_LAUNCH(ctx);
    void* args[] = {&A, &s_atom, &kappa, &b_vec, &d_vec, &r_vec, &p_vec, &q_vec, &t_atom, &part, &rtol, &cg_max, &jout};
    OMEN_CUDA(ctx, cudaLaunchCooperativeKernel((const void*)jcg_kernel, dim3(blocks), dim3(256), args, 0, st));
    step_kernel<<<gn, 256, 0, st>>>(phi, d_vec, n, part);
    OMEN_CHECK_LAUNCH(ctx);
    JcgOut ho{};
    OMEN_CUDA(ctx, cudaMemcpyAsync(&ho, jout, sizeof(JcgOut), cudaMemcpyDeviceToHost, st));
    OMEN_CUDA(ctx, cudaMemcpyAsync(hp.data(), part, sizeof(double) * gn, cudaMemcpyDeviceToHost, st));
    OMEN_CUDA(ctx, cudaStreamSynchronize(st));
    ++it;
    cg_total += ho.iterations;
    last = 0.0;
    for (unsigned b = 0; b < gn; ++b) last = std::max(last, hp[b]);
    if (!std::isfinite(last)) return set_err(ctx, OMEN_ENUMERIC, "Newton step is not finite");
    if (!ho.converged)
      return set_err(ctx, OMEN_ENOCONV, "Newton step %d: CG stopped at %d iterations (rel %.3e)", it, ho.iterations, ho.rel);
    if (last < o->tol_V) {
      converged = true;
      break;
    }
  }
  if (info) {
    info->iterations = it;
    info->converged = converged ? 1 : 0;
    info->last_step_V = last;
    info->cg_iterations = cg_total;
    info->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
  if (!converged) return set_err(ctx, OMEN_ENOCONV, "Newton-Raphson stopped at %d steps, last step %.3e V", it, last);
  return OMEN_OK;
}
