// Charge from eigenstates, grid deposit and gather, Fermi level (paper Section III-A item 2:
// the charge profile from filling the states at a given Fermi level, or charge and Fermi level
// together under charge neutrality).
#include <algorithm>
#include <cmath>
#include <type_traits>
#include <vector>

#include "omen_internal.h"
#include "sk_device.cuh"
#include "vec.cuh"
#include "cic.cuh"
#include "df.cuh"

// n_atom[i] += w * sum_n occ[n] * sum_o |psi_n[o*N + i]|^2
//
// The squares are summed on the FP32 pipe in double-float arithmetic (GB300's FP64 rate would
// otherwise bound the kernel, one FP64 FMA per 8-byte amplitude).  Each FP64 amplitude v is
// split, scaled by 2^32 (exact), into FP32 parts with integer operations only: hi keeps the
// sign, the exponent and the leading 24 significant bits, lo is the rest rounded to FP32 (48
// significant bits in all).  v^2 2^64 is then hi^2 (the FP32 product plus its exact FMA error)
// + 2 hi lo + lo^2, the terms added with TwoSum into an FP32 pair (about 1e-14 relative).  The
// scaling keeps amplitudes in [2^-83, 2^32) clear of FP32 underflow and overflow; smaller ones
// (contributing below 2^-166) count as zero, and so do occupations below 2^-126.  Infinite or
// NaN amplitudes (and finite ones of 2^96 or more) give NaN.
template <int kSplitShift>
__device__ __forceinline__ float2 split_fp64(double v) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  const unsigned hi32 = (unsigned)(b >> 32), lo32 = (unsigned)b;
  const int e = (int)((hi32 >> 20) & 0x7FFu);   // biased FP64 exponent
  // FP32 exponent of hi: e - 1023 + 127 + shift
  const int eh = e - 896 + kSplitShift;
  if (eh <= 0) return make_float2(0.f, 0.f);     // |v| < 2^-158, or zero
  if (eh >= 255) return make_float2(__int_as_float(0x7fc00000), 0.f);   // beyond FP32, inf or NaN: NaN
  const unsigned sign = hi32 & 0x80000000u;
  const unsigned top23 = ((hi32 & 0xFFFFFu) << 3) | (lo32 >> 29);
  const float hi = __uint_as_float(sign | ((unsigned)eh << 23) | top23);
  // the remaining 29 bits: rem * 2^(e - 1075 + shift)
  const unsigned rem = lo32 & 0x1FFFFFFFu;
  const int el = e - 948 + kSplitShift;
  const float scale = el > 0 ? __uint_as_float((unsigned)el << 23) : 0.f;
  const float lo = __fmul_rn(__uint2float_rn(rem), scale);
  return make_float2(hi, sign ? -lo : lo);
}

__device__ __forceinline__ void df_add_square(float& S, float& Cc, double v) {
  const float2 h = split_fp64<32>(v);
  const float p = __fmul_rn(h.x, h.x);
  float e = __fmaf_rn(h.x, h.x, -p);
  e = __fmaf_rn(__fmul_rn(2.f, h.x), h.y, e);
  e = __fmaf_rn(h.y, h.y, e);
  const float s = __fadd_rn(S, p);
  const float bb = __fsub_rn(s, S);
  const float t = __fadd_rn(__fsub_rn(S, __fsub_rn(s, bb)), __fsub_rn(p, bb));
  Cc = __fadd_rn(Cc, __fadd_rn(t, e));
  S = s;
}

template <bool C, int NB>
__global__ void __launch_bounds__(256) density_kernel(const void* __restrict__ psiv, long long nrows, int natoms,
                                                      int nb_rt, int nstates, const double* __restrict__ occ,
                                                      double w, double* __restrict__ n_atom) {
  using E = Elem<double, C>;
  const typename E::V* psi = static_cast<const typename E::V*>(psiv);
  const int nb = NB > 0 ? NB : nb_rt;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < natoms; i += gridDim.x * blockDim.x) {
    float AS = 0.f, AC = 0.f;   // sum over states of occ * (state's sum of squares)
    for (int s = 0; s < nstates; ++s) {
      const double f = occ[s];
      if (f == 0.0) continue;
      const typename E::V* ps = psi + (size_t)s * nrows + i;
      float S = 0.f, Cc = 0.f;
      if constexpr (NB > 0) {
        typename E::V v[NB];
#pragma unroll
        for (int o = 0; o < NB; ++o) v[o] = ps[(size_t)o * natoms];
#pragma unroll
        for (int o = 0; o < NB; ++o) {
          df_add_square(S, Cc, E::re(v[o]));
          if constexpr (C) df_add_square(S, Cc, E::im(v[o]));
        }
      } else {
        for (int o = 0; o < nb; ++o) {
          const typename E::V v = ps[(size_t)o * natoms];
          df_add_square(S, Cc, E::re(v));
          if constexpr (C) df_add_square(S, Cc, E::im(v));
        }
      }
      df_mac(AS, AC, df_norm(S, Cc), split_fp64<0>(f));
    }
    // the squares carry the factor 2^64 of the split
    n_atom[i] += w * (((double)AS + (double)AC) * 0x1p-64);
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
  // one thread per atom, the grid a whole number of waves of 152-SM-sized blocks
  const unsigned grid = (unsigned)std::max(1, std::min((N + 255) / 256, 152 * 8));
  auto launch = [&](auto cplx, auto nbc) {
    constexpr bool Cx = decltype(cplx)::value;
    constexpr int NB = decltype(nbc)::value;
    density_kernel<Cx, NB><<<grid, 256, 0, ctx->stream>>>(psi, h->nrows, N, h->nb, nstates, d_occ, w, n_atom);
  };
  using T_ = std::true_type;
  using F_ = std::false_type;
  using I1 = std::integral_constant<int, 1>;
  using I5 = std::integral_constant<int, 5>;
  using I10 = std::integral_constant<int, 10>;
  using I20 = std::integral_constant<int, 20>;
  using I0 = std::integral_constant<int, 0>;
  if (h->is_complex) {
    if (h->nb == 1) launch(T_{}, I1{});
    else if (h->nb == 5) launch(T_{}, I5{});
    else if (h->nb == 10) launch(T_{}, I10{});
    else if (h->nb == 20) launch(T_{}, I20{});
    else launch(T_{}, I0{});
  } else {
    if (h->nb == 1) launch(F_{}, I1{});
    else if (h->nb == 5) launch(F_{}, I5{});
    else if (h->nb == 10) launch(F_{}, I10{});
    else if (h->nb == 20) launch(F_{}, I20{});
    else launch(F_{}, I0{});
  }
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
