// Device-side Hamiltonian assembly (paper Section I: sp3s*/sp3d5s* tight binding with strain).
//
// 1. b0 table: the Slater–Koster block of every (species pair, bond direction) at d0,
//    from the Table I integrals (sk_device.cuh).
// 2. bond blocks: each existing bond slot gets (d0/d)^eta * b0[pair][dir], d = d0 (1 + strain),
//    stored in tiles of 32 consecutive slots with the entries of a tile contiguous
//    (blk[(tile*ne + e)*32 + lane]): a warp reads 32 slots of one entry with one coalesced
//    128-byte load, and one bond block of a warp is a single contiguous run.  Matrix-free Hamiltonians skip this step and H·X
//    regenerates the block from the b0 table, the two species and the strain.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "omen_internal.h"
#include "sk_device.cuh"

__constant__ int c_dir[4][3] = {{1, 1, 1}, {1, -1, -1}, {-1, 1, -1}, {-1, -1, 1}};

__global__ void b0_table_kernel(const double* __restrict__ V, int ns, int norb, double* __restrict__ b0,
                                float* __restrict__ b0_32) {
  const int total = ns * ns * 4 * norb * norb;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= total) return;
  const int e = t % (norb * norb);
  const int k = (t / (norb * norb)) % 4;
  const int pair = t / (norb * norb * 4);
  const int sa = pair / ns, sb = pair % ns;
  const double inv = 0.57735026918962576;  // 1/sqrt(3)
  const double c[3] = {c_dir[k][0] * inv, c_dir[k][1] * inv, c_dir[k][2] * inv};
  const int o1 = e / norb, o2 = e % norb;
  const double v = sk_element(sk_code(o1, norb), sk_code(o2, norb), c, V + (sa * ns + sb) * 14, V + (sb * ns + sa) * 14);
  b0[t] = v;
  b0_32[t] = (float)v;
}

__global__ void assemble_bonds_kernel(Geo g, NeighbourTables nt, const uint8_t* __restrict__ species,
                                      const double* __restrict__ strain, const double* __restrict__ b0,
                                      int ns, int norb, double eta, int slot_stride, double* __restrict__ blk64,
                                      float* __restrict__ blk32, float2* __restrict__ blkdf) {
  const int npad = 16 * slot_stride;
  const int pidx = blockIdx.x * blockDim.x + threadIdx.x;   // padded slot index
  if (pidx >= npad) return;
  const int cell = pidx % slot_stride;
  const int ks = pidx / slot_stride;  // k*4 + s
  const int ne = norb * norb;
  const size_t base = ((size_t)(pidx >> 5) * ne) * 32 + (pidx & 31);
  if (cell >= g.ncells) {  // padding
    for (int e = 0; e < ne; ++e) {
      if (blk64) blk64[base + (size_t)e * 32] = 0.0;
      if (blk32) blk32[base + (size_t)e * 32] = 0.0f;
      if (blkdf) blkdf[base + (size_t)e * 32] = make_float2(0.f, 0.f);
    }
    return;
  }
  const int slot = ks * g.ncells + cell;  // strain input layout
  const int k = ks >> 2, s = ks & 3;
  const int ix = cell % g.nx, iy = (cell / g.nx) % g.ny, iz = cell / (g.nx * g.ny);
  int cell2, wrap[3];
  const bool ok = shift_cell(g, ix, iy, iz, nt.a_to_b_off[s][k][0], nt.a_to_b_off[s][k][1], nt.a_to_b_off[s][k][2],
                             cell2, wrap);
  if (!ok) {
    for (int e = 0; e < ne; ++e) {
      if (blk64) blk64[base + (size_t)e * 32] = 0.0;
      if (blk32) blk32[base + (size_t)e * 32] = 0.0f;
      if (blkdf) blkdf[base + (size_t)e * 32] = make_float2(0.f, 0.f);
    }
    return;
  }
  const int sa = species[s * g.ncells + cell];
  const int sb = species[nt.a_to_b_site[s][k] * g.ncells + cell2];
  const double f = pow(1.0 + strain[slot], -eta);
  const double* tb = b0 + ((size_t)(sa * ns + sb) * 4 + k) * ne;
  for (int e = 0; e < ne; ++e) {
    const double v = f * tb[e];
    if (blk64) blk64[base + (size_t)e * 32] = v;
    if (blk32) blk32[base + (size_t)e * 32] = (float)v;
    if (blkdf) {
      const float hi = __double2float_rn(v);
      blkdf[base + (size_t)e * 32] = make_float2(hi, __double2float_rn(v - (double)hi));
    }
  }
}

// Matrix-free Hamiltonians: the bond-length factor (d0/d)^eta of every slot, d = d0 (1 + strain),
// kept in both precisions (the product regenerates each block as factor x b0[pair][dir]).
__global__ void mf_scale_kernel(const double* __restrict__ strain, long long nslots, double eta,
                                double* __restrict__ s64, float* __restrict__ s32) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nslots; i += (long long)gridDim.x * blockDim.x) {
    const double f = pow(1.0 + strain[i], -eta);
    s64[i] = f;
    s32[i] = (float)f;
  }
}

__global__ void max_species_kernel(const uint8_t* __restrict__ sp, int n, int* __restrict__ out) {
  int m = 0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) m = max(m, (int)sp[i]);
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, m);
}

static void free_ham_buffers(omen_ham* h) {
  cudaFree(h->d_blk64);
  cudaFree(h->d_blk32);
  cudaFree(h->d_blkdf);
  cudaFree(h->d_b0_64);
  cudaFree(h->d_b0_32);
  cudaFree(h->d_scale64);
  cudaFree(h->d_scale32);
  cudaFree(h->d_onsite);
  cudaFree(h->d_onsite32);
  cudaFree(h->d_onsite_df);
  cudaFree(h->d_U);
  cudaFree(h->d_U32);
  cudaFree(h->d_lambda);
}

extern "C" void omen_free_ham(omen_ham* h) {
  if (!h) return;
  free_ham_buffers(h);
  delete h;
}

#define ALLOC_OR_FAIL(ptr, bytes)                                                          \
  do {                                                                                     \
    if (cudaMalloc(&(ptr), (bytes)) != cudaSuccess) {                                      \
      cudaGetLastError();                                                                  \
      omen_free_ham(h);                                                                    \
      return set_err(ctx, OMEN_ENOMEM, "device allocation of %zu bytes failed", (size_t)(bytes)); \
    }                                                                                      \
  } while (0)

extern "C" omen_status omen_assemble_H(omen_ctx* ctx, const omen_lattice* lat, const omen_tb_params* p,
                                       const omen_ham_opts* opts, omen_ham** out) {
  if (!ctx || !lat || !p || !opts || !out) return set_err(ctx, OMEN_EINVAL, "null argument");
  *out = nullptr;
  if (p->basis != OMEN_SP3S && p->basis != OMEN_SP3D5S) return set_err(ctx, OMEN_EINVAL, "basis must be 5 or 10");
  if (p->nspecies < 1 || p->nspecies > 4) return set_err(ctx, OMEN_EINVAL, "nspecies must be 1..4");
  if (opts->precision < OMEN_F64 || opts->precision > OMEN_F64_DF)
    return set_err(ctx, OMEN_EINVAL, "unknown precision %d", opts->precision);
  if (opts->precision == OMEN_F64_DF && (opts->spin_orbit || opts->matrix_free || (opts->k && (lat->periodic[0] == OMEN_BLOCH || lat->periodic[1] == OMEN_BLOCH || lat->periodic[2] == OMEN_BLOCH))))
    return set_err(ctx, OMEN_EUNSUPPORTED, "double-float precision supports real stored Hamiltonians only");
  OMEN_CUDA(ctx, cudaSetDevice(ctx->device));
  {  // species indices must be < nspecies
    int* d_m = (int*)ctx->d_status;
    OMEN_CUDA(ctx, cudaMemsetAsync(d_m, 0, sizeof(int), ctx->stream));
    max_species_kernel<<<64, 256, 0, ctx->stream>>>(lat->d_species, lat->natoms, d_m);
    OMEN_CHECK_LAUNCH(ctx);
    int hm = 0;
    OMEN_CUDA(ctx, cudaMemcpyAsync(&hm, d_m, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    OMEN_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    if (hm >= p->nspecies) return set_err(ctx, OMEN_EINVAL, "species index %d >= nspecies %d", hm, p->nspecies);
  }
  auto* h = new omen_ham();
  h->lat = lat;
  h->norb = p->basis;
  h->spin_orbit = opts->spin_orbit ? 1 : 0;
  h->nspin = h->spin_orbit ? 2 : 1;
  h->nb = h->norb * h->nspin;
  h->precision = opts->precision;
  h->matrix_free = opts->matrix_free ? 1 : 0;
  h->nspecies = p->nspecies;
  h->eta = p->eta;
  h->nrows = (long long)h->nb * lat->natoms;
  h->bloch = 0;
  if (opts->k) {
    for (int d = 0; d < 3; ++d) h->kvec[d] = opts->k[d];
    for (int d = 0; d < 3; ++d)
      if (lat->periodic[d] == OMEN_BLOCH) h->bloch = 1;
  }
  const int ncell_d[3] = {lat->nx, lat->ny, lat->nz};
  for (int d = 0; d < 3; ++d) {
    double ph = 0.0;
    if (lat->periodic[d] == OMEN_BLOCH) ph = h->kvec[d] * ncell_d[d] * lat->a_nm;
    h->phase[d] = make_double2(cos(ph), sin(ph));
  }
  h->is_complex = (h->spin_orbit || h->bloch) ? 1 : 0;
  for (int s = 0; s < 4; ++s) h->lambda_so[s] = p->lambda_so[s];

  const int ns = p->nspecies, norb = p->basis, ne = norb * norb;
  h->slot_stride = (lat->ncells + 31) / 32 * 32;
  const size_t nslots = 16 * (size_t)h->slot_stride;
  const size_t ntab = (size_t)ns * ns * 4 * ne;
  ALLOC_OR_FAIL(h->d_b0_64, ntab * sizeof(double));
  ALLOC_OR_FAIL(h->d_b0_32, ntab * sizeof(float));
  ALLOC_OR_FAIL(h->d_onsite, sizeof(double) * ns * norb);
  ALLOC_OR_FAIL(h->d_onsite32, sizeof(float) * ns * norb);
  ALLOC_OR_FAIL(h->d_U, sizeof(double) * lat->natoms);
  ALLOC_OR_FAIL(h->d_lambda, sizeof(double) * 4);
  const bool need64 = !h->matrix_free && (h->precision == OMEN_F64 || h->precision == OMEN_F32_REFINE64);
  const bool need32 = !h->matrix_free && (h->precision == OMEN_F32 || h->precision == OMEN_F32_REFINE64);
  const bool needdf = h->precision == OMEN_F64_DF;
  if (need64) ALLOC_OR_FAIL(h->d_blk64, sizeof(double) * ne * nslots);
  if (need32) ALLOC_OR_FAIL(h->d_blk32, sizeof(float) * ne * nslots);
  if (needdf) ALLOC_OR_FAIL(h->d_blkdf, sizeof(float2) * ne * nslots);
  if (h->matrix_free) {
    ALLOC_OR_FAIL(h->d_scale64, sizeof(double) * 16 * (size_t)lat->ncells);
    ALLOC_OR_FAIL(h->d_scale32, sizeof(float) * 16 * (size_t)lat->ncells);
  }

  // parameter tables
  std::vector<double> V(ns * ns * 14), on(ns * norb);
  for (int a = 0; a < ns; ++a)
    for (int b = 0; b < ns; ++b)
      for (int q = 0; q < 14; ++q) V[(a * ns + b) * 14 + q] = p->V[a][b][q];
  for (int a = 0; a < ns; ++a) {
    int o = 0;
    on[a * norb + o++] = p->onsite[a][0];
    for (int i = 0; i < 3; ++i) on[a * norb + o++] = p->onsite[a][1];
    if (norb == 10)
      for (int i = 0; i < 5; ++i) on[a * norb + o++] = p->onsite[a][2];
    on[a * norb + o++] = p->onsite[a][3];
  }
  double* d_V = nullptr;
  if (cudaMalloc(&d_V, sizeof(double) * V.size()) != cudaSuccess) {
    omen_free_ham(h);
    return set_err(ctx, OMEN_ENOMEM, "device allocation failed");
  }
  cudaError_t e = cudaMemcpyAsync(d_V, V.data(), sizeof(double) * V.size(), cudaMemcpyHostToDevice, ctx->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h->d_onsite, on.data(), sizeof(double) * on.size(), cudaMemcpyHostToDevice, ctx->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h->d_lambda, p->lambda_so, sizeof(double) * 4, cudaMemcpyHostToDevice, ctx->stream);
  std::vector<float> on32(on.begin(), on.end());
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h->d_onsite32, on32.data(), sizeof(float) * on32.size(), cudaMemcpyHostToDevice, ctx->stream);
  std::vector<float2> ondf(on.size());
  if (e == cudaSuccess && needdf) {
    for (size_t i = 0; i < on.size(); ++i) {
      const float hi = (float)on[i];
      ondf[i] = make_float2(hi, (float)(on[i] - (double)hi));
    }
    if (cudaMalloc(&h->d_onsite_df, sizeof(float2) * ondf.size()) != cudaSuccess) {
      cudaGetLastError();
      cudaFree(d_V);
      omen_free_ham(h);
      return set_err(ctx, OMEN_ENOMEM, "device allocation failed");
    }
    e = cudaMemcpyAsync(h->d_onsite_df, ondf.data(), sizeof(float2) * ondf.size(), cudaMemcpyHostToDevice, ctx->stream);
  }
  if (e == cudaSuccess) {
    if (opts->U_atom_dev)
      e = cudaMemcpyAsync(h->d_U, opts->U_atom_dev, sizeof(double) * lat->natoms, cudaMemcpyDeviceToDevice, ctx->stream);
    else
      e = cudaMemsetAsync(h->d_U, 0, sizeof(double) * lat->natoms, ctx->stream);
  }
  if (e == cudaSuccess) {
    b0_table_kernel<<<(unsigned)((ntab + 255) / 256), 256, 0, ctx->stream>>>(d_V, ns, norb, h->d_b0_64, h->d_b0_32);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && h->matrix_free) {
    const long long n = 16ll * lat->ncells;
    mf_scale_kernel<<<(unsigned)std::min<long long>((n + 255) / 256, 65535), 256, 0, ctx->stream>>>(
        lat->d_strain, n, p->eta, h->d_scale64, h->d_scale32);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && (need64 || need32 || needdf)) {
    Geo g{lat->nx, lat->ny, lat->nz, lat->ncells, lat->natoms, {lat->periodic[0], lat->periodic[1], lat->periodic[2]}};
    assemble_bonds_kernel<<<(unsigned)((nslots + 255) / 256), 256, 0, ctx->stream>>>(
        g, host_neighbour_tables(), lat->d_species, lat->d_strain, h->d_b0_64, ns, norb, p->eta,
        h->slot_stride, h->d_blk64, h->d_blk32, h->d_blkdf);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  cudaFree(d_V);
  if (e != cudaSuccess) {
    omen_free_ham(h);
    return set_err(ctx, OMEN_ECUDA, "assembly failed: %s", cudaGetErrorString(e));
  }
  *out = h;
  return OMEN_OK;
}

extern "C" omen_status omen_ham_shape(const omen_ham* h, long long* nrows, int* is_complex, int* elem_bytes) {
  if (!h) return OMEN_EINVAL;
  if (nrows) *nrows = h->nrows;
  if (is_complex) *is_complex = h->is_complex;
  if (elem_bytes) *elem_bytes = (int)vec_elem_bytes(h, h->precision);
  return OMEN_OK;
}

extern "C" omen_status omen_ham_set_potential(omen_ctx* ctx, omen_ham* h, const double* U) {
  if (!ctx || !h) return set_err(ctx, OMEN_EINVAL, "null argument");
  if (h->effmass) return effmass_set_potential(ctx, h, U);
  if (U)
    OMEN_CUDA(ctx, cudaMemcpyAsync(h->d_U, U, sizeof(double) * h->lat->natoms, cudaMemcpyDeviceToDevice, ctx->stream));
  else
    OMEN_CUDA(ctx, cudaMemsetAsync(h->d_U, 0, sizeof(double) * h->lat->natoms, ctx->stream));
  return OMEN_OK;
}
