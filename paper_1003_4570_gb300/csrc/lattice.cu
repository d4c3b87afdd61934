// Structure on the device: species per atom, strain per bond slot, implicit neighbours.
//
// Paper Section II-A keeps, per subdomain, the atoms and their neighbour atoms without
// global position lists.  On one GPU the whole block is resident and the neighbour of an
// atom is computed from its cell index and the zincblende site tables below, so no
// neighbour list is stored or read.
#include <cstdarg>
#include <cstring>
#include <mutex>

#include "omen_internal.h"

omen_status set_err(omen_ctx* ctx, omen_status s, const char* fmt, ...) {
  if (ctx) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    ctx->err = buf;
  }
  return s;
}

// Site positions in units of a/4: A sites, then B = A + (1,1,1).
static const int kSite[8][3] = {{0, 0, 0}, {0, 2, 2}, {2, 0, 2}, {2, 2, 0},
                                {1, 1, 1}, {1, 3, 3}, {3, 1, 3}, {3, 3, 1}};
static const int kDir[4][3] = {{1, 1, 1}, {1, -1, -1}, {-1, 1, -1}, {-1, -1, 1}};

static int floor_div4(int q) { return q >= 0 ? q / 4 : -((-q + 3) / 4); }

static int site_at(const int p[3]) {
  for (int b = 0; b < 8; ++b)
    if (kSite[b][0] == p[0] && kSite[b][1] == p[1] && kSite[b][2] == p[2]) return b;
  return -1;
}

static NeighbourTables build_tables() {
  NeighbourTables t{};
  for (int s = 0; s < 4; ++s)
    for (int k = 0; k < 4; ++k) {
      int q[3], off[3], loc[3];
      // from A site s along +dir k to a B site
      for (int d = 0; d < 3; ++d) {
        q[d] = kSite[s][d] + kDir[k][d];
        off[d] = floor_div4(q[d]);
        loc[d] = q[d] - 4 * off[d];
        t.a_to_b_off[s][k][d] = off[d];
      }
      t.a_to_b_site[s][k] = site_at(loc);
      // from B site 4+s along -dir k to an A site
      for (int d = 0; d < 3; ++d) {
        q[d] = kSite[4 + s][d] - kDir[k][d];
        off[d] = floor_div4(q[d]);
        loc[d] = q[d] - 4 * off[d];
        t.b_to_a_off[s][k][d] = off[d];
      }
      t.b_to_a_site[s][k] = site_at(loc);
    }
  return t;
}

const NeighbourTables& host_neighbour_tables() {
  static NeighbourTables t = build_tables();
  return t;
}

static bool slot_exists(const omen_lattice* L, int s, int k, int ix, int iy, int iz) {
  const NeighbourTables& t = host_neighbour_tables();
  const int i[3] = {ix, iy, iz}, n[3] = {L->nx, L->ny, L->nz};
  for (int d = 0; d < 3; ++d) {
    int j = i[d] + t.a_to_b_off[s][k][d];
    if ((j < 0 || j >= n[d]) && L->periodic[d] == OMEN_HARD_WALL) return false;
  }
  return true;
}

extern "C" omen_status omen_build_lattice(omen_ctx* ctx, const omen_lattice_desc* d, omen_lattice** out) {
  if (!ctx || !d || !out) return set_err(ctx, OMEN_EINVAL, "null argument");
  *out = nullptr;
  if (d->nx < 1 || d->ny < 1 || d->nz < 1) return set_err(ctx, OMEN_EINVAL, "cell counts must be >= 1");
  if ((long long)d->nx * d->ny * d->nz * 16 > (1ll << 31) - 1)
    return set_err(ctx, OMEN_EINVAL, "structure too large for 32-bit slot indices");
  for (int i = 0; i < 3; ++i)
    if (d->periodic[i] < 0 || d->periodic[i] > 2) return set_err(ctx, OMEN_EINVAL, "periodic[%d] invalid", i);
  if (!(d->a_nm > 0)) return set_err(ctx, OMEN_EINVAL, "a_nm must be > 0");
  if (!d->species_host) return set_err(ctx, OMEN_EINVAL, "species_host is required");
  OMEN_CUDA(ctx, cudaSetDevice(ctx->device));
  auto* L = new omen_lattice();
  L->nx = d->nx; L->ny = d->ny; L->nz = d->nz;
  L->ncells = d->nx * d->ny * d->nz;
  L->natoms = 8 * L->ncells;
  for (int i = 0; i < 3; ++i) L->periodic[i] = d->periodic[i];
  L->a_nm = d->a_nm;
  cudaError_t e1 = cudaMalloc(&L->d_species, (size_t)L->natoms);
  cudaError_t e2 = cudaMalloc(&L->d_strain, sizeof(double) * 16 * (size_t)L->ncells);
  if (e1 != cudaSuccess || e2 != cudaSuccess) {
    omen_free_lattice(L);
    return set_err(ctx, OMEN_ENOMEM, "device allocation for the structure failed");
  }
  cudaError_t e = cudaMemcpyAsync(L->d_species, d->species_host, L->natoms, cudaMemcpyHostToDevice, ctx->stream);
  if (e == cudaSuccess) {
    if (d->strain_host)
      e = cudaMemcpyAsync(L->d_strain, d->strain_host, sizeof(double) * 16 * (size_t)L->ncells,
                          cudaMemcpyHostToDevice, ctx->stream);
    else
      e = cudaMemsetAsync(L->d_strain, 0, sizeof(double) * 16 * (size_t)L->ncells, ctx->stream);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) {
    omen_free_lattice(L);
    return set_err(ctx, OMEN_ECUDA, "structure upload failed: %s", cudaGetErrorString(e));
  }
  long long nb = 0;
  for (int iz = 0; iz < L->nz; ++iz)
    for (int iy = 0; iy < L->ny; ++iy)
      for (int ix = 0; ix < L->nx; ++ix)
        for (int s = 0; s < 4; ++s)
          for (int k = 0; k < 4; ++k) nb += slot_exists(L, s, k, ix, iy, iz);
  L->nbonds = nb;
  *out = L;
  return OMEN_OK;
}

extern "C" void omen_free_lattice(omen_lattice* L) {
  if (!L) return;
  cudaFree(L->d_species);
  cudaFree(L->d_strain);
  delete L;
}

extern "C" omen_status omen_lattice_counts(const omen_lattice* L, long long* natoms, long long* nbonds) {
  if (!L) return OMEN_EINVAL;
  if (natoms) *natoms = L->natoms;
  if (nbonds) *nbonds = L->nbonds;
  return OMEN_OK;
}

extern "C" omen_status omen_lattice_set_strain(omen_ctx* ctx, omen_lattice* L, const double* strain_dev) {
  if (!ctx || !L || !strain_dev) return set_err(ctx, OMEN_EINVAL, "null argument");
  OMEN_CUDA(ctx, cudaMemcpyAsync(L->d_strain, strain_dev, sizeof(double) * 16 * (size_t)L->ncells,
                                 cudaMemcpyDeviceToDevice, ctx->stream));
  return OMEN_OK;
}
