// Cloud-in-cell (trilinear) weights between the atoms of a zincblende structure and the nodes
// of the finite-difference grid (paper Section III-A items 2-3: the charge of the atoms goes to
// the Poisson grid, the potential comes back to the atoms).  Shared by the deposit/gather
// kernels and the Newton–Raphson Poisson solver.
#pragma once

#include <cmath>

#include "omen_internal.h"
#include "sk_device.cuh"

struct GridGeo {
  int nx, ny, nz;
  double hx, hy, hz;        // nm
  double vol_m3;
};

__device__ __forceinline__ void atom_position(const Geo& g, double a_nm, int atom, double p[3]) {
  const int sites[8][3] = {{0, 0, 0}, {0, 2, 2}, {2, 0, 2}, {2, 2, 0}, {1, 1, 1}, {1, 3, 3}, {3, 1, 3}, {3, 3, 1}};
  const int b = atom / g.ncells, cell = atom % g.ncells;
  const int ix = cell % g.nx, iy = (cell / g.nx) % g.ny, iz = cell / (g.nx * g.ny);
  const double q = 0.25 * a_nm;
  p[0] = (4 * ix + sites[b][0]) * q;
  p[1] = (4 * iy + sites[b][1]) * q;
  p[2] = (4 * iz + sites[b][2]) * q;
}

// trilinear (cloud-in-cell) stencil: node index into the full (nz+1, ny, nx) node array
__device__ __forceinline__ void cic(const GridGeo& G, const double p[3], long long idx[8], double w[8]) {
  const double tx = p[0] / G.hx, ty = p[1] / G.hy, tz = p[2] / G.hz;
  const int i0 = (int)floor(tx), j0 = (int)floor(ty), k0 = (int)floor(tz);
  const double fx = tx - i0, fy = ty - j0, fz = tz - k0;
  int c = 0;
  for (int dz = 0; dz < 2; ++dz)
    for (int dy = 0; dy < 2; ++dy)
      for (int dx = 0; dx < 2; ++dx) {
        int ii = (i0 + dx) % G.nx;
        if (ii < 0) ii += G.nx;
        int jj = (j0 + dy) % G.ny;
        if (jj < 0) jj += G.ny;
        int kk = min(max(k0 + dz, 0), G.nz);
        idx[c] = ((long long)kk * G.ny + jj) * G.nx + ii;
        w[c] = (dx ? fx : 1.0 - fx) * (dy ? fy : 1.0 - fy) * (dz ? fz : 1.0 - fz);
        ++c;
      }
}


inline GridGeo grid_geo(const omen_grid* gr) {
  GridGeo G;
  G.nx = gr->nx;
  G.ny = gr->ny;
  G.nz = gr->nz;
  G.hx = gr->Lx_nm / gr->nx;
  G.hy = gr->Ly_nm / gr->ny;
  G.hz = gr->Lz_nm / gr->nz;
  G.vol_m3 = G.hx * G.hy * G.hz * 1e-27;
  return G;
}

inline Geo lat_geo(const omen_lattice* L) {
  return Geo{L->nx, L->ny, L->nz, L->ncells, L->natoms, {L->periodic[0], L->periodic[1], L->periodic[2]}};
}

