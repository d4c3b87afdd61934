// Slater–Koster two-centre integrals on the device (Slater & Koster, Phys. Rev. 94, 1498
// (1954), Table I), the parity rule for reversed orbital order, and the zincblende
// neighbour geometry shared by the assembly and H·X kernels.
#pragma once

#include <cuda_runtime.h>

#include "omen_internal.h"

// Orbital codes: 0 s, 1 px, 2 py, 3 pz, 4 dyz, 5 dzx, 6 dxy, 7 dx2-y2, 8 d3z2-r2, 9 s*.
__host__ __device__ inline int sk_code(int o, int norb) { return norb == 10 ? o : (o == 4 ? 9 : o); }
__host__ __device__ inline int sk_l(int c) { return (c == 0 || c == 9) ? 0 : (c <= 3 ? 1 : 2); }

// Integral indices
enum { P_SS = 0, P_SSSS, P_SSS, P_SP, P_SSP, P_SD, P_SSD, P_PPS, P_PPP, P_PDS, P_PDP, P_DDS, P_DDP, P_DDD };

// E_{a,b}(c) for orbital a on atom 1, b on atom 2, with l(a) <= l(b); for l(a) == l(b) the
// pair must be in table order (s-like: (s,s) (s*,s*) (s,s*); d: t2g before x2-y2 before z2).
__host__ __device__ inline double sk_table(int a, int b, const double c[3], const double* V) {
  const double r3 = 1.7320508075688772;
  const double l = c[0], m = c[1], n = c[2];
  const int la = sk_l(a), lb = sk_l(b);
  if (la == 0 && lb == 0) {
    if (a == 0 && b == 0) return V[P_SS];
    if (a == 9 && b == 9) return V[P_SSSS];
    return V[P_SSS];  // (s, s*)
  }
  if (la == 0 && lb == 1) return c[b - 1] * V[a == 0 ? P_SP : P_SSP];
  if (la == 0 && lb == 2) {
    const double v = V[a == 0 ? P_SD : P_SSD];
    if (b <= 6) {  // t2g: index t = b-4: yz (m n), zx (n l), xy (l m)
      const int t = b - 4;
      return r3 * c[(t + 1) % 3] * c[(t + 2) % 3] * v;
    }
    if (b == 7) return 0.5 * r3 * (l * l - m * m) * v;
    return (n * n - 0.5 * (l * l + m * m)) * v;
  }
  if (la == 1 && lb == 1) {
    const int i = a - 1, j = b - 1;
    return c[i] * c[j] * (V[P_PPS] - V[P_PPP]) + (i == j ? V[P_PPP] : 0.0);
  }
  if (la == 1 && lb == 2) {
    const int i = a - 1;
    const double s = V[P_PDS], p = V[P_PDP];
    if (b <= 6) {
      const int t = b - 4, j = (t + 1) % 3, k = (t + 2) % 3;
      const double cijk = c[i] * c[j] * c[k];
      return r3 * cijk * s + ((i == j ? c[k] : 0.0) + (i == k ? c[j] : 0.0) - 2.0 * cijk) * p;
    }
    if (b == 7) {
      const double q = l * l - m * m;
      const double ai = (i == 0) ? l : (i == 1 ? -m : 0.0);
      return 0.5 * r3 * c[i] * q * s + (ai - c[i] * q) * p;
    }
    const double q = n * n - 0.5 * (l * l + m * m);
    const double bi = (i == 2) ? n : 0.0;
    return c[i] * q * s + r3 * (bi - c[i] * n * n) * p;
  }
  // d - d
  const double s = V[P_DDS], p = V[P_DDP], d = V[P_DDD];
  if (a <= 6 && b <= 6) {
    const int t = a - 4, u = b - 4;
    if (t == u) {
      const int i = t, j = (t + 1) % 3, k = (t + 2) % 3;
      const double cj2 = c[j] * c[j], ck2 = c[k] * c[k];
      return 3.0 * cj2 * ck2 * s + (cj2 + ck2 - 4.0 * cj2 * ck2) * p + (c[i] * c[i] + cj2 * ck2) * d;
    }
    // shared index: the one that appears in both pairs; the two others
    const int sh = 3 - t - u;  // index not equal to t or u is shared (t2g pair (t+1,t+2))
    const int pa = t, pb = u;  // d_t misses index t, so its other index is u, and vice versa
    const double cs2 = c[sh] * c[sh];
    return 3.0 * c[pb] * cs2 * c[pa] * s + c[pa] * c[pb] * (1.0 - 4.0 * cs2) * p + c[pa] * c[pb] * (cs2 - 1.0) * d;
  }
  if (a <= 6 && b == 7) {
    const double q = l * l - m * m;
    if (a == 6) return 1.5 * l * m * q * s + 2.0 * l * m * (m * m - l * l) * p + 0.5 * l * m * q * d;
    if (a == 4) return 1.5 * m * n * q * s - m * n * (1.0 + 2.0 * q) * p + m * n * (1.0 + 0.5 * q) * d;
    return 1.5 * n * l * q * s + n * l * (1.0 - 2.0 * q) * p - n * l * (1.0 - 0.5 * q) * d;
  }
  if (a <= 6 && b == 8) {
    const double q = n * n - 0.5 * (l * l + m * m);
    if (a == 6) return r3 * l * m * q * s - 2.0 * r3 * l * m * n * n * p + 0.5 * r3 * l * m * (1.0 + n * n) * d;
    if (a == 4) return r3 * m * n * q * s + r3 * m * n * (l * l + m * m - n * n) * p - 0.5 * r3 * m * n * (l * l + m * m) * d;
    return r3 * l * n * q * s + r3 * l * n * (l * l + m * m - n * n) * p - 0.5 * r3 * l * n * (l * l + m * m) * d;
  }
  if (a == 7 && b == 7) {
    const double q = l * l - m * m;
    return 0.75 * q * q * s + (l * l + m * m - q * q) * p + (n * n + 0.25 * q * q) * d;
  }
  if (a == 7 && b == 8) {
    const double q = l * l - m * m;
    return 0.5 * r3 * q * (n * n - 0.5 * (l * l + m * m)) * s + r3 * n * n * (m * m - l * l) * p + 0.25 * r3 * (1.0 + n * n) * q * d;
  }
  const double q = n * n - 0.5 * (l * l + m * m);  // (z2, z2)
  return q * q * s + 3.0 * n * n * (l * l + m * m) * p + 0.75 * (l * l + m * m) * (l * l + m * m) * d;
}

// <atom1 a | H | atom2 b>, c = unit vector from atom 1 to atom 2.  V12: first-named orbital on
// atom 1; V21: on atom 2.  Pairs out of table order use E_ab(c) = (-1)^(la+lb) E_ba(c; V21);
// same-l p-p and d-d pairs are symmetric and use V12 in table order.
__host__ __device__ inline double sk_element(int a, int b, const double c[3], const double* V12, const double* V21) {
  const int la = sk_l(a), lb = sk_l(b);
  if (la < lb) return sk_table(a, b, c, V12);
  if (la > lb) return (((la + lb) & 1) ? -1.0 : 1.0) * sk_table(b, a, c, V21);
  if (la == 0) {
    if (a == 9 && b == 0) return sk_table(0, 9, c, V21);
    return sk_table(a, b, c, V12);
  }
  if (la == 1) return sk_table(a, b, c, V12);
  // d-d: order t2g (4,5,6) < 7 < 8; same-l swap has even parity
  int ra = a, rb = b;
  const bool swap = (a >= 7 && b <= 6) || (a == 8 && b == 7);
  if (swap) { ra = b; rb = a; }
  return sk_table(ra, rb, c, V12);
}

// Geometry helpers ---------------------------------------------------------------------------
struct Geo {
  int nx, ny, nz, ncells, natoms;
  int periodic[3];
};

// Neighbour cell of (ix,iy,iz) shifted by off (components in {-1,0,1}).  Returns false if the
// shift leaves a hard-wall direction.  wrap_sign[d] = -1/+1 when the shift wrapped across the
// low/high face of a periodic direction, else 0.
__device__ __forceinline__ bool shift_cell(const Geo& g, int ix, int iy, int iz, int ox, int oy, int oz,
                                           int& cell, int wrap_sign[3]) {
  int j[3] = {ix + ox, iy + oy, iz + oz};
  const int n[3] = {g.nx, g.ny, g.nz};
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    wrap_sign[d] = 0;
    if (j[d] < 0) {
      if (g.periodic[d] == OMEN_HARD_WALL) return false;
      j[d] += n[d];
      wrap_sign[d] = -1;
    } else if (j[d] >= n[d]) {
      if (g.periodic[d] == OMEN_HARD_WALL) return false;
      j[d] -= n[d];
      wrap_sign[d] = 1;
    }
  }
  cell = (j[2] * g.ny + j[1]) * g.nx + j[0];
  return true;
}
