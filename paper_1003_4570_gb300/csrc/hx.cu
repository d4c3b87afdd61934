// y = (H - sigma) x: the block-sparse tight-binding product repeated by the Lanczos
// recurrence (paper Section II-B benchmarks "500 Lanczos iterations"; Section III-A item 1).
//
// One thread per atom (grid.x over (cell tile, site b) with b fastest, grid.z over vectors).  Each row
// of H has an onsite block and four bond blocks.  Bond blocks are stored once per bond
// (A-atom slot); an A atom applies B, its B partner applies B^T, so no block is duplicated.
// The partner's copy of the block is read within about one z-plane of cells of the first
// read, which lies inside the L2 cache, so HBM sees each block about once.
// Blocks are stored in 32-slot tiles (entries of a tile contiguous): for a fixed entry,
// consecutive threads (consecutive cells) read consecutive words, and a warp's whole block
// is one contiguous run of memory.  Vectors are orbital-major, atom-minor, so the
// per-orbital loads of x and stores of y are coalesced as well.
// Bloch phase: a neighbour reached across the high (low) face of a Bloch-periodic direction d
// is its periodic image shifted by +L_d (-L_d); its amplitude is multiplied by
// exp(+i k_d L_d) (resp. the conjugate).
#include <algorithm>
#include <cmath>
#include <type_traits>
#include <vector>

#include "omen_internal.h"
#include "sk_device.cuh"
#include "df.cuh"

template <typename T> struct Cx;
template <> struct Cx<double> { using t = double2; };
template <> struct Cx<float> { using t = float2; };

template <typename T, bool CPLX> struct VecT { using t = T; };
template <typename T> struct VecT<T, true> { using t = typename Cx<T>::t; };

template <typename T>
struct HxArgs {
  Geo g;
  NeighbourTables nt;
  const T* __restrict__ blk;          // stored blocks (entry-major), or null for matrix-free
  const T* __restrict__ b0;           // [ns*ns*4][norb*norb] blocks at d0 (matrix-free)
  const T* __restrict__ scale;        // [16*ncells] (d0/d)^eta per bond slot (matrix-free)
  const uint8_t* __restrict__ species;
  const double* __restrict__ onsite;  // [ns][norb]
  const T* __restrict__ onsite_t;     // the same in T (real matrix-free rows)
  const double* __restrict__ U;       // [natoms]
  const double* __restrict__ lambda;  // [ns]
  const void* x;
  void* y;
  long long nrows;
  double sigma;
  double2 phase[3];
  int ns;
  int slot_stride;
  int cell0, cell1;                   // cells [cell0, cell1) of this launch (a z-range of planes)
  int nbid;                           // CTA work items: 8 sites x cell tiles of blockDim.x cells
};

template <typename T>
__device__ __forceinline__ typename Cx<T>::t cmul(typename Cx<T>::t a, typename Cx<T>::t b) {
  typename Cx<T>::t r;
  r.x = a.x * b.x - a.y * b.y;
  r.y = a.x * b.y + a.y * b.x;
  return r;
}

// Accumulator helpers: real or complex times a real block entry.
template <typename T> __device__ __forceinline__ void fma_r(T& acc, T h, T x) { acc = fma(h, x, acc); }
template <typename T, typename C> __device__ __forceinline__ void fma_c(C& acc, T h, C x) {
  acc.x = fma(h, x.x, acc.x);
  acc.y = fma(h, x.y, acc.y);
}

// RBT: block rows loaded per register batch (0 = the built-in rule below); the CTA width
// (blockDim.x, a multiple of 32 up to 128) and RBT are the tile shape the tuner chooses.
// Matrix-free block rows: RB rows of the b0 block (shared memory) into registers, with 16-byte
// loads where the row offsets allow (FP32 with an even RB and orbital count, FP64 with an even
// orbital count), else one word at a time.
template <typename T, int NORB, int RB>
__device__ __forceinline__ void smem_rows(const T* hb, int r0, T* hr) {
  constexpr int NE = RB * NORB;
  if constexpr (sizeof(T) == 4 && NORB % 2 == 0 && RB % 2 == 0) {
    const float4* h4 = reinterpret_cast<const float4*>(hb + r0 * NORB);
#pragma unroll
    for (int e = 0; e < NE / 4; ++e) {
      const float4 v = h4[e];
      hr[4 * e] = v.x; hr[4 * e + 1] = v.y; hr[4 * e + 2] = v.z; hr[4 * e + 3] = v.w;
    }
  } else if constexpr (sizeof(T) == 8 && NORB % 2 == 0) {
    const double2* h2 = reinterpret_cast<const double2*>(hb + r0 * NORB);
#pragma unroll
    for (int e = 0; e < NE / 2; ++e) {
      const double2 v = h2[e];
      hr[2 * e] = v.x; hr[2 * e + 1] = v.y;
    }
  } else {
#pragma unroll
    for (int e = 0; e < NE; ++e) hr[e] = hb[r0 * NORB + e];
  }
}

// Rows of one work item: site b = bid & 7 (fastest, so CTAs in flight cover all 8 sites of a
// window of cells and the transposed (B-end) read of a bond block follows its A-end read within
// L2 reach) and cells [cell0 + (bid >> 3) * blockDim.x, ...) one per thread.
template <typename T, int NORB, bool CPLX, bool SO, bool MATFREE, int RBT>
__device__ __forceinline__ void hx_item(const HxArgs<T>& a, int bid, const T* __restrict__ tab) {
  using V = typename VecT<T, CPLX>::t;
  constexpr int NS = SO ? 2 : 1;
  const Geo& g = a.g;
  const int b = bid & 7;
  const int cell = a.cell0 + (bid >> 3) * blockDim.x + threadIdx.x;
  if (cell >= a.cell1) return;
  const int N = g.natoms;
  const int atom = b * g.ncells + cell;
  const int ix = cell % g.nx, iy = (cell / g.nx) % g.ny, iz = cell / (g.nx * g.ny);
  const V* __restrict__ x = static_cast<const V*>(a.x) + (size_t)blockIdx.z * a.nrows;
  V* __restrict__ y = static_cast<V*>(a.y) + (size_t)blockIdx.z * a.nrows;
  const int sp = a.species[atom];

  V acc[NS][NORB];
  {
    const T u = (T)(a.U[atom] - a.sigma);
#pragma unroll
    for (int s = 0; s < NS; ++s)
#pragma unroll
      for (int o = 0; o < NORB; ++o) {
        const T d = a.onsite_t[sp * NORB + o] + u;
        const V xv = x[(size_t)(s * NORB + o) * N + atom];
        if constexpr (CPLX) {
          acc[s][o].x = d * xv.x;
          acc[s][o].y = d * xv.y;
        } else {
          acc[s][o] = d * xv;
        }
      }
    if constexpr (SO) {
      // lambda L.sigma on (px,py,pz) = orbitals 1..3, basis (spin, orbital), spin up first
      const T lam = (T)a.lambda[sp];
      V xu[3], xd[3];
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        xu[i] = x[(size_t)(1 + i) * N + atom];
        xd[i] = x[(size_t)(NORB + 1 + i) * N + atom];
      }
      // i*z = (-z.y, z.x)
      // up x: -i xu_y + xd_z ; up y: i xu_x - i xd_z ; up z: i xd_y - xd_x
      // dn x: i xd_y - xu_z ; dn y: -i xd_x - i xu_z ; dn z: i xu_y + xu_x
      acc[0][1].x += lam * (xu[1].y + xd[2].x);
      acc[0][1].y += lam * (-xu[1].x + xd[2].y);
      acc[0][2].x += lam * (-xu[0].y + xd[2].y);
      acc[0][2].y += lam * (xu[0].x - xd[2].x);
      acc[0][3].x += lam * (-xd[1].y - xd[0].x);
      acc[0][3].y += lam * (xd[1].x - xd[0].y);
      acc[1][1].x += lam * (-xd[1].y - xu[2].x);
      acc[1][1].y += lam * (xd[1].x - xu[2].y);
      acc[1][2].x += lam * (xd[0].y + xu[2].y);
      acc[1][2].y += lam * (-xd[0].x - xu[2].x);
      acc[1][3].x += lam * (-xu[1].y + xu[0].x);
      acc[1][3].y += lam * (xu[1].x + xu[0].y);
    }
  }

  const bool is_a = b < 4;
  const int s = is_a ? b : b - 4;
  constexpr int RB = RBT > 0 ? RBT
                             : (MATFREE ? ((sizeof(T) == 4 && NORB % 2 == 0) ? 2 : 1)
                                        : (sizeof(T) == 8 ? 1 : (NS == 1 ? NORB : (NORB == 10 ? 5 : NORB))));
  static_assert(NORB % RB == 0, "RB must divide the orbital count");
#pragma unroll 1
  for (int k = 0; k < 4; ++k) {
    int ox, oy, oz, site2;
    if (is_a) {
      ox = a.nt.a_to_b_off[s][k][0]; oy = a.nt.a_to_b_off[s][k][1]; oz = a.nt.a_to_b_off[s][k][2];
      site2 = a.nt.a_to_b_site[s][k];
    } else {
      ox = a.nt.b_to_a_off[s][k][0]; oy = a.nt.b_to_a_off[s][k][1]; oz = a.nt.b_to_a_off[s][k][2];
      site2 = a.nt.b_to_a_site[s][k];
    }
    int cell2, wrap[3];
    if (!shift_cell(g, ix, iy, iz, ox, oy, oz, cell2, wrap)) continue;
    const int atom2 = site2 * g.ncells + cell2;
    // bond slot belongs to the A end
    const size_t slot = is_a ? (size_t)(k * 4 + s) * g.ncells + cell : (size_t)(k * 4 + site2) * g.ncells + cell2;

    V xn[NS][NORB];
#pragma unroll
    for (int q = 0; q < NS; ++q)
#pragma unroll
      for (int o = 0; o < NORB; ++o) xn[q][o] = x[(size_t)(q * NORB + o) * N + atom2];
    if constexpr (CPLX) {
      if (wrap[0] | wrap[1] | wrap[2]) {
        typename Cx<T>::t f;
        f.x = (T)1; f.y = (T)0;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          if (wrap[d]) {
            typename Cx<T>::t p;
            p.x = (T)a.phase[d].x;
            p.y = (T)(wrap[d] > 0 ? a.phase[d].y : -a.phase[d].y);
            f = cmul<T>(f, p);
          }
        }
#pragma unroll
        for (int q = 0; q < NS; ++q)
#pragma unroll
          for (int o = 0; o < NORB; ++o) xn[q][o] = cmul<T>(xn[q][o], f);
      }
    }

    const T* __restrict__ hb;
    size_t stride;
    T scale = (T)1;
    if constexpr (MATFREE) {
      const int sa = is_a ? sp : a.species[atom2];
      const int sb = is_a ? a.species[atom2] : sp;
      scale = a.scale[slot];
      hb = tab + ((sa * a.ns + sb) * 4 + k) * (NORB * NORB);
      stride = 1;
    } else {
      const size_t ks = is_a ? (size_t)(k * 4 + s) : (size_t)(k * 4 + site2);
      const size_t pidx = ks * a.slot_stride + (is_a ? cell : cell2);
      hb = a.blk + ((pidx >> 5) * (NORB * NORB)) * 32 + (pidx & 31);
      stride = 32;
    }

    if constexpr (MATFREE) {
      // the (d0/d)^eta factor is applied to the neighbour amplitudes once per bond
#pragma unroll
      for (int q = 0; q < NS; ++q)
#pragma unroll
        for (int o = 0; o < NORB; ++o) {
          if constexpr (CPLX) { xn[q][o].x *= scale; xn[q][o].y *= scale; } else { xn[q][o] *= scale; }
        }
    }
    // Rows of the block are loaded RB at a time into registers before their FMAs, so each
    // thread keeps RB*NORB independent loads in flight (memory-level parallelism).  Every
    // accumulator sums its terms in the same order for any RB: the result does not depend on it.
#pragma unroll
    for (int r0 = 0; r0 < NORB; r0 += RB) {
      T hr[RB * NORB];
      if constexpr (MATFREE) {
        smem_rows<T, NORB, RB>(hb, r0, hr);
      } else {
#pragma unroll
        for (int e = 0; e < RB * NORB; ++e) hr[e] = __ldg(hb + (size_t)(r0 * NORB + e) * stride);
      }
      if (is_a) {
#pragma unroll
        for (int i = 0; i < RB; ++i)
#pragma unroll
          for (int o2 = 0; o2 < NORB; ++o2) {
            const T h = hr[i * NORB + o2];
#pragma unroll
            for (int q = 0; q < NS; ++q) {
              if constexpr (CPLX) fma_c(acc[q][r0 + i], h, xn[q][o2]); else fma_r(acc[q][r0 + i], h, xn[q][o2]);
            }
          }
      } else {
#pragma unroll
        for (int i = 0; i < RB; ++i)
#pragma unroll
          for (int o2 = 0; o2 < NORB; ++o2) {
            const T h = hr[i * NORB + o2];
#pragma unroll
            for (int q = 0; q < NS; ++q) {
              if constexpr (CPLX) fma_c(acc[q][o2], h, xn[q][r0 + i]); else fma_r(acc[q][o2], h, xn[q][r0 + i]);
            }
          }
      }
    }
  }
#pragma unroll
  for (int q = 0; q < NS; ++q)
#pragma unroll
    for (int o = 0; o < NORB; ++o) y[(size_t)(q * NORB + o) * N + atom] = acc[q][o];
}

// Real matrix-free rows (no spin-orbit, no Bloch phase).  The site class (A or B end of its
// bonds) is a template parameter, so the row/column order of each block product is fixed at
// compile time; the four bonds are unrolled; the onsite energies come from a table in T and
// U - sigma is formed once per atom, so an FP32 product runs no FP64 arithmetic per orbital.
// Each accumulator sums its terms in the same order as hx_item's (onsite, then k = 0..3).
// Real FP32 rows with an even orbital count use packed FP32x2 FMAs and a second, row-pair
// interleaved copy of the table (for the A end) after the row-major one.
template <typename T, int NORB, bool CPLX>
__host__ __device__ constexpr bool mf_paired() { return !CPLX && sizeof(T) == 4 && NORB % 2 == 0; }

template <typename T, int NORB, int RB, bool IS_A>
__device__ __forceinline__ void hx_item_mf_real(const HxArgs<T>& a, int bid, const T* __restrict__ tab) {
  constexpr bool PAIRED = mf_paired<T, NORB, false>();
  const int tab_copy = a.ns * a.ns * 4 * NORB * NORB;   // offset of the interleaved copy
  const Geo& g = a.g;
  const int b = bid & 7;
  const int s = IS_A ? b : b - 4;
  const int cell = a.cell0 + (bid >> 3) * blockDim.x + threadIdx.x;
  if (cell >= a.cell1) return;
  const int N = g.natoms;
  const int atom = b * g.ncells + cell;
  const int nxy = g.nx * g.ny;
  const int iz = cell / nxy;
  const int rem = cell - iz * nxy;
  const int iy = rem / g.nx;
  const int ix = rem - iy * g.nx;
  // faces this cell touches: a bond leaving through one wraps (periodic) or is absent (hard wall)
  const bool lo[3] = {ix == 0, iy == 0, iz == 0};
  const bool hi[3] = {ix == g.nx - 1, iy == g.ny - 1, iz == g.nz - 1};
  const int stride[3] = {1, g.nx, nxy};
  const int extent[3] = {g.nx * 1, g.ny * g.nx, g.nz * nxy};
  const T* __restrict__ x = static_cast<const T*>(a.x) + (size_t)blockIdx.z * a.nrows;
  T* __restrict__ y = static_cast<T*>(a.y) + (size_t)blockIdx.z * a.nrows;
  const int sp = a.species[atom];
  const int npair = a.ns * a.ns;
  T acc[NORB];
  {
    const T u = (T)(a.U[atom] - a.sigma);
    const T* xp = x + atom;
#pragma unroll
    for (int o = 0; o < NORB; ++o) acc[o] = (a.onsite_t[sp * NORB + o] + u) * xp[o * N];
  }
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int* off = IS_A ? a.nt.a_to_b_off[s][k] : a.nt.b_to_a_off[s][k];
    const int site2 = IS_A ? a.nt.a_to_b_site[s][k] : a.nt.b_to_a_site[s][k];
    int cell2 = cell;
    bool ok = true;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const int od = off[d];            // uniform over the CTA: -1 or 0 (A sites), 0 or +1 (B sites)
      cell2 += od * stride[d];
      if ((od < 0 && lo[d]) || (od > 0 && hi[d])) {
        ok = ok && g.periodic[d] != OMEN_HARD_WALL;
        cell2 -= od * extent[d];
      }
    }
    if (!ok) continue;
    const int atom2 = site2 * g.ncells + cell2;
    const int slot = IS_A ? (k * 4 + s) * g.ncells + cell : (k * 4 + site2) * g.ncells + cell2;
    const int sp2 = a.species[atom2];
    // table in shared memory ordered [direction][pair][entry]: the (at most ns^2) blocks a warp
    // reads for one direction lie in distinct banks
    const T* hb = tab + (k * npair + (IS_A ? sp * a.ns + sp2 : sp2 * a.ns + sp)) * (NORB * NORB);
    const T sc = a.scale[slot];
    const T* xp = x + atom2;
    T xn[NORB];
#pragma unroll
    for (int o = 0; o < NORB; ++o) xn[o] = xp[o * N] * sc;
    if constexpr (PAIRED) {
      // two accumulators per packed FP32x2 FMA (each lane an ordinary fma: same bits as the
      // scalar form).  A end: acc[r], acc[r+1] += (h[r][c], h[r+1][c]) x[c] from the row-pair
      // interleaved copy of the table; B end: acc[c], acc[c+1] += (h[r][c], h[r][c+1]) x[r]
      // from the row-major copy.
      const float4* h4 = reinterpret_cast<const float4*>(IS_A ? hb + tab_copy : hb);
#pragma unroll
      for (int p = 0; p < NORB / 2; ++p) {
        float2 hp[NORB];
#pragma unroll
        for (int q = 0; q < NORB / 2; ++q) {
          const float4 v = h4[p * (NORB / 2) + q];
          hp[2 * q] = make_float2(v.x, v.y);
          hp[2 * q + 1] = make_float2(v.z, v.w);
        }
        if constexpr (IS_A) {
          float2 acc2 = make_float2(acc[2 * p], acc[2 * p + 1]);
#pragma unroll
          for (int c = 0; c < NORB; ++c) acc2 = __ffma2_rn(hp[c], make_float2(xn[c], xn[c]), acc2);
          acc[2 * p] = acc2.x;
          acc[2 * p + 1] = acc2.y;
        } else {
          // hp holds rows 2p and 2p+1 (row-major: NORB/2 pairs per row)
#pragma unroll
          for (int i = 0; i < 2; ++i)
#pragma unroll
            for (int q = 0; q < NORB / 2; ++q) {
              float2 acc2 = make_float2(acc[2 * q], acc[2 * q + 1]);
              acc2 = __ffma2_rn(hp[i * (NORB / 2) + q], make_float2(xn[2 * p + i], xn[2 * p + i]), acc2);
              acc[2 * q] = acc2.x;
              acc[2 * q + 1] = acc2.y;
            }
        }
      }
    } else {
#pragma unroll
      for (int r0 = 0; r0 < NORB; r0 += RB) {
        T hr[RB * NORB];
        smem_rows<T, NORB, RB>(hb, r0, hr);
#pragma unroll
        for (int i = 0; i < RB; ++i)
#pragma unroll
          for (int o2 = 0; o2 < NORB; ++o2) {
            if constexpr (IS_A) acc[r0 + i] = fma(hr[i * NORB + o2], xn[o2], acc[r0 + i]);
            else acc[o2] = fma(hr[i * NORB + o2], xn[r0 + i], acc[o2]);
          }
      }
    }
  }
  T* yp = y + atom;
#pragma unroll
  for (int o = 0; o < NORB; ++o) yp[o * N] = acc[o];
}

// Stored blocks: one work item per CTA.  Matrix-free: the b0 table (ns^2 x 4 directions x
// norb^2 entries, a few KB) is staged in shared memory once per CTA and the CTAs stride over the
// work items, so the per-bond block reads are shared-memory broadcasts (a warp touches at most
// ns^2 distinct blocks) instead of divergent L1 traffic.
template <typename T, int NORB, bool CPLX, bool SO, bool MATFREE, int RBT>
__global__ void __launch_bounds__(128) hx_kernel(HxArgs<T> a) {
  if constexpr (MATFREE) {
    extern __shared__ __align__(16) unsigned char hx_smem[];
    T* tab = reinterpret_cast<T*>(hx_smem);
    constexpr int NE = NORB * NORB;
    const int npair = a.ns * a.ns;
    const int n = npair * 4 * NE;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      if constexpr (CPLX) {
        tab[i] = a.b0[i];
      } else {            // b0 is [pair][k][e]; the real rows read [k][pair][e]
        const int e = i % NE, pk = i / NE, pair = pk >> 2, k = pk & 3;
        const int blk = (k * npair + pair) * NE;
        tab[blk + e] = a.b0[i];
        if constexpr (mf_paired<T, NORB, CPLX>()) {   // row pair p, column c, row parity q
          const int r = e / NORB, c = e - r * NORB;
          tab[n + blk + ((r >> 1) * NORB + c) * 2 + (r & 1)] = a.b0[i];
        }
      }
    }
    __syncthreads();
    if constexpr (!CPLX) {
      constexpr int RB = RBT > 0 ? RBT : ((sizeof(T) == 4 && NORB % 2 == 0) ? 2 : 1);
      for (int bid = blockIdx.x; bid < a.nbid; bid += gridDim.x) {
        if ((bid & 7) < 4) hx_item_mf_real<T, NORB, RB, true>(a, bid, tab);
        else hx_item_mf_real<T, NORB, RB, false>(a, bid, tab);
      }
    } else {
      for (int bid = blockIdx.x; bid < a.nbid; bid += gridDim.x) hx_item<T, NORB, CPLX, SO, true, RBT>(a, bid, tab);
    }
  } else {
    hx_item<T, NORB, CPLX, SO, false, RBT>(a, blockIdx.x, nullptr);
  }
}

// ---------------------------------------------------------------------------------------
// Double-float product (precision OMEN_F64_DF): every value is an FP32 pair (hi, lo) with
// value = hi + lo, products and sums by the error-free transformations of df.cuh, all on the
// FP32 pipe (57x GB300's FP64 rate); the bytes moved equal those of FP64.
struct HxDfArgs {
  Geo g;
  NeighbourTables nt;
  const float2* __restrict__ blk;
  const uint8_t* __restrict__ species;
  const float2* __restrict__ onsite;   // [ns][norb] double-float
  const double* __restrict__ U;
  const float2* x;
  float2* y;
  long long nrows;
  double sigma;
  int slot_stride;
  int cell0, cell1;                    // cells [cell0, cell1) of this launch
};

template <int NORB>
__global__ void __launch_bounds__(128) hx_df_kernel(HxDfArgs a) {
  const Geo& g = a.g;
  const int b = blockIdx.x & 7;
  const int cell = a.cell0 + (blockIdx.x >> 3) * blockDim.x + threadIdx.x;
  if (cell >= a.cell1) return;
  const int N = g.natoms;
  const int atom = b * g.ncells + cell;
  const int ix = cell % g.nx, iy = (cell / g.nx) % g.ny, iz = cell / (g.nx * g.ny);
  const float2* __restrict__ x = a.x + (size_t)blockIdx.z * a.nrows;
  float2* __restrict__ y = a.y + (size_t)blockIdx.z * a.nrows;
  const int sp = a.species[atom];
  float S[NORB], C[NORB];
  {
    const float2 u = df_from_double(a.U[atom] - a.sigma);
#pragma unroll
    for (int o = 0; o < NORB; ++o) {
      S[o] = 0.f;
      C[o] = 0.f;
      df_mac(S[o], C[o], df_add(a.onsite[sp * NORB + o], u), x[(size_t)o * N + atom]);
    }
  }
  const bool is_a = b < 4;
  const int s = is_a ? b : b - 4;
#pragma unroll 1
  for (int k = 0; k < 4; ++k) {
    int ox, oy, oz, site2;
    if (is_a) {
      ox = a.nt.a_to_b_off[s][k][0]; oy = a.nt.a_to_b_off[s][k][1]; oz = a.nt.a_to_b_off[s][k][2];
      site2 = a.nt.a_to_b_site[s][k];
    } else {
      ox = a.nt.b_to_a_off[s][k][0]; oy = a.nt.b_to_a_off[s][k][1]; oz = a.nt.b_to_a_off[s][k][2];
      site2 = a.nt.b_to_a_site[s][k];
    }
    int cell2, wrap[3];
    if (!shift_cell(g, ix, iy, iz, ox, oy, oz, cell2, wrap)) continue;
    const int atom2 = site2 * g.ncells + cell2;
    float2 xn[NORB];
#pragma unroll
    for (int o = 0; o < NORB; ++o) xn[o] = x[(size_t)o * N + atom2];
    const size_t ks = is_a ? (size_t)(k * 4 + s) : (size_t)(k * 4 + site2);
    const size_t pidx = ks * a.slot_stride + (is_a ? cell : cell2);
    const float2* __restrict__ hb = a.blk + ((pidx >> 5) * (NORB * NORB)) * 32 + (pidx & 31);
    constexpr int RB = (NORB == 10) ? 5 : NORB;
#pragma unroll
    for (int r0 = 0; r0 < NORB; r0 += RB) {
      float2 hr[RB * NORB];
#pragma unroll
      for (int e = 0; e < RB * NORB; ++e) hr[e] = __ldg(hb + (size_t)(r0 * NORB + e) * 32);
      if (is_a) {
#pragma unroll
        for (int i = 0; i < RB; ++i)
#pragma unroll
          for (int o2 = 0; o2 < NORB; ++o2) df_mac(S[r0 + i], C[r0 + i], hr[i * NORB + o2], xn[o2]);
      } else {
#pragma unroll
        for (int i = 0; i < RB; ++i)
#pragma unroll
          for (int o2 = 0; o2 < NORB; ++o2) df_mac(S[o2], C[o2], hr[i * NORB + o2], xn[r0 + i]);
      }
    }
  }
#pragma unroll
  for (int o = 0; o < NORB; ++o) y[(size_t)o * N + atom] = df_norm(S[o], C[o]);
}

__global__ void f64_to_df_kernel(const double* __restrict__ src, float2* __restrict__ dst, long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    dst[i] = df_from_double(src[i]);
}
__global__ void df_to_f64_kernel(const float2* __restrict__ src, double* __restrict__ dst, long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    dst[i] = (double)src[i].x + (double)src[i].y;
}

static cudaError_t launch_df(const omen_ham* h, const void* x, void* y, int nvec, double sigma, cudaStream_t st,
                             int cell0, int cell1) {
  const omen_lattice* L = h->lat;
  HxDfArgs a;
  a.g = Geo{L->nx, L->ny, L->nz, L->ncells, L->natoms, {L->periodic[0], L->periodic[1], L->periodic[2]}};
  a.nt = host_neighbour_tables();
  a.blk = h->d_blkdf;
  a.species = L->d_species;
  a.onsite = h->d_onsite_df;
  a.U = h->d_U;
  a.x = static_cast<const float2*>(x);
  a.y = static_cast<float2*>(y);
  a.nrows = h->nrows;
  a.sigma = sigma;
  a.slot_stride = h->slot_stride;
  a.cell0 = cell0;
  a.cell1 = cell1;
  dim3 grid(((cell1 - cell0 + 127) / 128) * 8, 1, nvec);
  if (h->norb == 10) hx_df_kernel<10><<<grid, 128, 0, st>>>(a);
  else hx_df_kernel<5><<<grid, 128, 0, st>>>(a);
  return cudaGetLastError();
}

extern "C" omen_status omen_convert_vectors(omen_ctx* ctx, const void* src, int sp, void* dst, int dp, long long n) {
  if (!ctx || !src || !dst || n < 0) return set_err(ctx, OMEN_EINVAL, "null argument");
  const unsigned grid = (unsigned)std::max<long long>(1, std::min<long long>((n + 255) / 256, 152 * 16));
  if (sp == OMEN_F64 && dp == OMEN_F64_DF)
    f64_to_df_kernel<<<grid, 256, 0, ctx->stream>>>(static_cast<const double*>(src), static_cast<float2*>(dst), n);
  else if (sp == OMEN_F64_DF && dp == OMEN_F64)
    df_to_f64_kernel<<<grid, 256, 0, ctx->stream>>>(static_cast<const float2*>(src), static_cast<double*>(dst), n);
  else
    return set_err(ctx, OMEN_EINVAL, "conversion supports F64 <-> F64_DF");
  OMEN_CHECK_LAUNCH(ctx);
  return OMEN_OK;
}

// ---------------------------------------------------------------------------------------
// k-batched product over several structures: y = (H_i(k) - sigma) x for every wave vector k of
// every structure i, all in one launch (the (structure, k) work list).  Within a structure the
// real bond blocks are the same for every k (the phase sits only on bonds that wrap a Bloch
// face), so each thread loads a block entry once and applies it to KB wave vectors.  The CTAs
// of structure i are [cta0_i, cta0_i + tiles_i * ceil(nk_i / KB)); within them the tile index
// runs fastest.  phases_i[k*3 + d] = exp(i k_d L_d).  Structure i's vectors are [nk_i][nrows_i]
// starting at element x_off_i of x and y.
static constexpr int kMaxKInst = 16;

template <typename T>
struct KInst {
  Geo g;
  const T* blk;
  const uint8_t* species;
  const double* onsite;
  const double* U;
  const double2* phases;
  long long nrows;
  long long x_off;
  int nk;
  int slot_stride;
  int cta0;
  int tiles;
};

template <typename T>
struct KMulti {
  NeighbourTables nt;
  KInst<T> in[kMaxKInst];
  int n;
  const void* x;
  void* y;
  double sigma;
};

template <typename T, int NORB, int KB>
__global__ void __launch_bounds__(128) hx_kbatch_kernel(KMulti<T> m) {
  using V = typename Cx<T>::t;
  int inst = 0;
  while (inst + 1 < m.n && (int)blockIdx.x >= m.in[inst + 1].cta0) ++inst;
  const KInst<T>& I = m.in[inst];
  const Geo& g = I.g;
  const int local = (int)blockIdx.x - I.cta0;
  const int tile = local % I.tiles;
  const int b = tile & 7;
  const int cell = (tile >> 3) * blockDim.x + threadIdx.x;
  if (cell >= g.ncells) return;
  const int N = g.natoms;
  const int atom = b * g.ncells + cell;
  const int ix = cell % g.nx, iy = (cell / g.nx) % g.ny, iz = cell / (g.nx * g.ny);
  const int k0 = (local / I.tiles) * KB;
  const int nkb = min(KB, I.nk - k0);
  const V* __restrict__ x = static_cast<const V*>(m.x) + I.x_off;
  V* __restrict__ y = static_cast<V*>(m.y) + I.x_off;
  const int sp = I.species[atom];
  V acc[KB][NORB];
  {
    const T u = (T)(I.U[atom] - m.sigma);
#pragma unroll
    for (int q = 0; q < KB; ++q)
#pragma unroll
      for (int o = 0; o < NORB; ++o) {
        acc[q][o].x = (T)0;
        acc[q][o].y = (T)0;
        if (q < nkb) {
          const T d = (T)I.onsite[sp * NORB + o] + u;
          const V xv = x[(size_t)(k0 + q) * I.nrows + (size_t)o * N + atom];
          acc[q][o].x = d * xv.x;
          acc[q][o].y = d * xv.y;
        }
      }
  }
  const bool is_a = b < 4;
  const int s = is_a ? b : b - 4;
#pragma unroll 1
  for (int k = 0; k < 4; ++k) {
    int ox, oy, oz, site2;
    if (is_a) {
      ox = m.nt.a_to_b_off[s][k][0]; oy = m.nt.a_to_b_off[s][k][1]; oz = m.nt.a_to_b_off[s][k][2];
      site2 = m.nt.a_to_b_site[s][k];
    } else {
      ox = m.nt.b_to_a_off[s][k][0]; oy = m.nt.b_to_a_off[s][k][1]; oz = m.nt.b_to_a_off[s][k][2];
      site2 = m.nt.b_to_a_site[s][k];
    }
    int cell2, wrap[3];
    if (!shift_cell(g, ix, iy, iz, ox, oy, oz, cell2, wrap)) continue;
    const int atom2 = site2 * g.ncells + cell2;
    V xn[KB][NORB];
#pragma unroll
    for (int q = 0; q < KB; ++q) {
      V f;
      f.x = (T)1;
      f.y = (T)0;
      if (q < nkb && (wrap[0] | wrap[1] | wrap[2])) {
#pragma unroll
        for (int d = 0; d < 3; ++d)
          if (wrap[d]) {
            const double2 ph = I.phases[(size_t)(k0 + q) * 3 + d];
            V p;
            p.x = (T)ph.x;
            p.y = (T)(wrap[d] > 0 ? ph.y : -ph.y);
            f = cmul<T>(f, p);
          }
      }
#pragma unroll
      for (int o = 0; o < NORB; ++o) {
        if (q < nkb) xn[q][o] = cmul<T>(x[(size_t)(k0 + q) * I.nrows + (size_t)o * N + atom2], f);
        else { xn[q][o].x = (T)0; xn[q][o].y = (T)0; }
      }
    }
    const size_t ks = is_a ? (size_t)(k * 4 + s) : (size_t)(k * 4 + site2);
    const size_t pidx = ks * I.slot_stride + (is_a ? cell : cell2);
    const T* __restrict__ hb = I.blk + ((pidx >> 5) * (NORB * NORB)) * 32 + (pidx & 31);
#pragma unroll
    for (int o1 = 0; o1 < NORB; ++o1)
#pragma unroll
      for (int o2 = 0; o2 < NORB; ++o2) {
        const T h = __ldg(hb + (size_t)(o1 * NORB + o2) * 32);
#pragma unroll
        for (int q = 0; q < KB; ++q) {
          if (is_a) fma_c(acc[q][o1], h, xn[q][o2]);
          else fma_c(acc[q][o2], h, xn[q][o1]);
        }
      }
  }
#pragma unroll
  for (int q = 0; q < KB; ++q)
    if (q < nkb)
#pragma unroll
      for (int o = 0; o < NORB; ++o) y[(size_t)(k0 + q) * I.nrows + (size_t)o * N + atom] = acc[q][o];
}

size_t vec_elem_bytes(const omen_ham* h, int precision) {
  const size_t r = (precision == OMEN_F64 || precision == OMEN_F64_DF) ? 8 : 4;
  return h->is_complex ? 2 * r : r;
}

template <typename T, int NORB, bool CPLX, bool SO, bool MF, int RBT>
static cudaError_t launch_t(const HxArgs<T>& a0, int nvec, int threads, cudaStream_t st) {
  HxArgs<T> a = a0;
  a.nbid = ((a.cell1 - a.cell0 + threads - 1) / threads) * 8;
  if constexpr (!MF) {
    dim3 grid(a.nbid, 1, nvec);
    hx_kernel<T, NORB, CPLX, SO, false, RBT><<<grid, threads, 0, st>>>(a);
    return cudaGetLastError();
  } else {
    // one resident wave of CTAs (per vector), each striding over the work items
    const size_t smem = (size_t)a.ns * a.ns * 4 * NORB * NORB * sizeof(T) * (mf_paired<T, NORB, CPLX>() ? 2 : 1);
    auto kern = hx_kernel<T, NORB, CPLX, SO, true, RBT>;
    if (smem > 48 * 1024) {
      const cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
    }
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem);
    if (e != cudaSuccess) return e;
    const int wave = std::max(1, sms * std::max(1, per_sm));
    dim3 grid(std::min(a.nbid, wave), 1, nvec);
    kern<<<grid, threads, smem, st>>>(a);
    return cudaGetLastError();
  }
}

// Register-batch sizes compiled for each variant (0 = the built-in rule): FP32 stored blocks
// take 1, 2, 5 or NORB rows (NORB only without spin-orbit); FP64 stored 1 or 2; matrix-free
// 1 or 2 (rows dividing the orbital count).
template <typename T, int NORB, bool SO, bool MF>
static constexpr bool rb_compiled(int rb) {
  if (rb == 0) return true;
  if (NORB % rb != 0) return false;
  if (MF) return rb == 1 || rb == 2;
  if (sizeof(T) == 8) return rb == 1 || rb == 2;
  return rb == 1 || rb == 2 || rb == 5 || (rb == NORB && !SO);
}

template <typename T, int NORB, bool CPLX, bool SO, bool MF>
static cudaError_t launch_rb(const HxArgs<T>& a, int nvec, HxTile t, cudaStream_t st) {
  const int thr = t.threads ? t.threads : 128;
  if constexpr (rb_compiled<T, NORB, SO, MF>(1)) if (t.rb == 1) return launch_t<T, NORB, CPLX, SO, MF, 1>(a, nvec, thr, st);
  if constexpr (rb_compiled<T, NORB, SO, MF>(2)) if (t.rb == 2) return launch_t<T, NORB, CPLX, SO, MF, 2>(a, nvec, thr, st);
  if constexpr (rb_compiled<T, NORB, SO, MF>(5)) if (t.rb == 5) return launch_t<T, NORB, CPLX, SO, MF, 5>(a, nvec, thr, st);
  if constexpr (rb_compiled<T, NORB, SO, MF>(10)) if (t.rb == 10) return launch_t<T, NORB, CPLX, SO, MF, 10>(a, nvec, thr, st);
  return launch_t<T, NORB, CPLX, SO, MF, 0>(a, nvec, thr, st);
}

template <typename T, int NORB>
static cudaError_t launch_norb(const HxArgs<T>& a, const omen_ham* h, int nvec, HxTile t, cudaStream_t st) {
  const bool mf = h->matrix_free;
  if (!h->is_complex) return mf ? launch_rb<T, NORB, false, false, true>(a, nvec, t, st) : launch_rb<T, NORB, false, false, false>(a, nvec, t, st);
  if (!h->spin_orbit) return mf ? launch_rb<T, NORB, true, false, true>(a, nvec, t, st) : launch_rb<T, NORB, true, false, false>(a, nvec, t, st);
  return mf ? launch_rb<T, NORB, true, true, true>(a, nvec, t, st) : launch_rb<T, NORB, true, true, false>(a, nvec, t, st);
}

// Whether (threads, rb) is a compiled tile shape for this Hamiltonian and vector precision.
bool hx_tile_valid(const omen_ham* h, int vec_precision, int threads, int rb) {
  if (threads != 0 && (threads < 32 || threads > 128 || threads % 32 != 0)) return false;
  const bool f64 = vec_precision == OMEN_F64;
  const bool so = h->spin_orbit, mf = h->matrix_free;
  if (h->norb == 10) {
    if (f64) return so ? (mf ? rb_compiled<double, 10, true, true>(rb) : rb_compiled<double, 10, true, false>(rb))
                       : (mf ? rb_compiled<double, 10, false, true>(rb) : rb_compiled<double, 10, false, false>(rb));
    return so ? (mf ? rb_compiled<float, 10, true, true>(rb) : rb_compiled<float, 10, true, false>(rb))
              : (mf ? rb_compiled<float, 10, false, true>(rb) : rb_compiled<float, 10, false, false>(rb));
  }
  if (f64) return so ? (mf ? rb_compiled<double, 5, true, true>(rb) : rb_compiled<double, 5, true, false>(rb))
                     : (mf ? rb_compiled<double, 5, false, true>(rb) : rb_compiled<double, 5, false, false>(rb));
  return so ? (mf ? rb_compiled<float, 5, true, true>(rb) : rb_compiled<float, 5, true, false>(rb))
            : (mf ? rb_compiled<float, 5, false, true>(rb) : rb_compiled<float, 5, false, false>(rb));
}

template <typename T>
static cudaError_t launch_prec(const omen_ham* h, const T* blk, const T* b0, const T* scale, const void* x, void* y,
                               int nvec, double sigma, cudaStream_t st, int cell0, int cell1) {
  const omen_lattice* L = h->lat;
  HxArgs<T> a;
  a.g = Geo{L->nx, L->ny, L->nz, L->ncells, L->natoms, {L->periodic[0], L->periodic[1], L->periodic[2]}};
  a.nt = host_neighbour_tables();
  a.blk = blk;
  a.b0 = b0;
  a.scale = scale;
  a.species = L->d_species;
  a.onsite = h->d_onsite;
  if constexpr (sizeof(T) == 8) a.onsite_t = reinterpret_cast<const T*>(h->d_onsite);
  else a.onsite_t = reinterpret_cast<const T*>(h->d_onsite32);
  a.U = h->d_U;
  a.lambda = h->d_lambda;
  a.x = x;
  a.y = y;
  a.nrows = h->nrows;
  a.sigma = sigma;
  for (int d = 0; d < 3; ++d) a.phase[d] = h->phase[d];
  a.ns = h->nspecies;
  a.slot_stride = h->slot_stride;
  a.cell0 = cell0;
  a.cell1 = cell1;
  const HxTile t = h->tile[sizeof(T) == 8 ? 0 : 1];
  return h->norb == 10 ? launch_norb<T, 10>(a, h, nvec, t, st) : launch_norb<T, 5>(a, h, nvec, t, st);
}

// y rows of the cells [cell0, cell1) (all orbitals, sites, vectors); the rest of y is untouched
static omen_status launch_hx_cells(omen_ctx* ctx, const omen_ham* h, const void* x, void* y, int nvec, double sigma,
                                   int vec_precision, int cell0, int cell1, cudaStream_t st) {
  if (nvec < 1 || nvec > 65535) return set_err(ctx, OMEN_EINVAL, "nvec must be 1..65535");
  if (cell1 <= cell0) return OMEN_OK;
  cudaError_t e;
  if (vec_precision == OMEN_F64_DF) {
    if (!h->d_blkdf) return set_err(ctx, OMEN_EINVAL, "Hamiltonian has no double-float blocks");
    e = launch_df(h, x, y, nvec, sigma, st, cell0, cell1);
  } else if (vec_precision == OMEN_F64) {
    if (!h->matrix_free && !h->d_blk64) return set_err(ctx, OMEN_EINVAL, "Hamiltonian has no FP64 blocks");
    e = launch_prec<double>(h, h->d_blk64, h->d_b0_64, h->d_scale64, x, y, nvec, sigma, st, cell0, cell1);
  } else {
    if (!h->matrix_free && !h->d_blk32) return set_err(ctx, OMEN_EINVAL, "Hamiltonian has no FP32 blocks");
    e = launch_prec<float>(h, h->d_blk32, h->d_b0_32, h->d_scale32, x, y, nvec, sigma, st, cell0, cell1);
  }
  if (e != cudaSuccess) return set_err(ctx, OMEN_ECUDA, "H·X launch failed: %s", cudaGetErrorString(e));
  return OMEN_OK;
}

omen_status launch_hx(omen_ctx* ctx, const omen_ham* h, const void* x, void* y, int nvec, double sigma, int vec_precision) {
  if (h->effmass) return launch_hx_effmass(ctx, h, x, y, nvec, sigma, vec_precision, ctx->stream);
  return launch_hx_cells(ctx, h, x, y, nvec, sigma, vec_precision, 0, h->lat->ncells, ctx->stream);
}

// The vector type of the Hamiltonian's products: FP32 for OMEN_F32 and OMEN_F32_REFINE64 (the
// refinement is internal to omen_eigs), double-float pairs for OMEN_F64_DF, else FP64.
static int native_precision(const omen_ham* h) {
  if (h->precision == OMEN_F64_DF) return OMEN_F64_DF;
  return (h->precision == OMEN_F32 || h->precision == OMEN_F32_REFINE64) ? OMEN_F32 : OMEN_F64;
}

extern "C" omen_status omen_hx(omen_ctx* ctx, const omen_ham* h, const void* x, void* y, int nvec, double sigma) {
  if (!ctx || !h || !x || !y) return set_err(ctx, OMEN_EINVAL, "null argument");
  return launch_hx(ctx, h, x, y, nvec, sigma, native_precision(h));
}

// Host-buffer product with the copies overlapped: the structure is cut into slabs of whole
// z-planes; slab i of x goes up on one copy stream, its rows of y are computed on the context's
// stream as soon as the planes they touch (the slab and one plane on each side) are on the
// device, and go down on the other copy stream while later slabs compute.  A slab of every
// vector is one strided copy: rows (vector, orbital, site) are ncells apart and a slab's cells
// are contiguous within each.  With a periodic z axis the first slab also needs the last
// plane, so it is computed last.
static omen_status hx_host_pipelined(omen_ctx* ctx, const omen_ham* h, const void* xh, void* yh, void* dx, void* dy,
                                     int nvec, double sigma) {
  const omen_lattice* L = h->lat;
  const int prec = native_precision(h);
  const size_t el = vec_elem_bytes(h, prec);
  const int plane = L->nx * L->ny;
  const int S = std::max(1, std::min(8, L->nz / 2));
  const size_t pitch = (size_t)L->ncells * el;
  const size_t rows = (size_t)nvec * (size_t)(h->nrows / L->ncells);   // (vector, orbital, site) runs
  for (int k = 0; k < 2; ++k)
    if (!ctx->copy_stream[k] && cudaStreamCreateWithFlags(&ctx->copy_stream[k], cudaStreamNonBlocking) != cudaSuccess) {
      ctx->copy_stream[k] = nullptr;
      return set_err(ctx, OMEN_ECUDA, "could not create a copy stream");
    }
  cudaStream_t sin = ctx->copy_stream[0], sout = ctx->copy_stream[1];
  omen_status st = OMEN_OK;
  while (st == OMEN_OK && ctx->host_events.size() < (size_t)(2 * S + 2)) {
    cudaEvent_t e = nullptr;
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) st = set_err(ctx, OMEN_ECUDA, "event creation failed");
    else ctx->host_events.push_back(e);
  }
  if (st != OMEN_OK) return st;
  std::vector<cudaEvent_t>& ev = ctx->host_events;
  auto z0 = [&](int i) { return (int)((long long)L->nz * i / S); };
  cudaEvent_t* ein = ev.data();
  cudaEvent_t* ecomp = ev.data() + S;
  cudaEvent_t start = ev[2 * S], done = ev[2 * S + 1];
  cudaError_t e = cudaSuccess;
  if (st == OMEN_OK) {
    // order the copy streams after the context's stream (earlier work on the buffers)
    e = cudaEventRecord(start, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(sin, start, 0);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(sout, start, 0);
  }
  for (int i = 0; i < S && st == OMEN_OK && e == cudaSuccess; ++i) {
    const size_t c0 = (size_t)z0(i) * plane, c1 = (size_t)z0(i + 1) * plane;
    e = cudaMemcpy2DAsync(static_cast<char*>(dx) + c0 * el, pitch, static_cast<const char*>(xh) + c0 * el, pitch,
                          (c1 - c0) * el, rows, cudaMemcpyHostToDevice, sin);
    if (e == cudaSuccess) e = cudaEventRecord(ein[i], sin);
  }
  const bool zper = L->periodic[2] != OMEN_HARD_WALL;
  for (int t = 0; t < S && st == OMEN_OK && e == cudaSuccess; ++t) {
    const int i = zper ? (t + 1) % S : t;     // periodic z: slab 0 last
    const int need = zper && i == 0 ? S - 1 : std::min(i + 1, S - 1);
    e = cudaStreamWaitEvent(ctx->stream, ein[need], 0);
    if (e != cudaSuccess) break;
    st = launch_hx_cells(ctx, h, dx, dy, nvec, sigma, prec, z0(i) * plane, z0(i + 1) * plane, ctx->stream);
    if (st != OMEN_OK) break;
    e = cudaEventRecord(ecomp[i], ctx->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(sout, ecomp[i], 0);
    const size_t c0 = (size_t)z0(i) * plane, c1 = (size_t)z0(i + 1) * plane;
    if (e == cudaSuccess)
      e = cudaMemcpy2DAsync(static_cast<char*>(yh) + c0 * el, pitch, static_cast<const char*>(dy) + c0 * el, pitch,
                            (c1 - c0) * el, rows, cudaMemcpyDeviceToHost, sout);
  }
  // the context's stream (and the caller's frees on it) wait for the last copy down
  if (st == OMEN_OK && e == cudaSuccess) e = cudaEventRecord(done, sout);
  if (st == OMEN_OK && e == cudaSuccess) e = cudaStreamWaitEvent(ctx->stream, done, 0);
  if (st == OMEN_OK && e != cudaSuccess) st = set_err(ctx, OMEN_ECUDA, "host H·X copies: %s", cudaGetErrorString(e));
  if (st != OMEN_OK) {
    // leave nothing in flight on the copy streams before the buffers go back
    cudaStreamSynchronize(sin);
    cudaStreamSynchronize(sout);
  }
  return st;
}

extern "C" omen_status omen_hx_host(omen_ctx* ctx, const omen_ham* h, const void* xh, void* yh, int nvec, double sigma) {
  if (!ctx || !h || !xh || !yh) return set_err(ctx, OMEN_EINVAL, "null argument");
  if (nvec < 1) return set_err(ctx, OMEN_EINVAL, "nvec must be >= 1");
  const size_t bytes = vec_elem_bytes(h, native_precision(h)) * (size_t)h->nrows * nvec;
  if (h->precision == OMEN_F64_DF) {
    // FP64 host arrays; double-float conversion on the device
    const long long n = h->nrows * nvec;
    void *dx = nullptr, *dy = nullptr, *fx = nullptr;
    if (cudaMallocAsync(&dx, bytes, ctx->stream) != cudaSuccess || cudaMallocAsync(&dy, bytes, ctx->stream) != cudaSuccess ||
        cudaMallocAsync(&fx, 8 * (size_t)n, ctx->stream) != cudaSuccess) {
      cudaGetLastError();
      return set_err(ctx, OMEN_ENOMEM, "device allocation of %zu bytes failed", bytes);
    }
    omen_status st = OMEN_OK;
    cudaError_t e = cudaMemcpyAsync(fx, xh, 8 * (size_t)n, cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess) st = omen_convert_vectors(ctx, fx, OMEN_F64, dx, OMEN_F64_DF, n);
    if (e == cudaSuccess && st == OMEN_OK) st = launch_hx(ctx, h, dx, dy, nvec, sigma, OMEN_F64_DF);
    if (e == cudaSuccess && st == OMEN_OK) st = omen_convert_vectors(ctx, dy, OMEN_F64_DF, fx, OMEN_F64, n);
    if (e == cudaSuccess && st == OMEN_OK) e = cudaMemcpyAsync(yh, fx, 8 * (size_t)n, cudaMemcpyDeviceToHost, ctx->stream);
    cudaFreeAsync(dx, ctx->stream);
    cudaFreeAsync(dy, ctx->stream);
    cudaFreeAsync(fx, ctx->stream);
    cudaError_t e2 = cudaStreamSynchronize(ctx->stream);
    if (st != OMEN_OK) return st;
    if (e != cudaSuccess || e2 != cudaSuccess)
      return set_err(ctx, OMEN_ECUDA, "host H·X failed: %s", cudaGetErrorString(e != cudaSuccess ? e : e2));
    return OMEN_OK;
  }
  const size_t half = (bytes + 255) / 256 * 256;
  if (ctx->host_scratch_bytes < 2 * half) {
    // grow the context's scratch (synchronises the device once; later calls reuse it)
    OMEN_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    if (ctx->host_scratch) cudaFree(ctx->host_scratch);
    ctx->host_scratch = nullptr;
    ctx->host_scratch_bytes = 0;
    if (cudaMalloc(&ctx->host_scratch, 2 * half) != cudaSuccess) {
      cudaGetLastError();
      ctx->host_scratch = nullptr;
      return set_err(ctx, OMEN_ENOMEM, "device allocation of %zu bytes failed", 2 * half);
    }
    ctx->host_scratch_bytes = 2 * half;
  }
  void* dx = ctx->host_scratch;
  void* dy = static_cast<char*>(ctx->host_scratch) + half;
  omen_status st = OMEN_OK;
  if (h->effmass) {
    // one copy up, the product, one copy down
    cudaError_t e = cudaMemcpyAsync(dx, xh, bytes, cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess) st = launch_hx(ctx, h, dx, dy, nvec, sigma, native_precision(h));
    if (e == cudaSuccess && st == OMEN_OK) e = cudaMemcpyAsync(yh, dy, bytes, cudaMemcpyDeviceToHost, ctx->stream);
    if (e != cudaSuccess && st == OMEN_OK) st = set_err(ctx, OMEN_ECUDA, "host H·X copies: %s", cudaGetErrorString(e));
  } else {
    st = hx_host_pipelined(ctx, h, xh, yh, dx, dy, nvec, sigma);
  }
  cudaError_t e2 = cudaStreamSynchronize(ctx->stream);
  if (st != OMEN_OK) return st;
  if (e2 != cudaSuccess) return set_err(ctx, OMEN_ECUDA, "host H·X failed: %s", cudaGetErrorString(e2));
  return OMEN_OK;
}

// Wave vectors per thread KB: 2 by default (the FP64 register budget: 2 x 10 complex
// amplitudes per bond); 1, 2, 4 compiled for FP32 and 1, 2 for FP64.
static constexpr int kKB = 2;
static bool kb_compiled(bool f64, int kb) { return kb == 0 || kb == 1 || kb == 2 || (!f64 && kb == 4); }

bool hx_kbatch_tile_valid(int vec_precision, int threads, int kb) {
  if (threads != 0 && (threads < 32 || threads > 128 || threads % 32 != 0)) return false;
  return kb_compiled(vec_precision == OMEN_F64, kb);
}

template <typename T, int KB>
static cudaError_t launch_kb(KMulti<T>& m, int norb, int threads, cudaStream_t st) {
  long long total = 0;
  for (int i = 0; i < m.n; ++i) {
    m.in[i].tiles = ((m.in[i].g.ncells + threads - 1) / threads) * 8;
    m.in[i].cta0 = (int)total;
    total += (long long)m.in[i].tiles * ((m.in[i].nk + KB - 1) / KB);
  }
  if (total > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
  if (norb == 10) hx_kbatch_kernel<T, 10, KB><<<(unsigned)total, threads, 0, st>>>(m);
  else hx_kbatch_kernel<T, 5, KB><<<(unsigned)total, threads, 0, st>>>(m);
  return cudaGetLastError();
}

template <typename T>
static cudaError_t launch_kmulti_prec(const KItem* items, int nitems, const void* x, void* y, double sigma,
                                      cudaStream_t st) {
  KMulti<T> m;
  m.nt = host_neighbour_tables();
  m.n = nitems;
  m.x = x;
  m.y = y;
  m.sigma = sigma;
  for (int i = 0; i < nitems; ++i) {
    const omen_ham* h = items[i].ham;
    const omen_lattice* L = h->lat;
    KInst<T>& I = m.in[i];
    I.g = Geo{L->nx, L->ny, L->nz, L->ncells, L->natoms, {L->periodic[0], L->periodic[1], L->periodic[2]}};
    if constexpr (sizeof(T) == 8) I.blk = h->d_blk64; else I.blk = h->d_blk32;
    I.species = L->d_species;
    I.onsite = h->d_onsite;
    I.U = h->d_U;
    I.phases = items[i].phases;
    I.nrows = h->nrows;
    I.x_off = items[i].x_off;
    I.nk = items[i].nk;
    I.slot_stride = h->slot_stride;
  }
  const HxTile t = items[0].ham->ktile[sizeof(T) == 8 ? 0 : 1];
  const int thr = t.threads ? t.threads : 128;
  if (t.rb == 1) return launch_kb<T, 1>(m, items[0].ham->norb, thr, st);
  if constexpr (sizeof(T) == 4) if (t.rb == 4) return launch_kb<T, 4>(m, items[0].ham->norb, thr, st);
  return launch_kb<T, kKB>(m, items[0].ham->norb, thr, st);
}

omen_status launch_hx_kmulti(omen_ctx* ctx, const KItem* items, int nitems, const void* x, void* y, double sigma,
                             int vec_precision) {
  if (nitems < 1 || nitems > kMaxKInst) return set_err(ctx, OMEN_EINVAL, "1..%d structures per k batch", kMaxKInst);
  const bool f64 = vec_precision == OMEN_F64;
  for (int i = 0; i < nitems; ++i) {
    const omen_ham* h = items[i].ham;
    if (!h || items[i].nk < 1 || items[i].nk > 65535) return set_err(ctx, OMEN_EINVAL, "structure %d: null or nk out of range", i);
    if (!h->bloch || h->matrix_free || h->spin_orbit)
      return set_err(ctx, OMEN_EUNSUPPORTED, "k batch needs Bloch structures with stored blocks and no spin-orbit");
    if (h->norb != items[0].ham->norb) return set_err(ctx, OMEN_EINVAL, "structures of one k batch share the basis");
    if (f64 ? !h->d_blk64 : !h->d_blk32) return set_err(ctx, OMEN_EINVAL, "structure %d has no blocks of this precision", i);
  }
  const cudaError_t e = f64 ? launch_kmulti_prec<double>(items, nitems, x, y, sigma, ctx->stream)
                            : launch_kmulti_prec<float>(items, nitems, x, y, sigma, ctx->stream);
  if (e != cudaSuccess) return set_err(ctx, OMEN_ECUDA, "k-batched H·X launch: %s", cudaGetErrorString(e));
  return OMEN_OK;
}

omen_status launch_hx_kbatch(omen_ctx* ctx, const omen_ham* h, int nk, const double2* phases_dev, const void* x, void* y,
                             double sigma, int vec_precision) {
  const KItem item{h, nk, phases_dev, 0};
  return launch_hx_kmulti(ctx, &item, 1, x, y, sigma, vec_precision);
}

omen_status make_phases(omen_ctx* ctx, const omen_ham* h, int nk, const double* k_host, double2** out) {
  const omen_lattice* L = h->lat;
  std::vector<double2> ph((size_t)nk * 3);
  const int nc[3] = {L->nx, L->ny, L->nz};
  for (int q = 0; q < nk; ++q)
    for (int d = 0; d < 3; ++d) {
      const double t = (L->periodic[d] == OMEN_BLOCH) ? k_host[q * 3 + d] * nc[d] * L->a_nm : 0.0;
      ph[(size_t)q * 3 + d] = make_double2(cos(t), sin(t));
    }
  if (cudaMallocAsync(out, sizeof(double2) * ph.size(), ctx->stream) != cudaSuccess) {
    cudaGetLastError();
    return set_err(ctx, OMEN_ENOMEM, "phase table");
  }
  OMEN_CUDA(ctx, cudaMemcpyAsync(*out, ph.data(), sizeof(double2) * ph.size(), cudaMemcpyHostToDevice, ctx->stream));
  return OMEN_OK;
}

extern "C" omen_status omen_hx_kbatch_multi(omen_ctx* ctx, int nitems, const omen_kbatch_item* it, const void* x, void* y,
                                            double sigma) {
  if (!ctx || !it || !x || !y || nitems < 1 || nitems > kMaxKInst) return set_err(ctx, OMEN_EINVAL, "null argument or 1..%d structures", kMaxKInst);
  std::vector<KItem> items(nitems);
  std::vector<double2*> ph(nitems, nullptr);
  long long off = 0;
  omen_status s = OMEN_OK;
  for (int i = 0; i < nitems && s == OMEN_OK; ++i) {
    if (!it[i].ham || !it[i].k_host || it[i].nk < 1) { s = set_err(ctx, OMEN_EINVAL, "structure %d: null argument or nk < 1", i); break; }
    if (it[i].ham->effmass) { s = set_err(ctx, OMEN_EUNSUPPORTED, "k batch runs on tight-binding Hamiltonians"); break; }
    if (!it[i].ham->bloch) { s = set_err(ctx, OMEN_EINVAL, "structure %d has no Bloch-periodic direction", i); break; }
    s = make_phases(ctx, it[i].ham, it[i].nk, it[i].k_host, &ph[i]);
    items[i] = KItem{it[i].ham, it[i].nk, ph[i], off};
    off += (long long)it[i].nk * it[i].ham->nrows;
  }
  if (s == OMEN_OK) {
    const omen_ham* h0 = it[0].ham;
    for (int i = 1; i < nitems && s == OMEN_OK; ++i)
      if (it[i].ham->precision != h0->precision) s = set_err(ctx, OMEN_EINVAL, "structures of one k batch share the precision");
    if (s == OMEN_OK) s = launch_hx_kmulti(ctx, items.data(), nitems, x, y, sigma, native_precision(h0));
  }
  for (double2* q : ph)
    if (q) cudaFreeAsync(q, ctx->stream);
  return s;
}

extern "C" omen_status omen_hx_kbatch(omen_ctx* ctx, const omen_ham* h, int nk, const double* k_host, const void* x,
                                      void* y, double sigma) {
  if (!ctx || !h || !k_host || !x || !y || nk < 1) return set_err(ctx, OMEN_EINVAL, "null argument or nk < 1");
  if (h->effmass) return set_err(ctx, OMEN_EUNSUPPORTED, "k batch runs on tight-binding Hamiltonians");
  if (!h->bloch) return set_err(ctx, OMEN_EINVAL, "k batch needs a structure with Bloch-periodic directions");
  double2* ph = nullptr;
  omen_status s = make_phases(ctx, h, nk, k_host, &ph);
  if (s != OMEN_OK) return s;
  s = launch_hx_kbatch(ctx, h, nk, ph, x, y, sigma, native_precision(h));
  cudaFreeAsync(ph, ctx->stream);
  return s;
}
