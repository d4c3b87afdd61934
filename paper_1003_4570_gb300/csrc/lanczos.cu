// Thick-restart block Lanczos with full reorthogonalisation, plain and folded spectrum
// (paper Section III-A item 1: "(block) Lanczos"; Section II-B: the Lanczos iteration is the
// benchmarked unit).
//
// Operator A = H (lowest eigenvalues) or A = (H - sigma)^2 (folded spectrum: eigenvalues of H
// nearest sigma, taken as Rayleigh quotients <x, H x>).  Each block step:
//   W = A V_j;  twice: h = V^H W, W -= V h (classical Gram–Schmidt, applied twice);
//   W = V_{j+1} R by Cholesky QR (twice);  T[:, j] = sum of h, T[j+1, j] = R.
// When the basis is full, the Rayleigh–Ritz pairs of T are computed on the host in FP64;
// the wanted Ritz vectors and the residual block are kept (Wu & Simon's thick restart, in
// block form) and the recurrence continues from them.
// Krylov vectors are FP64 or FP32 (complex when H is); all coefficients (h, R, T, Ritz
// values) are accumulated and kept in FP64.  OMEN_F32_REFINE64 finishes with FP64
// Rayleigh–Ritz steps on span{X, H X - X Lambda}.
#include <algorithm>
#include <array>
#include <omp.h>

#include <chrono>
#include <cmath>
#include <complex>
#include <cstring>
#include <map>
#include <mutex>
#include <type_traits>
#include <vector>

#include "dense_eig.h"
#include "omen_internal.h"
#include "vec.cuh"
#include "df.cuh"

using cd = std::complex<double>;

static constexpr int kMaxBlockCols = 16;   // columns handled per pass by the small kernels
static constexpr int kDotThreads = 256;

// ---------------------------------------------------------------------------------------
// P[chunk][i][j] = sum over rows of the chunk of conj(A_i[r]) * B_j[r]   (FP64 accumulators)
template <typename T, bool C>
__global__ void __launch_bounds__(kDotThreads) dots_partial_kernel(const void* Av, long long lda, int na,
                                                                   const void* Bv, long long ldb, int nb,
                                                                   long long n, int CH, double2* __restrict__ P) {
  using E = Elem<T, C>;
  using V = typename E::V;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V* Bs = reinterpret_cast<V*>(smem_raw);
  const V* A = static_cast<const V*>(Av);
  const V* B = static_cast<const V*>(Bv);
  const long long r0 = (long long)blockIdx.x * CH;
  const int len = (int)min((long long)CH, n - r0);
  for (int j = 0; j < nb; ++j)
    for (int t = threadIdx.x; t < len; t += blockDim.x) Bs[j * CH + t] = B[j * ldb + r0 + t];
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int i = warp; i < na; i += nw) {
    double ar[kMaxBlockCols], ai[kMaxBlockCols];
#pragma unroll
    for (int j = 0; j < kMaxBlockCols; ++j) { ar[j] = 0.0; ai[j] = 0.0; }
    const V* Ai = A + i * lda + r0;
    for (int t = lane; t < len; t += 32) {
      const V a = Ai[t];
      const double xr = E::re(a), xi = E::im(a);
#pragma unroll
      for (int j = 0; j < kMaxBlockCols; ++j) {
        if (j < nb) {
          const V bv = Bs[j * CH + t];
          const double yr = E::re(bv);
          ar[j] = fma(xr, yr, ar[j]);
          if constexpr (C) {
            const double yi = E::im(bv);
            ar[j] = fma(xi, yi, ar[j]);
            ai[j] = fma(xr, yi, ai[j]);
            ai[j] = fma(-xi, yr, ai[j]);
          }
        }
      }
    }
#pragma unroll
    for (int j = 0; j < kMaxBlockCols; ++j) {
      if (j < nb) {
        double sr = ar[j], si = ai[j];
        for (int o = 16; o > 0; o >>= 1) {
          sr += __shfl_xor_sync(0xffffffffu, sr, o);
          si += __shfl_xor_sync(0xffffffffu, si, o);
        }
        if (lane == 0) P[((size_t)blockIdx.x * na + i) * nb + j] = make_double2(sr, si);
      }
    }
  }
}

__global__ void reduce_partial_kernel(const double2* __restrict__ P, int nchunks, int count, double2* __restrict__ out) {
  const int e = blockIdx.x;
  double sr = 0.0, si = 0.0;
  for (int c = threadIdx.x; c < nchunks; c += blockDim.x) {
    const double2 v = P[(size_t)c * count + e];
    sr += v.x;
    si += v.y;
  }
  __shared__ double red[2][32];
  for (int o = 16; o > 0; o >>= 1) {
    sr += __shfl_xor_sync(0xffffffffu, sr, o);
    si += __shfl_xor_sync(0xffffffffu, si, o);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) { red[0][warp] = sr; red[1][warp] = si; }
  __syncthreads();
  if (warp == 0) {
    const int nw = blockDim.x >> 5;
    sr = lane < nw ? red[0][lane] : 0.0;
    si = lane < nw ? red[1][lane] : 0.0;
    for (int o = 16; o > 0; o >>= 1) {
      sr += __shfl_xor_sync(0xffffffffu, sr, o);
      si += __shfl_xor_sync(0xffffffffu, si, o);
    }
    if (lane == 0) out[e] = make_double2(sr, si);
  }
}

// Projections onto one vector, P[chunk][i] = sum_r conj(A_i[r]) b[r], for the common case of a
// single right-hand vector.  CTA (g, c) handles basis vectors 16g..16g+15 over row chunk c;
// each thread keeps 16 independent loads in flight per row.  Consecutive CTAs share a chunk,
// so b stays in L2 across the basis groups.  FP64 vectors accumulate in FP64; FP32 vectors
// accumulate each thread's rows in compensated FP32 (Kahan) before the FP64 block sum.
static constexpr int kIG = 16;
// basis vectors per CTA of dots1_kernel: 16 real, 8 complex (the complex accumulators would
// otherwise hold the kernel to one CTA per SM)
static constexpr int dots1_ig(bool cplx) { return cplx ? 8 : kIG; }
template <typename T, bool C, int IG>
__global__ void __launch_bounds__(256, C ? 1 : 2) dots1_kernel(const void* Av, long long lda, int na, const void* Bv,
                                                    long long n, int rows_per_cta, double2* __restrict__ P,
                                                    long long a_ps = 0, long long b_ps = 0, long long p_ps = 0,
                                                    const long long* __restrict__ poff = nullptr,
                                                    const long long* __restrict__ plen = nullptr,
                                                    const int* __restrict__ act = nullptr) {
  using E = Elem<T, C>;
  using V = typename E::V;
  using Acc = std::conditional_t<sizeof(T) == 8, double, float>;
  // IG basis vectors per CTA (at most dots1_ig(C)); chosen from na so that no accumulator
  // sits idle under a predicate (predicated-off FP64 FMAs still occupy the pipe)
  // grid.z = independent problems (batched Lanczos): offsets a_ps, b_ps (elements), p_ps
  // (partials) per problem, or per-problem element offsets poff and lengths plen
  const long long off = poff ? poff[blockIdx.z] : 0;
  if (act && !act[blockIdx.z]) return;   // a converged (frozen) problem of the batch
  if (plen) n = plen[blockIdx.z];
  const V* A = static_cast<const V*>(Av) + blockIdx.z * a_ps + off;
  const V* B = static_cast<const V*>(Bv) + blockIdx.z * b_ps + off;
  P += blockIdx.z * p_ps;
  const int i0 = blockIdx.x * IG;
  const int ni = min(IG, na - i0);
  const long long r0 = (long long)blockIdx.y * rows_per_cta;
  const long long r1 = min(n, r0 + rows_per_cta);
  Acc sr[IG], si[IG], cr[IG], ci[IG];
#pragma unroll
  for (int i = 0; i < IG; ++i) { sr[i] = 0; si[i] = 0; cr[i] = 0; ci[i] = 0; }
  for (long long r = r0 + threadIdx.x; r < r1; r += blockDim.x) {
    const V bv = B[r];
    V av[IG];
#pragma unroll
    for (int i = 0; i < IG; ++i)
      if (i < ni) av[i] = A[(size_t)(i0 + i) * lda + r];
#pragma unroll
    for (int i = 0; i < IG; ++i) {
      if (i < ni) {
        Acc pr, pi = 0;
        if constexpr (C) {
          pr = (Acc)av[i].x * (Acc)bv.x + (Acc)av[i].y * (Acc)bv.y;
          pi = (Acc)av[i].x * (Acc)bv.y - (Acc)av[i].y * (Acc)bv.x;
        } else {
          pr = (Acc)av[i] * (Acc)bv;
        }
        if constexpr (sizeof(T) == 8) {
          sr[i] += pr;
          si[i] += pi;
        } else {  // Kahan-compensated FP32 sums
          const Acc yr = pr - cr[i], tr = sr[i] + yr;
          cr[i] = (tr - sr[i]) - yr;
          sr[i] = tr;
          const Acc yi = pi - ci[i], ti = si[i] + yi;
          ci[i] = (ti - si[i]) - yi;
          si[i] = ti;
        }
      }
    }
  }
  __shared__ double red[8][IG > 0 ? IG : 1][2];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int i = 0; i < IG; ++i) {
    double vr = (double)sr[i] - (double)cr[i], vi = (double)si[i] - (double)ci[i];
    for (int o = 16; o > 0; o >>= 1) {
      vr += __shfl_xor_sync(0xffffffffu, vr, o);
      if constexpr (C) vi += __shfl_xor_sync(0xffffffffu, vi, o);
    }
    if (lane == 0) { red[warp][i][0] = vr; red[warp][i][1] = vi; }
  }
  __syncthreads();
  if (threadIdx.x < ni) {
    double vr = 0.0, vi = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { vr += red[w][threadIdx.x][0]; vi += red[w][threadIdx.x][1]; }
    P[(size_t)blockIdx.y * na + i0 + threadIdx.x] = make_double2(vr, C ? vi : 0.0);
  }
}

// y = beta*y + sum_i A_i Ms_i over this CTA's rows (Ms: coefficients in shared memory, alpha
// already applied), 8 basis loads in flight per row.
template <typename T, bool C, typename A2>
__device__ __forceinline__ void combine1_rows(const typename Elem<T, C>::V* __restrict__ A, long long lda, int na,
                                              const A2* __restrict__ Ms, typename Elem<T, C>::V* __restrict__ Y,
                                              long long n, T rbeta, bool use_beta) {
  using V = typename Elem<T, C>::V;
  using R = T;
  for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (long long)gridDim.x * blockDim.x) {
    R yr = 0, yi = 0;
    int i = 0;
    for (; i + 8 <= na; i += 8) {
      V av[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) av[k] = A[(size_t)(i + k) * lda + r];
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const A2 m = Ms[i + k];
        if constexpr (C) {
          yr = fma(av[k].x, m.x, yr);
          yr = fma(-av[k].y, m.y, yr);
          yi = fma(av[k].x, m.y, yi);
          yi = fma(av[k].y, m.x, yi);
        } else {
          yr = fma(av[k], m.x, yr);
        }
      }
    }
    for (; i < na; ++i) {
      const V a = A[(size_t)i * lda + r];
      const A2 m = Ms[i];
      if constexpr (C) {
        yr = fma(a.x, m.x, yr);
        yr = fma(-a.y, m.y, yr);
        yi = fma(a.x, m.y, yi);
        yi = fma(a.y, m.x, yi);
      } else {
        yr = fma(a, m.x, yr);
      }
    }
    V out;
    if constexpr (C) {
      out.x = yr;
      out.y = yi;
      if (use_beta) {
        out.x = fma(rbeta, Y[r].x, out.x);
        out.y = fma(rbeta, Y[r].y, out.y);
      }
    } else {
      out = yr;
      if (use_beta) out = fma(rbeta, Y[r], out);
    }
    Y[r] = out;
  }
}

// y = beta*y + alpha * sum_i A_i m_i for one output vector.
// FP64 vectors accumulate in FP64; FP32 vectors in FP32 (coefficients rounded once from their
// FP64 values; the result is stored in FP32), which keeps them off GB300's slow FP64 pipe.
template <typename T, bool C>
__global__ void __launch_bounds__(256) combine1_kernel(const void* Av, long long lda, int na, const double2* __restrict__ M,
                                                       void* Yv, long long n, double alpha, double beta,
                                                       long long a_ps = 0, long long m_ps = 0, long long y_ps = 0,
                                                       const long long* __restrict__ poff = nullptr,
                                                       const long long* __restrict__ plen = nullptr,
                                                       const int* __restrict__ act = nullptr) {
  using E = Elem<T, C>;
  using V = typename E::V;
  using A2 = std::conditional_t<sizeof(T) == 8, double2, float2>;
  using R = T;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  A2* Ms = reinterpret_cast<A2*>(smem_raw);
  M += blockIdx.y * m_ps;
  for (int t = threadIdx.x; t < na; t += blockDim.x) {
    A2 m;
    m.x = (R)(alpha * M[t].x);
    m.y = (R)(alpha * M[t].y);
    Ms[t] = m;
  }
  __syncthreads();
  const long long off = poff ? poff[blockIdx.y] : 0;
  if (act && !act[blockIdx.y]) return;
  if (plen) n = plen[blockIdx.y];
  const V* A = static_cast<const V*>(Av) + blockIdx.y * a_ps + off;
  V* Y = static_cast<V*>(Yv) + blockIdx.y * y_ps + off;
  combine1_rows<T, C, A2>(A, lda, na, Ms, Y, n, (R)beta, beta != 0.0);
}

// The update w -= V h of the full Gram–Schmidt pass, applied only where it is needed to keep
// the basis semi-orthogonal (Simon, Math. Comp. 42 (1984) 115): when some |h_i| exceeds
// eta * ||w|| (eta = square root of the vectors' unit roundoff; ||w||^2 read from nrm2), or
// when the previous step applied its pass (a correction is always repeated once, since the
// vector it repairs feeds the next step).  gate[parity] records whether this step applied it,
// gate[parity ^ 1] is the previous step's record.  When applied, h is also added into column
// Tcol of the projected matrix.
template <typename T, bool C>
__global__ void __launch_bounds__(256) combine1_gated_kernel(const void* Av, int na, const double2* __restrict__ M,
                                                             void* Yv, long long n, const double2* __restrict__ nrm2,
                                                             double eta, int* __restrict__ gate, int parity,
                                                             double2* __restrict__ Tcol) {
  using E = Elem<T, C>;
  using V = typename E::V;
  using A2 = std::conditional_t<sizeof(T) == 8, double2, float2>;
  using R = T;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  A2* Ms = reinterpret_cast<A2*>(smem_raw);
  __shared__ int any;
  if (threadIdx.x == 0) any = 0;
  __syncthreads();
  const double lim = eta * eta * fmax(nrm2->x, 0.0);
  int mine = 0;
  for (int t = threadIdx.x; t < na; t += blockDim.x) {
    const double2 h = M[t];
    if (h.x * h.x + h.y * h.y > lim || !(h.x == h.x) || !(h.y == h.y)) mine = 1;
    A2 m;
    m.x = (R)(-h.x);
    m.y = (R)(-h.y);
    Ms[t] = m;
  }
  if (mine) any = 1;
  __syncthreads();
  const bool run = any || gate[parity ^ 1];
  if (blockIdx.x == 0 && threadIdx.x == 0) gate[parity] = run ? 1 : 0;
  if (!run) return;
  if (blockIdx.x == 0)
    for (int t = threadIdx.x; t < na; t += blockDim.x) {
      Tcol[t].x += M[t].x;
      Tcol[t].y += M[t].y;
    }
  combine1_rows<T, C, A2>(static_cast<const V*>(Av), n, na, Ms, static_cast<V*>(Yv), n, (R)1, true);
}

// Projections onto NB right-hand columns at once (2 <= NB <= 4): CTA (g, c) handles basis
// vectors IG*g .. IG*g + IG-1 (IG = 16 / NB real, 8 / NB complex) over row chunk c; every basis load serves all NB
// columns.  Partials P[chunk][i][j].
template <typename T, bool C, int NB>
__global__ void __launch_bounds__(256) dotsn_kernel(const void* Av, long long lda, int na, const void* Bv, long long ldb,
                                                    int nb, long long n, int rows_per_cta, double2* __restrict__ P) {
  using E = Elem<T, C>;
  using V = typename E::V;
  using Acc = std::conditional_t<sizeof(T) == 8, double, float>;
  constexpr int IG = dots1_ig(C) / NB;
  const V* A = static_cast<const V*>(Av);
  const V* B = static_cast<const V*>(Bv);
  const int i0 = blockIdx.x * IG;
  const int ni = min(IG, na - i0);
  const long long r0 = (long long)blockIdx.y * rows_per_cta;
  const long long r1 = min(n, r0 + rows_per_cta);
  Acc sr[IG][NB], si[IG][NB], cr[IG][NB], ci[IG][NB];   // c*: Kahan compensation (FP32 only)
#pragma unroll
  for (int i = 0; i < IG; ++i)
#pragma unroll
    for (int j = 0; j < NB; ++j) { sr[i][j] = 0; si[i][j] = 0; cr[i][j] = 0; ci[i][j] = 0; }
  for (long long r = r0 + threadIdx.x; r < r1; r += blockDim.x) {
    V bv[NB], av[IG];
#pragma unroll
    for (int j = 0; j < NB; ++j)
      if (j < nb) bv[j] = B[(size_t)j * ldb + r];
#pragma unroll
    for (int i = 0; i < IG; ++i)
      if (i < ni) av[i] = A[(size_t)(i0 + i) * lda + r];
#pragma unroll
    for (int i = 0; i < IG; ++i)
#pragma unroll
      for (int j = 0; j < NB; ++j)
        if (i < ni && j < nb) {
          Acc pr, pi = 0;
          if constexpr (C) {
            pr = (Acc)av[i].x * (Acc)bv[j].x + (Acc)av[i].y * (Acc)bv[j].y;
            pi = (Acc)av[i].x * (Acc)bv[j].y - (Acc)av[i].y * (Acc)bv[j].x;
          } else {
            pr = (Acc)av[i] * (Acc)bv[j];
          }
          if constexpr (sizeof(T) == 8) {
            sr[i][j] += pr;
            si[i][j] += pi;
          } else {
            const Acc yr = pr - cr[i][j], tr = sr[i][j] + yr;
            cr[i][j] = (tr - sr[i][j]) - yr;
            sr[i][j] = tr;
            const Acc yi = pi - ci[i][j], ti = si[i][j] + yi;
            ci[i][j] = (ti - si[i][j]) - yi;
            si[i][j] = ti;
          }
        }
  }
  __shared__ double red[8][16][2];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int i = 0; i < IG; ++i)
#pragma unroll
    for (int j = 0; j < NB; ++j) {
      double vr = (double)sr[i][j] - (double)cr[i][j], vi = (double)si[i][j] - (double)ci[i][j];
      for (int o = 16; o > 0; o >>= 1) {
        vr += __shfl_xor_sync(0xffffffffu, vr, o);
        if constexpr (C) vi += __shfl_xor_sync(0xffffffffu, vi, o);
      }
      if (lane == 0) { red[warp][i * NB + j][0] = vr; red[warp][i * NB + j][1] = vi; }
    }
  __syncthreads();
  if (threadIdx.x < IG * NB) {
    const int i = threadIdx.x / NB, j = threadIdx.x % NB;
    if (i < ni && j < nb) {
      double vr = 0.0, vi = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { vr += red[w][threadIdx.x][0]; vi += red[w][threadIdx.x][1]; }
      P[((size_t)blockIdx.y * na + i0 + i) * nb + j] = make_double2(vr, C ? vi : 0.0);
    }
  }
}

// Y_j = beta Y_j + alpha sum_i A_i M[i + j*na] for NB (<= 4) columns at once, every basis
// load serving all NB columns.  Arithmetic in the vectors' precision, as in combine1_kernel
// (coefficients alpha*M rounded once), so FP32 vectors stay off the FP64 pipe.
template <typename T, bool C, int NB>
__global__ void __launch_bounds__(256) combinen_kernel(const void* Av, long long lda, int na, const double2* __restrict__ M,
                                                       int nb, void* Yv, long long ldy, long long n, double alpha, double beta) {
  using E = Elem<T, C>;
  using V = typename E::V;
  using A2 = std::conditional_t<sizeof(T) == 8, double2, float2>;
  using R = T;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  A2* Ms = reinterpret_cast<A2*>(smem_raw);
  for (int t = threadIdx.x; t < na * nb; t += blockDim.x) {
    A2 m;
    m.x = (R)(alpha * M[t].x);
    m.y = (R)(alpha * M[t].y);
    Ms[t] = m;
  }
  __syncthreads();
  const V* A = static_cast<const V*>(Av);
  V* Y = static_cast<V*>(Yv);
  const R rbeta = (R)beta;
  for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (long long)gridDim.x * blockDim.x) {
    R yr[NB], yi[NB];
#pragma unroll
    for (int j = 0; j < NB; ++j) { yr[j] = 0; yi[j] = 0; }
    int i = 0;
    for (; i + 4 <= na; i += 4) {
      V av[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) av[k] = A[(size_t)(i + k) * lda + r];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const R xr = E::re(av[k]), xi = E::im(av[k]);
#pragma unroll
        for (int j = 0; j < NB; ++j)
          if (j < nb) {
            const A2 m = Ms[i + k + j * na];
            yr[j] = fma(xr, m.x, yr[j]);
            if constexpr (C) {
              yr[j] = fma(-xi, m.y, yr[j]);
              yi[j] = fma(xr, m.y, yi[j]);
              yi[j] = fma(xi, m.x, yi[j]);
            }
          }
      }
    }
    for (; i < na; ++i) {
      const V a = A[(size_t)i * lda + r];
      const R xr = E::re(a), xi = E::im(a);
#pragma unroll
      for (int j = 0; j < NB; ++j)
        if (j < nb) {
          const A2 m = Ms[i + j * na];
          yr[j] = fma(xr, m.x, yr[j]);
          if constexpr (C) {
            yr[j] = fma(-xi, m.y, yr[j]);
            yi[j] = fma(xr, m.y, yi[j]);
            yi[j] = fma(xi, m.x, yi[j]);
          }
        }
    }
#pragma unroll
    for (int j = 0; j < NB; ++j)
      if (j < nb) {
        V& out = Y[(size_t)j * ldy + r];
        R orr = yr[j], oi = yi[j];
        if (beta != 0.0) {
          orr = fma(rbeta, (R)E::re(out), orr);
          oi = fma(rbeta, (R)E::im(out), oi);
        }
        out = E::make(orr, oi);
      }
  }
}

// Many-output combination of real FP64 vectors (restarts: kk Ritz vectors from m basis
// vectors): nb FMAs per element read would hold it to GB300's FP64 rate, so each element is
// split once into a double-float pair (one FP64 subtraction) and the nb products and sums run in
// double-float arithmetic on the FP32 pipe; each result is rounded back to FP64 (about 48 of its
// 53 bits exact — the next step re-orthogonalises anyway).
template <int NBT>
__global__ void __launch_bounds__(256) combine_split_kernel(const double* __restrict__ A, long long lda, int na,
                                                            const double2* __restrict__ M, int nb, double* __restrict__ Y,
                                                            long long ldy, long long n, double alpha, double beta) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* Ms = reinterpret_cast<float2*>(smem_raw);
  for (int t = threadIdx.x; t < na * nb; t += blockDim.x) Ms[t] = df_from_double(alpha * M[t].x);
  __syncthreads();
  for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (long long)gridDim.x * blockDim.x) {
    float S[NBT], Cc[NBT];
#pragma unroll
    for (int j = 0; j < NBT; ++j) { S[j] = 0.f; Cc[j] = 0.f; }
    for (int i = 0; i < na; ++i) {
      const float2 a = df_from_double(A[(size_t)i * lda + r]);
#pragma unroll
      for (int j = 0; j < NBT; ++j)
        if (j < nb) df_mac(S[j], Cc[j], a, Ms[i + j * na]);
    }
#pragma unroll
    for (int j = 0; j < NBT; ++j)
      if (j < nb) {
        double v = (double)S[j] + (double)Cc[j];
        if (beta != 0.0) v = fma(beta, Y[(size_t)j * ldy + r], v);
        Y[(size_t)j * ldy + r] = v;
      }
  }
}

// Column-wise inner products <A_j, B_j> (j < ncols, columns n apart): CTA (c, j) sums chunk c of
// column j; partials P[c][j] for reduce_dev_kernel (na = ncols, nb = 1).  The Rayleigh quotients
// and residual norms of a set of vectors need only these, not the full Gram matrices.
template <typename T, bool C>
__global__ void __launch_bounds__(256) dots_cols_kernel(const void* Av, const void* Bv, long long n, int ncols,
                                                        int rows_per_cta, double2* __restrict__ P) {
  using E = Elem<T, C>;
  using V = typename E::V;
  const int j = blockIdx.y;
  const V* A = static_cast<const V*>(Av) + (size_t)j * n;
  const V* B = static_cast<const V*>(Bv) + (size_t)j * n;
  const long long r0 = (long long)blockIdx.x * rows_per_cta;
  const long long r1 = min(n, r0 + rows_per_cta);
  double sr = 0.0, si = 0.0;
  for (long long r = r0 + threadIdx.x; r < r1; r += blockDim.x) {
    const double ar = E::re(A[r]), ai = E::im(A[r]), br = E::re(B[r]), bi = E::im(B[r]);
    sr = fma(ar, br, sr);
    if constexpr (C) {
      sr = fma(ai, bi, sr);
      si = fma(ar, bi, si);
      si = fma(-ai, br, si);
    }
  }
  __shared__ double red[2][8];
  for (int o = 16; o > 0; o >>= 1) {
    sr += __shfl_xor_sync(0xffffffffu, sr, o);
    si += __shfl_xor_sync(0xffffffffu, si, o);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) { red[0][warp] = sr; red[1][warp] = si; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { a += red[0][w]; b += red[1][w]; }
    P[(size_t)blockIdx.x * ncols + j] = make_double2(a, b);
  }
}

__global__ void dots_cols_df_kernel(const float2* __restrict__ A, const float2* __restrict__ B, long long n, int ncols,
                                    int rows_per_cta, double2* __restrict__ P) {
  const int j = blockIdx.y;
  A += (size_t)j * n;
  B += (size_t)j * n;
  const long long r0 = (long long)blockIdx.x * rows_per_cta;
  const long long r1 = min(n, r0 + rows_per_cta);
  float S = 0.f, Cc = 0.f;
  for (long long r = r0 + threadIdx.x; r < r1; r += blockDim.x) df_mac(S, Cc, A[r], B[r]);
  double v = (double)S + (double)Cc;
  __shared__ double red[8];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) a += red[w];
    P[(size_t)blockIdx.x * ncols + j] = make_double2(a, 0.0);
  }
}

// ---- double-float Krylov kernels (precision OMEN_F64_DF): real vectors of (hi, lo) pairs,
// products and sums in double-float arithmetic on the FP32 pipe (df.cuh); partial sums and
// coefficients cross to and from FP64 once per thread and row respectively.

// Projections of NB (1, 2 or 4) right-hand columns on IG = 16 / NB basis vectors per CTA;
// partials P[chunk][i][j] as dotsn_kernel writes them.
template <int NB, int IG>
__global__ void __launch_bounds__(256) dots_df_kernel(const float2* __restrict__ A, long long lda, int na,
                                                      const float2* __restrict__ B, long long ldb, int nb, long long n,
                                                      int rows_per_cta, double2* __restrict__ P,
                                                      const int* __restrict__ gate = nullptr) {
  if (gate && !*gate) return;   // a pass the overlap estimates skip
  const int i0 = blockIdx.x * IG;
  const int ni = min(IG, na - i0);
  const long long r0 = (long long)blockIdx.y * rows_per_cta;
  const long long r1 = min(n, r0 + rows_per_cta);
  float S[IG][NB], Cc[IG][NB];
#pragma unroll
  for (int i = 0; i < IG; ++i)
#pragma unroll
    for (int j = 0; j < NB; ++j) { S[i][j] = 0.f; Cc[i][j] = 0.f; }
  for (long long r = r0 + threadIdx.x; r < r1; r += blockDim.x) {
    float2 bv[NB], av[IG];
#pragma unroll
    for (int j = 0; j < NB; ++j) bv[j] = (j < nb) ? B[(size_t)j * ldb + r] : make_float2(0.f, 0.f);
#pragma unroll
    for (int i = 0; i < IG; ++i) av[i] = (i < ni) ? A[(size_t)(i0 + i) * lda + r] : make_float2(0.f, 0.f);
#pragma unroll
    for (int i = 0; i < IG; ++i)
#pragma unroll
      for (int j = 0; j < NB; ++j) df_mac(S[i][j], Cc[i][j], av[i], bv[j]);
  }
  __shared__ double red[8][16];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int i = 0; i < IG; ++i)
#pragma unroll
    for (int j = 0; j < NB; ++j) {
      double v = (double)S[i][j] + (double)Cc[i][j];
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane == 0) red[warp][i * NB + j] = v;
    }
  __syncthreads();
  if (threadIdx.x < IG * NB) {
    const int i = threadIdx.x / NB, j = threadIdx.x % NB;
    if (i < ni && j < nb) {
      double v = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += red[w][threadIdx.x];
      P[((size_t)blockIdx.y * na + i0 + i) * nb + j] = make_double2(v, 0.0);
    }
  }
}

// Y_j = beta Y_j + alpha sum_i A_i M[i + j*na] for NB (1, 2 or 4) columns; coefficients
// alpha*M (FP64) become double-float pairs once per CTA.
template <int NB>
__global__ void __launch_bounds__(256) combine_df_kernel(const float2* __restrict__ A, long long lda, int na,
                                                         const double2* __restrict__ M, int nb, float2* __restrict__ Y,
                                                         long long ldy, long long n, double alpha, double beta,
                                                         const int* __restrict__ gate = nullptr) {
  if (gate && !*gate) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* Ms = reinterpret_cast<float2*>(smem_raw);
  for (int t = threadIdx.x; t < na * nb; t += blockDim.x) Ms[t] = df_from_double(alpha * M[t].x);
  __syncthreads();
  const float2 b2 = df_from_double(beta);
  for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (long long)gridDim.x * blockDim.x) {
    float S[NB], Cc[NB];
#pragma unroll
    for (int j = 0; j < NB; ++j) { S[j] = 0.f; Cc[j] = 0.f; }
    int i = 0;
    for (; i + 4 <= na; i += 4) {
      float2 av[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) av[k] = A[(size_t)(i + k) * lda + r];
#pragma unroll
      for (int k = 0; k < 4; ++k)
#pragma unroll
        for (int j = 0; j < NB; ++j)
          if (j < nb) df_mac(S[j], Cc[j], av[k], Ms[i + k + j * na]);
    }
    for (; i < na; ++i) {
      const float2 a = A[(size_t)i * lda + r];
#pragma unroll
      for (int j = 0; j < NB; ++j)
        if (j < nb) df_mac(S[j], Cc[j], a, Ms[i + j * na]);
    }
#pragma unroll
    for (int j = 0; j < NB; ++j)
      if (j < nb) {
        float2& out = Y[(size_t)j * ldy + r];
        if (beta != 0.0) df_mac(S[j], Cc[j], out, b2);
        out = df_norm(S[j], Cc[j]);
      }
  }
}

// V = W / ||W|| (double-float), ||W||^2 read from the device; the norm goes into T[row, col]
__global__ void normalize_df_kernel(const float2* __restrict__ W, float2* __restrict__ Vo, long long n,
                                    const double2* __restrict__ nrm2, double2* __restrict__ Tm, int ldT, int row, int col,
                                    int* __restrict__ flag) {
  const double b = sqrt(fmax(nrm2->x, 0.0));
  const float2 inv = df_from_double((b > 1e-300) ? 1.0 / b : 0.0);
  for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (long long)gridDim.x * blockDim.x) {
    float S = 0.f, Cc = 0.f;
    df_mac(S, Cc, W[r], inv);
    Vo[r] = df_norm(S, Cc);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    if (Tm) Tm[row + (size_t)col * ldT] = make_double2(b, 0.0);
    if (!(b > 1e-300) || !isfinite(b)) *flag = 1;
  }
}

// Partial reorthogonalisation (Simon, Math. Comp. 42 (1984) 115; the estimate recurrence as in
// Larsen's PROPACK): om holds estimates omega_i[k] of the overlaps v_i . v_k of the two newest
// basis vectors (vector i in row i & 1 of om, ldT entries each; om[2 ldT] a running estimate of
// ||A||).  With A v_k = sum_l T[l, k] v_l for every earlier basis vector (the columns of the
// projected matrix, thick-restart arrowhead included), the new vector
// beta' v_{j+1} = A v_j - alpha_j v_j - beta_j v_{j-1} has
//   beta' omega_{j+1}[k] = sum_l T[l, k] omega_j[l] - alpha_j omega_j[k] - beta_j omega_{j-1}[k]
// plus a rounding term eps1 ||A|| (added with the sign of the estimate).  The overlaps with v_j
// and v_{j-1} are removed exactly by the three-term step.  When the largest estimate exceeds
// delta (the square root of the unit roundoff) the full Gram–Schmidt pass runs for this vector
// and the next one, and the estimates restart at eps1.  gate[0]: this step's pass; gate[1]: the
// pass of the next step is forced.
template <bool C>
__global__ void omega_kernel(const double2* __restrict__ T, int ldT, int j, const double2* __restrict__ nrm2,
                             double* __restrict__ om, int* __restrict__ gate, double eps1, double delta) {
  // estimates are complex for complex vectors: omega_i[k] = v_k^H v_i, and v_k^H A v_j =
  // sum_l conj(T[l, k]) omega_j[l] since A is Hermitian
  constexpr int S = C ? 2 : 1;                          // doubles per estimate
  double* wj = om + (size_t)(j & 1) * S * ldT;          // omega_j
  double* wn = om + (size_t)((j + 1) & 1) * S * ldT;    // omega_{j-1} in, omega_{j+1} out
  const double bn = sqrt(fmax(nrm2->x, 0.0));
  const double aj = T[j + (size_t)j * ldT].x;
  const double bj = j > 0 ? T[j + (size_t)(j - 1) * ldT].x : 0.0;
  __shared__ double red[32];
  __shared__ int run_s;
  const double anorm = fmax(om[2 * S * ldT], fabs(aj) + fabs(bj) + bn);
  const double ib = 1.0 / fmax(bn, 1e-300);
  double mx = 0.0;
  for (int k = threadIdx.x; k < j - 1; k += blockDim.x) {
    double sr = 0.0, si = 0.0;
    for (int l = 0; l <= j; ++l) {
      const double2 t = T[l + (size_t)k * ldT];
      if constexpr (C) {
        const double wr = wj[2 * l], wi = wj[2 * l + 1];
        sr += t.x * wr + t.y * wi;          // conj(t) * w
        si += t.x * wi - t.y * wr;
      } else {
        sr += t.x * wj[l];
      }
    }
    if constexpr (C) {
      double vr = sr - aj * wj[2 * k] - bj * wn[2 * k];
      double vi = si - aj * wj[2 * k + 1] - bj * wn[2 * k + 1];
      const double a = hypot(vr, vi);
      const double g = a > 0.0 ? (a + eps1 * anorm) / a : 0.0;
      vr = a > 0.0 ? vr * g : eps1 * anorm;
      vi = a > 0.0 ? vi * g : 0.0;
      wn[2 * k] = vr * ib;
      wn[2 * k + 1] = vi * ib;
      mx = fmax(mx, hypot(vr, vi) * ib);
    } else {
      double v = sr - aj * wj[k] - bj * wn[k];
      v = (v + copysign(eps1 * anorm, v)) * ib;
      wn[k] = v;
      mx = fmax(mx, fabs(v));
    }
  }
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    double m = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = fmax(m, red[w]);
    const int forced = gate[1];
    const int run = (m > delta || !(m == m) || forced) ? 1 : 0;
    gate[0] = run;
    gate[1] = (run && !forced) ? 1 : 0;
    run_s = run;
    om[2 * S * ldT] = anorm;
  }
  __syncthreads();
  for (int k = threadIdx.x; k <= j; k += blockDim.x)
    if (run_s || k >= j - 1) {
      wn[S * k] = eps1;
      if (C) wn[S * k + 1] = 0.0;
    }
  if (threadIdx.x == 0) {
    wn[S * (j + 1)] = 1.0;
    if (C) wn[S * (j + 1) + 1] = 0.0;
  }
}

// After full passes: vectors i1 - 1 and i1 orthogonal to all earlier ones (estimates eps1), and
// the next step's pass forced (a restart's kept vectors are only semi-orthogonal among themselves).
template <bool C>
__global__ void omega_reset_kernel(double* __restrict__ om, int ldT, int i1, double eps1, int* __restrict__ gate) {
  constexpr int S = C ? 2 : 1;
  double* a = om + (size_t)(i1 & 1) * S * ldT;
  double* b = om + (size_t)((i1 - 1) & 1) * S * ldT;
  for (int k = threadIdx.x; k < ldT; k += blockDim.x) {
    a[S * k] = (k == i1) ? 1.0 : eps1;
    if (C) a[S * k + 1] = 0.0;
    if (i1 >= 1) {
      b[S * k] = (k == i1 - 1) ? 1.0 : eps1;
      if (C) b[S * k + 1] = 0.0;
    }
  }
  if (threadIdx.x == 0) {
    gate[0] = 1;
    gate[1] = 1;
  }
}

// Device-side reduction of the partials into out (na x nb, column-major) and, optionally,
// into columns col0.. of the projected matrix T (ldT x ldT, column-major).
__global__ void reduce_dev_kernel(const double2* __restrict__ P, int nchunks, int na, int nb, double2* __restrict__ out,
                                  double2* __restrict__ accT, int ldT, int col0, long long p_ps = 0,
                                  long long out_ps = 0, long long t_ps = 0, const int* __restrict__ act = nullptr) {
  if (act && !act[blockIdx.y]) return;
  const int e = blockIdx.x;
  P += blockIdx.y * p_ps;
  out += blockIdx.y * out_ps;
  if (accT) accT += blockIdx.y * t_ps;
  const int count = na * nb;
  double sr = 0.0, si = 0.0;
  for (int c = threadIdx.x; c < nchunks; c += blockDim.x) {
    const double2 v = P[(size_t)c * count + e];
    sr += v.x;
    si += v.y;
  }
  __shared__ double red[2][32];
  for (int o = 16; o > 0; o >>= 1) {
    sr += __shfl_xor_sync(0xffffffffu, sr, o);
    si += __shfl_xor_sync(0xffffffffu, si, o);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) { red[0][warp] = sr; red[1][warp] = si; }
  __syncthreads();
  if (threadIdx.x == 0) {
    sr = 0.0;
    si = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { sr += red[0][w]; si += red[1][w]; }
    const int i = e / nb, j = e % nb;
    out[i + (size_t)j * na] = make_double2(sr, si);
    if (accT) {
      double2* t = accT + i + (size_t)(col0 + j) * ldT;
      t->x += sr;
      t->y += si;
    }
  }
}

// V = W / ||W|| with ||W||^2 read from the device; the norm goes into T[row, col].
template <typename T, bool C>
__global__ void normalize_kernel(const void* Wv, void* Vv, long long n, const double2* __restrict__ nrm2,
                                 double2* __restrict__ Tm, int ldT, int row, int col, int* __restrict__ flag,
                                 long long w_ps = 0, long long v_ps = 0, long long n_ps = 0, long long t_ps = 0,
                                 const long long* __restrict__ poff = nullptr,
                                 const long long* __restrict__ plen = nullptr,
                                 const int* __restrict__ act = nullptr) {
  using E = Elem<T, C>;
  using V = typename E::V;
  nrm2 += blockIdx.y * n_ps;
  if (Tm) Tm += blockIdx.y * t_ps;
  const double b = sqrt(fmax(nrm2->x, 0.0));
  const double inv = (b > 1e-300) ? 1.0 / b : 0.0;
  if (act && !act[blockIdx.y]) return;
  const long long off = poff ? poff[blockIdx.y] : 0;
  if (plen) n = plen[blockIdx.y];
  const V* W = static_cast<const V*>(Wv) + blockIdx.y * w_ps + off;
  V* Vo = static_cast<V*>(Vv) + blockIdx.y * v_ps + off;
  for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (long long)gridDim.x * blockDim.x)
    Vo[r] = E::make(E::re(W[r]) * inv, E::im(W[r]) * inv);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    if (Tm) Tm[row + (size_t)col * ldT] = make_double2(b, 0.0);
    if (!(b > 1e-300) || !isfinite(b)) *flag = 1;
  }
}

// Y_j[r] = beta * Y_j[r] + alpha * sum_i A_i[r] M[i + j*na]   (M complex FP64, column-major)
template <typename T, bool C>
__global__ void combine_kernel(const void* Av, long long lda, int na, const double2* __restrict__ M, int nb,
                               void* Yv, long long ldy, long long n, double alpha, double beta) {
  // arithmetic in the vectors' precision (coefficients alpha*M rounded once): FP32 vectors keep
  // their nb products per element off GB300's FP64 pipe
  using E = Elem<T, C>;
  using V = typename E::V;
  using A2 = std::conditional_t<sizeof(T) == 8, double2, float2>;
  using R = T;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  A2* Ms = reinterpret_cast<A2*>(smem_raw);
  for (int t = threadIdx.x; t < na * nb; t += blockDim.x) {
    A2 m;
    m.x = (R)(alpha * M[t].x);
    m.y = (R)(alpha * M[t].y);
    Ms[t] = m;
  }
  __syncthreads();
  const V* A = static_cast<const V*>(Av);
  V* Y = static_cast<V*>(Yv);
  const R rbeta = (R)beta;
  for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (long long)gridDim.x * blockDim.x) {
    R yr[kMaxBlockCols], yi[kMaxBlockCols];
#pragma unroll
    for (int j = 0; j < kMaxBlockCols; ++j) { yr[j] = 0; yi[j] = 0; }
    for (int i0 = 0; i0 < na; i0 += 4) {
      V av[4];
#pragma unroll
      for (int k = 0; k < 4; ++k)
        if (i0 + k < na) av[k] = A[(size_t)(i0 + k) * lda + r];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        if (i0 + k >= na) break;
        const int i = i0 + k;
        const R xr = (R)E::re(av[k]), xi = (R)E::im(av[k]);
#pragma unroll
        for (int j = 0; j < kMaxBlockCols; ++j) {
          if (j < nb) {
            const A2 m = Ms[i + j * na];
            yr[j] = fma(xr, m.x, yr[j]);
            if constexpr (C) {
              yr[j] = fma(-xi, m.y, yr[j]);
              yi[j] = fma(xr, m.y, yi[j]);
              yi[j] = fma(xi, m.x, yi[j]);
            }
          }
        }
      }
    }
#pragma unroll
    for (int j = 0; j < kMaxBlockCols; ++j) {
      if (j < nb) {
        V& out = Y[j * ldy + r];
        R orr = yr[j], oi = yi[j];
        if (beta != 0.0) {
          orr = fma(rbeta, (R)E::re(out), orr);
          oi = fma(rbeta, (R)E::im(out), oi);
        }
        out = E::make(orr, oi);
      }
    }
  }
}

// SplitMix64 (Steele, Lea & Flood, OOPSLA 2014) keyed by (seed, index): uniform [-1, 1).
__device__ __forceinline__ unsigned long long splitmix64(unsigned long long z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
template <typename T, bool C>
__global__ void random_fill_kernel(void* Xv, long long n, unsigned long long seed) {
  using E = Elem<T, C>;
  using V = typename E::V;
  V* X = static_cast<V*>(Xv);
  for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (long long)gridDim.x * blockDim.x) {
    const unsigned long long h1 = splitmix64(seed * 0x100000001B3ull + 2 * (unsigned long long)r);
    const unsigned long long h2 = splitmix64(seed * 0x100000001B3ull + 2 * (unsigned long long)r + 1);
    const double u1 = (double)(h1 >> 11) * (1.0 / 9007199254740992.0) * 2.0 - 1.0;
    const double u2 = (double)(h2 >> 11) * (1.0 / 9007199254740992.0) * 2.0 - 1.0;
    X[r] = E::make(u1, u2);
  }
}

__global__ void random_fill_df_kernel(float2* __restrict__ X, long long n, unsigned long long seed) {
  for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (long long)gridDim.x * blockDim.x) {
    const unsigned long long h = splitmix64(seed * 0x100000001B3ull + 2 * (unsigned long long)r);
    X[r] = df_from_double((double)(h >> 11) * (1.0 / 9007199254740992.0) * 2.0 - 1.0);
  }
}

template <typename Tin, typename Tout, bool C>
__global__ void convert_kernel(const void* Xv, void* Yv, long long n) {
  using Ei = Elem<Tin, C>;
  using Eo = Elem<Tout, C>;
  const typename Ei::V* X = static_cast<const typename Ei::V*>(Xv);
  typename Eo::V* Y = static_cast<typename Eo::V*>(Yv);
  for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (long long)gridDim.x * blockDim.x)
    Y[r] = Eo::make(Ei::re(X[r]), Ei::im(X[r]));
}

// cudaFuncSetAttribute costs a driver call: raise a kernel's dynamic shared-memory limit only
// when a launch needs more than the largest value already set for it.
template <typename K>
static void smem_limit(K kernel, size_t bytes) {
  static std::mutex mu;
  static std::map<std::pair<int, const void*>, size_t> current;   // per (device, kernel)
  if (bytes <= 48 * 1024) return;
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lock(mu);
  size_t& cur = current[{dev, reinterpret_cast<const void*>(kernel)}];
  if (bytes > cur) {
    cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    cur = bytes;
  }
}

// ---------------------------------------------------------------------------------------
// Host-side helpers bound to one vector type.
// basis vectors per CTA for a projection on na of them: the smallest power of two >= na,
// capped at `cap`
static int dots_ig_for(int na, int cap) {
  int ig = 1;
  while (ig < na && ig < cap) ig *= 2;
  return ig;
}

template <typename T, bool C>
static void launch_dots1(int ig, dim3 grid, cudaStream_t st, const void* A, long long lda, int na, const void* B,
                         long long n, int rows, double2* P, long long a_ps = 0, long long b_ps = 0, long long p_ps = 0,
                         const long long* poff = nullptr, const long long* plen = nullptr, const int* act = nullptr) {
  switch (ig) {
    case 1: dots1_kernel<T, C, 1><<<grid, 256, 0, st>>>(A, lda, na, B, n, rows, P, a_ps, b_ps, p_ps, poff, plen, act); break;
    case 2: dots1_kernel<T, C, 2><<<grid, 256, 0, st>>>(A, lda, na, B, n, rows, P, a_ps, b_ps, p_ps, poff, plen, act); break;
    case 4: dots1_kernel<T, C, 4><<<grid, 256, 0, st>>>(A, lda, na, B, n, rows, P, a_ps, b_ps, p_ps, poff, plen, act); break;
    case 8: dots1_kernel<T, C, 8><<<grid, 256, 0, st>>>(A, lda, na, B, n, rows, P, a_ps, b_ps, p_ps, poff, plen, act); break;
    default:
      if constexpr (!C) dots1_kernel<T, C, 16><<<grid, 256, 0, st>>>(A, lda, na, B, n, rows, P, a_ps, b_ps, p_ps, poff, plen, act);
      else dots1_kernel<T, C, 8><<<grid, 256, 0, st>>>(A, lda, na, B, n, rows, P, a_ps, b_ps, p_ps, poff, plen, act);
  }
}

struct KrylovOps {
  omen_ctx* ctx;
  const omen_ham* ham;
  int prec;            // OMEN_F64 or OMEN_F32 (element precision of these vectors)
  bool cplx;
  long long n;         // rows
  size_t el;           // bytes per element
  double2* d_partial = nullptr;
  size_t partial_cap = 0;  // in double2
  double2* d_small = nullptr;  // reduced results / small matrices
  size_t small_cap = 0;
  void* qr_tmp = nullptr;      // copy of a block during Cholesky QR
  size_t qr_cap = 0;
  double2* d_hs = nullptr;     // projection sums of the block path
  size_t hs_cap = 0;
  int sm_count = 148;

  omen_status init() {
    el = vec_elem_bytes(ham, prec);
    cudaDeviceGetAttribute(&sm_count, cudaDevAttrMultiProcessorCount, ctx->device);
    small_cap = 1 << 18;
    if (cudaMalloc(&d_small, small_cap * sizeof(double2)) != cudaSuccess) {
      cudaGetLastError();
      return set_err(ctx, OMEN_ENOMEM, "small work buffer");
    }
    return OMEN_OK;
  }
  void release() {
    cudaFree(d_partial);
    cudaFree(d_small);
    cudaFree(qr_tmp);
    cudaFree(d_hs);
  }
  char* col(void* base, long long j) const { return static_cast<char*>(base) + (size_t)j * n * el; }

  int chunk_rows(int nb) const {
    // rows per CTA so that nb columns of B fit in ~96 KB of shared memory
    long long ch = (96 * 1024) / ((long long)nb * el);
    ch = std::min<long long>(ch, 8192);
    ch = std::max<long long>(ch, 64);
    return (int)(ch / 32 * 32);
  }

  // out (host, na x nb column-major complex) = A^H B   (A: na columns, B: nb columns)
  omen_status dots(const void* A, int na, const void* B, int nb, std::vector<cd>& out) {
    out.assign((size_t)na * nb, cd(0));
    if ((nb <= 4 || prec == OMEN_F64_DF) && (size_t)na * nb <= small_cap) {
      omen_status s1 = dots_dev(A, na, B, nb, d_small, nullptr, 0, 0);
      if (s1 != OMEN_OK) return s1;
      OMEN_CUDA(ctx, cudaMemcpyAsync(out.data(), d_small, (size_t)na * nb * sizeof(double2), cudaMemcpyDeviceToHost, ctx->stream));
      OMEN_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
      for (const cd& v : out)
        if (!std::isfinite(v.real()) || !std::isfinite(v.imag()))
          return set_err(ctx, OMEN_ENUMERIC, "non-finite value in a Krylov inner product");
      return OMEN_OK;
    }
    for (int j0 = 0; j0 < nb; j0 += kMaxBlockCols) {
      const int nbj = std::min(kMaxBlockCols, nb - j0);
      const int CH = chunk_rows(nbj);
      const long long nchunks = (n + CH - 1) / CH;
      const size_t need = (size_t)nchunks * na * nbj;
      omen_status se = ensure_partial(need);
      if (se != OMEN_OK) return se;
      if ((size_t)na * nbj > small_cap) return set_err(ctx, OMEN_EINVAL, "projection too large");
      const size_t shm = (size_t)nbj * CH * el;
      const void* Bj = col(const_cast<void*>(B), j0);
#define DOTS_LAUNCH(T, Cc)                                                                          \
  do {                                                                                              \
    smem_limit(dots_partial_kernel<T, Cc>, shm); \
    dots_partial_kernel<T, Cc><<<(unsigned)nchunks, kDotThreads, shm, ctx->stream>>>(A, n, na, Bj, n, nbj, n, CH, d_partial); \
  } while (0)
      if (prec == OMEN_F64) { if (cplx) DOTS_LAUNCH(double, true); else DOTS_LAUNCH(double, false); }
      else { if (cplx) DOTS_LAUNCH(float, true); else DOTS_LAUNCH(float, false); }
#undef DOTS_LAUNCH
      OMEN_CHECK_LAUNCH(ctx);
      const int count = na * nbj;
      reduce_partial_kernel<<<count, 256, 0, ctx->stream>>>(d_partial, (int)nchunks, count, d_small);
      OMEN_CHECK_LAUNCH(ctx);
      std::vector<cd> tmp(count);
      OMEN_CUDA(ctx, cudaMemcpyAsync(tmp.data(), d_small, count * sizeof(double2), cudaMemcpyDeviceToHost, ctx->stream));
      OMEN_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
      // partial layout [i][j]
      for (int i = 0; i < na; ++i)
        for (int j = 0; j < nbj; ++j) out[i + (size_t)(j0 + j) * na] = tmp[(size_t)i * nbj + j];
    }
    for (const cd& v : out)
      if (!std::isfinite(v.real()) || !std::isfinite(v.imag()))
        return set_err(ctx, OMEN_ENUMERIC, "non-finite value in a Krylov inner product");
    return OMEN_OK;
  }

  // Y = beta*Y + alpha * A M   (M host na x nb column-major)
  omen_status combine(const void* A, int na, const std::vector<cd>& M, int nb, void* Y, double alpha, double beta) {
    if ((nb <= 4 || prec == OMEN_F64_DF) && (size_t)na * nb <= small_cap) {
      // pageable source: the copy has consumed M when the call returns; stream order protects d_small
      OMEN_CUDA(ctx, cudaMemcpyAsync(d_small, M.data(), (size_t)na * nb * sizeof(double2), cudaMemcpyHostToDevice, ctx->stream));
      return combine_dev(A, na, d_small, nb, Y, alpha, beta);
    }
    if ((size_t)na * kMaxBlockCols > small_cap) return set_err(ctx, OMEN_EINVAL, "combination too large");
    for (int j0 = 0; j0 < nb; j0 += kMaxBlockCols) {
      const int nbj = std::min(kMaxBlockCols, nb - j0);
      std::vector<cd> Mj((size_t)na * nbj);
      for (int j = 0; j < nbj; ++j)
        for (int i = 0; i < na; ++i) Mj[i + (size_t)j * na] = M[i + (size_t)(j0 + j) * na];
      OMEN_CUDA(ctx, cudaMemcpyAsync(d_small, Mj.data(), Mj.size() * sizeof(double2), cudaMemcpyHostToDevice, ctx->stream));
      const size_t shm = Mj.size() * sizeof(double2);
      const unsigned grid = (unsigned)std::min<long long>((n + 255) / 256, (long long)sm_count * 8);
      void* Yj = col(Y, j0);
#define COMB_LAUNCH(T, Cc)                                                                           \
  do {                                                                                               \
    smem_limit(combine_kernel<T, Cc>, shm); \
    combine_kernel<T, Cc><<<grid, 256, shm, ctx->stream>>>(A, n, na, d_small, nbj, Yj, n, n, alpha, beta); \
  } while (0)
      if (prec == OMEN_F64 && !cplx) {
        const size_t shs = (size_t)na * nbj * sizeof(float2);
        const double* Ad = static_cast<const double*>(A);
        double* Yd = static_cast<double*>(Yj);
        if (nbj <= 8) {
          smem_limit(combine_split_kernel<8>, shs);
          combine_split_kernel<8><<<grid, 256, shs, ctx->stream>>>(Ad, n, na, d_small, nbj, Yd, n, n, alpha, beta);
        } else {
          smem_limit(combine_split_kernel<16>, shs);
          combine_split_kernel<16><<<grid, 256, shs, ctx->stream>>>(Ad, n, na, d_small, nbj, Yd, n, n, alpha, beta);
        }
      } else if (prec == OMEN_F64) COMB_LAUNCH(double, true);
      else { if (cplx) COMB_LAUNCH(float, true); else COMB_LAUNCH(float, false); }
#undef COMB_LAUNCH
      OMEN_CHECK_LAUNCH(ctx);
      // the small buffer is reused by the next chunk: wait for this kernel to read it
      OMEN_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    }
    return OMEN_OK;
  }

  // Rows per CTA of the projection kernels (na basis vectors, ig of them per CTA): enough row
  // chunks that the grid covers every SM about twice (small problems would otherwise run on a
  // handful of CTAs), at most 8192 rows per chunk, at most 65535 chunks.
  long long dot_rows(int na, int ig) const {
    const long long groups = std::max(1, (na + ig - 1) / ig);
    const long long want = std::max<long long>(1, (2LL * sm_count + groups - 1) / groups);
    long long rows = (n + want - 1) / want;
    rows = std::min<long long>(8192, std::max<long long>(256, (rows + 255) / 256 * 256));
    while ((n + rows - 1) / rows > 65535) rows *= 2;
    return rows;
  }
  // the largest partial-sum count a projection of up to na_max basis vectors asks for
  size_t max_partials(int na_max) const {
    size_t need = 0;
    for (int na = 1; na <= na_max; ++na)
      for (int ig : {kIG, 8, 4, 2}) {
        const long long rows = dot_rows(na, ig);
        need = std::max(need, (size_t)((n + rows - 1) / rows) * na * 4);
      }
    return need;
  }

  // out (host, ncols) = <A_j, B_j> for each column j
  omen_status dots_cols(const void* A, const void* B, int ncols, std::vector<cd>& out) {
    out.assign(ncols, cd(0));
    if ((size_t)ncols > small_cap) return set_err(ctx, OMEN_EINVAL, "too many columns");
    const long long rows = dot_rows(ncols, 1);
    const long long nchunks = (n + rows - 1) / rows;
    omen_status s1 = ensure_partial((size_t)nchunks * ncols);
    if (s1 != OMEN_OK) return s1;
    dim3 grid((unsigned)nchunks, ncols);
    if (prec == OMEN_F64_DF)
      dots_cols_df_kernel<<<grid, 256, 0, ctx->stream>>>(static_cast<const float2*>(A), static_cast<const float2*>(B), n, ncols,
                                                          (int)rows, d_partial);
    else if (prec == OMEN_F64) {
      if (cplx) dots_cols_kernel<double, true><<<grid, 256, 0, ctx->stream>>>(A, B, n, ncols, (int)rows, d_partial);
      else dots_cols_kernel<double, false><<<grid, 256, 0, ctx->stream>>>(A, B, n, ncols, (int)rows, d_partial);
    } else {
      if (cplx) dots_cols_kernel<float, true><<<grid, 256, 0, ctx->stream>>>(A, B, n, ncols, (int)rows, d_partial);
      else dots_cols_kernel<float, false><<<grid, 256, 0, ctx->stream>>>(A, B, n, ncols, (int)rows, d_partial);
    }
    reduce_dev_kernel<<<ncols, 256, 0, ctx->stream>>>(d_partial, (int)nchunks, ncols, 1, d_small, nullptr, 0, 0);
    OMEN_CHECK_LAUNCH(ctx);
    OMEN_CUDA(ctx, cudaMemcpyAsync(out.data(), d_small, sizeof(double2) * ncols, cudaMemcpyDeviceToHost, ctx->stream));
    OMEN_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    for (const cd& v : out)
      if (!std::isfinite(v.real()) || !std::isfinite(v.imag()))
        return set_err(ctx, OMEN_ENUMERIC, "non-finite value in a Krylov inner product");
    return OMEN_OK;
  }

  // grows geometrically (cudaFree synchronises the device, so it must not happen per step)
  omen_status ensure_partial(size_t need) {
    if (need <= partial_cap) return OMEN_OK;
    const size_t cap = std::max<size_t>({need, 2 * partial_cap, (size_t)1 << 18});
    cudaFree(d_partial);
    d_partial = nullptr;
    partial_cap = 0;
    if (cudaMalloc(&d_partial, cap * sizeof(double2)) != cudaSuccess) {
      cudaGetLastError();
      return set_err(ctx, OMEN_ENOMEM, "partial-sum buffer");
    }
    partial_cap = cap;
    return OMEN_OK;
  }

  // out_dev (na x nb, column-major) = A^H B on the device, optionally added into T columns;
  // nothing is copied to the host and the stream is not synchronised.
  omen_status dots_dev(const void* A, int na, const void* B, int nb, double2* out_dev, double2* accT, int ldT, int col0) {
    if (nb > kMaxBlockCols) return set_err(ctx, OMEN_EINVAL, "dots_dev: too many columns");
    if (prec == OMEN_F64_DF) {
      // double-float vectors: up to 4 right-hand columns per launch
      for (int j0 = 0; j0 < nb; j0 += 4) {
        const int nbj = std::min(4, nb - j0);
        const int NBk = nbj == 1 ? 1 : (nbj == 2 ? 2 : 4);
        const int ig = dots_ig_for(na, 16 / NBk);
        const int rows = (int)dot_rows(na, ig);
        const long long nchunks = (n + rows - 1) / rows;
        omen_status s1 = ensure_partial((size_t)nchunks * na * nbj);
        if (s1 != OMEN_OK) return s1;
        dim3 grid((na + ig - 1) / ig, (unsigned)nchunks);
        const float2* Af = static_cast<const float2*>(A);
        const float2* Bf = static_cast<const float2*>(B) + (size_t)j0 * n;
#define DDF(NBc, IGc) dots_df_kernel<NBc, IGc><<<grid, 256, 0, ctx->stream>>>(Af, n, na, Bf, n, nbj, n, rows, d_partial)
        if (NBk == 1) {
          if (ig == 1) DDF(1, 1); else if (ig == 2) DDF(1, 2); else if (ig == 4) DDF(1, 4); else if (ig == 8) DDF(1, 8); else DDF(1, 16);
        } else if (NBk == 2) {
          if (ig == 1) DDF(2, 1); else if (ig == 2) DDF(2, 2); else if (ig == 4) DDF(2, 4); else DDF(2, 8);
        } else {
          if (ig == 1) DDF(4, 1); else if (ig == 2) DDF(4, 2); else DDF(4, 4);
        }
#undef DDF
        reduce_dev_kernel<<<na * nbj, 256, 0, ctx->stream>>>(d_partial, (int)nchunks, na, nbj, out_dev + (size_t)j0 * na, accT,
                                                           ldT, col0 + j0);
        OMEN_CHECK_LAUNCH(ctx);
      }
      return OMEN_OK;
    }
    if (nb > 1 && nb <= 4) {
      // a few right-hand columns: one launch, each basis load serving every column
      const int ig = dots1_ig(cplx) / ((nb <= 2) ? 2 : 4);
      const int rows = (int)dot_rows(na, ig);
      const long long nchunks = (n + rows - 1) / rows;
      omen_status s1 = ensure_partial((size_t)nchunks * na * nb);
      if (s1 != OMEN_OK) return s1;
      dim3 grid((na + ig - 1) / ig, (unsigned)nchunks);
#define DOTSN(T, Cc)                                                                                     \
  do {                                                                                                   \
    if (nb <= 2) dotsn_kernel<T, Cc, 2><<<grid, 256, 0, ctx->stream>>>(A, n, na, B, n, nb, n, rows, d_partial); \
    else dotsn_kernel<T, Cc, 4><<<grid, 256, 0, ctx->stream>>>(A, n, na, B, n, nb, n, rows, d_partial);        \
  } while (0)
      if (prec == OMEN_F64) { if (cplx) DOTSN(double, true); else DOTSN(double, false); }
      else { if (cplx) DOTSN(float, true); else DOTSN(float, false); }
#undef DOTSN
      reduce_dev_kernel<<<na * nb, 256, 0, ctx->stream>>>(d_partial, (int)nchunks, na, nb, out_dev, accT, ldT, col0);
      OMEN_CHECK_LAUNCH(ctx);
      return OMEN_OK;
    }
    if (nb == 1) {
      const int ig1 = dots_ig_for(na, dots1_ig(cplx));
      const int rows = (int)dot_rows(na, ig1);
      const long long nchunks = (n + rows - 1) / rows;
      omen_status s1 = ensure_partial((size_t)nchunks * na);
      if (s1 != OMEN_OK) return s1;
      dim3 grid((na + ig1 - 1) / ig1, (unsigned)nchunks);
      if (prec == OMEN_F64) {
        if (cplx) launch_dots1<double, true>(ig1, grid, ctx->stream, A, n, na, B, n, rows, d_partial);
        else launch_dots1<double, false>(ig1, grid, ctx->stream, A, n, na, B, n, rows, d_partial);
      } else {
        if (cplx) launch_dots1<float, true>(ig1, grid, ctx->stream, A, n, na, B, n, rows, d_partial);
        else launch_dots1<float, false>(ig1, grid, ctx->stream, A, n, na, B, n, rows, d_partial);
      }
      reduce_dev_kernel<<<na, 256, 0, ctx->stream>>>(d_partial, (int)nchunks, na, 1, out_dev, accT, ldT, col0);
      OMEN_CHECK_LAUNCH(ctx);
      return OMEN_OK;
    }
    const int CH = chunk_rows(nb);
    const long long nchunks = (n + CH - 1) / CH;
    omen_status s = ensure_partial((size_t)nchunks * na * nb);
    if (s != OMEN_OK) return s;
    const size_t shm = (size_t)nb * CH * el;
#define DOTS_LAUNCH2(T, Cc)                                                                         \
  do {                                                                                              \
    smem_limit(dots_partial_kernel<T, Cc>, shm); \
    dots_partial_kernel<T, Cc><<<(unsigned)nchunks, kDotThreads, shm, ctx->stream>>>(A, n, na, B, n, nb, n, CH, d_partial); \
  } while (0)
    if (prec == OMEN_F64) { if (cplx) DOTS_LAUNCH2(double, true); else DOTS_LAUNCH2(double, false); }
    else { if (cplx) DOTS_LAUNCH2(float, true); else DOTS_LAUNCH2(float, false); }
#undef DOTS_LAUNCH2
    reduce_dev_kernel<<<na * nb, 256, 0, ctx->stream>>>(d_partial, (int)nchunks, na, nb, out_dev, accT, ldT, col0);
    OMEN_CHECK_LAUNCH(ctx);
    return OMEN_OK;
  }

  // Y = beta*Y + alpha * A M with M (na x nb, column-major) already on the device
  omen_status combine_dev(const void* A, int na, const double2* M_dev, int nb, void* Y, double alpha, double beta) {
    if (prec == OMEN_F64_DF) {
      const unsigned grid = (unsigned)std::min<long long>((n + 255) / 256, (long long)sm_count * 8);
      for (int j0 = 0; j0 < nb; j0 += 4) {
        const int nbj = std::min(4, nb - j0);
        const size_t shm = (size_t)na * nbj * sizeof(float2);
        const float2* Af = static_cast<const float2*>(A);
        float2* Yf = static_cast<float2*>(Y) + (size_t)j0 * n;
        const double2* Mj = M_dev + (size_t)j0 * na;
#define COMBDF(NBk)                                                                                     \
  do {                                                                                                  \
    smem_limit(combine_df_kernel<NBk>, shm);                                                            \
    combine_df_kernel<NBk><<<grid, 256, shm, ctx->stream>>>(Af, n, na, Mj, nbj, Yf, n, n, alpha, beta); \
  } while (0)
        if (nbj == 1) COMBDF(1);
        else if (nbj == 2) COMBDF(2);
        else COMBDF(4);
#undef COMBDF
        OMEN_CHECK_LAUNCH(ctx);
      }
      return OMEN_OK;
    }
    if (nb > kMaxBlockCols) return set_err(ctx, OMEN_EINVAL, "combine_dev: too many columns");
    if (nb > 1 && nb <= 4) {
      const size_t shmn = (size_t)na * nb * sizeof(double2);
      const unsigned gridn = (unsigned)std::min<long long>((n + 255) / 256, (long long)sm_count * 8);
#define COMBN(T, Cc)                                                                                        \
  do {                                                                                                      \
    if (nb <= 2) {                                                                                          \
      smem_limit(combinen_kernel<T, Cc, 2>, shmn);                                                          \
      combinen_kernel<T, Cc, 2><<<gridn, 256, shmn, ctx->stream>>>(A, n, na, M_dev, nb, Y, n, n, alpha, beta); \
    } else {                                                                                                \
      smem_limit(combinen_kernel<T, Cc, 4>, shmn);                                                          \
      combinen_kernel<T, Cc, 4><<<gridn, 256, shmn, ctx->stream>>>(A, n, na, M_dev, nb, Y, n, n, alpha, beta); \
    }                                                                                                       \
  } while (0)
      if (prec == OMEN_F64) { if (cplx) COMBN(double, true); else COMBN(double, false); }
      else { if (cplx) COMBN(float, true); else COMBN(float, false); }
#undef COMBN
      OMEN_CHECK_LAUNCH(ctx);
      return OMEN_OK;
    }
    if (nb == 1) {
      const size_t shm1 = (size_t)na * sizeof(double2);
      const unsigned grid1 = (unsigned)std::min<long long>((n + 255) / 256, (long long)sm_count * 8);
#define COMB1(T, Cc)                                                                                  \
  do {                                                                                                \
    smem_limit(combine1_kernel<T, Cc>, shm1);                                                         \
    combine1_kernel<T, Cc><<<grid1, 256, shm1, ctx->stream>>>(A, n, na, M_dev, Y, n, alpha, beta);       \
  } while (0)
      if (prec == OMEN_F64) { if (cplx) COMB1(double, true); else COMB1(double, false); }
      else { if (cplx) COMB1(float, true); else COMB1(float, false); }
#undef COMB1
      OMEN_CHECK_LAUNCH(ctx);
      return OMEN_OK;
    }
    const size_t shm = (size_t)na * nb * sizeof(double2);
    const unsigned grid = (unsigned)std::min<long long>((n + 255) / 256, (long long)sm_count * 8);
#define COMB_LAUNCH2(T, Cc)                                                                          \
  do {                                                                                               \
    smem_limit(combine_kernel<T, Cc>, shm); \
    combine_kernel<T, Cc><<<grid, 256, shm, ctx->stream>>>(A, n, na, M_dev, nb, Y, n, n, alpha, beta); \
  } while (0)
    if (prec == OMEN_F64) { if (cplx) COMB_LAUNCH2(double, true); else COMB_LAUNCH2(double, false); }
    else { if (cplx) COMB_LAUNCH2(float, true); else COMB_LAUNCH2(float, false); }
#undef COMB_LAUNCH2
    OMEN_CHECK_LAUNCH(ctx);
    return OMEN_OK;
  }

  // w -= V h only where semi-orthogonality needs it (combine1_gated_kernel); h added into Tcol then
  omen_status combine_gated(const void* A, int na, const double2* h_dev, void* W, const double2* nrm2, int parity,
                            double2* Tcol) {
    const double eta = prec == OMEN_F64 ? 1.0536712127723509e-08 : 2.44140625e-04;  // sqrt(2^-53), sqrt(2^-24)
    const size_t shm = (size_t)na * sizeof(double2);
    const unsigned grid = (unsigned)std::min<long long>((n + 255) / 256, (long long)sm_count * 8);
    int* gate = ctx->d_status + 2;
#define GATED(T, Cc)                                                                                  \
  do {                                                                                                \
    smem_limit(combine1_gated_kernel<T, Cc>, shm);                                                    \
    combine1_gated_kernel<T, Cc><<<grid, 256, shm, ctx->stream>>>(A, na, h_dev, W, n, nrm2, eta, gate, parity, Tcol); \
  } while (0)
    if (prec == OMEN_F64) { if (cplx) GATED(double, true); else GATED(double, false); }
    else { if (cplx) GATED(float, true); else GATED(float, false); }
#undef GATED
    OMEN_CHECK_LAUNCH(ctx);
    return OMEN_OK;
  }
  // Partial reorthogonalisation: the full pass h = V^H w (added into T column js), w -= V h for
  // one real vector, every kernel skipped unless gate[0] (set by omega_kernel) is nonzero.
  omen_status pass_gated(const void* Vb, int na, void* W, double2* h_dev, double2* Tm, int ldT, int js, const int* gate) {
    if (prec == OMEN_F64_DF) {
      const int ig = dots_ig_for(na, 16);
      const int rows = (int)dot_rows(na, ig);
      const long long nchunks = (n + rows - 1) / rows;
      omen_status s1 = ensure_partial((size_t)nchunks * na);
      if (s1 != OMEN_OK) return s1;
      dim3 grid((na + ig - 1) / ig, (unsigned)nchunks);
      const float2* Af = static_cast<const float2*>(Vb);
      const float2* Bf = static_cast<const float2*>(W);
#define DDFG(IGc) dots_df_kernel<1, IGc><<<grid, 256, 0, ctx->stream>>>(Af, n, na, Bf, n, 1, n, rows, d_partial, gate)
      if (ig == 1) DDFG(1); else if (ig == 2) DDFG(2); else if (ig == 4) DDFG(4); else if (ig == 8) DDFG(8); else DDFG(16);
#undef DDFG
      reduce_dev_kernel<<<na, 256, 0, ctx->stream>>>(d_partial, (int)nchunks, na, 1, h_dev, Tm, ldT, js, 0, 0, 0, gate);
      const unsigned gridc = (unsigned)std::min<long long>((n + 255) / 256, (long long)sm_count * 8);
      const size_t shm = (size_t)na * sizeof(float2);
      smem_limit(combine_df_kernel<1>, shm);
      combine_df_kernel<1><<<gridc, 256, shm, ctx->stream>>>(Af, n, na, h_dev, 1, static_cast<float2*>(W), n, n, -1.0, 1.0,
                                                            gate);
      OMEN_CHECK_LAUNCH(ctx);
      return OMEN_OK;
    }
    const int ig1 = dots_ig_for(na, dots1_ig(cplx));
    const int rows = (int)dot_rows(na, ig1);
    const long long nchunks = (n + rows - 1) / rows;
    omen_status s1 = ensure_partial((size_t)nchunks * na);
    if (s1 != OMEN_OK) return s1;
    dim3 grid((na + ig1 - 1) / ig1, (unsigned)nchunks);
    const size_t shm1 = (size_t)na * sizeof(double2);
    const unsigned grid1 = (unsigned)std::min<long long>((n + 255) / 256, (long long)sm_count * 8);
#define PASSG(Tt, Cc)                                                                                            \
  do {                                                                                                           \
    launch_dots1<Tt, Cc>(ig1, grid, ctx->stream, Vb, n, na, W, n, rows, d_partial, 0, 0, 0, nullptr, nullptr, gate); \
    reduce_dev_kernel<<<na, 256, 0, ctx->stream>>>(d_partial, (int)nchunks, na, 1, h_dev, Tm, ldT, js, 0, 0, 0, gate); \
    smem_limit(combine1_kernel<Tt, Cc>, shm1);                                                                   \
    combine1_kernel<Tt, Cc><<<grid1, 256, shm1, ctx->stream>>>(Vb, n, na, h_dev, W, n, -1.0, 1.0, 0, 0, 0, nullptr, \
                                                              nullptr, gate);                                   \
  } while (0)
    if (prec == OMEN_F64) { if (cplx) PASSG(double, true); else PASSG(double, false); }
    else { if (cplx) PASSG(float, true); else PASSG(float, false); }
#undef PASSG
    OMEN_CHECK_LAUNCH(ctx);
    return OMEN_OK;
  }

  // the next gated pass (parity) is applied unconditionally (after a restart's full passes)
  omen_status force_next_pass(int parity) {
    OMEN_CUDA(ctx, cudaMemsetAsync(ctx->d_status + 2 + (parity ^ 1), 1, sizeof(int), ctx->stream));
    return OMEN_OK;
  }

  omen_status normalize_dev(const void* W, void* V, const double2* nrm2, double2* Tm, int ldT, int row, int col) {
    const unsigned grid = (unsigned)std::min<long long>((n + 255) / 256, (long long)sm_count * 8);
    int* flag = ctx->d_status + 1;
    if (prec == OMEN_F64_DF) {
      normalize_df_kernel<<<grid, 256, 0, ctx->stream>>>(static_cast<const float2*>(W), static_cast<float2*>(V), n, nrm2, Tm,
                                                         ldT, row, col, flag);
      OMEN_CHECK_LAUNCH(ctx);
      return OMEN_OK;
    }
    if (prec == OMEN_F64) {
      if (cplx) normalize_kernel<double, true><<<grid, 256, 0, ctx->stream>>>(W, V, n, nrm2, Tm, ldT, row, col, flag);
      else normalize_kernel<double, false><<<grid, 256, 0, ctx->stream>>>(W, V, n, nrm2, Tm, ldT, row, col, flag);
    } else {
      if (cplx) normalize_kernel<float, true><<<grid, 256, 0, ctx->stream>>>(W, V, n, nrm2, Tm, ldT, row, col, flag);
      else normalize_kernel<float, false><<<grid, 256, 0, ctx->stream>>>(W, V, n, nrm2, Tm, ldT, row, col, flag);
    }
    OMEN_CHECK_LAUNCH(ctx);
    return OMEN_OK;
  }

  // ---- batched: P independent problems.  Problem p's part of a vector slot starts at element
  // b_off[p] and has b_len[p] rows (device arrays; b_nmax = the longest).  A: na basis slots with
  // stride lda between slots; B, out, T per problem. ----
  const long long* b_off = nullptr;
  const long long* b_len = nullptr;
  const int* b_act = nullptr;   // per-problem 0/1: frozen problems are skipped
  long long b_nmax = 0;

  omen_status dots_dev_batch(int P, const void* A, long long lda, int na, const void* B, double2* out_dev,
                             long long out_ps, double2* accT, int ldT, long long t_ps, int col0) {
    // the P problems share the grid: chunks sized for about two CTAs per SM over the batch
    const int igb = dots_ig_for(na, dots1_ig(cplx));
    const long long groups = (na + igb - 1) / igb;
    const long long want = std::max<long long>(1, (2LL * sm_count + groups * P - 1) / (groups * P));
    long long rows = (b_nmax + want - 1) / want;
    rows = std::min<long long>(8192, std::max<long long>(256, (rows + 255) / 256 * 256));
    while ((b_nmax + rows - 1) / rows > 65535) rows *= 2;
    const long long nchunks = (b_nmax + rows - 1) / rows;
    const long long pps = nchunks * na;
    omen_status s1 = ensure_partial((size_t)pps * P);
    if (s1 != OMEN_OK) return s1;
    dim3 grid((unsigned)groups, (unsigned)nchunks, P);
#define DOTSB(T, Cc) \
  launch_dots1<T, Cc>(igb, grid, ctx->stream, A, lda, na, B, b_nmax, (int)rows, d_partial, 0, 0, pps, b_off, b_len, b_act)
    if (prec == OMEN_F64) { if (cplx) DOTSB(double, true); else DOTSB(double, false); }
    else { if (cplx) DOTSB(float, true); else DOTSB(float, false); }
#undef DOTSB
    reduce_dev_kernel<<<dim3(na, P), 256, 0, ctx->stream>>>(d_partial, (int)nchunks, na, 1, out_dev, accT, ldT, col0, pps,
                                                            out_ps, t_ps, b_act);
    OMEN_CHECK_LAUNCH(ctx);
    return OMEN_OK;
  }

  omen_status combine_dev_batch(int P, const void* A, long long lda, int na, const double2* M_dev, long long m_ps, void* Y,
                                double alpha, double beta) {
    const size_t shm1 = (size_t)na * sizeof(double2);
    const unsigned gx = (unsigned)std::max<long long>(1, std::min<long long>((b_nmax + 255) / 256, (long long)sm_count * 8 / std::max(1, P) + 1));
    dim3 grid(gx, P);
#define COMB1B(T, Cc)                                                                                 \
  do {                                                                                                \
    smem_limit(combine1_kernel<T, Cc>, shm1);                                                         \
    combine1_kernel<T, Cc><<<grid, 256, shm1, ctx->stream>>>(A, lda, na, M_dev, Y, b_nmax, alpha, beta, 0, m_ps, 0, b_off, b_len, b_act); \
  } while (0)
    if (prec == OMEN_F64) { if (cplx) COMB1B(double, true); else COMB1B(double, false); }
    else { if (cplx) COMB1B(float, true); else COMB1B(float, false); }
#undef COMB1B
    OMEN_CHECK_LAUNCH(ctx);
    return OMEN_OK;
  }

  omen_status normalize_dev_batch(int P, const void* W, void* Vo, const double2* nrm2, double2* Tm, int ldT,
                                  long long t_ps, int row, int col) {
    const unsigned gx = (unsigned)std::max<long long>(1, std::min<long long>((b_nmax + 255) / 256, (long long)sm_count * 8 / std::max(1, P) + 1));
    dim3 grid(gx, P);
    int* flag = ctx->d_status + 1;
#define NORMB(T, Cc) \
  normalize_kernel<T, Cc><<<grid, 256, 0, ctx->stream>>>(W, Vo, b_nmax, nrm2, Tm, ldT, row, col, flag, 0, 0, 1, t_ps, b_off, b_len, b_act)
    if (prec == OMEN_F64) { if (cplx) NORMB(double, true); else NORMB(double, false); }
    else { if (cplx) NORMB(float, true); else NORMB(float, false); }
#undef NORMB
    OMEN_CHECK_LAUNCH(ctx);
    return OMEN_OK;
  }

  omen_status random_fill(void* X, int ncols, unsigned long long seed) {
    const long long total = n * ncols;
    const unsigned grid = (unsigned)std::min<long long>((total + 255) / 256, (long long)sm_count * 8);
    if (prec == OMEN_F64_DF) {
      random_fill_df_kernel<<<grid, 256, 0, ctx->stream>>>(static_cast<float2*>(X), total, seed);
      OMEN_CHECK_LAUNCH(ctx);
      return OMEN_OK;
    }
    if (prec == OMEN_F64) {
      if (cplx) random_fill_kernel<double, true><<<grid, 256, 0, ctx->stream>>>(X, total, seed);
      else random_fill_kernel<double, false><<<grid, 256, 0, ctx->stream>>>(X, total, seed);
    } else {
      if (cplx) random_fill_kernel<float, true><<<grid, 256, 0, ctx->stream>>>(X, total, seed);
      else random_fill_kernel<float, false><<<grid, 256, 0, ctx->stream>>>(X, total, seed);
    }
    OMEN_CHECK_LAUNCH(ctx);
    return OMEN_OK;
  }

  // operator: W = A X, A = H (folded = false) or (H - sigma)^2
  bool negate = false;   // operator -H (highest eigenvalues)
  // locking: the nlock vectors at lock_X (columns) are projected out after every product, so
  // the recurrence sees the operator restricted to their orthogonal complement
  const void* lock_X = nullptr;
  int nlock = 0;
  double2* d_lock = nullptr;   // [nlock] projections (single column)
  unsigned long long lock_seed = 0;   // start vector of a locked solve: a new draw every time
  // a solve may stop early once its lowest Ritz value minus its residual exceeds this line
  bool has_line = false;
  double stop_line = 0.0;

  omen_status deflate(void* W) {
    if (nlock == 0) return OMEN_OK;
    omen_status s1 = dots_dev(lock_X, nlock, W, 1, d_lock, nullptr, 0, 0);
    if (s1 == OMEN_OK) s1 = combine_dev(lock_X, nlock, d_lock, 1, W, -1.0, 1.0);
    return s1;
  }

  omen_status apply(const void* X, void* W, void* tmp, int nb, bool folded, double sigma, long long& count) {
    if (nlock > 0) {
      if (nb != 1 || negate) return set_err(ctx, OMEN_EUNSUPPORTED, "locking needs the single-vector lowest solve");
      omen_status s = apply_raw(X, W, tmp, nb, folded, sigma, count);
      return s == OMEN_OK ? deflate(W) : s;
    }
    return apply_raw(X, W, tmp, nb, folded, sigma, count);
  }

  omen_status apply_raw(const void* X, void* W, void* tmp, int nb, bool folded, double sigma, long long& count) {
    if (!folded) {
      count += nb;
      omen_status s = launch_hx(ctx, ham, X, W, nb, 0.0, prec);
      if (s != OMEN_OK || !negate) return s;
      std::vector<cd> m1((size_t)nb * nb, cd(0));
      for (int j = 0; j < nb; ++j) m1[j + (size_t)j * nb] = cd(-1.0);
      // W = -W via a copy: W <- 0*W + (-1) * tmp where tmp holds H X
      OMEN_CUDA(ctx, cudaMemcpyAsync(tmp, W, (size_t)nb * n * el, cudaMemcpyDeviceToDevice, ctx->stream));
      return combine(tmp, nb, m1, nb, W, 1.0, 0.0);
    }
    omen_status s = launch_hx(ctx, ham, X, tmp, nb, sigma, prec);
    if (s != OMEN_OK) return s;
    count += 2 * nb;
    return launch_hx(ctx, ham, tmp, W, nb, sigma, prec);
  }

  // Orthonormalise the nb columns of W in place (Cholesky QR, twice): W_in = W_out R.
  // Returns 1 in `deficient` if the block is numerically rank deficient.
  omen_status cholqr(void* W, int nb, std::vector<cd>& R, int& deficient) {
    R.assign((size_t)nb * nb, cd(0));
    for (int i = 0; i < nb; ++i) R[i + (size_t)i * nb] = 1.0;
    deficient = 0;
    std::vector<cd> G, Rk((size_t)nb * nb), Ri((size_t)nb * nb);
    for (int pass = 0; pass < 2; ++pass) {
      omen_status s = dots(W, nb, W, nb, G);
      if (s != OMEN_OK) return s;
      // Hermitian part
      for (int j = 0; j < nb; ++j)
        for (int i = 0; i < nb; ++i)
          if (i > j) {
            cd a = 0.5 * (G[i + (size_t)j * nb] + std::conj(G[j + (size_t)i * nb]));
            G[i + (size_t)j * nb] = a;
            G[j + (size_t)i * nb] = std::conj(a);
          }
      double gmax = 0;
      for (int i = 0; i < nb; ++i) gmax = std::max(gmax, std::real(G[i + (size_t)i * nb]));
      for (int i = 0; i < nb; ++i)
        if (std::real(G[i + (size_t)i * nb]) <= 1e-28 * std::max(gmax, 1e-300) || gmax == 0.0) { deficient = 1; return OMEN_OK; }
      if (cholesky_upper(nb, G.data(), Rk.data())) { deficient = 1; return OMEN_OK; }
      // ill-conditioned after the first pass means the block lost rank
      if (pass == 1) {
        double dmin = 1e300, dmax = 0;
        for (int i = 0; i < nb; ++i) {
          dmin = std::min(dmin, std::abs(Rk[i + (size_t)i * nb]));
          dmax = std::max(dmax, std::abs(Rk[i + (size_t)i * nb]));
        }
        if (dmin < 1e-6 * dmax) { deficient = 1; return OMEN_OK; }
      }
      upper_inverse(nb, Rk.data(), Ri.data());
      // W <- W Ri from a copy of W (the combination may not alias its input)
      const size_t need = (size_t)nb * n * el;
      if (need > qr_cap) {
        cudaFree(qr_tmp);
        qr_tmp = nullptr;
        qr_cap = 0;
        if (cudaMalloc(&qr_tmp, need) != cudaSuccess) {
          cudaGetLastError();
          return set_err(ctx, OMEN_ENOMEM, "QR work vectors");
        }
        qr_cap = need;
      }
      OMEN_CUDA(ctx, cudaMemcpyAsync(qr_tmp, W, need, cudaMemcpyDeviceToDevice, ctx->stream));
      omen_status s2 = combine(qr_tmp, nb, Ri, nb, W, 1.0, 0.0);
      if (s2 != OMEN_OK) return s2;
      // R <- Rk R
      std::vector<cd> Rn((size_t)nb * nb, cd(0));
      for (int j = 0; j < nb; ++j)
        for (int i = 0; i < nb; ++i) {
          cd s3 = 0;
          for (int k = 0; k < nb; ++k) s3 += Rk[i + (size_t)k * nb] * R[k + (size_t)j * nb];
          Rn[i + (size_t)j * nb] = s3;
        }
      R = Rn;
    }
    return OMEN_OK;
  }

  // Orthogonalise W (nb cols) against the first nv columns of V (twice); adds the
  // coefficients into hsum (nv x nb).
  // Block three-term step: W -= V_j (V_j^H W) and W -= V_{j-1} Mprev (the known coupling), then
  // one full classical Gram–Schmidt pass over the nv basis vectors.  hsum (nv x nb) receives
  // every coefficient removed, Mprev included.
  omen_status orthogonalise3(const void* V, int nv, int jstart, int jprev, const std::vector<cd>& Mprev, void* W, int nb,
                             std::vector<cd>& hsum) {
    hsum.assign((size_t)nv * nb, cd(0));
    const size_t need = (size_t)nv * nb * 2 + (size_t)nb * nb;
    if (need > hs_cap) {
      cudaFree(d_hs);
      d_hs = nullptr;
      hs_cap = 0;
      if (cudaMalloc(&d_hs, need * sizeof(double2)) != cudaSuccess) {
        cudaGetLastError();
        return set_err(ctx, OMEN_ENOMEM, "projection sums");
      }
      hs_cap = need;
    }
    double2* h = d_hs;
    double2* sum = d_hs + (size_t)nv * nb;
    double2* mp = sum + (size_t)nv * nb;
    OMEN_CUDA(ctx, cudaMemsetAsync(sum, 0, sizeof(double2) * nv * nb, ctx->stream));
    omen_status s = dots_dev(col(const_cast<void*>(V), jstart), nb, W, nb, h, sum + jstart, nv, 0);
    if (s == OMEN_OK) s = combine_dev(col(const_cast<void*>(V), jstart), nb, h, nb, W, -1.0, 1.0);
    if (s != OMEN_OK) return s;
    if (jprev >= 0) {
      OMEN_CUDA(ctx, cudaMemcpyAsync(mp, Mprev.data(), sizeof(double2) * nb * nb, cudaMemcpyHostToDevice, ctx->stream));
      s = combine_dev(col(const_cast<void*>(V), jprev), nb, mp, nb, W, -1.0, 1.0);
      if (s != OMEN_OK) return s;
    }
    s = dots_dev(V, nv, W, nb, h, sum, nv, 0);
    if (s == OMEN_OK) s = combine_dev(V, nv, h, nb, W, -1.0, 1.0);
    if (s != OMEN_OK) return s;
    OMEN_CUDA(ctx, cudaMemcpyAsync(hsum.data(), sum, sizeof(double2) * nv * nb, cudaMemcpyDeviceToHost, ctx->stream));
    OMEN_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    if (jprev >= 0)
      for (int j = 0; j < nb; ++j)
        for (int i = 0; i < nb; ++i) hsum[(jprev + i) + (size_t)j * nv] += Mprev[i + (size_t)j * nb];
    for (const cd& v : hsum)
      if (!std::isfinite(v.real()) || !std::isfinite(v.imag()))
        return set_err(ctx, OMEN_ENUMERIC, "non-finite value in a Krylov inner product");
    return OMEN_OK;
  }

  omen_status orthogonalise(const void* V, int nv, void* W, int nb, std::vector<cd>* hsum) {
    if (hsum) hsum->assign((size_t)nv * nb, cd(0));
    if (nv == 0) return OMEN_OK;
    if (nb > kMaxBlockCols) return set_err(ctx, OMEN_EINVAL, "orthogonalise: too many columns");
    const size_t need = (size_t)nv * nb * 2;   // per-pass coefficients + running sums
    if (need > hs_cap) {
      cudaFree(d_hs);
      d_hs = nullptr;
      hs_cap = 0;
      if (cudaMalloc(&d_hs, need * sizeof(double2)) != cudaSuccess) {
        cudaGetLastError();
        return set_err(ctx, OMEN_ENOMEM, "projection sums");
      }
      hs_cap = need;
    }
    double2* h = d_hs;
    double2* sum = d_hs + (size_t)nv * nb;
    OMEN_CUDA(ctx, cudaMemsetAsync(sum, 0, sizeof(double2) * nv * nb, ctx->stream));
    for (int pass = 0; pass < 2; ++pass) {
      omen_status s = dots_dev(V, nv, W, nb, h, sum, nv, 0);
      if (s != OMEN_OK) return s;
      s = combine_dev(V, nv, h, nb, W, -1.0, 1.0);
      if (s != OMEN_OK) return s;
    }
    if (hsum) {
      OMEN_CUDA(ctx, cudaMemcpyAsync(hsum->data(), sum, sizeof(double2) * nv * nb, cudaMemcpyDeviceToHost, ctx->stream));
      OMEN_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
      for (const cd& v : *hsum)
        if (!std::isfinite(v.real()) || !std::isfinite(v.imag()))
          return set_err(ctx, OMEN_ENUMERIC, "non-finite value in a Krylov inner product");
    }
    return OMEN_OK;
  }

};

// ---------------------------------------------------------------------------------------
static int max_iter_of(const omen_eig_opts* o) { return o->max_iter; }

struct RitzResult {
  std::vector<double> lam;   // eigenvalues of H (ascending)
  std::vector<double> res;   // FP64 ||H x - lam x||
  std::vector<double> bound; // min(res, res^2/gap)
};

// Error bound per pair from residuals and the spread of the computed values: Weyl (r) or
// Kato–Temple (r^2 / gap) with the gap to the nearest value outside the pair's cluster.
static void error_bounds(const std::vector<double>& lam_all, const std::vector<double>& lam,
                         const std::vector<double>& res, std::vector<double>& bound) {
  bound.resize(lam.size());
  for (size_t i = 0; i < lam.size(); ++i) {
    const double clus = 1e-7 * std::max(1.0, std::fabs(lam[i]));
    double gap = 1e300;
    for (double v : lam_all) {
      const double d = std::fabs(v - lam[i]);
      if (d > clus) gap = std::min(gap, d);
    }
    const double r = res[i];
    bound[i] = (gap < 1e299) ? std::min(r, r * r / gap) : r;
  }
}

// Rayleigh quotients and FP64-accumulated residual norms of the k columns of X (H X in HX).
static omen_status rayleigh_residuals(KrylovOps& op, void* X, void* HX, void* R, int k, std::vector<double>& lam,
                                      std::vector<double>& res) {
  // all k columns at once: diag(X^H X), diag(X^H HX), then R = HX - X diag(lam), diag(R^H R)
  lam.assign(k, 0.0);
  res.assign(k, 0.0);
  std::vector<double> xx(k), rr(k);
  for (int j0 = 0; j0 < k; j0 += kMaxBlockCols) {
    const int nb = std::min(kMaxBlockCols, k - j0);
    std::vector<cd> g, gh;
    // only the diagonals of X^H X, X^H HX and R^H R are needed: column-wise products
    omen_status s = op.dots_cols(op.col(X, j0), op.col(X, j0), nb, g);
    if (s != OMEN_OK) return s;
    s = op.dots_cols(op.col(X, j0), op.col(HX, j0), nb, gh);
    if (s != OMEN_OK) return s;
    for (int j = 0; j < nb; ++j) {
      xx[j0 + j] = std::real(g[j]);
      lam[j0 + j] = std::real(gh[j]) / xx[j0 + j];
    }
    OMEN_CUDA(op.ctx, cudaMemcpyAsync(op.col(R, j0), op.col(HX, j0), (size_t)nb * op.n * op.el, cudaMemcpyDeviceToDevice,
                                      op.ctx->stream));
    // R_j -= lam_j X_j, one column at a time (the coefficient matrix is diagonal)
    std::vector<double2> lj(nb);
    for (int j = 0; j < nb; ++j) lj[j] = make_double2(lam[j0 + j], 0.0);
    OMEN_CUDA(op.ctx, cudaMemcpyAsync(op.d_small, lj.data(), sizeof(double2) * nb, cudaMemcpyHostToDevice, op.ctx->stream));
    for (int j = 0; j < nb && s == OMEN_OK; ++j)
      s = op.combine_dev(op.col(X, j0 + j), 1, op.d_small + j, 1, op.col(R, j0 + j), -1.0, 1.0);
    if (s != OMEN_OK) return s;
    s = op.dots_cols(op.col(R, j0), op.col(R, j0), nb, g);
    if (s != OMEN_OK) return s;
    for (int j = 0; j < nb; ++j) res[j0 + j] = std::sqrt(std::max(0.0, std::real(g[j])) / xx[j0 + j]);
  }
  return OMEN_OK;
}

struct DevBuf {
  void* p = nullptr;
  ~DevBuf() { if (p) cudaFree(p); }
};

// Solve in the vector precision of `op`; on return X holds k Ritz vectors (columns) with
// their eigenvalues in rr.lam, sorted ascending.
static omen_status lanczos_solve(KrylovOps& op, const omen_eig_opts* o, void* X, int k_out, RitzResult& rr,
                                 omen_eig_info* info, const void* v0_host, bool& converged) {
  omen_ctx* ctx = op.ctx;
  const int b = o->block;
  const int m = o->basis;
  const bool folded = (o->which == OMEN_NEAREST);
  const long long n = op.n;
  DevBuf Vb, Wb, Tb, Xb, HXb, Rb;
  const size_t vbytes = (size_t)n * op.el;
  if (cudaMalloc(&Vb.p, (size_t)(m + b) * vbytes) != cudaSuccess || cudaMalloc(&Wb.p, (size_t)b * vbytes) != cudaSuccess ||
      cudaMalloc(&Tb.p, (size_t)std::max(b, k_out) * vbytes) != cudaSuccess ||
      cudaMalloc(&Xb.p, (size_t)m * vbytes) != cudaSuccess) {
    cudaGetLastError();
    return set_err(ctx, OMEN_ENOMEM, "Lanczos basis (%d vectors of %lld rows)", m + b, n);
  }
  void* V = Vb.p;
  void* W = Wb.p;
  void* tmp = Tb.p;
  // start block
  if (o->v0_dev) {
    OMEN_CUDA(ctx, cudaMemcpyAsync(V, o->v0_dev, (size_t)b * vbytes, cudaMemcpyDeviceToDevice, ctx->stream));
  } else if (v0_host) {
    OMEN_CUDA(ctx, cudaMemcpyAsync(V, v0_host, (size_t)b * vbytes, cudaMemcpyHostToDevice, ctx->stream));
  } else {
    omen_status s = op.random_fill(V, b, 0x5EEDull);
    if (s != OMEN_OK) return s;
  }
  std::vector<cd> R;
  int deficient = 0;
  omen_status s = op.cholqr(V, b, R, deficient);
  if (s != OMEN_OK) return s;
  if (deficient) return set_err(ctx, OMEN_EINVAL, "start block is rank deficient");

  const int ldT = m + b;
  std::vector<cd> T((size_t)ldT * ldT, cd(0));
  auto Tat = [&](int i, int j) -> cd& { return T[i + (size_t)j * ldT]; };
  int jstart = 0, nbas = b;   // current block = V[jstart, jstart+b), basis = V[0, nbas)
  long long hx = 0;
  int iter = 0, restarts = 0;
  const int max_iter = o->max_iter;
  double gateA = -1.0;
  converged = false;
  std::vector<double> theta;
  std::vector<cd> Y;
  std::vector<cd> Rlast;
  unsigned long long reseed = 1;
  auto t_start = std::chrono::steady_clock::now();
  bool fresh = true;   // first step of a cycle: the new block couples to every kept vector

  while (true) {
    // expand
    s = op.apply(op.col(V, jstart), W, tmp, b, folded, o->sigma, hx);
    if (s != OMEN_OK) return s;
    std::vector<cd> hsum;
    if (fresh || jstart < b) {
      // two full classical Gram–Schmidt passes
      s = op.orthogonalise(V, nbas, W, b, &hsum);
    } else {
      // three-term block step (against the current and previous blocks), then one full pass
      const int jprev = jstart - b;
      std::vector<cd> Mprev((size_t)b * b);
      for (int j = 0; j < b; ++j)
        for (int i = 0; i < b; ++i) Mprev[i + (size_t)j * b] = Tat(jprev + i, jstart + j);
      s = op.orthogonalise3(V, nbas, jstart, jprev, Mprev, W, b, hsum);
    }
    fresh = false;
    if (s != OMEN_OK) return s;
    for (int j = 0; j < b; ++j)
      for (int i = 0; i < nbas; ++i) {
        const cd v = hsum[i + (size_t)j * nbas];
        Tat(i, jstart + j) = v;
        Tat(jstart + j, i) = std::conj(v);
      }
    for (int j = 0; j < b; ++j)
      for (int i = 0; i < b; ++i) {  // Hermitian average of the diagonal block
        const cd a = 0.5 * (Tat(jstart + i, jstart + j) + std::conj(Tat(jstart + j, jstart + i)));
        Tat(jstart + i, jstart + j) = a;
        Tat(jstart + j, jstart + i) = std::conj(a);
      }
    s = op.cholqr(W, b, R, deficient);
    if (s != OMEN_OK) return s;
    if (deficient) {
      // invariant subspace found: continue with fresh directions, no coupling
      s = op.random_fill(W, b, 0xABCD0000ull + reseed++);
      if (s != OMEN_OK) return s;
      s = op.orthogonalise(V, nbas, W, b, nullptr);
      if (s != OMEN_OK) return s;
      s = op.orthogonalise(V, nbas, W, b, nullptr);
      if (s != OMEN_OK) return s;
      std::vector<cd> Rd;
      s = op.cholqr(W, b, Rd, deficient);
      if (s != OMEN_OK) return s;
      if (deficient) return set_err(ctx, OMEN_ENUMERIC, "could not extend the Krylov basis");
      R.assign((size_t)b * b, cd(0));
    }
    OMEN_CUDA(ctx, cudaMemcpyAsync(op.col(V, nbas), W, (size_t)b * vbytes, cudaMemcpyDeviceToDevice, ctx->stream));
    for (int j = 0; j < b; ++j)
      for (int i = 0; i < b; ++i) {
        Tat(nbas + i, jstart + j) = R[i + (size_t)j * b];
        Tat(jstart + j, nbas + i) = std::conj(R[i + (size_t)j * b]);
      }
    Rlast = R;
    ++iter;
    const bool full = nbas + b > m;
    const bool check = full || iter >= max_iter || (iter % std::max(4, (m / b) / 2) == 0 && nbas >= o->nev + b);
    if (check && nbas >= o->nev) {
      // Rayleigh–Ritz on T[0:nbas, 0:nbas]
      std::vector<cd> Tn((size_t)nbas * nbas);
      for (int j = 0; j < nbas; ++j)
        for (int i = 0; i < nbas; ++i) Tn[i + (size_t)j * nbas] = Tat(i, j);
      theta.assign(nbas, 0.0);
      Y.assign((size_t)nbas * nbas, cd(0));
      if (hermitian_eig(nbas, Tn.data(), theta.data(), Y.data()))
        return set_err(ctx, OMEN_ENUMERIC, "projected eigenproblem did not converge");
      std::vector<double> resA(nbas);
      for (int i = 0; i < nbas; ++i) {
        double acc = 0;
        for (int r = 0; r < b; ++r) {
          cd v = 0;
          for (int c = 0; c < b; ++c) v += Rlast[r + (size_t)c * b] * Y[(jstart + c) + (size_t)i * nbas];
          acc += std::norm(v);
        }
        resA[i] = std::sqrt(acc);
      }
      const int nev = o->nev;
      bool done = false;
      if (!folded) {
        std::vector<double> lam(theta.begin(), theta.begin() + nev), res(resA.begin(), resA.begin() + nev), bd;
        error_bounds(theta, lam, res, bd);
        done = *std::max_element(bd.begin(), bd.end()) <= o->tol;
      } else {
        double rmax = *std::max_element(resA.begin(), resA.begin() + nev);
        if (gateA < 0) gateA = std::max(o->tol, 1e-12) * 1e3;
        if (rmax <= gateA || iter >= max_iter) {
          // explicit check on H for the nev (+ b) Ritz vectors of smallest theta
          const int kc = std::min(nbas, nev + b);
          std::vector<cd> Yk((size_t)nbas * kc);
          for (int j = 0; j < kc; ++j)
            for (int i = 0; i < nbas; ++i) Yk[i + (size_t)j * nbas] = Y[i + (size_t)j * nbas];
          s = op.combine(V, nbas, Yk, kc, Xb.p, 1.0, 0.0);
          if (s != OMEN_OK) return s;
          if (!HXb.p && (cudaMalloc(&HXb.p, (size_t)(o->nev + b) * vbytes) != cudaSuccess ||
                         cudaMalloc(&Rb.p, (size_t)(o->nev + b) * vbytes) != cudaSuccess)) {
            cudaGetLastError();
            return set_err(ctx, OMEN_ENOMEM, "Ritz check vectors");
          }
          s = launch_hx(ctx, op.ham, Xb.p, HXb.p, kc, 0.0, op.prec);
          if (s != OMEN_OK) return s;
          hx += kc;
          std::vector<double> lamk, resk, bd;
          s = rayleigh_residuals(op, Xb.p, HXb.p, Rb.p, kc, lamk, resk);
          if (s != OMEN_OK) return s;
          std::vector<double> lam(lamk.begin(), lamk.begin() + nev), res(resk.begin(), resk.begin() + nev);
          error_bounds(lamk, lam, res, bd);
          done = *std::max_element(bd.begin(), bd.end()) <= o->tol;
          if (!done) gateA = std::min(gateA, rmax) * 0.01;
        }
      }
      if (done || iter >= max_iter) {
        converged = done;
        break;
      }
      if (full) {
        // thick restart: keep kk Ritz vectors of smallest theta and the residual block
        const int kk = std::min(m - b, std::max(o->nev + b, (nbas / 2 / b) * b));
        std::vector<cd> Yk((size_t)nbas * kk);
        for (int j = 0; j < kk; ++j)
          for (int i = 0; i < nbas; ++i) Yk[i + (size_t)j * nbas] = Y[i + (size_t)j * nbas];
        s = op.combine(V, nbas, Yk, kk, Xb.p, 1.0, 0.0);
        if (s != OMEN_OK) return s;
        OMEN_CUDA(ctx, cudaMemcpyAsync(V, Xb.p, (size_t)kk * vbytes, cudaMemcpyDeviceToDevice, ctx->stream));
        OMEN_CUDA(ctx, cudaMemcpyAsync(op.col(V, kk), op.col(V, nbas), (size_t)b * vbytes, cudaMemcpyDeviceToDevice, ctx->stream));
        std::fill(T.begin(), T.end(), cd(0));
        for (int i = 0; i < kk; ++i) Tat(i, i) = theta[i];
        for (int i = 0; i < kk; ++i)
          for (int r = 0; r < b; ++r) {
            cd v = 0;
            for (int c = 0; c < b; ++c) v += Rlast[r + (size_t)c * b] * Y[(jstart + c) + (size_t)i * nbas];
            Tat(kk + r, i) = v;
            Tat(i, kk + r) = std::conj(v);
          }
        jstart = kk;
        nbas = kk + b;
        ++restarts;
        fresh = true;
        continue;
      }
    }
    jstart = nbas;
    nbas += b;
  }

  // outputs: k_out Ritz vectors of smallest theta, eigenvalues of H from Rayleigh quotients
  const int kc = std::min(nbas, k_out);
  std::vector<cd> Yk((size_t)nbas * kc);
  for (int j = 0; j < kc; ++j)
    for (int i = 0; i < nbas; ++i) Yk[i + (size_t)j * nbas] = Y[i + (size_t)j * nbas];
  s = op.combine(V, nbas, Yk, kc, X, 1.0, 0.0);
  if (s != OMEN_OK) return s;
  if (info) {
    info->iterations = iter;
    info->hx_count = hx;
    info->restarts = restarts;
    info->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
  }
  (void)rr;
  return OMEN_OK;
}

// Single-vector thick-restart Lanczos with the recurrence kept on the device: the
// projection coefficients accumulate into a device copy of T and the norm of the new
// direction is applied from device memory, so a step issues kernels only and the host
// synchronises once per convergence check (every few steps / at each restart).
// Executable graphs of step sequences, keyed by what fixes their kernel arguments (first step's
// basis index, basis size, fresh flag, number of steps).  Captured on the context's private
// stream, replayed on the caller's stream; destroyed (after the stream drains) with the solve.
struct SegmentGraphs {
  omen_ctx* ctx;
  std::map<std::array<int, 4>, cudaGraphExec_t> cache;
  explicit SegmentGraphs(omen_ctx* c) : ctx(c) {}
  ~SegmentGraphs() {
    if (cache.empty()) return;
    cudaStreamSynchronize(ctx->stream);
    for (auto& kv : cache) cudaGraphExecDestroy(kv.second);
  }
  template <typename F>
  omen_status run(const std::array<int, 4>& key, F&& enqueue) {
    auto it = cache.find(key);
    if (it == cache.end()) {
      if (!ctx->cap_stream && cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
        ctx->cap_stream = nullptr;
        return set_err(ctx, OMEN_ECUDA, "could not create the capture stream");
      }
      cudaStream_t user = ctx->stream;
      ctx->stream = ctx->cap_stream;
      cudaError_t e = cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeRelaxed);
      omen_status s = (e == cudaSuccess) ? enqueue() : OMEN_ECUDA;
      cudaGraph_t g = nullptr;
      if (e == cudaSuccess) e = cudaStreamEndCapture(ctx->cap_stream, &g);
      ctx->stream = user;
      if (s != OMEN_OK || e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        return s != OMEN_OK ? s : set_err(ctx, OMEN_ECUDA, "Lanczos step capture: %s", cudaGetErrorString(e));
      }
      cudaGraphExec_t ex = nullptr;
      e = cudaGraphInstantiate(&ex, g, 0);
      cudaGraphDestroy(g);
      if (e != cudaSuccess) return set_err(ctx, OMEN_ECUDA, "Lanczos graph instantiation: %s", cudaGetErrorString(e));
      it = cache.emplace(key, ex).first;
    }
    const cudaError_t e = cudaGraphLaunch(it->second, ctx->stream);
    if (e != cudaSuccess) return set_err(ctx, OMEN_ECUDA, "Lanczos graph launch: %s", cudaGetErrorString(e));
    return OMEN_OK;
  }
};

static omen_status lanczos_solve_single(KrylovOps& op, const omen_eig_opts* o, void* X, int k_out,
                                        omen_eig_info* info, bool& converged) {
  omen_ctx* ctx = op.ctx;
  const int m = o->basis;
  const bool folded = (o->which == OMEN_NEAREST);
  const size_t vbytes = (size_t)op.n * op.el;
  const int ldT = m + 1;
  DevBuf Vb, Wb, Tb, Xb, Td, Hd, HXb, Rb;
  if (cudaMalloc(&Vb.p, (size_t)(m + 1) * vbytes) != cudaSuccess || cudaMalloc(&Wb.p, vbytes) != cudaSuccess ||
      cudaMalloc(&Tb.p, std::max<size_t>(1, k_out) * vbytes) != cudaSuccess ||
      cudaMalloc(&Xb.p, (size_t)m * vbytes) != cudaSuccess ||
      cudaMalloc(&Td.p, sizeof(double2) * ldT * ldT) != cudaSuccess ||
      cudaMalloc(&Hd.p, sizeof(double2) * (ldT + 2)) != cudaSuccess) {
    cudaGetLastError();
    return set_err(ctx, OMEN_ENOMEM, "Lanczos basis (%d vectors of %lld rows)", m + 1, op.n);
  }
  void* V = Vb.p;
  void* W = Wb.p;
  void* tmp = Tb.p;
  double2* dT = static_cast<double2*>(Td.p);
  double2* dh = static_cast<double2*>(Hd.p);
  double2* dn = dh + ldT;
  OMEN_CUDA(ctx, cudaMemsetAsync(dT, 0, sizeof(double2) * ldT * ldT, ctx->stream));
  OMEN_CUDA(ctx, cudaMemsetAsync(ctx->d_status + 1, 0, sizeof(int), ctx->stream));
  if (o->v0_dev || o->v0_host) {
    if (o->v0_dev) OMEN_CUDA(ctx, cudaMemcpyAsync(W, o->v0_dev, vbytes, cudaMemcpyDeviceToDevice, ctx->stream));
    else OMEN_CUDA(ctx, cudaMemcpyAsync(W, o->v0_host, vbytes, cudaMemcpyHostToDevice, ctx->stream));
    if (op.prec == OMEN_F64_DF) {
      // the start vector comes in FP64: split it into double-float pairs in place (same size)
      omen_status sc = omen_convert_vectors(ctx, W, OMEN_F64, W, OMEN_F64_DF, op.n);
      if (sc != OMEN_OK) return sc;
    }
  } else {
    omen_status s = op.random_fill(W, 1, op.nlock ? 0x5EEDull + 0x9E3779B97F4A7C15ull * (op.lock_seed + 1) : 0x5EEDull);
    if (s != OMEN_OK) return s;
  }
  for (int pass = 0; pass < 2 && op.nlock; ++pass) {
    omen_status sd = op.deflate(W);
    if (sd != OMEN_OK) return sd;
  }
  omen_status s = op.dots_dev(W, 1, W, 1, dn, nullptr, 0, 0);
  if (s != OMEN_OK) return s;
  s = op.normalize_dev(W, V, dn, nullptr, 0, 0, 0);
  if (s != OMEN_OK) return s;

  std::vector<cd> Th((size_t)ldT * ldT);
  int jstart = 0, nbas = 1;
  long long hx = 0;
  int iter = 0, restarts = 0, since_check = 0;
  const int check_every = std::max(4, std::min(32, m / 4));
  double gateA = -1.0;
  converged = false;
  std::vector<double> theta;
  std::vector<cd> Y;
  auto t_start = std::chrono::steady_clock::now();
  bool fresh = true;   // first step of a cycle: the new vector couples to every kept vector
  bool line_crossed = false;
  // One step on the device: W = A v_js, orthogonalise W against v_0..v_{nb-1} (T column js),
  // v_nb = W / ||W|| (T[nb, js] = ||W||).  No host synchronisation.
  const bool semi = ctx->reorth == OMEN_REORTH_SEMI && op.prec != OMEN_F64_DF;
  // partial reorthogonalisation by overlap estimates (real FP64 / FP32 vectors)
  // (FP64 vectors only: an FP32 basis driven past its rounding floor, as the FP32 phase of a
  // refined solve is, loses orthogonality faster than the estimates follow, and double-float
  // bases drifted from the fully orthogonalised run's Ritz values)
  const bool pro = ctx->reorth == OMEN_REORTH_PARTIAL && op.prec == OMEN_F64;
  const double unit = 1.1102230246251565e-16;                      // 2^-53
  const double eps1 = 0.5 * unit * std::sqrt((double)op.n);
  const double delta = std::sqrt(unit);                            // semi-orthogonality
  int* pgate = ctx->d_status + 6;
  DevBuf Om;
  if (pro) {
    const size_t omb = sizeof(double) * (4 * (size_t)ldT + 1);   // complex estimates, two vectors
    if (cudaMalloc(&Om.p, omb) != cudaSuccess) {
      cudaGetLastError();
      return set_err(ctx, OMEN_ENOMEM, "overlap estimates");
    }
    OMEN_CUDA(ctx, cudaMemsetAsync(Om.p, 0, omb, ctx->stream));
  }
  double* om = static_cast<double*>(Om.p);
  auto enqueue_step = [&](int js, int nb, bool fr) -> omen_status {
    long long unused = 0;
    omen_status s2 = op.apply(op.col(V, js), W, tmp, 1, folded, o->sigma, unused);
    if (s2 != OMEN_OK) return s2;
    if (fr) {
      // two full classical Gram–Schmidt passes
      for (int pass = 0; pass < 2 && s2 == OMEN_OK; ++pass) {
        s2 = op.dots_dev(V, nb, W, 1, dh, dT, ldT, js);
        if (s2 == OMEN_OK) s2 = op.combine_dev(V, nb, dh, 1, W, -1.0, 1.0);
      }
      if (s2 == OMEN_OK && semi) s2 = op.force_next_pass((js + 1) & 1);
      if (s2 == OMEN_OK && pro) {
        if (op.cplx) omega_reset_kernel<true><<<1, 256, 0, ctx->stream>>>(om, ldT, nb, eps1, pgate);
        else omega_reset_kernel<false><<<1, 256, 0, ctx->stream>>>(om, ldT, nb, eps1, pgate);
        OMEN_CHECK_LAUNCH(ctx);
      }
    } else if (pro) {
      // three-term step, then the full pass only when the overlap estimates call for it
      s2 = op.dots_dev(op.col(V, js), 1, W, 1, dh, dT + js, ldT, js);
      if (s2 == OMEN_OK) s2 = op.combine_dev(op.col(V, js), 1, dh, 1, W, -1.0, 1.0);
      if (s2 == OMEN_OK) s2 = op.combine_dev(op.col(V, js - 1), 1, dT + js + (size_t)(js - 1) * ldT, 1, W, -1.0, 1.0);
      if (s2 != OMEN_OK) return s2;
      OMEN_CUDA(ctx, cudaMemcpyAsync(dT + (js - 1) + (size_t)js * ldT, dT + js + (size_t)(js - 1) * ldT,
                                     sizeof(double2), cudaMemcpyDeviceToDevice, ctx->stream));
      s2 = op.dots_dev(W, 1, W, 1, dn, nullptr, 0, 0);
      if (s2 != OMEN_OK) return s2;
      if (op.cplx) omega_kernel<true><<<1, 256, 0, ctx->stream>>>(dT, ldT, js, dn, om, pgate, eps1, delta);
      else omega_kernel<false><<<1, 256, 0, ctx->stream>>>(dT, ldT, js, dn, om, pgate, eps1, delta);
      OMEN_CHECK_LAUNCH(ctx);
      s2 = op.pass_gated(V, nb, W, dh, dT, ldT, js, pgate);
    } else {
      // three-term step against v_j (alpha) and v_{j-1} (beta, already in T), then one full
      // pass that removes what rounding left along every basis vector (under the
      // semi-orthogonality policy: only when the measured overlaps call for it)
      s2 = op.dots_dev(op.col(V, js), 1, W, 1, dh, dT + js, ldT, js);
      if (s2 == OMEN_OK) s2 = op.combine_dev(op.col(V, js), 1, dh, 1, W, -1.0, 1.0);
      if (s2 == OMEN_OK) s2 = op.combine_dev(op.col(V, js - 1), 1, dT + js + (size_t)(js - 1) * ldT, 1, W, -1.0, 1.0);
      if (s2 != OMEN_OK) return s2;
      OMEN_CUDA(ctx, cudaMemcpyAsync(dT + (js - 1) + (size_t)js * ldT, dT + js + (size_t)(js - 1) * ldT,
                                     sizeof(double2), cudaMemcpyDeviceToDevice, ctx->stream));
      if (semi) {
        s2 = op.dots_dev(V, nb, W, 1, dh, nullptr, 0, 0);
        if (s2 == OMEN_OK) s2 = op.dots_dev(W, 1, W, 1, dn, nullptr, 0, 0);
        if (s2 == OMEN_OK) s2 = op.combine_gated(V, nb, dh, W, dn, js & 1, dT + (size_t)js * ldT);
      } else {
        s2 = op.dots_dev(V, nb, W, 1, dh, dT, ldT, js);
        if (s2 == OMEN_OK) s2 = op.combine_dev(V, nb, dh, 1, W, -1.0, 1.0);
      }
    }
    if (s2 == OMEN_OK) s2 = op.dots_dev(W, 1, W, 1, dn, nullptr, 0, 0);
    if (s2 == OMEN_OK) s2 = op.normalize_dev(W, op.col(V, nb), dn, dT, ldT, nb, js);
    return s2;
  };
  // a host check follows the step that leaves nb basis vectors when this holds
  auto check_after = [&](int nb, int it, int since) {
    const bool full_ = nb + 1 > m;
    return (full_ || it >= max_iter_of(o) || (since >= check_every && nb >= o->nev + 1)) && nb >= o->nev;
  };
  SegmentGraphs graphs(ctx);
  const bool use_graphs = ctx->use_graphs && !op.negate;
  if (use_graphs) {
    // the partial-sum buffer must not move under a captured graph: size it for the widest pass
    s = op.ensure_partial(op.max_partials(m + 1));
    if (s != OMEN_OK) return s;
  }
  while (true) {
    // the steps up to and including the next host check run as one segment
    int nseg = 0;
    for (int nb = nbas, it = iter, sc = since_check;; ++nb) {
      ++nseg;
      if (check_after(nb, ++it, ++sc)) break;
    }
    auto run_segment = [&]() -> omen_status {
      int js = jstart, nb = nbas;
      bool fr = fresh;
      for (int i = 0; i < nseg; ++i, fr = false, js = nb, ++nb) {
        omen_status s2 = enqueue_step(js, nb, fr);
        if (s2 != OMEN_OK) return s2;
      }
      return OMEN_OK;
    };
    if (use_graphs && nseg >= 2) s = graphs.run({jstart, nbas, fresh ? 1 : 0, nseg}, run_segment);
    else s = run_segment();
    if (s != OMEN_OK) return s;
    hx += (long long)nseg * (folded ? 2 : 1);
    iter += nseg;
    since_check += nseg;
    nbas += nseg - 1;
    jstart = nbas - 1;
    fresh = false;
    const bool full = nbas + 1 > m;
    {
      since_check = 0;
      OMEN_CUDA(ctx, cudaMemcpyAsync(Th.data(), dT, sizeof(double2) * ldT * ldT, cudaMemcpyDeviceToHost, ctx->stream));
      int flag = 0;
      OMEN_CUDA(ctx, cudaMemcpyAsync(&flag, ctx->d_status + 1, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
      OMEN_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
      if (flag) return set_err(ctx, OMEN_ENUMERIC, "Lanczos breakdown or non-finite value (zero or NaN norm)");
      // Hermitian projected matrix from the column data (row i <= column j)
      std::vector<cd> Tn((size_t)nbas * nbas);
      for (int j = 0; j < nbas; ++j)
        for (int i = 0; i <= j; ++i) {
          cd v = Th[i + (size_t)j * ldT];
          if (i == j) v = cd(std::real(v), 0.0);
          Tn[i + (size_t)j * nbas] = v;
          Tn[j + (size_t)i * nbas] = std::conj(v);
        }
      for (const cd& v : Tn)
        if (!std::isfinite(v.real()) || !std::isfinite(v.imag())) return set_err(ctx, OMEN_ENUMERIC, "non-finite projected matrix");
      const double beta = std::real(Th[nbas + (size_t)jstart * ldT]);
      theta.assign(nbas, 0.0);
      Y.assign((size_t)nbas * nbas, cd(0));
      if (hermitian_eig(nbas, Tn.data(), theta.data(), Y.data()))
        return set_err(ctx, OMEN_ENUMERIC, "projected eigenproblem did not converge");
      std::vector<double> resA(nbas);
      for (int i = 0; i < nbas; ++i) resA[i] = std::fabs(beta) * std::abs(Y[jstart + (size_t)i * nbas]);
      const int nev = o->nev;
      bool done = false;
      // explicit check on H for the nev (+1) Ritz vectors of smallest theta: true FP64 residuals
      auto explicit_check = [&](bool& ok) -> omen_status {
        const int kc = std::min(nbas, nev + 1);
        std::vector<cd> Yk((size_t)nbas * kc);
        for (int j = 0; j < kc; ++j)
          for (int i = 0; i < nbas; ++i) Yk[i + (size_t)j * nbas] = Y[i + (size_t)j * nbas];
        omen_status s3 = op.combine(V, nbas, Yk, kc, Xb.p, 1.0, 0.0);
        if (s3 != OMEN_OK) return s3;
        if (!HXb.p && (cudaMalloc(&HXb.p, (size_t)(o->nev + 1) * vbytes) != cudaSuccess ||
                       cudaMalloc(&Rb.p, (size_t)(o->nev + 1) * vbytes) != cudaSuccess)) {
          cudaGetLastError();
          return set_err(ctx, OMEN_ENOMEM, "Ritz check vectors");
        }
        s3 = launch_hx(ctx, op.ham, Xb.p, HXb.p, kc, 0.0, op.prec);
        if (s3 != OMEN_OK) return s3;
        hx += kc;
        std::vector<double> lamk, resk, bd;
        s3 = rayleigh_residuals(op, Xb.p, HXb.p, Rb.p, kc, lamk, resk);
        if (s3 != OMEN_OK) return s3;
        if (op.negate)
          for (double& l : lamk) l = -l;
        std::vector<double> lam(lamk.begin(), lamk.begin() + nev), res(resk.begin(), resk.begin() + nev);
        error_bounds(lamk, lam, res, bd);
        ok = *std::max_element(bd.begin(), bd.end()) <= o->tol;
        return OMEN_OK;
      };
      if (!folded) {
        std::vector<double> lam(theta.begin(), theta.begin() + nev), res(resA.begin(), resA.begin() + nev), bd;
        error_bounds(theta, lam, res, bd);
        done = *std::max_element(bd.begin(), bd.end()) <= o->tol;
        // under partial reorthogonalisation the projected matrix is only as good as the basis's
        // orthogonality, which restarts erode: confirm on H before stopping
        if (done && pro) {
          s = explicit_check(done);
          if (s != OMEN_OK) return s;
        }
        // nothing of the operator below the line (Weyl): no lower eigenvalue left to find
        if (op.has_line && theta[0] - resA[0] > op.stop_line) {
          done = true;
          line_crossed = true;
        }
      } else if (op.has_line && theta[0] - resA[0] > op.stop_line) {
        // folded operator: nothing of it below the line, so no state nearer sigma is missing
        done = true;
        line_crossed = true;
      } else {
        const double rmax = *std::max_element(resA.begin(), resA.begin() + nev);
        if (gateA < 0) gateA = std::max(o->tol, 1e-12) * 1e3;
        if (rmax <= gateA || iter >= max_iter_of(o)) {
          s = explicit_check(done);
          if (s != OMEN_OK) return s;
          if (!done) gateA = std::min(gateA, rmax) * 0.01;
        }
      }
      if (done || iter >= max_iter_of(o)) {
        converged = done && !line_crossed;
        break;
      }
      if (full) {
        const int kk = std::min(m - 1, std::max(o->nev + 1, nbas / 2));
        std::vector<cd> Yk((size_t)nbas * kk);
        for (int j = 0; j < kk; ++j)
          for (int i = 0; i < nbas; ++i) Yk[i + (size_t)j * nbas] = Y[i + (size_t)j * nbas];
        s = op.combine(V, nbas, Yk, kk, Xb.p, 1.0, 0.0);
        if (s != OMEN_OK) return s;
        OMEN_CUDA(ctx, cudaMemcpyAsync(V, Xb.p, (size_t)kk * vbytes, cudaMemcpyDeviceToDevice, ctx->stream));
        OMEN_CUDA(ctx, cudaMemcpyAsync(op.col(V, kk), op.col(V, nbas), vbytes, cudaMemcpyDeviceToDevice, ctx->stream));
        std::fill(Th.begin(), Th.end(), cd(0));
        for (int i = 0; i < kk; ++i) Th[i + (size_t)i * ldT] = theta[i];
        for (int i = 0; i < kk; ++i) {
          const cd c = beta * Y[jstart + (size_t)i * nbas];
          Th[kk + (size_t)i * ldT] = c;
          Th[i + (size_t)kk * ldT] = std::conj(c);
        }
        // column kk is accumulated again by the next projection: start it at zero
        for (int i = 0; i <= kk; ++i) Th[i + (size_t)kk * ldT] = cd(0);
        OMEN_CUDA(ctx, cudaMemcpyAsync(dT, Th.data(), sizeof(double2) * ldT * ldT, cudaMemcpyHostToDevice, ctx->stream));
        OMEN_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
        jstart = kk;
        nbas = kk + 1;
        ++restarts;
        fresh = true;
        continue;
      }
    }
    jstart = nbas;
    nbas += 1;
  }
  const int kc = std::min(nbas, k_out);
  std::vector<cd> Yk((size_t)nbas * kc);
  for (int j = 0; j < kc; ++j)
    for (int i = 0; i < nbas; ++i) Yk[i + (size_t)j * nbas] = Y[i + (size_t)j * nbas];
  s = op.combine(V, nbas, Yk, kc, X, 1.0, 0.0);
  if (s != OMEN_OK) return s;
  if (info) {
    info->iterations = iter;
    info->hx_count = hx;
    info->restarts = restarts;
    info->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
  }
  return OMEN_OK;
}

// Sort the k columns of X (and HX) by the key and permute lam/res accordingly.
static omen_status sort_columns(KrylovOps& op, void* X, int k, std::vector<double>& key, std::vector<double>* a1,
                                std::vector<double>* a2) {
  std::vector<int> ord(k);
  for (int i = 0; i < k; ++i) ord[i] = i;
  std::stable_sort(ord.begin(), ord.end(), [&](int x, int y) { return key[x] < key[y]; });
  bool ident = true;
  for (int i = 0; i < k; ++i) ident &= ord[i] == i;
  if (ident) return OMEN_OK;
  DevBuf tb;
  if (cudaMalloc(&tb.p, (size_t)k * op.n * op.el) != cudaSuccess) {
    cudaGetLastError();
    return set_err(op.ctx, OMEN_ENOMEM, "sort buffer");
  }
  for (int i = 0; i < k; ++i)
    OMEN_CUDA(op.ctx, cudaMemcpyAsync(op.col(tb.p, i), op.col(X, ord[i]), op.n * op.el, cudaMemcpyDeviceToDevice, op.ctx->stream));
  OMEN_CUDA(op.ctx, cudaMemcpyAsync(X, tb.p, (size_t)k * op.n * op.el, cudaMemcpyDeviceToDevice, op.ctx->stream));
  OMEN_CUDA(op.ctx, cudaStreamSynchronize(op.ctx->stream));
  auto perm = [&](std::vector<double>& v) {
    std::vector<double> t(k);
    for (int i = 0; i < k; ++i) t[i] = v[ord[i]];
    v = t;
  };
  perm(key);
  if (a1) perm(*a1);
  if (a2) perm(*a2);
  return OMEN_OK;
}

// FP64 Rayleigh–Ritz refinement on span{X, H X - X Lambda}: X (k columns, FP64) in/out.
static omen_status refine64(KrylovOps& op, void* X, int k, const omen_eig_opts* o, std::vector<double>& lam,
                            std::vector<double>& res, std::vector<double>& bound, long long& hx) {
  omen_ctx* ctx = op.ctx;
  const size_t vb = (size_t)op.n * op.el;
  DevBuf Sb, HSb, Rb;
  if (cudaMalloc(&Sb.p, 2 * k * vb) != cudaSuccess || cudaMalloc(&HSb.p, 2 * k * vb) != cudaSuccess ||
      cudaMalloc(&Rb.p, (size_t)k * vb) != cudaSuccess) {
    cudaGetLastError();
    return set_err(ctx, OMEN_ENOMEM, "refinement vectors");
  }
  const bool nearest = o->which == OMEN_NEAREST;
  omen_status s;
  for (int it = 0; it < 12; ++it) {
    // S = [X, R], R = H X - X Lambda
    OMEN_CUDA(ctx, cudaMemcpyAsync(Sb.p, X, k * vb, cudaMemcpyDeviceToDevice, ctx->stream));
    std::vector<cd> Rq;
    int def = 0;
    s = op.cholqr(Sb.p, k, Rq, def);
    if (s != OMEN_OK) return s;
    if (def) return set_err(ctx, OMEN_ENUMERIC, "refinement basis lost rank");
    s = launch_hx(ctx, op.ham, Sb.p, HSb.p, k, 0.0, OMEN_F64);
    if (s != OMEN_OK) return s;
    hx += k;
    s = rayleigh_residuals(op, Sb.p, HSb.p, Rb.p, k, lam, res);
    if (s != OMEN_OK) return s;
    error_bounds(lam, lam, res, bound);
    const double bmax = *std::max_element(bound.begin(), bound.end());
    if (it > 0 && bmax <= o->tol) {
      OMEN_CUDA(ctx, cudaMemcpyAsync(X, Sb.p, k * vb, cudaMemcpyDeviceToDevice, ctx->stream));
      return OMEN_OK;
    }
    // append the residuals, orthogonalise them against X and each other
    OMEN_CUDA(ctx, cudaMemcpyAsync(op.col(Sb.p, k), Rb.p, k * vb, cudaMemcpyDeviceToDevice, ctx->stream));
    for (int j0 = 0; j0 < k && s == OMEN_OK; j0 += kMaxBlockCols)
      s = op.orthogonalise(Sb.p, k, op.col(Sb.p, k + j0), std::min(kMaxBlockCols, k - j0), nullptr);
    if (s != OMEN_OK) return s;
    std::vector<cd> R2;
    s = op.cholqr(op.col(Sb.p, k), k, R2, def);
    if (s != OMEN_OK) return s;
    const int ns = def ? k : 2 * k;
    s = launch_hx(ctx, op.ham, Sb.p, HSb.p, ns, 0.0, OMEN_F64);
    if (s != OMEN_OK) return s;
    hx += ns;
    std::vector<cd> G;
    s = op.dots(Sb.p, ns, HSb.p, ns, G);
    if (s != OMEN_OK) return s;
    for (int j = 0; j < ns; ++j)
      for (int i = 0; i < j; ++i) {
        cd a = 0.5 * (G[i + (size_t)j * ns] + std::conj(G[j + (size_t)i * ns]));
        G[i + (size_t)j * ns] = a;
        G[j + (size_t)i * ns] = std::conj(a);
      }
    for (int i = 0; i < ns; ++i) G[i + (size_t)i * ns] = std::real(G[i + (size_t)i * ns]);
    std::vector<double> w(ns);
    std::vector<cd> Z((size_t)ns * ns);
    if (hermitian_eig(ns, G.data(), w.data(), Z.data())) return set_err(ctx, OMEN_ENUMERIC, "refinement eigenproblem");
    // choose k Ritz values: lowest, or nearest sigma
    std::vector<int> ord(ns);
    for (int i = 0; i < ns; ++i) ord[i] = i;
    if (nearest)
      std::stable_sort(ord.begin(), ord.end(), [&](int a, int b2) { return std::fabs(w[a] - o->sigma) < std::fabs(w[b2] - o->sigma); });
    else if (o->which == OMEN_HIGHEST)
      std::stable_sort(ord.begin(), ord.end(), [&](int a, int b2) { return w[a] > w[b2]; });
    std::vector<cd> Zk((size_t)ns * k);
    std::vector<int> pick(ord.begin(), ord.begin() + k);
    std::sort(pick.begin(), pick.end(), [&](int a, int b2) { return w[a] < w[b2]; });
    for (int j = 0; j < k; ++j)
      for (int i = 0; i < ns; ++i) Zk[i + (size_t)j * ns] = Z[i + (size_t)pick[j] * ns];
    s = op.combine(Sb.p, ns, Zk, k, X, 1.0, 0.0);
    if (s != OMEN_OK) return s;
  }
  // final evaluation
  s = launch_hx(ctx, op.ham, X, HSb.p, k, 0.0, OMEN_F64);
  if (s != OMEN_OK) return s;
  hx += k;
  s = rayleigh_residuals(op, X, HSb.p, Rb.p, k, lam, res);
  if (s != OMEN_OK) return s;
  error_bounds(lam, lam, res, bound);
  return OMEN_OK;
}

// out[j] = sum_n c_jn X[n], j < nout, with fixed pseudo-random coefficients c_jn in +-[0.5, 1]:
// a start block that lies (nearly) in the span of the k given vectors, e.g. the eigenvectors
// of the previous self-consistent iteration.
omen_status krylov_start_from(omen_ctx* ctx, const omen_ham* ham, int prec, const void* X, int k, void* out, int nout,
                              unsigned long long seed) {
  KrylovOps op{ctx, ham, prec, (bool)ham->is_complex, ham->nrows};
  omen_status s = op.init();
  if (s != OMEN_OK) return s;
  std::vector<cd> M((size_t)k * nout);
  unsigned long long z = seed;
  for (auto& c : M) {
    z += 0x9E3779B97F4A7C15ull;
    unsigned long long t = z;
    t = (t ^ (t >> 30)) * 0xBF58476D1CE4E5B9ull;
    t = (t ^ (t >> 27)) * 0x94D049BB133111EBull;
    t ^= t >> 31;
    const double u = (double)(t >> 11) * (1.0 / 9007199254740992.0);
    c = cd((u < 0.5 ? -1.0 : 1.0) * (0.5 + std::fabs(u - 0.5)), 0.0);
  }
  s = op.combine(X, k, M, nout, out, 1.0, 0.0);
  op.release();
  return s;
}

extern "C" omen_status omen_eigs(omen_ctx* ctx, const omen_ham* ham, const omen_eig_opts* o, double* evals_host,
                                 void* evecs_dev, omen_eig_info* info) {
  if (!ctx || !ham || !o || !evals_host) return set_err(ctx, OMEN_EINVAL, "null argument");
  const int b = o->block;
  if (o->nev < 1) return set_err(ctx, OMEN_EINVAL, "nev must be >= 1");
  if (b < 1 || b > kMaxBlockCols) return set_err(ctx, OMEN_EINVAL, "block must be 1..%d", kMaxBlockCols);
  if (o->basis % b != 0 || o->basis < o->nev + 2 * b) return set_err(ctx, OMEN_EINVAL, "basis must be a multiple of block and >= nev + 2*block");
  if (o->basis > 2048) return set_err(ctx, OMEN_EINVAL, "basis must be <= 2048");
  if (o->which != OMEN_LOWEST && o->which != OMEN_NEAREST && o->which != OMEN_HIGHEST)
    return set_err(ctx, OMEN_EINVAL, "which must be LOWEST, NEAREST or HIGHEST");
  if (!(o->tol > 0)) return set_err(ctx, OMEN_EINVAL, "tol must be > 0");
  if (o->max_iter < 1 || (long long)o->max_iter * b < o->nev)
    return set_err(ctx, OMEN_EINVAL, "max_iter * block must be >= nev");
  if ((long long)o->basis + b > ham->nrows) return set_err(ctx, OMEN_EINVAL, "basis larger than the problem");
  if (ham->precision == OMEN_F64_DF && b != 1)
    return set_err(ctx, OMEN_EUNSUPPORTED, "double-float Krylov vectors are single-vector (block 1) only");
  OMEN_CUDA(ctx, cudaSetDevice(ctx->device));
  auto t0 = std::chrono::steady_clock::now();
  omen_eig_info local{};
  omen_eig_info* inf = info ? info : &local;
  std::memset(inf, 0, sizeof(*inf));

  const int solve_prec = (ham->precision == OMEN_F64 || ham->precision == OMEN_F64_DF) ? ham->precision : OMEN_F32;
  KrylovOps op{ctx, ham, solve_prec, (bool)ham->is_complex, ham->nrows};
  omen_status s = op.init();
  if (s != OMEN_OK) return s;
  op.negate = (o->which == OMEN_HIGHEST);
  const int kout = std::min<long long>(o->nev + b, o->basis);
  DevBuf Xb;
  if (cudaMalloc(&Xb.p, (size_t)kout * ham->nrows * op.el) != cudaSuccess) {
    cudaGetLastError();
    op.release();
    return set_err(ctx, OMEN_ENOMEM, "Ritz vectors");
  }
  // An FP32 solve that the FP64 refinement polishes runs to a tighter target: the refinement
  // (Rayleigh–Ritz on [X, residuals]) removes the FP32 rounding of the vectors quickly but an
  // unconverged Krylov direction only slowly, so the FP32 phase should end near its own floor.
  omen_eig_opts oin = *o;
  if (ham->precision == OMEN_F32_REFINE64) oin.tol = o->tol * 1e-2;
  RitzResult rr;
  bool conv = false;
  s = (b == 1) ? lanczos_solve_single(op, &oin, Xb.p, kout, inf, conv)
               : lanczos_solve(op, &oin, Xb.p, kout, rr, inf, o->v0_host, conv);
  if (s != OMEN_OK) { op.release(); return s; }
  // evaluate the kout Ritz vectors in the solve precision
  DevBuf HXb, Rb;
  if (cudaMalloc(&HXb.p, (size_t)kout * ham->nrows * op.el) != cudaSuccess ||
      cudaMalloc(&Rb.p, (size_t)kout * ham->nrows * op.el) != cudaSuccess) {
    cudaGetLastError();
    op.release();
    return set_err(ctx, OMEN_ENOMEM, "Ritz evaluation");
  }
  s = launch_hx(ctx, ham, Xb.p, HXb.p, kout, 0.0, solve_prec);
  if (s == OMEN_OK) s = rayleigh_residuals(op, Xb.p, HXb.p, Rb.p, kout, rr.lam, rr.res);
  if (s != OMEN_OK) { op.release(); return s; }
  inf->hx_count += kout;
  // the nev wanted among the kout: lowest, or nearest sigma.  For the folded operator the key is
  // the square root of its Rayleigh quotient, ||(H - sigma) x||^2 = r^2 + (lambda - sigma)^2 (r the
  // H residual, orthogonal to x): an unconverged extra vector that mixes levels on both sides of
  // sigma has lambda near sigma but a large r, and must not displace a converged pair.
  std::vector<double> key(kout);
  for (int i = 0; i < kout; ++i)
    key[i] = (o->which == OMEN_NEAREST) ? std::hypot(rr.lam[i] - o->sigma, rr.res[i])
                                        : (o->which == OMEN_HIGHEST ? -rr.lam[i] : rr.lam[i]);
  s = sort_columns(op, Xb.p, kout, key, &rr.lam, &rr.res);
  if (s != OMEN_OK) { op.release(); return s; }
  error_bounds(rr.lam, rr.lam, rr.res, rr.bound);
  const int nev = o->nev;
  std::vector<double> lam(rr.lam.begin(), rr.lam.begin() + nev), res(rr.res.begin(), rr.res.begin() + nev);
  std::vector<double> bound(rr.bound.begin(), rr.bound.begin() + nev);
  if (b == 1 && (o->which == OMEN_LOWEST || o->which == OMEN_NEAREST) && ctx->lock_check && conv) {
    // A single-vector Krylov space holds one direction of each eigenspace: of a degenerate
    // level it finds one copy and may report the next eigenvalue in place of the others.  Check
    // with the nev vectors found locked (projected out of every product): the lowest eigenvalue
    // of what is left either lies above the nev-th (within tol: done) or is a missed one, which
    // is inserted in order, the last pair dropping out; then check again.
    DevBuf Zb, HZb, RZb, Lk;
    const int kz = 2;
    if (cudaMalloc(&Zb.p, (size_t)kz * ham->nrows * op.el) != cudaSuccess ||
        cudaMalloc(&HZb.p, (size_t)ham->nrows * op.el) != cudaSuccess ||
        cudaMalloc(&RZb.p, (size_t)ham->nrows * op.el) != cudaSuccess ||
        cudaMalloc(&Lk.p, sizeof(double2) * nev) != cudaSuccess) {
      cudaGetLastError();
      op.release();
      return set_err(ctx, OMEN_ENOMEM, "locking check vectors");
    }
    omen_eig_opts o1 = oin;
    o1.nev = 1;
    o1.basis = std::min(o->basis, std::max(16, nev + 8));
    o1.v0_dev = nullptr;
    o1.v0_host = nullptr;
    // distance of a level from the target: its value (lowest) or |lambda - sigma| (nearest); the
    // nev found are in increasing distance here
    const bool near = o->which == OMEN_NEAREST;
    auto dist = [&](double l) { return near ? std::fabs(l - o->sigma) : l; };
    // computed values outside the nev kept (extra Ritz values, levels pushed out, the last
    // check's value): they give the error bounds their gaps
    std::vector<double> outside(rr.lam.begin() + nev, rr.lam.end());
    auto rebound = [&]() {
      std::vector<double> all(lam);
      all.insert(all.end(), outside.begin(), outside.end());
      error_bounds(all, lam, res, bound);
    };
    for (int round = 0; round < nev; ++round) {
      op.lock_X = Xb.p;
      op.nlock = nev;
      op.d_lock = static_cast<double2*>(Lk.p);
      op.has_line = true;
      const double dmax = dist(lam[nev - 1]);
      // the line in the operator's own values: H (lowest) or (H - sigma)^2 (nearest)
      op.stop_line = near ? std::pow(std::max(dmax - o->tol, 0.0), 2) : dmax - o->tol;
      op.lock_seed = (unsigned long long)round;   // the previous start has no component left in a level partly found
      omen_eig_info i1{};
      bool c1 = false;
      s = lanczos_solve_single(op, &o1, Zb.p, 1, &i1, c1);
      op.nlock = 0;
      op.has_line = false;
      if (s != OMEN_OK) { op.release(); return s; }
      inf->iterations += i1.iterations;
      inf->hx_count += i1.hx_count + 1;
      std::vector<double> lz, rz;
      s = launch_hx(ctx, ham, Zb.p, HZb.p, 1, 0.0, solve_prec);
      if (s == OMEN_OK) s = rayleigh_residuals(op, Zb.p, HZb.p, RZb.p, 1, lz, rz);
      if (s != OMEN_OK) { op.release(); return s; }
      if (!(c1 && dist(lz[0]) < dist(lam[nev - 1]) - o->tol)) {
        outside.push_back(lz[0]);
        rebound();
        break;
      }
      outside.push_back(lam[nev - 1]);
      int j = nev - 1;
      while (j > 0 && dist(lam[j - 1]) > dist(lz[0])) {
        lam[j] = lam[j - 1];
        res[j] = res[j - 1];
        OMEN_CUDA(ctx, cudaMemcpyAsync(op.col(Xb.p, j), op.col(Xb.p, j - 1), (size_t)ham->nrows * op.el,
                                       cudaMemcpyDeviceToDevice, ctx->stream));
        --j;
      }
      lam[j] = lz[0];
      res[j] = rz[0];
      OMEN_CUDA(ctx, cudaMemcpyAsync(op.col(Xb.p, j), Zb.p, (size_t)ham->nrows * op.el, cudaMemcpyDeviceToDevice,
                                     ctx->stream));
      rebound();
    }
  }
  inf->max_residual_raw = *std::max_element(res.begin(), res.end());
  void* Xfinal = Xb.p;
  DevBuf X64;
  if (ham->precision == OMEN_F32_REFINE64) {
    KrylovOps op64{ctx, ham, OMEN_F64, (bool)ham->is_complex, ham->nrows};
    s = op64.init();
    if (s != OMEN_OK) { op.release(); return s; }
    if (cudaMalloc(&X64.p, (size_t)nev * ham->nrows * op64.el) != cudaSuccess) {
      cudaGetLastError();
      op.release();
      op64.release();
      return set_err(ctx, OMEN_ENOMEM, "refinement vectors");
    }
    const long long tot = (long long)nev * ham->nrows;
    const unsigned grid = (unsigned)std::min<long long>((tot + 255) / 256, 152 * 8);
    if (ham->is_complex) convert_kernel<float, double, true><<<grid, 256, 0, ctx->stream>>>(Xb.p, X64.p, tot);
    else convert_kernel<float, double, false><<<grid, 256, 0, ctx->stream>>>(Xb.p, X64.p, tot);
    long long hx = 0;
    s = refine64(op64, X64.p, nev, o, lam, res, bound, hx);
    inf->hx_count += hx;
    if (s == OMEN_OK) {
      std::vector<double> key2 = lam;
      s = sort_columns(op64, X64.p, nev, key2, &res, &bound);
      lam = key2;
    }
    op64.release();
    if (s != OMEN_OK) { op.release(); return s; }
    Xfinal = X64.p;
  } else {
    std::vector<double> key2 = lam;
    s = sort_columns(op, Xb.p, nev, key2, &res, &bound);
    lam = key2;
    if (s != OMEN_OK) { op.release(); return s; }
  }
  for (int i = 0; i < nev; ++i) evals_host[i] = lam[i];
  inf->max_residual = *std::max_element(res.begin(), res.end());
  inf->max_error_bound = *std::max_element(bound.begin(), bound.end());
  inf->converged = conv && inf->max_error_bound <= o->tol;
  if (evecs_dev && solve_prec == OMEN_F64_DF) {
    // double-float Krylov vectors: the eigenvectors are returned in FP64
    s = omen_convert_vectors(ctx, Xfinal, OMEN_F64_DF, evecs_dev, OMEN_F64, (long long)nev * ham->nrows);
  } else if (evecs_dev) {
    const size_t eb = (ham->precision == OMEN_F32_REFINE64) ? vec_elem_bytes(ham, OMEN_F64) : op.el;
    s = OMEN_OK;
    cudaError_t e = cudaMemcpyAsync(evecs_dev, Xfinal, (size_t)nev * ham->nrows * eb, cudaMemcpyDeviceToDevice, ctx->stream);
    if (e != cudaSuccess) s = set_err(ctx, OMEN_ECUDA, "copy of eigenvectors: %s", cudaGetErrorString(e));
  }
  cudaError_t e2 = cudaStreamSynchronize(ctx->stream);
  op.release();
  if (s != OMEN_OK) return s;
  if (e2 != cudaSuccess) return set_err(ctx, OMEN_ECUDA, "eigensolve: %s", cudaGetErrorString(e2));
  inf->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  if (!inf->converged) return set_err(ctx, OMEN_ENOCONV, "not converged: error bound %.3e > tol %.3e after %d block steps",
                                      inf->max_error_bound, o->tol, inf->iterations);
  return OMEN_OK;
}

// ---------------------------------------------------------------------------------------
// k-batched eigen-solve (paper Section II-C: k-space grouping; here all k of one structure in
// lockstep on one GPU).  nk independent single-vector thick-restart Lanczos recurrences, one per
// Bloch wave vector, advance together: every step is one k-batched H·X launch (bond blocks
// shared by all k) plus batched projection / update / normalisation launches.  Vectors are laid
// out [basis vector][k][row], so the current Lanczos vectors of all k are contiguous.
// Convergence (checked per k on the host): LOWEST - the Weyl / Kato–Temple bound on the Ritz
// values; NEAREST - the H residual estimated from the folded residual, r_A / (2 sqrt(theta)).
// ---- k-batched lockstep Lanczos over several structures ------------------------------------
// Every (structure, wave vector) pair is an independent problem p with its own basis, T matrix
// and convergence test; all of them advance one step per iteration, their H·X in one launch
// over the (structure, k) work list and their projections, updates and normalisations in one
// launch each (blockIdx over problems).  A vector slot holds every problem's vector: problem p
// at element off[p], len[p] = its structure's row count, structures in the given order and
// their wave vectors in order within each.
struct KbatchInput {
  const omen_ham* ham;
  int nk;
  const double* k_host;
};

namespace {
struct PhaseTables {
  omen_ctx* ctx;
  std::vector<double2*> p;
  ~PhaseTables() {
    for (double2* q : p)
      if (q) cudaFreeAsync(q, ctx->stream);
  }
};
struct OpsGuard {
  KrylovOps& op;
  ~OpsGuard() { op.release(); }
};
}  // namespace

// Deflation and stopping rule of one lockstep run: Lanczos on the operator with the nlock
// vectors of X (slots, the batch layout) projected out after every product; a problem also
// counts as done once its lowest Ritz value minus its residual exceeds stop_above[p] (no
// eigenvalue of the deflated operator lies below that line).
struct KLock {
  const void* X = nullptr;
  int n = 0;
  const std::vector<double>* stop_above = nullptr;
  const std::vector<char>* only = nullptr;   // run just these problems (the others count as done)
  unsigned long long seed = 0x5EEDull;
};
// Results of one run: the nev Ritz vectors of every problem in ascending order (slots of Xout),
// their Rayleigh quotients and residual norms [p][nev], and per-problem convergence.
struct KOut {
  void* Xout = nullptr;
  std::vector<double> lam, res;
  std::vector<char> conv;
  int iterations = 0, restarts = 0;
  long long hx = 0;
};

static omen_status kbatch_core(omen_ctx* ctx, const std::vector<KbatchInput>& in, const omen_eig_opts* o, int nev,
                               const KLock& lock, KOut& out) {
  if (!ctx) return OMEN_EINVAL;
  if (!o || in.empty() || (int)in.size() > 16) return set_err(ctx, OMEN_EINVAL, "null argument or 1..16 structures");
  const omen_ham* h0 = in[0].ham;
  for (size_t i = 0; i < in.size(); ++i) {
    const omen_ham* h = in[i].ham;
    if (!h || !in[i].k_host || in[i].nk < 1) return set_err(ctx, OMEN_EINVAL, "structure %zu: null argument or nk < 1", i);
    if (h->effmass) return set_err(ctx, OMEN_EUNSUPPORTED, "k batch runs on tight-binding Hamiltonians");
    if (!h->bloch || h->spin_orbit || h->matrix_free)
      return set_err(ctx, OMEN_EINVAL, "k batch needs Bloch Hamiltonians with stored blocks and no spin-orbit");
    if (h->precision == OMEN_F32_REFINE64) return set_err(ctx, OMEN_EUNSUPPORTED, "k batch runs in F64 or F32");
    if (h->precision != h0->precision || h->norb != h0->norb)
      return set_err(ctx, OMEN_EINVAL, "structures of one k batch share precision and basis");
    if ((long long)o->basis + 1 > h->nrows) return set_err(ctx, OMEN_EINVAL, "basis larger than structure %zu", i);
  }
  if (o->block != 1) return set_err(ctx, OMEN_EINVAL, "k batch uses block size 1");
  if (o->which != OMEN_LOWEST && o->which != OMEN_NEAREST) return set_err(ctx, OMEN_EINVAL, "which must be LOWEST or NEAREST");
  if (nev < 1 || o->basis < nev + 2 || o->basis > 2048 || !(o->tol > 0) || o->max_iter < nev)
    return set_err(ctx, OMEN_EINVAL, "invalid eigen options");
  OMEN_CUDA(ctx, cudaSetDevice(ctx->device));
  const int m = o->basis, ldT = m + 1;
  const bool folded = o->which == OMEN_NEAREST;
  const int prec = h0->precision == OMEN_F32 ? OMEN_F32 : OMEN_F64;
  // problems
  std::vector<long long> off, len;
  std::vector<KItem> items(in.size());
  long long Ntot = 0, nmax = 0;
  for (size_t i = 0; i < in.size(); ++i) {
    items[i] = KItem{in[i].ham, in[i].nk, nullptr, Ntot};
    for (int q = 0; q < in[i].nk; ++q) {
      off.push_back(Ntot);
      len.push_back(in[i].ham->nrows);
      Ntot += in[i].ham->nrows;
    }
    nmax = std::max(nmax, in[i].ham->nrows);
  }
  const int P = (int)off.size();
  KrylovOps op{ctx, h0, prec, true, Ntot};
  omen_status s = op.init();
  if (s != OMEN_OK) return s;
  OpsGuard og{op};
  PhaseTables pt{ctx, std::vector<double2*>(in.size(), nullptr)};
  for (size_t i = 0; i < in.size(); ++i) {
    s = make_phases(ctx, in[i].ham, in[i].nk, in[i].k_host, &pt.p[i]);
    if (s != OMEN_OK) return s;
    items[i].phases = pt.p[i];
  }
  const size_t blk = (size_t)Ntot * op.el;   // one slot: every problem's vector
  DevBuf Vb, Wb, Tb, Xb, Xf, Td, Hd, Ob, Lk;
  if (cudaMalloc(&Vb.p, (size_t)(m + 1) * blk) != cudaSuccess || cudaMalloc(&Wb.p, blk) != cudaSuccess ||
      cudaMalloc(&Tb.p, blk) != cudaSuccess || cudaMalloc(&Xb.p, (size_t)m * blk) != cudaSuccess ||
      cudaMalloc(&Xf.p, (size_t)nev * blk) != cudaSuccess ||
      cudaMalloc(&Td.p, sizeof(double2) * ldT * ldT * P) != cudaSuccess ||
      cudaMalloc(&Hd.p, sizeof(double2) * (ldT + 1) * P) != cudaSuccess ||
      cudaMalloc(&Ob.p, sizeof(long long) * 3 * P) != cudaSuccess ||
      cudaMalloc(&Lk.p, sizeof(double2) * (size_t)P * std::max(1, lock.n)) != cudaSuccess) {
    cudaGetLastError();
    return set_err(ctx, OMEN_ENOMEM, "k-batched Lanczos basis (%d slots of %lld elements)", m + 1, Ntot);
  }
  long long* d_off = static_cast<long long*>(Ob.p);
  OMEN_CUDA(ctx, cudaMemcpyAsync(d_off, off.data(), sizeof(long long) * P, cudaMemcpyHostToDevice, ctx->stream));
  OMEN_CUDA(ctx, cudaMemcpyAsync(d_off + P, len.data(), sizeof(long long) * P, cudaMemcpyHostToDevice, ctx->stream));
  int* d_act = reinterpret_cast<int*>(d_off + 2 * P);
  double2* d_lk = static_cast<double2*>(Lk.p);   // projections onto the locked vectors
  std::vector<int> act(P, 1);
  if (lock.only)
    for (int p = 0; p < P; ++p) act[p] = (*lock.only)[p] ? 1 : 0;
  OMEN_CUDA(ctx, cudaMemcpyAsync(d_act, act.data(), sizeof(int) * P, cudaMemcpyHostToDevice, ctx->stream));
  op.b_off = d_off;
  op.b_len = d_off + P;
  op.b_act = d_act;
  op.b_nmax = nmax;
  // problem -> structure, and the structures that still have an unconverged problem
  std::vector<int> owner;
  for (size_t i = 0; i < in.size(); ++i)
    for (int q = 0; q < in[i].nk; ++q) owner.push_back((int)i);
  std::vector<KItem> live;
  for (size_t i = 0; i < items.size(); ++i) {
    bool any = false;
    for (int p = 0; p < P; ++p) any = any || (owner[p] == (int)i && act[p]);
    if (any) live.push_back(items[i]);
  }
  char* V = static_cast<char*>(Vb.p);
  auto slot = [&](int j) { return V + (size_t)j * blk; };
  double2* dT = static_cast<double2*>(Td.p);
  double2* dh = static_cast<double2*>(Hd.p);
  double2* dn = dh + (size_t)ldT * P;
  const long long tps = (long long)ldT * ldT;
  const long long lda = Ntot;   // stride between basis slots
  OMEN_CUDA(ctx, cudaMemsetAsync(dT, 0, sizeof(double2) * tps * P, ctx->stream));
  OMEN_CUDA(ctx, cudaMemsetAsync(ctx->d_status + 1, 0, sizeof(int), ctx->stream));
  long long hx = 0;
  const int nitems = (int)items.size();
  int nactive = 0;
  for (int p = 0; p < P; ++p) nactive += act[p];
  // y -= X_lock (X_lock^H y) for every problem
  auto deflate = [&](void* Y) -> omen_status {
    if (lock.n == 0) return OMEN_OK;
    omen_status s2 = op.dots_dev_batch(P, lock.X, lda, lock.n, Y, d_lk, lock.n, nullptr, 0, 0, 0);
    if (s2 == OMEN_OK) s2 = op.combine_dev_batch(P, lock.X, lda, lock.n, d_lk, lock.n, Y, -1.0, 1.0);
    return s2;
  };
  auto apply = [&](const void* X, void* Y) -> omen_status {
    const int nl = (int)live.size();
    omen_status s2;
    if (!folded) {
      hx += nactive;
      s2 = launch_hx_kmulti(ctx, live.data(), nl, X, Y, 0.0, prec);
      return s2 == OMEN_OK ? deflate(Y) : s2;
    }
    s2 = launch_hx_kmulti(ctx, live.data(), nl, X, Tb.p, o->sigma, prec);
    if (s2 == OMEN_OK) s2 = deflate(Tb.p);
    if (s2 != OMEN_OK) return s2;
    hx += 2 * nactive;
    s2 = launch_hx_kmulti(ctx, live.data(), nl, Tb.p, Y, o->sigma, prec);
    return s2 == OMEN_OK ? deflate(Y) : s2;
  };
  if (o->v0_dev && lock.n == 0) OMEN_CUDA(ctx, cudaMemcpyAsync(Wb.p, o->v0_dev, blk, cudaMemcpyDeviceToDevice, ctx->stream));
  else if ((s = op.random_fill(Wb.p, 1, lock.seed)) != OMEN_OK) return s;
  for (int pass = 0; pass < 2 && s == OMEN_OK; ++pass) s = deflate(Wb.p);
  if (s == OMEN_OK) s = op.dots_dev_batch(P, Wb.p, lda, 1, Wb.p, dn, 1, nullptr, 0, 0, 0);
  if (s == OMEN_OK) s = op.normalize_dev_batch(P, Wb.p, slot(0), dn, nullptr, 0, 0, 0, 0);
  if (s != OMEN_OK) return s;

  // problem p's basis vectors i0.. combined by its coefficients M (nbas x nbj) into slots j0.. of Out
  auto combine_problem = [&](int p, int nbas, const std::vector<cd>& M, int nbj, char* Out, int j0) -> omen_status {
    OMEN_CUDA(ctx, cudaMemcpyAsync(op.d_small, M.data(), M.size() * sizeof(double2), cudaMemcpyHostToDevice, ctx->stream));
    const size_t shm = M.size() * sizeof(double2);
    const long long n = len[p];
    const unsigned grid = (unsigned)std::min<long long>((n + 255) / 256, (long long)op.sm_count * 8);
    char* Yout = Out + (size_t)j0 * blk + (size_t)off[p] * op.el;
    const char* Ain = V + (size_t)off[p] * op.el;
    if (prec == OMEN_F64) {
      smem_limit(combine_kernel<double, true>, shm);
      combine_kernel<double, true><<<grid, 256, shm, ctx->stream>>>(Ain, lda, nbas, op.d_small, nbj, Yout, lda, n, 1.0, 0.0);
    } else {
      smem_limit(combine_kernel<float, true>, shm);
      combine_kernel<float, true><<<grid, 256, shm, ctx->stream>>>(Ain, lda, nbas, op.d_small, nbj, Yout, lda, n, 1.0, 0.0);
    }
    OMEN_CHECK_LAUNCH(ctx);
    // the small buffer is reused by the next call
    OMEN_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return OMEN_OK;
  };

  std::vector<cd> Th((size_t)tps * P);
  std::vector<std::vector<double>> theta(P);
  std::vector<std::vector<cd>> Y(P);
  std::vector<char> conv(P, 0), frozen(P, 0);
  for (int p = 0; p < P; ++p)
    if (!act[p]) conv[p] = frozen[p] = 1;
  // a converged problem is frozen: its nev Ritz vectors go to Xf and it drops out of every
  // later launch (its structure's H·X too, once all of that structure's problems are frozen)
  auto freeze = [&](int p, int nb) -> omen_status {
    for (int j0 = 0; j0 < nev; j0 += kMaxBlockCols) {
      const int nbj = std::min(kMaxBlockCols, nev - j0);
      std::vector<cd> M((size_t)nb * nbj);
      for (int j = 0; j < nbj; ++j)
        for (int i = 0; i < nb; ++i) M[i + (size_t)j * nb] = Y[p][i + (size_t)(j0 + j) * nb];
      omen_status s2 = combine_problem(p, nb, M, nbj, static_cast<char*>(Xf.p), j0);
      if (s2 != OMEN_OK) return s2;
    }
    frozen[p] = 1;
    act[p] = 0;
    return OMEN_OK;
  };
  int jstart = 0, nbas = 1, iter = 0, restarts = 0, since = 0;
  const int check_every = std::max(8, m / 2);
  bool fresh = true;   // first step of a cycle: the new vector couples to every kept vector
  while (true) {
    s = apply(slot(jstart), Wb.p);
    if (fresh) {
      // two full classical Gram–Schmidt passes
      for (int pass = 0; pass < 2 && s == OMEN_OK; ++pass) {
        s = op.dots_dev_batch(P, V, lda, nbas, Wb.p, dh, ldT, dT, ldT, tps, jstart);
        if (s == OMEN_OK) s = op.combine_dev_batch(P, V, lda, nbas, dh, ldT, Wb.p, -1.0, 1.0);
      }
      fresh = false;
    } else if (s == OMEN_OK) {
      // three-term step (alpha against v_j, beta against v_{j-1} from T), then one full pass
      s = op.dots_dev_batch(P, slot(jstart), lda, 1, Wb.p, dh, ldT, dT + jstart, ldT, tps, jstart);
      if (s == OMEN_OK) s = op.combine_dev_batch(P, slot(jstart), lda, 1, dh, ldT, Wb.p, -1.0, 1.0);
      if (s == OMEN_OK)
        s = op.combine_dev_batch(P, slot(jstart - 1), lda, 1, dT + jstart + (size_t)(jstart - 1) * ldT, tps, Wb.p, -1.0, 1.0);
      if (s == OMEN_OK)
        OMEN_CUDA(ctx, cudaMemcpy2DAsync(dT + (jstart - 1) + (size_t)jstart * ldT, tps * sizeof(double2),
                                         dT + jstart + (size_t)(jstart - 1) * ldT, tps * sizeof(double2), sizeof(double2), P,
                                         cudaMemcpyDeviceToDevice, ctx->stream));
      if (s == OMEN_OK) s = op.dots_dev_batch(P, V, lda, nbas, Wb.p, dh, ldT, dT, ldT, tps, jstart);
      if (s == OMEN_OK) s = op.combine_dev_batch(P, V, lda, nbas, dh, ldT, Wb.p, -1.0, 1.0);
    }
    if (s == OMEN_OK) s = op.dots_dev_batch(P, Wb.p, lda, 1, Wb.p, dn, 1, nullptr, 0, 0, 0);
    if (s == OMEN_OK) s = op.normalize_dev_batch(P, Wb.p, slot(nbas), dn, dT, ldT, tps, nbas, jstart);
    if (s != OMEN_OK) return s;
    ++iter;
    ++since;
    const bool full = nbas + 1 > m;
    if (!(full || iter >= o->max_iter || (since >= check_every && nbas >= nev + 1)) || nbas < nev) {
      jstart = nbas;
      nbas += 1;
      continue;
    }
    since = 0;
    OMEN_CUDA(ctx, cudaMemcpyAsync(Th.data(), dT, sizeof(double2) * tps * P, cudaMemcpyDeviceToHost, ctx->stream));
    int flag = 0;
    OMEN_CUDA(ctx, cudaMemcpyAsync(&flag, ctx->d_status + 1, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    OMEN_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    if (flag) return set_err(ctx, OMEN_ENUMERIC, "Lanczos breakdown or non-finite value in the k batch");
    std::vector<double> betas(P);
    std::vector<int> bad(P, 0);
    // the P projected eigenproblems are independent: one host thread each
#pragma omp parallel for schedule(dynamic)
    for (int p = 0; p < P; ++p) {
      if (frozen[p]) continue;
      const cd* T = Th.data() + (size_t)p * tps;
      std::vector<cd> Tn((size_t)nbas * nbas);
      for (int j = 0; j < nbas; ++j)
        for (int i = 0; i <= j; ++i) {
          cd v = T[i + (size_t)j * ldT];
          if (i == j) v = cd(std::real(v), 0.0);
          Tn[i + (size_t)j * nbas] = v;
          Tn[j + (size_t)i * nbas] = std::conj(v);
        }
      betas[p] = std::real(T[nbas + (size_t)jstart * ldT]);
      theta[p].assign(nbas, 0.0);
      Y[p].assign((size_t)nbas * nbas, cd(0));
      if (hermitian_eig(nbas, Tn.data(), theta[p].data(), Y[p].data())) { bad[p] = 1; continue; }
      std::vector<double> lam(nev), res(nev), bd;
      for (int i = 0; i < nev; ++i) {
        const double rA = std::fabs(betas[p]) * std::abs(Y[p][jstart + (size_t)i * nbas]);
        lam[i] = theta[p][i];
        res[i] = folded ? rA / (2.0 * std::sqrt(std::max(theta[p][i], 0.0)) + 1e-300) : rA;
      }
      if (folded) {
        bd = res;
      } else {
        error_bounds(theta[p], lam, res, bd);
      }
      conv[p] = *std::max_element(bd.begin(), bd.end()) <= o->tol;
      // nothing of the deflated operator below the line: done (Weyl: an eigenvalue lies
      // within the residual of the lowest Ritz value, and Lanczos finds the lowest first)
      if (lock.stop_above) {
        // the line is in the operator's own values: H, or (H - sigma)^2 for the folded solve
        const double r0 = folded ? std::fabs(betas[p]) * std::abs(Y[p][jstart]) : res[0];
        if (theta[p][0] - r0 > (*lock.stop_above)[p]) conv[p] = 1;
      }
    }
    bool all = true;
    for (int p = 0; p < P; ++p) {
      if (bad[p]) return set_err(ctx, OMEN_ENUMERIC, "projected eigenproblem of problem %d did not converge", p);
      if (!frozen[p] && (conv[p] || iter >= o->max_iter) && (s = freeze(p, nbas)) != OMEN_OK) return s;
      all = all && conv[p];
    }
    if (all || iter >= o->max_iter) break;
    // drop frozen problems (and structures with nothing left) from the launches
    nactive = 0;
    live.clear();
    for (int p = 0; p < P; ++p) nactive += act[p];
    for (int i = 0; i < nitems; ++i) {
      bool any = false;
      for (int p = 0; p < P; ++p) any = any || (owner[p] == i && act[p]);
      if (any) live.push_back(items[i]);
    }
    OMEN_CUDA(ctx, cudaMemcpyAsync(d_act, act.data(), sizeof(int) * P, cudaMemcpyHostToDevice, ctx->stream));
    if (full) {
      const int kk = std::min(m - 1, std::max(nev + 1, nbas / 2));
      for (int p = 0; p < P; ++p) {
        if (frozen[p]) continue;
        for (int j0 = 0; j0 < kk; j0 += kMaxBlockCols) {
          const int nbj = std::min(kMaxBlockCols, kk - j0);
          std::vector<cd> M((size_t)nbas * nbj);
          for (int j = 0; j < nbj; ++j)
            for (int i = 0; i < nbas; ++i) M[i + (size_t)j * nbas] = Y[p][i + (size_t)(j0 + j) * nbas];
          if ((s = combine_problem(p, nbas, M, nbj, static_cast<char*>(Xb.p), j0)) != OMEN_OK) return s;
        }
      }
      OMEN_CUDA(ctx, cudaMemcpyAsync(V, Xb.p, (size_t)kk * blk, cudaMemcpyDeviceToDevice, ctx->stream));
      OMEN_CUDA(ctx, cudaMemcpyAsync(slot(kk), slot(nbas), blk, cudaMemcpyDeviceToDevice, ctx->stream));
      std::fill(Th.begin(), Th.end(), cd(0));
      for (int p = 0; p < P; ++p) {
        if (frozen[p]) continue;   // its theta / Y are stale or (never run) empty
        cd* T = Th.data() + (size_t)p * tps;
        for (int i = 0; i < kk; ++i) T[i + (size_t)i * ldT] = theta[p][i];
        for (int i = 0; i < kk; ++i) T[kk + (size_t)i * ldT] = betas[p] * Y[p][jstart + (size_t)i * nbas];
      }
      OMEN_CUDA(ctx, cudaMemcpyAsync(dT, Th.data(), sizeof(double2) * tps * P, cudaMemcpyHostToDevice, ctx->stream));
      OMEN_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
      jstart = kk;
      nbas = kk + 1;
      ++restarts;
      fresh = true;
      continue;
    }
    jstart = nbas;
    nbas += 1;
  }
  // every problem is frozen now: its Ritz vectors are in slots 0..nev-1 of Xf.
  // evaluate all of them: lam = <x,Hx>/<x,x>, r = ||Hx - lam x|| / ||x||
  op.b_act = nullptr;
  std::vector<double> lam((size_t)P * nev), res((size_t)P * nev);
  double2* dq = dh;  // reuse: P values
  std::vector<double2> hq(P), hn(P), hr(P);
  for (int i = 0; i < nev; ++i) {
    char* Xi = static_cast<char*>(Xf.p) + (size_t)i * blk;
    s = launch_hx_kmulti(ctx, items.data(), nitems, Xi, Wb.p, 0.0, prec);
    hx += P;
    if (s == OMEN_OK) s = op.dots_dev_batch(P, Xi, lda, 1, Wb.p, dq, 1, nullptr, 0, 0, 0);
    if (s != OMEN_OK) return s;
    OMEN_CUDA(ctx, cudaMemcpyAsync(hq.data(), dq, sizeof(double2) * P, cudaMemcpyDeviceToHost, ctx->stream));
    if ((s = op.dots_dev_batch(P, Xi, lda, 1, Xi, dq, 1, nullptr, 0, 0, 0)) != OMEN_OK) return s;
    OMEN_CUDA(ctx, cudaMemcpyAsync(hn.data(), dq, sizeof(double2) * P, cudaMemcpyDeviceToHost, ctx->stream));
    OMEN_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    std::vector<double2> mlam(P);
    for (int p = 0; p < P; ++p) {
      lam[(size_t)p * nev + i] = hq[p].x / hn[p].x;
      mlam[p] = make_double2(lam[(size_t)p * nev + i], 0.0);
    }
    OMEN_CUDA(ctx, cudaMemcpyAsync(dq, mlam.data(), sizeof(double2) * P, cudaMemcpyHostToDevice, ctx->stream));
    if ((s = op.combine_dev_batch(P, Xi, lda, 1, dq, 1, Wb.p, -1.0, 1.0)) != OMEN_OK) return s;  // W = HX - lam X
    if ((s = op.dots_dev_batch(P, Wb.p, lda, 1, Wb.p, dq, 1, nullptr, 0, 0, 0)) != OMEN_OK) return s;
    OMEN_CUDA(ctx, cudaMemcpyAsync(hr.data(), dq, sizeof(double2) * P, cudaMemcpyDeviceToHost, ctx->stream));
    OMEN_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    for (int p = 0; p < P; ++p) res[(size_t)p * nev + i] = std::sqrt(std::max(0.0, hr[p].x) / hn[p].x);
  }
  // ascending order per problem: values into out.lam / out.res, vectors into the slots of Xout
  out.lam.assign((size_t)P * nev, 0.0);
  out.res.assign((size_t)P * nev, 0.0);
  for (int p = 0; p < P; ++p) {
    std::vector<int> ord(nev);
    for (int i = 0; i < nev; ++i) ord[i] = i;
    std::sort(ord.begin(), ord.end(), [&](int a, int b) { return lam[(size_t)p * nev + a] < lam[(size_t)p * nev + b]; });
    for (int i = 0; i < nev; ++i) {
      out.lam[(size_t)p * nev + i] = lam[(size_t)p * nev + ord[i]];
      out.res[(size_t)p * nev + i] = res[(size_t)p * nev + ord[i]];
      OMEN_CUDA(ctx, cudaMemcpyAsync(static_cast<char*>(out.Xout) + (size_t)i * blk + (size_t)off[p] * op.el,
                                     static_cast<char*>(Xf.p) + (size_t)ord[i] * blk + (size_t)off[p] * op.el,
                                     (size_t)len[p] * op.el, cudaMemcpyDeviceToDevice, ctx->stream));
    }
  }
  OMEN_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  out.conv = conv;
  out.iterations = iter;
  out.restarts = restarts;
  out.hx = hx;
  return OMEN_OK;
}

// The lockstep solve, then (lowest eigenvalues) a check for eigenvalues it missed.  A
// single-vector Krylov space holds one direction of each eigenspace, so of a degenerate pair —
// common in symmetric supercells, e.g. every band at the zone boundary of a Bloch axis — it finds
// one copy and may report the next eigenvalue in place of the other.  The check runs the
// lockstep solver again for the lowest eigenvalue of each problem's operator with its current
// nev vectors projected out (locking), from a new start vector; where that eigenvalue lies below
// the current nev-th by more than the tolerance, it is inserted in order and the last one
// dropped.  Repeated until no problem changes (at most nev rounds).
static omen_status kbatch_solve(omen_ctx* ctx, const std::vector<KbatchInput>& in, const omen_eig_opts* o,
                                double* evals_host, void* evecs_dev, omen_eig_info* info) {
  if (!ctx) return OMEN_EINVAL;
  if (!o || !evals_host || in.empty()) return set_err(ctx, OMEN_EINVAL, "null argument or no structures");
  auto t0 = std::chrono::steady_clock::now();
  const int nev = o->nev;
  std::vector<long long> off, len;
  long long Ntot = 0;
  for (const KbatchInput& it : in) {
    if (!it.ham || it.nk < 1) return set_err(ctx, OMEN_EINVAL, "null Hamiltonian or nk < 1");
    for (int q = 0; q < it.nk; ++q) {
      off.push_back(Ntot);
      len.push_back(it.ham->nrows);
      Ntot += it.ham->nrows;
    }
  }
  const int P = (int)off.size();
  const size_t el = vec_elem_bytes(in[0].ham, in[0].ham->precision == OMEN_F32 ? OMEN_F32 : OMEN_F64);
  const size_t blk = (size_t)Ntot * el;
  DevBuf X, Z;
  if (cudaMalloc(&X.p, (size_t)std::max(1, nev) * blk) != cudaSuccess || cudaMalloc(&Z.p, blk) != cudaSuccess) {
    cudaGetLastError();
    return set_err(ctx, OMEN_ENOMEM, "k-batch eigenvectors (%d slots of %lld elements)", nev + 1, Ntot);
  }
  KOut main;
  main.Xout = X.p;
  omen_status s = kbatch_core(ctx, in, o, nev, KLock{}, main);
  if (s != OMEN_OK) return s;
  int iters = main.iterations, restarts = main.restarts, rounds = 0, inserted = 0;
  long long hx = main.hx;
  std::vector<char> conv = main.conv;
  if (o->which == OMEN_LOWEST || o->which == OMEN_NEAREST) {
    const double margin = o->tol;
    const bool near = o->which == OMEN_NEAREST;
    auto dist = [&](double l) { return near ? std::fabs(l - o->sigma) : l; };
    // the kept level farthest from the target (the last for the lowest eigenvalues)
    auto farthest = [&](int p) {
      const double* lp = main.lam.data() + (size_t)p * nev;
      int f = nev - 1;
      for (int i = 0; i < nev; ++i)
        if (dist(lp[i]) > dist(lp[f])) f = i;
      return f;
    };
    omen_eig_opts o1 = *o;
    o1.nev = 1;
    o1.v0_dev = nullptr;
    o1.basis = std::min(o->basis, std::max(16, nev + 8));
    // a problem whose deflated operator had nothing below its line is settled: later rounds
    // run only the problems the previous round changed
    std::vector<char> todo(P, 1);
    for (; rounds < nev; ++rounds) {
      std::vector<double> line(P), dline(P);
      for (int p = 0; p < P; ++p) {
        dline[p] = dist(main.lam[(size_t)p * nev + farthest(p)]) - margin;
        line[p] = near ? std::pow(std::max(dline[p], 0.0), 2) : dline[p];
      }
      KLock lk;
      lk.X = X.p;
      lk.n = nev;
      lk.stop_above = &line;
      lk.only = &todo;
      lk.seed = 0x5EEDull + 0x9E3779B97F4A7C15ull * (unsigned long long)(rounds + 1);
      KOut chk;
      chk.Xout = Z.p;
      s = kbatch_core(ctx, in, &o1, 1, lk, chk);
      if (s != OMEN_OK) return s;
      iters += chk.iterations;
      hx += chk.hx;
      bool changed = false;
      for (int p = 0; p < P; ++p) {
        if (!todo[p]) continue;
        todo[p] = 0;
        const double mu = chk.lam[p];
        if (!(dist(mu) < dline[p])) continue;
        if (!chk.conv[p]) { conv[p] = 0; continue; }
        // the farthest kept pair drops out; mu goes in at its place in the ascending list
        double* lp = main.lam.data() + (size_t)p * nev;
        double* rp = main.res.data() + (size_t)p * nev;
        for (int i = farthest(p); i < nev - 1; ++i) {
          lp[i] = lp[i + 1];
          rp[i] = rp[i + 1];
          OMEN_CUDA(ctx, cudaMemcpyAsync(static_cast<char*>(X.p) + (size_t)i * blk + (size_t)off[p] * el,
                                         static_cast<char*>(X.p) + (size_t)(i + 1) * blk + (size_t)off[p] * el,
                                         (size_t)len[p] * el, cudaMemcpyDeviceToDevice, ctx->stream));
        }
        int j = nev - 1;
        while (j > 0 && lp[j - 1] > mu) {
          lp[j] = lp[j - 1];
          rp[j] = rp[j - 1];
          OMEN_CUDA(ctx, cudaMemcpyAsync(static_cast<char*>(X.p) + (size_t)j * blk + (size_t)off[p] * el,
                                         static_cast<char*>(X.p) + (size_t)(j - 1) * blk + (size_t)off[p] * el,
                                         (size_t)len[p] * el, cudaMemcpyDeviceToDevice, ctx->stream));
          --j;
        }
        lp[j] = mu;
        rp[j] = chk.res[p];
        OMEN_CUDA(ctx, cudaMemcpyAsync(static_cast<char*>(X.p) + (size_t)j * blk + (size_t)off[p] * el,
                                       static_cast<char*>(Z.p) + (size_t)off[p] * el, (size_t)len[p] * el,
                                       cudaMemcpyDeviceToDevice, ctx->stream));
        changed = true;
        todo[p] = 1;
        ++inserted;
      }
      if (!changed) break;
    }
  }
  double maxres = 0.0, maxbd = 0.0;
  for (int p = 0; p < P; ++p) {
    std::vector<double> lp(main.lam.begin() + (size_t)p * nev, main.lam.begin() + (size_t)(p + 1) * nev);
    std::vector<double> rp(main.res.begin() + (size_t)p * nev, main.res.begin() + (size_t)(p + 1) * nev), bd;
    error_bounds(lp, lp, rp, bd);
    for (int i = 0; i < nev; ++i) {
      evals_host[(size_t)p * nev + i] = lp[i];
      maxres = std::max(maxres, rp[i]);
      maxbd = std::max(maxbd, bd[i]);
    }
    // eigenvectors: problem p's nev vectors of len[p] rows from element nev*off[p]
    if (evecs_dev)
      for (int i = 0; i < nev; ++i)
        OMEN_CUDA(ctx, cudaMemcpyAsync(static_cast<char*>(evecs_dev) + ((size_t)nev * off[p] + (size_t)i * len[p]) * el,
                                       static_cast<char*>(X.p) + (size_t)i * blk + (size_t)off[p] * el,
                                       (size_t)len[p] * el, cudaMemcpyDeviceToDevice, ctx->stream));
  }
  OMEN_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  bool allc = true;
  for (char c : conv) allc = allc && c;
  if (info) {
    std::memset(info, 0, sizeof(*info));
    info->iterations = iters;
    info->hx_count = hx;
    info->restarts = restarts;
    info->converged = allc;
    info->max_residual = maxres;
    info->max_error_bound = maxbd;
    info->max_residual_raw = maxres;
    info->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
  if (!allc)
    return set_err(ctx, OMEN_ENOCONV, "k batch: not every wave vector converged in %d steps (%d check rounds, %d inserted)",
                   iters, rounds, inserted);
  return OMEN_OK;
}



extern "C" omen_status omen_eigs_kbatch(omen_ctx* ctx, const omen_ham* ham, int nk, const double* k_host,
                                        const omen_eig_opts* o, double* evals_host, void* evecs_dev,
                                        omen_eig_info* info) {
  if (!ctx || !ham || !k_host) return set_err(ctx, OMEN_EINVAL, "null argument");
  return kbatch_solve(ctx, {KbatchInput{ham, nk, k_host}}, o, evals_host, evecs_dev, info);
}

extern "C" omen_status omen_eigs_kbatch_multi(omen_ctx* ctx, int nitems, const omen_kbatch_item* items,
                                              const omen_eig_opts* o, double* evals_host, void* evecs_dev,
                                              omen_eig_info* info) {
  if (!ctx || !items || nitems < 1) return set_err(ctx, OMEN_EINVAL, "null argument or no structures");
  std::vector<KbatchInput> in;
  for (int i = 0; i < nitems; ++i) in.push_back(KbatchInput{items[i].ham, items[i].nk, items[i].k_host});
  return kbatch_solve(ctx, in, o, evals_host, evecs_dev, info);
}
