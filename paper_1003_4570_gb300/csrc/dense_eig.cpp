// Host dense Hermitian eigensolver for the projected Lanczos matrix (m <= a few hundred).
//
// Householder reduction to tridiagonal form (Golub & Van Loan, Matrix Computations, 4th ed.,
// Alg. 8.3.1, complex Hermitian variant), a diagonal phase change that makes the
// off-diagonal real, then implicit symmetric QR steps with Wilkinson shifts and deflation
// (GvL Alg. 8.3.2 / 8.3.3), accumulating the Givens rotations.  FP64 throughout.
#include <algorithm>
#include <cmath>
#include <complex>
#include <numeric>
#include <vector>

#include "dense_eig.h"

using cd = std::complex<double>;

// A: n x n Hermitian, column-major (A[i + j*n] = A_ij); only the full matrix is read.
// On return w[0..n) ascending and Z (column-major, columns = eigenvectors).
int hermitian_eig(int n, const cd* A_in, double* w, cd* Z) {
  if (n <= 0) return 0;
  std::vector<cd> A(A_in, A_in + (size_t)n * n);
  auto a = [&](int i, int j) -> cd& { return A[i + (size_t)j * n]; };
  // Q accumulates the Householder reflectors: A = Q T Q^H
  std::vector<cd> Q((size_t)n * n, cd(0));
  for (int i = 0; i < n; ++i) Q[i + (size_t)i * n] = 1.0;
  std::vector<cd> v(n), p(n), q(n);
  for (int k = 0; k + 2 < n; ++k) {
    double xnorm = 0;
    for (int i = k + 1; i < n; ++i) xnorm += std::norm(a(i, k));
    xnorm = std::sqrt(xnorm);
    if (xnorm == 0.0) continue;
    const cd x0 = a(k + 1, k);
    const cd ph = (std::abs(x0) > 0) ? x0 / std::abs(x0) : cd(1);
    const cd alpha = -ph * xnorm;
    std::fill(v.begin(), v.end(), cd(0));
    for (int i = k + 1; i < n; ++i) v[i] = a(i, k);
    v[k + 1] -= alpha;
    double vn = 0;
    for (int i = k + 1; i < n; ++i) vn += std::norm(v[i]);
    if (vn == 0.0) continue;
    // H = I - 2 v v^H / (v^H v);  A <- H A H
    const double tau = 2.0 / vn;
    // p = tau * A v  (A Hermitian, restricted to rows/cols >= k)
    for (int i = k; i < n; ++i) {
      cd s = 0;
      for (int j = k + 1; j < n; ++j) s += a(i, j) * v[j];
      p[i] = tau * s;
    }
    // K = tau/2 * v^H p
    cd K = 0;
    for (int i = k + 1; i < n; ++i) K += std::conj(v[i]) * p[i];
    K *= 0.5 * tau;
    for (int i = k; i < n; ++i) q[i] = p[i] - K * v[i];
    // A <- A - v q^H - q v^H   (v zero at index k)
    for (int j = k; j < n; ++j)
      for (int i = k; i < n; ++i) a(i, j) -= v[i] * std::conj(q[j]) + q[i] * std::conj(v[j]);
    // Q <- Q H
    for (int i = 0; i < n; ++i) {
      cd s = 0;
      for (int j = k + 1; j < n; ++j) s += Q[i + (size_t)j * n] * v[j];
      s *= tau;
      for (int j = k + 1; j < n; ++j) Q[i + (size_t)j * n] -= s * std::conj(v[j]);
    }
  }
  // phases so that the sub-diagonal is real and non-negative: T' = D^H T D
  std::vector<double> d(n), e(n, 0.0);
  std::vector<cd> D(n);
  D[0] = 1.0;
  for (int i = 0; i < n; ++i) d[i] = std::real(a(i, i));
  for (int i = 0; i + 1 < n; ++i) {
    const cd t = a(i + 1, i);
    const double r = std::abs(t);
    e[i] = r;
    D[i + 1] = (r > 0) ? D[i] * (t / r) : D[i];
  }
  for (int j = 0; j < n; ++j)
    for (int i = 0; i < n; ++i) Q[i + (size_t)j * n] *= D[j];
  // implicit symmetric QR steps with a Wilkinson shift (bulge chasing by Givens rotations),
  // deflating converged off-diagonal entries from the bottom; Zr accumulates the rotations.
  std::vector<double> Zr((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) Zr[i + (size_t)i * n] = 1.0;
  const double eps = 2.220446049250313e-16;
  int hi = n - 1, sweeps = 0;
  while (hi > 0) {
    if (std::fabs(e[hi - 1]) <= eps * (std::fabs(d[hi - 1]) + std::fabs(d[hi])) || e[hi - 1] == 0.0) {
      e[hi - 1] = 0.0;
      --hi;
      continue;
    }
    int lo = hi - 1;
    while (lo > 0 && std::fabs(e[lo - 1]) > eps * (std::fabs(d[lo - 1]) + std::fabs(d[lo]))) --lo;
    if (lo > 0) e[lo - 1] = 0.0;
    if (++sweeps > 60 * n) return 1;
    // Wilkinson shift from the trailing 2x2 block of the unreduced segment [lo, hi]
    const double half = 0.5 * (d[hi - 1] - d[hi]);
    const double bb = e[hi - 1];
    const double den = half + (half >= 0 ? 1.0 : -1.0) * std::hypot(half, bb);
    const double mu = (den != 0.0) ? d[hi] - bb * bb / den : d[hi] - std::fabs(bb);
    double x = d[lo] - mu, z = e[lo];
    for (int k = lo; k < hi; ++k) {
      const double r = std::hypot(x, z);
      const double c = (r == 0.0) ? 1.0 : x / r, s = (r == 0.0) ? 0.0 : z / r;
      if (k > lo) e[k - 1] = r;
      const double p = d[k], q = e[k], t = d[k + 1];
      d[k] = c * c * p + 2.0 * c * s * q + s * s * t;
      d[k + 1] = s * s * p - 2.0 * c * s * q + c * c * t;
      e[k] = c * s * (t - p) + (c * c - s * s) * q;
      if (k + 1 < hi) {
        z = s * e[k + 1];        // bulge at (k, k+2)
        e[k + 1] *= c;
        x = e[k];
      }
      double* zk = &Zr[(size_t)k * n];
      double* zk1 = &Zr[(size_t)(k + 1) * n];
      for (int i = 0; i < n; ++i) {
        const double u = zk[i], w1 = zk1[i];
        zk[i] = c * u + s * w1;
        zk1[i] = -s * u + c * w1;
      }
    }
  }
  std::vector<int> order(n);
  std::iota(order.begin(), order.end(), 0);
  std::sort(order.begin(), order.end(), [&](int x, int y) { return d[x] < d[y]; });
  for (int jj = 0; jj < n; ++jj) {
    const int j = order[jj];
    w[jj] = d[j];
    for (int i = 0; i < n; ++i) {
      cd s = 0;
      for (int k = 0; k < n; ++k) s += Q[i + (size_t)k * n] * Zr[k + (size_t)j * n];
      Z[i + (size_t)jj * n] = s;
    }
  }
  return 0;
}

// Cholesky G = R^H R (R upper), column-major b x b.  Returns nonzero if not positive definite.
int cholesky_upper(int b, const cd* G, cd* R) {
  for (int i = 0; i < b * b; ++i) R[i] = 0;
  for (int j = 0; j < b; ++j) {
    cd s = G[j + (size_t)j * b];
    for (int k = 0; k < j; ++k) s -= std::conj(R[k + (size_t)j * b]) * R[k + (size_t)j * b];
    const double djj = std::real(s);
    if (!(djj > 0.0) || !std::isfinite(djj)) return 1;
    const double rjj = std::sqrt(djj);
    R[j + (size_t)j * b] = rjj;
    for (int i = j + 1; i < b; ++i) {
      cd t = G[j + (size_t)i * b];
      for (int k = 0; k < j; ++k) t -= std::conj(R[k + (size_t)j * b]) * R[k + (size_t)i * b];
      R[j + (size_t)i * b] = t / rjj;
    }
  }
  return 0;
}

// Inverse of an upper-triangular b x b matrix (column-major).
void upper_inverse(int b, const cd* R, cd* Ri) {
  for (int i = 0; i < b * b; ++i) Ri[i] = 0;
  for (int j = 0; j < b; ++j) {
    Ri[j + (size_t)j * b] = 1.0 / R[j + (size_t)j * b];
    for (int i = j - 1; i >= 0; --i) {
      cd s = 0;
      for (int k = i + 1; k <= j; ++k) s += R[i + (size_t)k * b] * Ri[k + (size_t)j * b];
      Ri[i + (size_t)j * b] = -s / R[i + (size_t)i * b];
    }
  }
}
