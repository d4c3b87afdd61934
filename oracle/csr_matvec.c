/*
 * Plain compressed-sparse-row product y = A x (oracle; test infrastructure).
 *
 * The textbook CSR loop: row i sums data[j] * x[indices[j]] for j in indptr[i] .. indptr[i+1]-1,
 * in that order, the same definition scipy's CSR product follows.  Rows are independent, so an
 * OpenMP loop over rows gives the host-core timing of the oracle's product without changing
 * any row's sum.  This is the CPU reference of the paper's repeated operation (the Hamiltonian-
 * vector product inside the Lanczos recurrence, Section II-B, Section III-A item 1); nothing in
 * the library links it.
 */
#include <omp.h>

void oracle_csr_matvec(long long nrows, const int* indptr, const int* indices, const double* data, const double* x,
                       double* y, int nthreads) {
  if (nthreads < 1) nthreads = omp_get_max_threads();
#pragma omp parallel for num_threads(nthreads) schedule(static)
  for (long long i = 0; i < nrows; ++i) {
    double s = 0.0;
    for (int j = indptr[i]; j < indptr[i + 1]; ++j) s += data[j] * x[indices[j]];
    y[i] = s;
  }
}

int oracle_max_threads(void) { return omp_get_max_threads(); }
