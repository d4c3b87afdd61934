// Host dense linear algebra for the small projected problems of the Krylov solver.
#pragma once
#include <complex>

int hermitian_eig(int n, const std::complex<double>* A, double* w, std::complex<double>* Z);
int cholesky_upper(int b, const std::complex<double>* G, std::complex<double>* R);
void upper_inverse(int b, const std::complex<double>* R, std::complex<double>* Ri);
