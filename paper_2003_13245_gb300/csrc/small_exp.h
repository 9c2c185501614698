// Small exponentials of a Lanczos matrix on the host (small_exp.cpp; no CUDA).
#pragma once
#include <complex>
#include <vector>

namespace tdmrg {

typedef std::complex<double> Cx;

// Eigendecomposition of a dense real symmetric k x k matrix A (row-major, destroyed) by cyclic
// Jacobi rotations: eigenvalues w[k], eigenvectors in the columns of Z (row-major k x k).
void symmetric_eigen(int k, std::vector<double>& A, std::vector<double>& w, std::vector<double>& Z);

// out[s][0..k) = exp(z_s T) e_1 for T = tridiag(beta, alpha, beta) (alpha[k] diagonal,
// beta[k-1] off-diagonal), s < nz.
void tridiag_exp_e1(int k, const double* alpha, const double* beta, int nz, const Cx* z, Cx* out);

// Gauss-Legendre nodes s[n] (ascending) and weights w[n] on [0, 1], n <= 64.
void gauss_legendre01(int n, std::vector<double>& s, std::vector<double>& w);

// Smallest node count n in [min(2, nmax), nmax] for which the n-point Gauss-Legendre error bound
// on [0, 1], (n!)^4 / ((2n + 1) ((2n)!)^3) max|f^(2n)|, is at most eps for an integrand with
// |f^(2n)| <= r^(2n) e^r (the Frechet integrand s -> e^{sA} E e^{(1-s)A} with r = 2 |A|, in
// units of |E|); nmax when no smaller count meets it.
int gauss_legendre_nodes_for(double r, int nmax, double eps);

}  // namespace tdmrg
