// Host-side small exponentials of a Lanczos matrix: exp(z T) e_1 for a real symmetric
// tridiagonal T (k <= 64) at many complex z, from one eigendecomposition of T.  Pure C++, no
// CUDA.  The eigendecomposition is the cyclic Jacobi method: plane rotations chosen to zero one
// off-diagonal entry at a time, swept over all pairs until the off-diagonal part is below
// rounding; the accumulated rotations are the eigenvectors.
#include "small_exp.h"

#include <cmath>
#include <stdexcept>
#include <vector>

namespace tdmrg {

void symmetric_eigen(int k, std::vector<double>& A, std::vector<double>& w,
                     std::vector<double>& Z) {
  Z.assign((size_t)k * k, 0.0);
  for (int i = 0; i < k; ++i) Z[(size_t)i * k + i] = 1.0;
  auto a = [&](int i, int j) -> double& { return A[(size_t)i * k + j]; };
  double scale = 0.0;
  for (double x : A) scale = std::max(scale, std::fabs(x));
  // the off-diagonal part settles at rounding size (about eps times the largest entry)
  for (int sweep = 0; sweep < 60; ++sweep) {
    double off = 0.0;
    for (int p = 0; p < k; ++p)
      for (int q = p + 1; q < k; ++q) off += a(p, q) * a(p, q);
    if (std::sqrt(off) <= 2.3e-16 * std::max(scale, 1e-300)) break;
    for (int p = 0; p < k; ++p)
      for (int q = p + 1; q < k; ++q) {
        const double apq = a(p, q);
        if (apq == 0.0) continue;
        // rotation angle with tan(2 phi) = 2 a_pq / (a_qq - a_pp), the smaller root
        const double theta = (a(q, q) - a(p, p)) / (2.0 * apq);
        const double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
        for (int r = 0; r < k; ++r) {          // columns p, q of A
          const double arp = a(r, p), arq = a(r, q);
          a(r, p) = c * arp - s * arq;
          a(r, q) = s * arp + c * arq;
        }
        for (int r = 0; r < k; ++r) {          // rows p, q of A
          const double apr = a(p, r), aqr = a(q, r);
          a(p, r) = c * apr - s * aqr;
          a(q, r) = s * apr + c * aqr;
        }
        for (int r = 0; r < k; ++r) {          // eigenvectors
          const double zrp = Z[(size_t)r * k + p], zrq = Z[(size_t)r * k + q];
          Z[(size_t)r * k + p] = c * zrp - s * zrq;
          Z[(size_t)r * k + q] = s * zrp + c * zrq;
        }
      }
  }
  w.resize(k);
  for (int i = 0; i < k; ++i) w[i] = a(i, i);
}

void tridiag_exp_e1(int k, const double* alpha, const double* beta, int nz, const Cx* z, Cx* out) {
  if (k < 1 || k > 64 || nz < 0) throw std::invalid_argument("tridiag_exp_e1: need 1 <= k <= 64");
  std::vector<double> A((size_t)k * k, 0.0), w, Z;
  for (int i = 0; i < k; ++i) {
    A[(size_t)i * k + i] = alpha[i];
    if (i + 1 < k) A[(size_t)i * k + i + 1] = A[(size_t)(i + 1) * k + i] = beta[i];
  }
  symmetric_eigen(k, A, w, Z);
  // exp(z T) e_1 = Z diag(exp(z w)) Z^T e_1; the largest exponent is factored out per z so
  // that no term overflows before the sum (the result itself is returned unscaled)
  for (int s = 0; s < nz; ++s) {
    double emax = -INFINITY;
    for (int i = 0; i < k; ++i) emax = std::max(emax, (z[s] * w[i]).real());
    std::vector<Cx> f(k);
    for (int i = 0; i < k; ++i) f[i] = std::exp(z[s] * w[i] - emax) * Z[i];   // Z[0][i]
    const double big = std::exp(emax);
    for (int r = 0; r < k; ++r) {
      Cx acc(0.0, 0.0);
      for (int i = 0; i < k; ++i) acc += Z[(size_t)r * k + i] * f[i];
      out[(size_t)s * k + r] = acc * big;
    }
  }
}

// Gauss-Legendre nodes and weights on [0, 1] (n <= 64): Newton iteration on the three-term
// recurrence of the Legendre polynomials from the usual cosine first guesses.
void gauss_legendre01(int n, std::vector<double>& s, std::vector<double>& w) {
  s.assign(n, 0.0);
  w.assign(n, 0.0);
  const double pi = 3.14159265358979323846;
  for (int i = 0; i < (n + 1) / 2; ++i) {
    double z = std::cos(pi * (i + 0.75) / (n + 0.5)), pp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p1 = 1.0, p2 = 0.0;
      for (int j = 1; j <= n; ++j) {
        const double p3 = p2;
        p2 = p1;
        p1 = ((2.0 * j - 1.0) * z * p2 - (j - 1.0) * p3) / j;
      }
      pp = n * (z * p1 - p2) / (z * z - 1.0);
      const double dz = p1 / pp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    const double wi = 2.0 / ((1.0 - z * z) * pp * pp);
    s[i] = 0.5 * (1.0 - z);            // ascending on [0, 1]
    s[n - 1 - i] = 0.5 * (1.0 + z);
    w[i] = w[n - 1 - i] = 0.5 * wi;
  }
}

int gauss_legendre_nodes_for(double r, int nmax, double eps) {
  const int n0 = nmax < 2 ? nmax : 2;
  if (!(r > 0.0)) return n0;
  const double lr = std::log(r), le = std::log(eps);
  for (int n = n0; n < nmax; ++n) {
    const double lc = 4.0 * std::lgamma(n + 1.0) - std::log(2.0 * n + 1.0) -
                      3.0 * std::lgamma(2.0 * n + 1.0);
    if (lc + 2.0 * n * lr + r <= le) return n;
  }
  return nmax;
}

}  // namespace tdmrg
