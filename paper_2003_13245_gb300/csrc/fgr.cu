// Hopping-limit (Fermi golden rule) mobility of Eq. 7 for a batch of parameter sets.
//
// For the current of Eq. 3 on the ring, to second order in V, the correlation function is
//   C(t) = 2 V^2 exp{-sum_m 2 g_m^2 [(2 n_m + 1) - n_m e^{i w_m t} - (n_m + 1) e^{-i w_m t}]}
//        = 2 V^2 exp{-sum_m 2 g_m^2 (2 n_m + 1)(1 - cos w_m t)} exp{-i sum_m 2 g_m^2 sin w_m t},
// n_m = 1 / (e^{w_m / kT} - 1): a hop relaxes the modes of both molecules, each carrier has two
// neighbours, and C(t) = Tr[rho j(t) j] carries the opposite time phase to the printed Eq. 7.
// The mobility is Eq. 2 with it, mu = (1 / kT) int_0^{t_max} Re C dt (trapezoid on the grid
// t_i = i dt, i < nt).  One block per parameter set; each thread sums a strided subset of the
// grid in a fixed order and the block adds the partial sums in a fixed tree, so the result is
// the same on every run.
#include <cmath>

#include "../../include/tdmrg.h"
#include "tdmrg_internal.cuh"

namespace tdmrg {

namespace {
constexpr int kFgrThreads = 256;

__global__ void __launch_bounds__(kFgrThreads)
fgr_mobility_kernel(int K, const double* __restrict__ omega, const double* __restrict__ g,
                    const double* __restrict__ V, const double* __restrict__ kT, double dt,
                    int nt, double* __restrict__ mu) {
  __shared__ double a2[64], coth[64], w[64];
  __shared__ double red[kFgrThreads];
  const int p = blockIdx.x;
  const double T = kT[p];
  for (int m = threadIdx.x; m < K; m += blockDim.x) {
    const double om = omega[(long long)p * K + m], gm = g[(long long)p * K + m];
    const double n = 1.0 / expm1(om / T);
    w[m] = om;
    a2[m] = 2.0 * gm * gm;
    coth[m] = 2.0 * n + 1.0;
  }
  __syncthreads();
  double acc = 0.0;
  for (int i = threadIdx.x; i < nt; i += blockDim.x) {
    const double t = i * dt;
    double re = 0.0, ph = 0.0;
    for (int m = 0; m < K; ++m) {
      double s, c;
      sincos(w[m] * t, &s, &c);
      re += a2[m] * coth[m] * (1.0 - c);
      ph += a2[m] * s;
    }
    const double weight = (i == 0 || i == nt - 1) ? 0.5 * dt : dt;
    acc += weight * exp(-re) * cos(ph);
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int s = kFgrThreads / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) mu[p] = 2.0 * V[p] * V[p] * red[0] / T;
}
}  // namespace

cudaError_t fgr_mobility(int P, int K, const double* omega, const double* g, const double* V,
                         const double* kT, double dt, int nt, double* mu, cudaStream_t s) {
  count_launch();
  fgr_mobility_kernel<<<P, kFgrThreads, 0, s>>>(K, omega, g, V, kT, dt, nt, mu);
  return cudaGetLastError();
}

}  // namespace tdmrg
