// exp(tau T_k) e_1 for the real symmetric tridiagonal matrix T_k of a Lanczos run, on one
// warp: lane i holds row i (diagonal a, off-diagonals bl on its left and br on its right;
// rows >= k are zero).  Taylor series with scaling (Moler & Van Loan, "Nineteen dubious
// ways to compute the exponential of a matrix", method 1, with the squaring replaced by
// repeated sub-steps): s = ceil(|tau| ||T - sigma||_inf / 0.5) sub-steps after a shift by
// the Gershgorin centre sigma, each summed until the term falls below 1e-19 of the
// sub-step's starting maximum.  Shared by the host-driven Lanczos and the fused bond
// exponential so that both take the same small exponential.
#pragma once

#include <cuda_runtime.h>

namespace tdmrg {

__device__ __forceinline__ double lz_warp_max(double v) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ double lz_warp_min(double v) {
  for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// 1/q for the Taylor terms (q <= 60), rounded once by the compiler
#define LZ_R4(q) 1.0 / (q), 1.0 / ((q) + 1), 1.0 / ((q) + 2), 1.0 / ((q) + 3)
static __constant__ double kLzInvQ[64] = {
    0.0, LZ_R4(1.0), LZ_R4(5.0), LZ_R4(9.0), LZ_R4(13.0), LZ_R4(17.0), LZ_R4(21.0),
    LZ_R4(25.0), LZ_R4(29.0), LZ_R4(33.0), LZ_R4(37.0), LZ_R4(41.0), LZ_R4(45.0), LZ_R4(49.0),
    LZ_R4(53.0), LZ_R4(57.0), 1.0 / 61.0, 1.0 / 62.0, 1.0 / 63.0};
#undef LZ_R4

// exp(tau T) e_1 for a T whose rows are given per lane (a: diagonal, bl/br: off-diagonals);
// tnorm = ||T||_inf.  All 32 lanes call it; returns the lane's entry in (yr, yi).
__device__ __forceinline__ void lz_taylor_exp(double a, double bl, double br, double tnorm,
                                              double tr, double ti, double& yr, double& yi) {
  const int lane = threadIdx.x & 31;
  const double tabs = sqrt(tr * tr + ti * ti);
  int nsub = (int)ceil(tabs * tnorm / 0.5);
  if (nsub < 1) nsub = 1;
  const double sr = tr / nsub, si = ti / nsub;
  yr = (lane == 0) ? 1.0 : 0.0;
  yi = 0.0;
  for (int st = 0; st < nsub; ++st) {
    // over one sub-step ||exp(tau T / s)|| >= e^-0.5, so the result keeps at least
    // e^-0.5 / sqrt(32) of the starting maximum: terms are compared against that maximum
    const double am = lz_warp_max(fabs(yr) + fabs(yi));
    double tr_ = yr, ti_ = yi, ar = yr, ai = yi;
    for (int q = 1; q <= 60; ++q) {
      const double ur = __shfl_up_sync(0xffffffffu, tr_, 1);
      const double ui = __shfl_up_sync(0xffffffffu, ti_, 1);
      const double dr = __shfl_down_sync(0xffffffffu, tr_, 1);
      const double di = __shfl_down_sync(0xffffffffu, ti_, 1);
      const double xr = a * tr_ + (lane >= 1 ? bl * ur : 0.0) + (lane < 31 ? br * dr : 0.0);
      const double xi = a * ti_ + (lane >= 1 ? bl * ui : 0.0) + (lane < 31 ? br * di : 0.0);
      // term <- (tau / nsub) (T term) / q
      const double cr = sr * kLzInvQ[q], ci = si * kLzInvQ[q];
      tr_ = cr * xr - ci * xi;
      ti_ = cr * xi + ci * xr;
      ar += tr_;
      ai += ti_;
      const double tm = lz_warp_max(fabs(tr_) + fabs(ti_));
      if (tm <= 1e-19 * am) break;
    }
    yr = ar;
    yi = ai;
  }
}

// exp(tau T_k) e_1 for the Lanczos tridiagonal T_k (rows >= k zero).  T_k is shifted by the
// centre sigma of its Gershgorin interval, exp(tau T) = e^(tau sigma) exp(tau (T - sigma)),
// so that the number of sub-steps follows the spread of the spectrum rather than its offset
// (the energy of the state, often much larger than the spread).
__device__ __forceinline__ void lz_exp_tridiag(double a, double bl, double br, int k, double tr,
                                               double ti, double& yr, double& yi) {
  const int lane = threadIdx.x & 31;
  const bool in = lane < k;
  const double rad = fabs(bl) + fabs(br);
  const double lo = lz_warp_min(in ? a - rad : 1e300);
  const double hi = lz_warp_max(in ? a + rad : -1e300);
  const double sigma = 0.5 * (lo + hi);
  const double as = in ? a - sigma : 0.0;
  const double tnorm = lz_warp_max(fabs(as) + rad);
  double zr, zi;
  lz_taylor_exp(as, bl, br, tnorm, tr, ti, zr, zi);
  const double er = exp(tr * sigma);
  double sn, cs;
  sincos(ti * sigma, &sn, &cs);
  const double fr = er * cs, fi = er * sn;
  yr = zr * fr - zi * fi;
  yi = zr * fi + zi * fr;
}

}  // namespace tdmrg
