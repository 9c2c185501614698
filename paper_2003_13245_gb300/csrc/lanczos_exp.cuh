// exp(tau T_k) e_1 for the real symmetric tridiagonal matrix T_k of a Lanczos run, on one
// warp: lane i holds row i (diagonal a, off-diagonals bl on its left and br on its right;
// rows >= k are zero).  Taylor series with scaling (Moler & Van Loan, "Nineteen dubious
// ways to compute the exponential of a matrix", method 1, with the squaring replaced by
// repeated sub-steps): s = ceil(|tau| ||T||_inf / 0.5) sub-steps, each summed until the
// term falls below 1e-18 of the partial sum.  Shared by the host-driven Lanczos and the
// fused bond exponential so that both take the same small exponential.
#pragma once

#include <cuda_runtime.h>

namespace tdmrg {

__device__ __forceinline__ double lz_warp_max(double v) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// All 32 lanes call it; returns the lane's entry of exp(tau T) e_1 in (yr, yi).
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
    double tr_ = yr, ti_ = yi, ar = yr, ai = yi;
    for (int q = 1; q <= 60; ++q) {
      const double ur = __shfl_up_sync(0xffffffffu, tr_, 1);
      const double ui = __shfl_up_sync(0xffffffffu, ti_, 1);
      const double dr = __shfl_down_sync(0xffffffffu, tr_, 1);
      const double di = __shfl_down_sync(0xffffffffu, ti_, 1);
      const double xr = a * tr_ + (lane >= 1 ? bl * ur : 0.0) + (lane < 31 ? br * dr : 0.0);
      const double xi = a * ti_ + (lane >= 1 ? bl * ui : 0.0) + (lane < 31 ? br * di : 0.0);
      // term <- (tau / nsub) * (T term) / q
      tr_ = (sr * xr - si * xi) / q;
      ti_ = (sr * xi + si * xr) / q;
      ar += tr_;
      ai += ti_;
      const double tm = lz_warp_max(fabs(tr_) + fabs(ti_));
      const double am = lz_warp_max(fabs(ar) + fabs(ai));
      if (tm <= 1e-18 * am) break;
    }
    yr = ar;
    yi = ai;
  }
}

}  // namespace tdmrg
