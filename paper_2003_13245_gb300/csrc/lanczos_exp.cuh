// exp(tau T_k) e_1 for the real symmetric tridiagonal matrix T_k of a Lanczos run, on one
// warp: lane i holds row i (diagonal a, off-diagonals bl on its left and br on its right;
// rows >= k are zero).  Taylor series with scaling (Moler & Van Loan, "Nineteen dubious
// ways to compute the exponential of a matrix", method 1, with the squaring replaced by
// repeated sub-steps): s = ceil(|tau| ||T - sigma||_inf) sub-steps after a shift by the
// Gershgorin centre sigma, each a Taylor sum with a term count fixed by the sub-step's norm.
// Shared by the Lanczos drivers so that all take the same small exponential.
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

constexpr int LZ_MAX_SUBSTEPS = 4096;

// 1/q for the Taylor terms (q <= 60), rounded once by the compiler
#define LZ_R4(q) 1.0 / (q), 1.0 / ((q) + 1), 1.0 / ((q) + 2), 1.0 / ((q) + 3)
static __constant__ double kLzInvQ[64] = {
    0.0, LZ_R4(1.0), LZ_R4(5.0), LZ_R4(9.0), LZ_R4(13.0), LZ_R4(17.0), LZ_R4(21.0),
    LZ_R4(25.0), LZ_R4(29.0), LZ_R4(33.0), LZ_R4(37.0), LZ_R4(41.0), LZ_R4(45.0), LZ_R4(49.0),
    LZ_R4(53.0), LZ_R4(57.0), 1.0 / 61.0, 1.0 / 62.0, 1.0 / 63.0};
#undef LZ_R4

// Product of the tridiagonal rows with a lane-distributed vector: (T u)_lane.
__device__ __forceinline__ double lz_tri(double a, double bl, double br, double u) {
  const int lane = threadIdx.x & 31;
  const double up = __shfl_up_sync(0xffffffffu, u, 1);
  const double dn = __shfl_down_sync(0xffffffffu, u, 1);
  return a * u + (lane >= 1 ? bl * up : 0.0) + (lane < 31 ? br * dn : 0.0);
}

// exp(tau T) e_1 for a T whose rows are given per lane (a: diagonal, bl/br: off-diagonals);
// tnorm = ||T||_inf.  All 32 lanes call it; returns the lane's entry in (yr, yi).
// Sub-steps of norm x = |tau| tnorm / s <= 1; the number of Taylor terms q is fixed in advance
// from x so that the first neglected term x^(q+1)/(q+1)! stays below 1e-18 (no per-term
// reduction across the warp).  T is real, so a real tau keeps the series real, and an
// imaginary tau = i theta needs only real tridiagonal products: in the first sub-step (start
// vector e_1, real) the terms alternate between real and imaginary (one product per term),
// afterwards the real and imaginary parts each take one product.
__device__ __forceinline__ void lz_taylor_exp(double a, double bl, double br, double tnorm,
                                              double tr, double ti, double& yr, double& yi) {
  const int lane = threadIdx.x & 31;
  const double tabs = sqrt(tr * tr + ti * ti);
  // sub-steps bounded: |tau| ||T|| is ~1..100 for a healthy Lanczos run; a non-finite or
  // absurd norm (a state that already overflowed) gets a bounded, meaningless result instead
  // of a loop of billions of sub-steps, and the non-finite norm check reports the state
  const double want = ceil(tabs * tnorm);
  int nsub = (want >= 1.0 && want <= (double)LZ_MAX_SUBSTEPS) ? (int)want
             : (want > (double)LZ_MAX_SUBSTEPS ? LZ_MAX_SUBSTEPS : 1);
  const double x = fmin(tabs * tnorm / nsub, 1.0);
  const int nq = x > 0.5 ? 20 : x > 0.25 ? 16 : x > 0.1 ? 14 : x > 0.01 ? 11 : x > 1e-3 ? 8 : 6;
  const double sr = tr / nsub, si = ti / nsub;
  yr = (lane == 0) ? 1.0 : 0.0;
  yi = 0.0;
  if (ti == 0.0) {
    // real tau: real series
    for (int st = 0; st < nsub; ++st) {
      double t = yr, acc = yr;
      for (int q = 1; q <= nq; ++q) {
        t = (sr * kLzInvQ[q]) * lz_tri(a, bl, br, t);
        acc += t;
      }
      yr = acc;
    }
    return;
  }
  if (tr == 0.0) {
    // imaginary tau = i theta.  First sub-step: term q = (i theta/s)^q T^q e_1 / q!, kept as
    // the real r_q = (theta/s)^q T^q e_1 / q! and added with the phase i^q.
    {
      double r = yr, ar = yr, ai = 0.0;
      for (int q = 1; q <= nq; ++q) {
        r = (si * kLzInvQ[q]) * lz_tri(a, bl, br, r);
        switch (q & 3) {
          case 1: ai += r; break;
          case 2: ar -= r; break;
          case 3: ai -= r; break;
          default: ar += r; break;
        }
      }
      yr = ar;
      yi = ai;
    }
    for (int st = 1; st < nsub; ++st) {
      double ur = yr, ui = yi, ar = yr, ai = yi;
      for (int q = 1; q <= nq; ++q) {
        const double c = si * kLzInvQ[q];
        const double xr = lz_tri(a, bl, br, ur), xi = lz_tri(a, bl, br, ui);
        ur = -c * xi;                 // (i c)(xr + i xi)
        ui = c * xr;
        ar += ur;
        ai += ui;
      }
      yr = ar;
      yi = ai;
    }
    return;
  }
  for (int st = 0; st < nsub; ++st) {
    double tr_ = yr, ti_ = yi, ar = yr, ai = yi;
    for (int q = 1; q <= nq; ++q) {
      const double xr = lz_tri(a, bl, br, tr_), xi = lz_tri(a, bl, br, ti_);
      // term <- (tau / nsub) (T term) / q
      const double cr = sr * kLzInvQ[q], ci = si * kLzInvQ[q];
      tr_ = cr * xr - ci * xi;
      ti_ = cr * xi + ci * xr;
      ar += tr_;
      ai += ti_;
    }
    yr = ar;
    yi = ai;
  }
}

// exp(tau (T_k - sigma)) e_1 for the Lanczos tridiagonal T_k (rows >= k zero), sigma the
// centre of its Gershgorin interval; exp(tau T) = e^(tau sigma) exp(tau (T - sigma)), so the
// number of sub-steps follows the spread of the spectrum rather than its offset (the energy
// of the state, often much larger than the spread).  The factor e^(tau sigma) is applied by
// lz_shift_factor: its modulus e^(Re(tau) sigma) whenever Re(tau) != 0, its phase only where
// the caller needs the vector itself (the phase does not change |y|).
__device__ __forceinline__ double lz_exp_shifted(double a, double bl, double br, int k,
                                                 double tr, double ti, double& yr, double& yi) {
  const int lane = threadIdx.x & 31;
  const bool in = lane < k;
  const double rad = fabs(bl) + fabs(br);
  const double lo = lz_warp_min(in ? a - rad : 1e300);
  const double hi = lz_warp_max(in ? a + rad : -1e300);
  const double sigma = 0.5 * (lo + hi);
  const double as = in ? a - sigma : 0.0;
  const double tnorm = lz_warp_max(fabs(as) + rad);
  lz_taylor_exp(as, bl, br, tnorm, tr, ti, yr, yi);
  return sigma;
}

// y *= e^(Re(tau) sigma) (modulus) and, when `phase`, y *= e^(i Im(tau) sigma)
__device__ __forceinline__ void lz_shift_factor(double sigma, double tr, double ti, bool phase,
                                                double& yr, double& yi) {
  if (tr != 0.0) {
    const double m = exp(tr * sigma);
    yr *= m;
    yi *= m;
  }
  if (phase && ti != 0.0) {
    double sn, cs;
    sincos(ti * sigma, &sn, &cs);
    const double r = yr * cs - yi * sn;
    yi = yr * sn + yi * cs;
    yr = r;
  }
}

}  // namespace tdmrg
