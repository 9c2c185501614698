// Building blocks of a Lanczos step run by a cooperative grid (CTA g owns the contiguous slice
// [e0, e0 + len) of every vector): a bounded grid barrier, per-slice dot products against the
// Krylov basis, fixed-order cross-CTA reductions that every CTA evaluates identically, the
// projection, the norm, and the tridiagonal bookkeeping with the small exponential.  Used by
// the fused bond exponential (bond_krylov.cu) and the fused site-Lanczos step
// (lanczos_step.cu).  All sums have a fixed order, so results do not depend on timing.
#pragma once

#include "tdmrg_internal.cuh"
#include "lanczos_exp.cuh"

namespace tdmrg {
namespace lzc {

constexpr int NV = KMAX + 1;                      // partial-dot slots per CTA

__device__ __forceinline__ double wsum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Grid barrier on one monotonic counter: barrier number e is passed once the counter reaches
// e * nblocks (one atomic per CTA; the launcher clears the counter).  Bounded: gives up after
// `limit` clock cycles (kBarrierWaitCycles, ~2 s, unless a test lowers it), sets *status = 1,
// and every CTA then leaves.
__device__ __forceinline__ bool barrier(unsigned* bar, unsigned nblocks, unsigned& epoch,
                                        int* status, long long limit) {
  __syncthreads();
  __shared__ int s_ok;
  ++epoch;
  if (threadIdx.x == 0) {
    volatile unsigned* vbar = bar;
    volatile int* vstat = status;
    const unsigned target = epoch * nblocks;
    __threadfence();
    atomicAdd(bar, 1u);
    int ok = 1;
    const long long t0 = clock64();
    while (*vbar < target) {
      if (*vstat) { ok = 0; break; }
      if (clock64() - t0 > limit) {
        atomicExch(status, 1);
        ok = 0;
        break;
      }
    }
    __threadfence();
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// Warp wv computes the partial dots conj(q_i) . w over the own slice for i = i0 + wv,
// i0 + wv + nwarps, ... < i1 (lanes stride the slice, fixed warp tree) and stores them at
// part[blockIdx.x * NV + i].  V holds the basis (vector i at V + i * n); w points at the own
// slice of w (shared or global memory).
__device__ __forceinline__ void slice_dots(const cplx* V, long long n, const cplx* w,
                                           long long e0, int len, int i0, int i1, cplx* part) {
  const int lane = threadIdx.x & 31, wv = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int i = i0 + wv; i < i1; i += nw) {
    const cplx* q = V + (size_t)i * n + e0;
    double sr = 0.0, si = 0.0;
    for (int e = lane; e < len; e += 32) {
      const cplx a = q[e], b = w[e];
      sr = fma(a.x, b.x, sr);
      sr = fma(a.y, b.y, sr);
      si = fma(a.x, b.y, si);
      si = fma(-a.y, b.x, si);
    }
    sr = wsum(sr);
    si = wsum(si);
    if (lane == 0) part[(size_t)blockIdx.x * NV + i] = make_double2(sr, si);
  }
}

// The same partial dots with every thread of the CTA on every vector (for large slices): the
// vectors are taken four at a time, each thread sums its elements (stride blockDim), then a
// warp tree and the warps in order.  red: 8 * (blockDim / 32) doubles of shared memory.
__device__ __forceinline__ void slice_dots_block(const cplx* V, long long n, const cplx* w,
                                                 long long e0, int len, int i0, int i1,
                                                 cplx* part, double* red) {
  const int lane = threadIdx.x & 31, wv = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int c0 = i0; c0 < i1; c0 += 4) {
    const int nv = min(4, i1 - c0);
    double sr[4] = {0.0, 0.0, 0.0, 0.0}, si[4] = {0.0, 0.0, 0.0, 0.0};
    for (int e = threadIdx.x; e < len; e += blockDim.x) {
      const cplx b = w[e];
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        if (v < nv) {
          const cplx a = V[(size_t)(c0 + v) * n + e0 + e];
          sr[v] = fma(a.x, b.x, sr[v]);
          sr[v] = fma(a.y, b.y, sr[v]);
          si[v] = fma(a.x, b.y, si[v]);
          si[v] = fma(-a.y, b.x, si[v]);
        }
      }
    }
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      if (v < nv) {                 // uniform across the CTA
        sr[v] = wsum(sr[v]);
        si[v] = wsum(si[v]);
        if (lane == 0) {
          red[(wv * 4 + v) * 2] = sr[v];
          red[(wv * 4 + v) * 2 + 1] = si[v];
        }
      }
    }
    __syncthreads();
    if ((int)threadIdx.x < nv) {
      double x = 0.0, y = 0.0;
      for (int u = 0; u < nw; ++u) {
        x += red[(u * 4 + threadIdx.x) * 2];
        y += red[(u * 4 + threadIdx.x) * 2 + 1];
      }
      part[(size_t)blockIdx.x * NV + c0 + threadIdx.x] = make_double2(x, y);
    }
    __syncthreads();
  }
}

// h[i] = sum_g part[g * NV + i] for i in [i0, i1), every CTA in the same order.
__device__ __forceinline__ void reduce_dots(const cplx* part, int G, int i0, int i1, cplx* h) {
  const int lane = threadIdx.x & 31, wv = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int i = i0 + wv; i < i1; i += nw) {
    double sr = 0.0, si = 0.0;
    for (int g = lane; g < G; g += 32) {
      const cplx p = __ldcg(&part[(size_t)g * NV + i]);
      sr += p.x;
      si += p.y;
    }
    sr = wsum(sr);
    si = wsum(si);
    if (lane == 0) h[i] = make_double2(sr, si);
  }
  __syncthreads();
}

// w[e] -= sum_{i in [i0, i1)} h[i] q_i[e] on the own slice
__device__ __forceinline__ void slice_project(const cplx* V, long long n, cplx* w, long long e0,
                                              int len, int i0, int i1, const cplx* h) {
  for (int e = threadIdx.x; e < len; e += blockDim.x) {
    double ax = w[e].x, ay = w[e].y;
    for (int i = i0; i < i1; ++i) {
      const cplx q = V[(size_t)i * n + e0 + e], c = h[i];
      ax = fma(-q.x, c.x, ax);
      ax = fma(q.y, c.y, ax);
      ay = fma(-q.x, c.y, ay);
      ay = fma(-q.y, c.x, ay);
    }
    w[e] = make_double2(ax, ay);
  }
  __syncthreads();
}

// partn[blockIdx.x] = ||w||^2 over the own slice (red: blockDim/32 doubles of shared memory)
__device__ __forceinline__ void slice_norm(const cplx* w, int len, double* red, double* partn) {
  double s = 0.0;
  for (int e = threadIdx.x; e < len; e += blockDim.x)
    s = fma(w[e].x, w[e].x, fma(w[e].y, w[e].y, s));
  s = wsum(s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int v = 0; v < (int)(blockDim.x >> 5); ++v) t += red[v];
    partn[blockIdx.x] = t;
  }
}

// *dst = sum over CTAs of partn (warp 0, fixed order), visible to the CTA on return
__device__ __forceinline__ void reduce_norm(const double* partn, int G, double* dst) {
  if (threadIdx.x < 32) {
    double s = 0.0;
    for (int g = threadIdx.x; g < G; g += 32) s += __ldcg(&partn[g]);
    s = wsum(s);
    if (threadIdx.x == 0) *dst = s;
  }
  __syncthreads();
}

// Lanczos vector j done: alpha_j = Re(h1[j] + h2[j]), beta_{j+1} = sqrt(nrm2).  Warp 0 extends
// the tridiagonal T (alpha[0..j), beta[1..j] read from `alpha`, `beta`; alpha[j], beta[j+1]
// stored there when `store`), evaluates y = exp(tau T) e_1 (lane i returns y_i in yr, yi) and
// decides whether to stop: breakdown, kcap vectors, or beta_{j+1} |y_j| < tol unless the
// dimension is fixed.  Every lane returns the same done / err / breakdown.  Call from the 32
// lanes of one warp.
__device__ __forceinline__ void tridiag_step(int j, double aj, double nrm2, double tr, double ti,
                                             double tol, int kcap, int fixed, double* alpha,
                                             double* beta, bool store, double& yr, double& yi,
                                             bool& done, double& err, bool& breakdown) {
  const int lane = threadIdx.x & 31;
  const int kk = j + 1;
  const double nb = sqrt(nrm2);
  const double a = lane < j ? alpha[lane] : (lane == j ? aj : 0.0);
  const double bl = (lane >= 1 && lane < kk) ? beta[lane] : 0.0;
  const double br = (lane + 1 < kk) ? beta[lane + 1] : 0.0;
  __syncwarp();
  if (store && lane == 0) {
    alpha[j] = aj;
    beta[j + 1] = nb;
  }
  const double scale = lz_warp_max(fmax(fabs(a), fabs(bl)));
  const double sigma = lz_exp_shifted(a, bl, br, kk, tr, ti, yr, yi);
  lz_shift_factor(sigma, tr, ti, false, yr, yi);       // modulus only: enough for the test
  const double ylr = __shfl_sync(0xffffffffu, yr, kk - 1);
  const double yli = __shfl_sync(0xffffffffu, yi, kk - 1);
  err = nb * sqrt(ylr * ylr + yli * yli);
  breakdown = nb <= 1e-12 * fmax(scale, 1e-300);
  done = breakdown || kk >= kcap || (!fixed && err < tol);
  if (done) lz_shift_factor(sigma, 0.0, ti, true, yr, yi);   // the phase, for the result
  __syncwarp();
}

}  // namespace lzc
}  // namespace tdmrg
