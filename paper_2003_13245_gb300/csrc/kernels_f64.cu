// FP64 kernels of the TDVP sweep: strided batched complex GEMM (the contractions of H_eff,
// the environment updates and the bond step), sparse MPO channel mixing, the one-launch
// norm, the start and final combination of a Lanczos run, and the column-wise cooperative
// gauge QR (completion pass and kernel-level entry points).
#include "tdmrg_internal.cuh"

#include <atomic>
#include <cooperative_groups.h>
#include <cmath>

namespace tdmrg {

static std::atomic<long long> g_launches{0};
long long launch_count() { return g_launches.load(); }
void count_launch(int n) { g_launches += n; }

__device__ __forceinline__ cplx cmul(cplx a, cplx b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ cplx cmulc(cplx a, cplx b) {   // conj(a) * b
  return make_double2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ void cfma(cplx& acc, cplx a, cplx b) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(a.y, b.x, acc.y);
}
__device__ __forceinline__ cplx cadd(cplx a, cplx b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ cplx csub(cplx a, cplx b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ cplx cconj_if(cplx a, int c) { return c ? make_double2(a.x, -a.y) : a; }

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_max(double v) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// ------------------------------------------------------------------------------------
// complex GEMM: 64 x 64 output tile, 16-deep k slices, 256 threads, 4 x 4 outputs/thread
// ------------------------------------------------------------------------------------
constexpr int GT = 64;
constexpr int GK = 16;

__global__ void __launch_bounds__(256) zgemm_kernel(int m, int n, int k, int nred, cplx alpha,
                                                    MatRef A, MatRef B, cplx beta, cplx* C,
                                                    long long ldc, long long sc,
                                                    const int* skip) {
  if (skip && *skip) return;
  __shared__ cplx As[GK][GT + 1];
  __shared__ cplx Bs[GK][GT + 1];
  const int t = threadIdx.x;
  const int tx = t & 15, ty = t >> 4;
  const int bm = blockIdx.y * GT, bn = blockIdx.x * GT;
  const long long b = blockIdx.z;
  cplx acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = make_double2(0.0, 0.0);

  const bool a_kcontig = (A.cs == 1);
  const bool b_kcontig = (B.rs == 1);
  for (int r = 0; r < nred; ++r) {
    const cplx* Ap = A.p + b * A.sb + (long long)r * A.sr;
    const cplx* Bp = B.p + b * B.sb + (long long)r * B.sr;
    for (int k0 = 0; k0 < k; k0 += GK) {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        int i, kk;
        if (a_kcontig) { kk = t & 15; i = (t >> 4) + 16 * q; }
        else { i = t & 63; kk = (t >> 6) + 4 * q; }
        const int gi = bm + i, gk = k0 + kk;
        cplx v = make_double2(0.0, 0.0);
        if (gi < m && gk < k) v = cconj_if(Ap[gi * A.rs + gk * A.cs], A.conj);
        As[kk][i] = v;
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        int j, kk;
        if (b_kcontig) { kk = t & 15; j = (t >> 4) + 16 * q; }
        else { j = t & 63; kk = (t >> 6) + 4 * q; }
        const int gj = bn + j, gk = k0 + kk;
        cplx v = make_double2(0.0, 0.0);
        if (gj < n && gk < k) v = cconj_if(Bp[gk * B.rs + gj * B.cs], B.conj);
        Bs[kk][j] = v;
      }
      __syncthreads();
#pragma unroll 4
      for (int kk = 0; kk < GK; ++kk) {
        cplx av[4], bv[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) av[i] = As[kk][ty + 16 * i];
#pragma unroll
        for (int j = 0; j < 4; ++j) bv[j] = Bs[kk][tx + 16 * j];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) cfma(acc[i][j], av[i], bv[j]);
      }
      __syncthreads();
    }
  }
  cplx* Cb = C + b * sc;
  const bool use_beta = (beta.x != 0.0 || beta.y != 0.0);
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int gi = bm + ty + 16 * i;
    if (gi >= m) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int gj = bn + tx + 16 * j;
      if (gj >= n) continue;
      cplx v = cmul(alpha, acc[i][j]);
      if (use_beta) v = cadd(v, cmul(beta, Cb[gi * ldc + gj]));
      Cb[gi * ldc + gj] = v;
    }
  }
}

cudaError_t zgemm(int m, int n, int k, int nbatch, int nred, cplx alpha, MatRef A, MatRef B,
                  cplx beta, cplx* C, long long ldc, long long sc, const int* skip,
                  cudaStream_t s) {
  if (m <= 0 || n <= 0 || nbatch <= 0) return cudaSuccess;
  dim3 grid((n + GT - 1) / GT, (m + GT - 1) / GT, nbatch);
  count_launch();
  zgemm_kernel<<<grid, 256, 0, s>>>(m, n, k, nred, alpha, A, B, beta, C, ldc, sc, skip);
  return cudaGetLastError();
}

// ------------------------------------------------------------------------------------
// MPO channel mixing
// ------------------------------------------------------------------------------------
__global__ void mpo_mix_kernel(int Dout, int Ma, int d, int Mb, const int* start,
                               const int* chan, const cplx* ops, const cplx* X, long long xs,
                               cplx* Y, long long ys, const int* skip) {
  if (skip && *skip) return;
  const long long per = (long long)Ma * d * d * Mb;
  const long long total = per * Dout;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    long long r = e;
    const int b = (int)(r % Mb); r /= Mb;
    const int tau = (int)(r % d); r /= d;
    const int sig = (int)(r % d); r /= d;
    const int a = (int)(r % Ma);
    const int wo = (int)(r / Ma);
    cplx acc = make_double2(0.0, 0.0);
    for (int blk = start[wo]; blk < start[wo + 1]; ++blk) {
      const cplx* op = ops + (long long)blk * d * d + sig * d;
      const cplx* x = X + chan[blk] * xs + ((long long)a * d * d + tau) * Mb + b;
      for (int u = 0; u < d; ++u) {
        const cplx o = op[u];
        if (o.x != 0.0 || o.y != 0.0) cfma(acc, o, x[(long long)u * d * Mb]);
      }
    }
    Y[wo * ys + (e - (long long)wo * per)] = acc;
  }
}

cudaError_t mpo_mix(const MixTable& T, int Ma, int d, int Mb, const cplx* X, long long xs,
                    cplx* Y, long long ys, const int* skip, cudaStream_t s) {
  const long long total = (long long)T.Dout * Ma * d * d * Mb;
  if (total <= 0) return cudaSuccess;
  long long blocks = (total + 255) / 256;
  if (blocks > 152 * 32) blocks = 152 * 32;
  count_launch();
  mpo_mix_kernel<<<(int)blocks, 256, 0, s>>>(T.Dout, Ma, d, Mb, T.start, T.chan, T.ops, X, xs,
                                              Y, ys, skip);
  return cudaGetLastError();
}

// ------------------------------------------------------------------------------------
// reductions (two stages, fixed order: deterministic)
// ------------------------------------------------------------------------------------
__device__ __forceinline__ cplx block_sum_c(cplx v, cplx* sh) {
  double re = warp_sum(v.x), im = warp_sum(v.y);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) sh[w] = make_double2(re, im);
  __syncthreads();
  cplx out = make_double2(0.0, 0.0);
  if (threadIdx.x < 32) {
    cplx x = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : make_double2(0.0, 0.0);
    out.x = warp_sum(x.x);
    out.y = warp_sum(x.y);
  }
  __syncthreads();
  return out;
}

// Cross-block sums (znorm2): block x writes its partial, the last block (ticket counter)
// sums the partials in index order -- deterministic, no second launch.
constexpr int RED_BLOCKS = 304;      // partial blocks per vector (2 per SM)

__device__ __forceinline__ bool last_block(unsigned* counter, unsigned nblocks) {
  __shared__ int s_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned t = atomicAdd(counter, 1u);
    s_last = (t == nblocks - 1);
  }
  __syncthreads();
  return s_last != 0;
}

__global__ void znorm2_kernel(long long n, const cplx* x, double* out, double* partial,
                              unsigned* counter, const int* skip) {
  if (skip && *skip) return;
  __shared__ cplx sh[32];
  double a = 0.0, b = 0.0;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x) {
    const cplx v = x[e];
    a = fma(v.x, v.x, a);
    b = fma(v.y, v.y, b);
  }
  cplx s = block_sum_c(make_double2(a + b, 0.0), sh);
  if (threadIdx.x == 0) partial[blockIdx.x] = s.x;
  if (!last_block(counter, gridDim.x)) return;
  double r = 0.0;
  for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) r += __ldcg(&partial[i]);
  cplx t = block_sum_c(make_double2(r, 0.0), sh);
  if (threadIdx.x == 0) {
    *out = t.x;
    *counter = 0;
  }
}

cudaError_t znorm2(long long n, const cplx* x, double* out, double* partial, unsigned* counter,
                   const int* skip, cudaStream_t s) {
  int g = (int)((n + 255) / 256);
  if (g > RED_BLOCKS) g = RED_BLOCKS;
  if (g < 1) g = 1;
  count_launch();
  znorm2_kernel<<<g, 256, 0, s>>>(n, x, out, partial, counter, skip);
  return cudaGetLastError();
}

// x *= 1/sqrt(*nrm2); *logacc += log(*nrm2)  (imaginary-time renormalisation of the center)
__global__ void znormalize_log_kernel(long long n, cplx* x, const double* nrm2, double* logacc) {
  const double s = *nrm2;
  if (!(s > 0.0)) return;
  const double f = 1.0 / sqrt(s);
  if (blockIdx.x == 0 && threadIdx.x == 0) *logacc += log(s);
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x) {
    x[e].x *= f;
    x[e].y *= f;
  }
}

cudaError_t znormalize_log(long long n, cplx* x, const double* nrm2, double* logacc,
                           cudaStream_t s) {
  long long blocks = (n + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  if (blocks < 1) blocks = 1;
  count_launch();
  znormalize_log_kernel<<<(int)blocks, 256, 0, s>>>(n, x, nrm2, logacc);
  return cudaGetLastError();
}

__global__ void zconj_kernel(long long n, cplx* x) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x)
    x[e].y = -x[e].y;
}

__global__ void zaxpy_kernel(long long n, cplx alpha, const cplx* x, cplx* y) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x) {
    const cplx v = x[e];
    y[e].x = fma(alpha.x, v.x, fma(-alpha.y, v.y, y[e].x));
    y[e].y = fma(alpha.x, v.y, fma(alpha.y, v.x, y[e].y));
  }
}

cudaError_t zaxpy(long long n, cplx alpha, const cplx* x, cplx* y, cudaStream_t s) {
  long long blocks = (n + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  if (blocks < 1) blocks = 1;
  count_launch();
  zaxpy_kernel<<<(int)blocks, 256, 0, s>>>(n, alpha, x, y);
  return cudaGetLastError();
}

// S = the Hermitian matrix with the strictly lower triangle of M, its conjugate mirror above
// the diagonal and Re(M_ii) on it (n x n, row-major)
__global__ void herm_lower_kernel(int n, const cplx* M, cplx* S) {
  const long long nn = (long long)n * n;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < nn;
       e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e / n), j = (int)(e % n);
    cplx v;
    if (i > j) v = M[e];
    else if (i < j) v = make_double2(M[(long long)j * n + i].x, -M[(long long)j * n + i].y);
    else v = make_double2(M[e].x, 0.0);
    S[e] = v;
  }
}

cudaError_t herm_lower(int n, const cplx* M, cplx* S, cudaStream_t s) {
  long long blocks = ((long long)n * n + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  if (blocks < 1) blocks = 1;
  count_launch();
  herm_lower_kernel<<<(int)blocks, 256, 0, s>>>(n, M, S);
  return cudaGetLastError();
}

// X[r][:] R^H = B[r][:] for every row r (R n x n upper triangular, row-major): back
// substitution, one thread per row, x_j = (b_j - sum_{k>j} x_k conj(R_jk)) / conj(R_jj)
__global__ void solve_rh_kernel(int m, int n, const cplx* R, const cplx* B, cplx* X) {
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < m; r += gridDim.x * blockDim.x) {
    const cplx* b = B + (size_t)r * n;
    cplx* x = X + (size_t)r * n;
    for (int j = n - 1; j >= 0; --j) {
      double ar = b[j].x, ai = b[j].y;
      for (int k = j + 1; k < n; ++k) {
        const cplx q = R[(size_t)j * n + k], v = x[k];
        ar -= v.x * q.x + v.y * q.y;
        ai -= v.y * q.x - v.x * q.y;
      }
      const cplx dj = R[(size_t)j * n + j];          // divide by conj(dj) = multiply by dj/|dj|^2
      const double nd = dj.x * dj.x + dj.y * dj.y;
      x[j] = make_double2((ar * dj.x - ai * dj.y) / nd, (ai * dj.x + ar * dj.y) / nd);
    }
  }
}

cudaError_t solve_rh(int m, int n, const cplx* R, const cplx* B, cplx* X, cudaStream_t s) {
  int blocks = (m + 127) / 128;
  if (blocks < 1) blocks = 1;
  count_launch();
  solve_rh_kernel<<<blocks, 128, 0, s>>>(m, n, R, B, X);
  return cudaGetLastError();
}

// triu: zero the strictly lower triangle of an n x n matrix in place
__global__ void triu_kernel(int n, cplx* A) {
  const long long nn = (long long)n * n;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < nn;
       e += (long long)gridDim.x * blockDim.x)
    if (e / n > e % n) A[e] = make_double2(0.0, 0.0);
}

cudaError_t triu_inplace(int n, cplx* A, cudaStream_t s) {
  long long blocks = ((long long)n * n + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  if (blocks < 1) blocks = 1;
  count_launch();
  triu_kernel<<<(int)blocks, 256, 0, s>>>(n, A);
  return cudaGetLastError();
}

cudaError_t zconj(long long n, cplx* x, cudaStream_t s) {
  long long blocks = (n + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  if (blocks < 1) blocks = 1;
  count_launch();
  zconj_kernel<<<(int)blocks, 256, 0, s>>>(n, x);
  return cudaGetLastError();
}

__global__ void zscale_by_kernel(long long n, cplx* x, const double* factor, const int* skip) {
  if (skip && *skip) return;
  const double f = *factor;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x) {
    x[e].x *= f;
    x[e].y *= f;
  }
}

cudaError_t zscale_by(long long n, cplx* x, const double* factor, const int* skip,
                      cudaStream_t s) {
  long long blocks = (n + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  if (blocks < 1) blocks = 1;
  count_launch();
  zscale_by_kernel<<<(int)blocks, 256, 0, s>>>(n, x, factor, skip);
  return cudaGetLastError();
}

// ------------------------------------------------------------------------------------
// Lanczos bookkeeping: the start of a run and the final combination (the orthogonalisation
// steps themselves are one cooperative launch each, lanczos_step.cu).
// ------------------------------------------------------------------------------------
__global__ void lz_start_kernel(LzState* S, const double* nrm2) {
  if (threadIdx.x == 0) {
    const double b0 = sqrt(*nrm2);
    S->b0 = b0;
    S->inv = b0 > 0.0 ? 1.0 / b0 : 0.0;
    S->k = 0;
    S->done = (b0 == 0.0) ? 1 : 0;
    S->noconv = 0;
    S->err = 0.0;
    if (b0 == 0.0) {
      for (int i = 0; i < KMAX; ++i) S->c[i] = make_double2(0.0, 0.0);
    }
  }
}

cudaError_t lz_start(LzState* S, const double* nrm2, cudaStream_t s) {
  count_launch();
  lz_start_kernel<<<1, 32, 0, s>>>(S, nrm2);
  return cudaGetLastError();
}

__global__ void zcombine_kernel(long long n, const LzState* S, const cplx* V, long long ldv,
                                cplx* out) {
  const int k = S->k;
  __shared__ cplx c[KMAX];
  if (threadIdx.x < KMAX) c[threadIdx.x] = S->c[threadIdx.x];
  __syncthreads();
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x) {
    cplx acc = make_double2(0.0, 0.0);
    for (int i = 0; i < k; ++i) cfma(acc, c[i], V[i * ldv + e]);
    out[e] = acc;
  }
}

cudaError_t zcombine(long long n, const LzState* S, const cplx* V, long long ldv, cplx* out,
                     cudaStream_t s) {
  long long blocks = (n + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  if (blocks < 1) blocks = 1;
  count_launch();
  zcombine_kernel<<<(int)blocks, 256, 0, s>>>(n, S, V, ldv, out);
  return cudaGetLastError();
}

// ------------------------------------------------------------------------------------
// Gauge QR: Gram-Schmidt (twice) column by column with skipped columns and deterministic
// completion.  One cooperative launch; CTA g owns a contiguous block of rows of Y, Q and
// of the working vector, so the only cross-CTA traffic is the partial dot products and
// norms, exchanged through double-buffered global arrays and a bounded grid barrier.
// ------------------------------------------------------------------------------------
constexpr int QR_THREADS = 256;

__device__ __forceinline__ bool grid_barrier(unsigned* bar, unsigned nblocks, int* status,
                                             long long limit) {
  __syncthreads();
  __shared__ int s_ok;
  if (threadIdx.x == 0) {
    volatile unsigned* vgen = bar + 1;
    volatile int* vstat = status;
    const unsigned gen = *vgen;
    __threadfence();
    const unsigned prev = atomicAdd(bar, 1u);
    int ok = 1;
    if (prev == nblocks - 1) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      const long long t0 = clock64();
      while (*vgen == gen) {
        if (*vstat) { ok = 0; break; }
        if (clock64() - t0 > limit) {
          atomicExch(status, 1);
          ok = 0;
          break;
        }
      }
    }
    __threadfence();
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

__device__ __forceinline__ cplx qr_load(const QrRef& Y, long long r, long long c) {
  const long long off = r * Y.rs + (c % Y.cb) * Y.cs + (c / Y.cb) * Y.cbs;
  return cconj_if(Y.p[off], Y.conj);
}

struct QrKernelArgs {
  int m, n, p;
  QrRef Y, E;
  cplx* Q;
  cplx* R;
  cplx* part;
  double* partn;
  unsigned* bar;
  int* status;
  long long wait;                // grid-barrier wait limit (clock cycles)
  double rank_tol, complete_tol;
  const unsigned char* acc_in;   // completion only: accepted flags of a factorisation done
                                 // elsewhere (Q, R already written; only skipped columns filled)
  int* src_out = nullptr;        // if set: per completed position, the candidate that filled it
                                 // (i < p: column i of E, p + i: unit vector e_i)
};

// Sum of the G per-block partial doubles at stride `stride` (fixed order per lane, then a
// fixed warp tree): evaluated by warp 0, result broadcast through red[slot].
__device__ __forceinline__ void qr_sum_partials(const double* base, long long stride, unsigned G,
                                                double* red, int slot) {
  if (threadIdx.x < 32) {
    double a = 0.0, b = 0.0;
    unsigned gg = threadIdx.x;
    for (; gg + 32 < G; gg += 64) {
      a += __ldcg(&base[gg * stride]);
      b += __ldcg(&base[(gg + 32) * stride]);
    }
    if (gg < G) a += __ldcg(&base[gg * stride]);
    a = warp_sum(a + b);
    if (threadIdx.x == 0) red[slot] = a;
  }
}

// One Gram-Schmidt pass of v (own rows) against the accepted columns of Q below `lim`:
// h = Q^H v reduced over all CTAs (together with ||v||^2 before the pass), v -= Q h,
// hacc += h.  Returns ||v_before||^2 in *vv_before and sum |h|^2 in *hh (identical in all
// CTAs: same partials, same summation order).  Every phase splits its sums over several
// threads with independent accumulators, because FP64 dependency latency dominates here.
__device__ bool qr_pass(const QrKernelArgs& A, int r0, int nr, int lim, cplx* v, cplx* h,
                        cplx* hacc, const unsigned char* acc, int& buf, unsigned G, double* red,
                        cplx* sm, double* vv_before, double* hh) {
  const int n = A.n;
  const int g = blockIdx.x;
  const int T = blockDim.x;
  // (1) partial dots of this CTA's rows: P threads per column, 4 accumulators each
  {
    int P = lim > 0 ? T / lim : 1;
    if (P < 1) P = 1;
    if (P > 8) P = 8;
    for (int idx = threadIdx.x; idx < lim * P; idx += T) {
      const int i = idx % lim, part = idx / lim;
      double ax = 0.0, bx = 0.0, ay = 0.0, by = 0.0;
      if (acc[i]) {
        for (int r = part; r < nr; r += P) {
          const cplx q = A.Q[(long long)(r0 + r) * n + i];
          const cplx x = v[r];
          ax = fma(q.x, x.x, ax);
          bx = fma(q.y, x.y, bx);
          ay = fma(q.x, x.y, ay);
          by = fma(-q.y, x.x, by);
        }
      }
      if (lim * P <= T) sm[part * lim + i] = make_double2(ax + bx, ay + by);
      else A.part[((long long)buf * G + g) * (n + 1) + i] = make_double2(ax + bx, ay + by);
    }
    __syncthreads();
    if (lim * P <= T) {
      for (int i = threadIdx.x; i < lim; i += T) {
        cplx s = make_double2(0.0, 0.0);
        for (int part = 0; part < P; ++part) s = cadd(s, sm[part * lim + i]);
        A.part[((long long)buf * G + g) * (n + 1) + i] = s;
      }
    }
  }
  // partial ||v||^2 of this CTA's rows, stored after the n dot products
  double vv = 0.0;
  for (int r = threadIdx.x; r < nr; r += T) vv += v[r].x * v[r].x + v[r].y * v[r].y;
  vv = warp_sum(vv);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = vv;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (T >> 5); ++w) t += red[w];
    A.part[((long long)buf * G + g) * (n + 1) + n] = make_double2(t, 0.0);
  }
  if (!grid_barrier(A.bar, G, A.status, A.wait)) return false;
  // (2) reduce the G partials of every column: P threads per column, 2 accumulators each
  {
    const cplx* base = A.part + (long long)buf * G * (n + 1);
    int P = lim > 0 ? T / lim : 1;
    if (P < 1) P = 1;
    if (P > 8) P = 8;
    for (int idx = threadIdx.x; idx < lim * P; idx += T) {
      const int i = idx % lim, part = idx / lim;
      cplx s0 = make_double2(0.0, 0.0), s1 = make_double2(0.0, 0.0);
      if (acc[i]) {
        unsigned gg = part;
        for (; gg + P < G; gg += 2 * P) {
          s0 = cadd(s0, __ldcg(&base[(long long)gg * (n + 1) + i]));
          s1 = cadd(s1, __ldcg(&base[(long long)(gg + P) * (n + 1) + i]));
        }
        if (gg < G) s0 = cadd(s0, __ldcg(&base[(long long)gg * (n + 1) + i]));
      }
      const cplx s = cadd(s0, s1);
      if (lim * P <= T) sm[part * lim + i] = s;
      else h[i] = s;
    }
    __syncthreads();
    double hsq = 0.0;
    for (int i = threadIdx.x; i < lim; i += T) {
      cplx s;
      if (lim * P <= T) {
        s = make_double2(0.0, 0.0);
        for (int part = 0; part < P; ++part) s = cadd(s, sm[part * lim + i]);
        h[i] = s;
      } else {
        s = h[i];
      }
      hacc[i] = cadd(hacc[i], s);
      hsq += s.x * s.x + s.y * s.y;
    }
    hsq = warp_sum(hsq);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = hsq;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int w = 0; w < (T >> 5); ++w) t += red[w];
      red[32] = t;
    }
    qr_sum_partials(&base[n].x, 2LL * (n + 1), G, red, 33);
  }
  buf ^= 1;
  __syncthreads();
  *hh = red[32];
  *vv_before = red[33];
  // (3) v -= Q h: P3 (a power of two <= 32) threads per row, 2 accumulators each
  {
    int P3 = 1;
    while (P3 < 32 && 2 * P3 * nr <= T) P3 *= 2;
    const int total = nr * P3;
    for (int base_i = 0; base_i < total; base_i += T) {
      const int idx = base_i + threadIdx.x;
      const bool on = idx < total;
      const int r = on ? idx / P3 : 0, part = idx % P3;
      double ar = 0.0, br = 0.0, ai = 0.0, bi = 0.0;
      if (on) {
        for (int i = part; i < lim; i += P3) {
          const cplx q = A.Q[(long long)(r0 + r) * n + i];
          const cplx c = h[i];
          ar = fma(q.x, c.x, ar);
          br = fma(-q.y, c.y, br);
          ai = fma(q.x, c.y, ai);
          bi = fma(q.y, c.x, bi);
        }
      }
      double sr = ar + br, si = ai + bi;
      for (int o = P3 >> 1; o > 0; o >>= 1) {
        sr += __shfl_xor_sync(0xffffffffu, sr, o);
        si += __shfl_xor_sync(0xffffffffu, si, o);
      }
      if (on && part == 0) v[r] = make_double2(v[r].x - sr, v[r].y - si);
    }
  }
  __syncthreads();
  return true;
}

__device__ bool qr_norm(const QrKernelArgs& A, int nr, const cplx* v, double& out, int& buf,
                        unsigned G, double* red) {
  double s = 0.0;
  for (int r = threadIdx.x; r < nr; r += blockDim.x) s += v[r].x * v[r].x + v[r].y * v[r].y;
  s = warp_sum(s);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) red[warp] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    A.partn[buf * G + blockIdx.x] = t;
  }
  if (!grid_barrier(A.bar, G, A.status, A.wait)) return false;
  qr_sum_partials(A.partn + buf * G, 1, G, red, 32);   // reads through L2 (other CTAs)
  __syncthreads();
  out = sqrt(red[32]);
  buf ^= 1;
  __syncthreads();
  return true;
}

// Residual norm of v against the accepted columns below `lim`, Gram-Schmidt with
// re-orthogonalisation only when needed: after one pass, if sum|h|^2 <= 0.75 ||v||^2 the
// residual norm is taken from Pythagoras (no cancellation beyond a factor 4); otherwise a
// second pass is made and the norm is computed directly ("twice is enough").  On return v holds
// the residual and *nrm its norm.
__device__ bool qr_residual(const QrKernelArgs& A, int r0, int nr, int lim, cplx* v, cplx* h,
                            cplx* hacc, const unsigned char* acc, int& buf, unsigned G,
                            double* red, cplx* sm, double* nrm) {
  double vv, hh;
  if (!qr_pass(A, r0, nr, lim, v, h, hacc, acc, buf, G, red, sm, &vv, &hh)) return false;
  if (hh <= 0.75 * vv) {
    *nrm = sqrt(fmax(vv - hh, 0.0));
    return true;
  }
  if (!qr_pass(A, r0, nr, lim, v, h, hacc, acc, buf, G, red, sm, &vv, &hh)) return false;
  return qr_norm(A, nr, v, *nrm, buf, G, red);
}

__global__ void __launch_bounds__(QR_THREADS) gauge_qr_kernel(QrKernelArgs A) {
  extern __shared__ unsigned char smem[];
  const int m = A.m, n = A.n;
  const unsigned G = gridDim.x;
  const int rows = (m + G - 1) / G;
  const int r0 = blockIdx.x * rows;
  const int nr = max(0, min(m, r0 + rows) - r0);
  cplx* v = reinterpret_cast<cplx*>(smem);
  cplx* h = v + rows;
  cplx* hacc = h + n;
  double* red = reinterpret_cast<double*>(hacc + n);            // 34 doubles
  cplx* sm = reinterpret_cast<cplx*>(red + 34);                  // QR_THREADS entries
  unsigned char* acc = reinterpret_cast<unsigned char*>(sm + QR_THREADS);
  int buf = 0;

  if (A.acc_in) {
    // completion only: nothing to do unless a column was skipped (same decision in all CTAs)
    __shared__ int s_missing;
    if (threadIdx.x == 0) s_missing = 0;
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      acc[i] = A.acc_in[i];
      if (!acc[i]) atomicOr(&s_missing, 1);
    }
    __syncthreads();
    if (!s_missing) return;
  }
  if (!A.acc_in) {
  for (long long e = threadIdx.x; e < (long long)nr * n; e += blockDim.x)
    A.Q[(long long)r0 * n + e] = make_double2(0.0, 0.0);
  if (blockIdx.x == 0)
    for (long long e = threadIdx.x; e < (long long)n * n; e += blockDim.x)
      A.R[e] = make_double2(0.0, 0.0);
  for (int i = threadIdx.x; i < n; i += blockDim.x) acc[i] = 0;
  // ||Y||_F
  double ynorm2 = 0.0;
  for (long long e = threadIdx.x; e < (long long)nr * n; e += blockDim.x) {
    const cplx y = qr_load(A.Y, r0 + e / n, e % n);
    ynorm2 += y.x * y.x + y.y * y.y;
  }
  ynorm2 = warp_sum(ynorm2);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = ynorm2;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    A.partn[buf * G + blockIdx.x] = t;
  }
  if (!grid_barrier(A.bar, G, A.status, A.wait)) return;
  qr_sum_partials(A.partn + buf * G, 1, G, red, 33);
  __syncthreads();
  const double thr = A.rank_tol * sqrt(red[33]);
  buf ^= 1;
  __syncthreads();

  // accepted columns
  for (int j = 0; j < n; ++j) {
    for (int r = threadIdx.x; r < nr; r += blockDim.x) v[r] = qr_load(A.Y, r0 + r, j);
    for (int i = threadIdx.x; i < n; i += blockDim.x) hacc[i] = make_double2(0.0, 0.0);
    __syncthreads();
    double nrm;
    if (!qr_residual(A, r0, nr, j, v, h, hacc, acc, buf, G, red, sm, &nrm)) return;
    const bool take = nrm > thr;
    if (take) {
      const double inv = 1.0 / nrm;
      for (int r = threadIdx.x; r < nr; r += blockDim.x)
        A.Q[(long long)(r0 + r) * n + j] = make_double2(v[r].x * inv, v[r].y * inv);
    }
    if (blockIdx.x == 0) {
      for (int i = threadIdx.x; i < j; i += blockDim.x) A.R[(long long)i * n + j] = hacc[i];
      if (threadIdx.x == 0 && take) A.R[(long long)j * n + j] = make_double2(nrm, 0.0);
    }
    __syncthreads();
    if (threadIdx.x == 0 && take) acc[j] = 1;
    __syncthreads();
  }
  }
  // completion of skipped positions
  long long cand = 0;
  for (int j = 0; j < n; ++j) {
    if (acc[j]) continue;
    bool found = false;
    while (!found) {
      if (cand >= (long long)A.p + m) {
        if (threadIdx.x == 0 && blockIdx.x == 0) atomicExch(A.status, 2);
        return;
      }
      double n0;
      if (cand < A.p) {
        for (int r = threadIdx.x; r < nr; r += blockDim.x) v[r] = qr_load(A.E, r0 + r, cand);
        __syncthreads();
        if (!qr_norm(A, nr, v, n0, buf, G, red)) return;
      } else {
        const long long unit = cand - A.p;
        for (int r = threadIdx.x; r < nr; r += blockDim.x)
          v[r] = make_double2((r0 + r) == unit ? 1.0 : 0.0, 0.0);
        __syncthreads();
        n0 = 1.0;
      }
      ++cand;
      if (n0 == 0.0) continue;
      double nc;
      if (!qr_residual(A, r0, nr, n, v, h, hacc, acc, buf, G, red, sm, &nc)) return;
      if (nc > A.complete_tol * n0) {
        const double inv = 1.0 / nc;
        for (int r = threadIdx.x; r < nr; r += blockDim.x)
          A.Q[(long long)(r0 + r) * n + j] = make_double2(v[r].x * inv, v[r].y * inv);
        __syncthreads();
        if (threadIdx.x == 0) acc[j] = 1;
        if (A.src_out && threadIdx.x == 0 && blockIdx.x == 0) A.src_out[j] = (int)(cand - 1);
        __syncthreads();
        found = true;
      }
    }
  }
}

// per device: the SM count (one CTA per SM keeps the barrier cheap) and whether the kernel's
// shared-memory limit has been raised on that device
constexpr int kQrMaxDevices = 64;
static int g_qr_coop_blocks[kQrMaxDevices];
static bool g_qr_attr_set[kQrMaxDevices];

static int qr_device() {
  int dev = 0;
  cudaGetDevice(&dev);
  return (dev >= 0 && dev < kQrMaxDevices) ? dev : 0;
}

int gauge_qr_grid(int m) {
  const int dev = qr_device();
  if (g_qr_coop_blocks[dev] < 1) {
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    g_qr_coop_blocks[dev] = sms > 0 ? sms : 1;
  }
  int g = (m + 15) / 16;
  if (g > g_qr_coop_blocks[dev]) g = g_qr_coop_blocks[dev];
  if (g < 1) g = 1;
  return g;
}

size_t gauge_qr_smem(int m, int n, int G) {
  const int rows = (m + G - 1) / G;
  return (size_t)rows * sizeof(cplx) + 2 * (size_t)n * sizeof(cplx) + 34 * sizeof(double) +
         QR_THREADS * sizeof(cplx) + (size_t)n + 16;
}

static cudaError_t qr_allow_smem() {
  const int dev = qr_device();
  if (g_qr_attr_set[dev]) return cudaSuccess;
  const cudaError_t e = cudaFuncSetAttribute(
      gauge_qr_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kQrMaxSmem);
  if (e == cudaSuccess) g_qr_attr_set[dev] = true;
  return e;
}

cudaError_t gauge_qr(int m, int n, QrRef Y, int p, QrRef E, cplx* Q, cplx* R,
                     const QrScratch& W, int* status, cudaStream_t s, int gcap, double rank_tol,
                     int* src) {
  int G = gauge_qr_grid(m);
  if (gcap > 0 && G > gcap) G = gcap;
  if (G > W.gmax || n > W.nmax) return cudaErrorInvalidValue;
  const size_t smem = gauge_qr_smem(m, n, G);
  if (smem > kQrMaxSmem) return cudaErrorInvalidValue;
  cudaError_t e = qr_allow_smem();
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(W.bar, 0, 2 * sizeof(unsigned), s);
  if (e != cudaSuccess) return e;
  QrKernelArgs a;
  a.m = m; a.n = n; a.p = p;
  a.Y = Y; a.E = E;
  if (p == 0) { a.E = Y; }
  a.Q = Q; a.R = R;
  a.part = W.part; a.partn = W.partn; a.bar = W.bar; a.status = status;
  a.wait = W.wait > 0 ? W.wait : kBarrierWaitCycles;
  a.rank_tol = rank_tol;
  a.complete_tol = 1e-2;
  a.acc_in = nullptr;
  a.src_out = src;
  // cooperative launch through cudaLaunchKernelEx (also valid inside a stream capture)
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(G);
  cfg.blockDim = dim3(QR_THREADS);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  count_launch();
  return cudaLaunchKernelEx(&cfg, gauge_qr_kernel, a);
}

cudaError_t gauge_qr_complete(int m, int n, int p, QrRef E, cplx* Q, const unsigned char* acc,
                              const QrScratch& W, int* status, cudaStream_t s, int gcap,
                              int* src) {
  int G = gauge_qr_grid(m);
  if (gcap > 0 && G > gcap) G = gcap;
  if (G > W.gmax || n > W.nmax) return cudaErrorInvalidValue;
  const size_t smem = gauge_qr_smem(m, n, G);
  if (smem > kQrMaxSmem) return cudaErrorInvalidValue;
  cudaError_t e = qr_allow_smem();
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(W.bar, 0, 2 * sizeof(unsigned), s);
  if (e != cudaSuccess) return e;
  QrKernelArgs a;
  a.m = m; a.n = n; a.p = p;
  a.Y = E; a.E = E;
  a.Q = Q; a.R = nullptr;
  a.part = W.part; a.partn = W.partn; a.bar = W.bar; a.status = status;
  a.wait = W.wait > 0 ? W.wait : kBarrierWaitCycles;
  a.rank_tol = 1e-12;
  a.complete_tol = 1e-2;
  a.acc_in = acc;
  a.src_out = src;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(G);
  cfg.blockDim = dim3(QR_THREADS);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  count_launch();
  return cudaLaunchKernelEx(&cfg, gauge_qr_kernel, a);
}

// ------------------------------------------------------------------------------------
// small helpers
// ------------------------------------------------------------------------------------
__global__ void ztranspose_kernel(int m, int n, const cplx* src, cplx* dst, int conj) {
  __shared__ cplx tile[32][33];
  const int bx = blockIdx.x * 32, by = blockIdx.y * 32;
  for (int yy = threadIdx.y; yy < 32; yy += 8) {
    const int i = by + yy, j = bx + threadIdx.x;
    if (i < m && j < n) tile[yy][threadIdx.x] = cconj_if(src[(long long)i * n + j], conj);
  }
  __syncthreads();
  for (int yy = threadIdx.y; yy < 32; yy += 8) {
    const int j = bx + yy, i = by + threadIdx.x;
    if (i < m && j < n) dst[(long long)j * m + i] = tile[threadIdx.x][yy];
  }
}

cudaError_t ztranspose(int m, int n, const cplx* src, cplx* dst, int conj, cudaStream_t s) {
  dim3 grid((n + 31) / 32, (m + 31) / 32);
  count_launch();
  ztranspose_kernel<<<grid, dim3(32, 8), 0, s>>>(m, n, src, dst, conj);
  return cudaGetLastError();
}

// entries: triples (a, s, b) of unit coefficients; the tensor is zeroed first by the caller
__global__ void fill_entries_kernel(cplx* A, int D, int Mr, const int* entries, int nent) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nent; e += gridDim.x * blockDim.x) {
    const int a = entries[3 * e], s = entries[3 * e + 1], b = entries[3 * e + 2];
    A[((long long)a * D + s) * Mr + b] = make_double2(1.0, 0.0);
  }
}

cudaError_t zfill_identity_mps(cplx* A, int Ml, int D, int Mr, const int* entries, int nent,
                               cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(A, 0, sizeof(cplx) * (size_t)Ml * D * Mr, s);
  if (e != cudaSuccess) return e;
  if (nent > 0) count_launch();
  if (nent > 0) fill_entries_kernel<<<(nent + 255) / 256, 256, 0, s>>>(A, D, Mr, entries, nent);
  return cudaGetLastError();
}


// out = sum_b E[b][b] of an M x M matrix (one block, fixed summation order)
__global__ void __launch_bounds__(256) ztrace_kernel(const cplx* E, int M, cplx* out) {
  __shared__ double sr[256], si[256];
  double re = 0.0, im = 0.0;
  for (int b = threadIdx.x; b < M; b += 256) {
    const cplx e = E[(long long)b * M + b];
    re += e.x;
    im += e.y;
  }
  sr[threadIdx.x] = re;
  si[threadIdx.x] = im;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      sr[threadIdx.x] += sr[threadIdx.x + w];
      si[threadIdx.x] += si[threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = make_double2(sr[0], si[0]);
}

cudaError_t ztrace(const cplx* E, int M, cplx* out, cudaStream_t s) {
  count_launch();
  ztrace_kernel<<<1, 256, 0, s>>>(E, M, out);
  return cudaGetLastError();
}


// FP64 FMA throughput probe: every thread runs 8 independent chains of `iters` FMAs
// (x <- x * a + b with |a| < 1, so the chains stay finite) and stores their sum.
__global__ void __launch_bounds__(256) dfma_loop_kernel(long long iters, double a, double b,
                                                        double* sink) {
  double x0 = threadIdx.x * 1e-3, x1 = x0 + 0.1, x2 = x0 + 0.2, x3 = x0 + 0.3;
  double x4 = x0 + 0.4, x5 = x0 + 0.5, x6 = x0 + 0.6, x7 = x0 + 0.7;
  for (long long i = 0; i < iters; ++i) {
    x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
    x4 = fma(x4, a, b); x5 = fma(x5, a, b); x6 = fma(x6, a, b); x7 = fma(x7, a, b);
  }
  sink[blockIdx.x * (long long)blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
}

cudaError_t dfma_loop(int blocks, long long iters, double* sink, cudaStream_t s) {
  count_launch();
  dfma_loop_kernel<<<blocks, 256, 0, s>>>(iters, 0.999999, 1e-6, sink);
  return cudaGetLastError();
}


// Parameter cotangent of a site operator H_eff(L, W, R) between a and b:
//   G[w][v][s][u] += k * sum_{x,t,c} U[w][x][u][t][c] V[v][x][s][t][c],
//   U[w][x][u][t][c] = sum_y L[w,x,y] b[y,u,t,c],  V[v][x][s][t][c] = sum_b' conj(a[x,s,t,b']) R[v,b',c],
// so that <a, H_eff(L, dW, R) b> = sum dW[w,v,s,u] G[w,v,s,u].  One block per (w, v, s), the
// threads striding over (x, t, c) with c fastest (coalesced), d accumulators per thread, a
// fixed-order block reduction and one writer per entry.
constexpr int GRAM_MAX_D = 16;
__global__ void __launch_bounds__(256) param_gram_kernel(int Dl, int Dr, int Ml, int d, int Mr,
                                                         const cplx* U, const cplx* V, cplx k,
                                                         cplx* G) {
  __shared__ double red[2 * GRAM_MAX_D][8];
  const int s = blockIdx.x % d;
  const int v = (blockIdx.x / d) % Dr;
  const int w = blockIdx.x / (d * Dr);
  const long long D = (long long)d * d;
  const long long K = (long long)Ml * d * Mr;
  double ar[GRAM_MAX_D], ai[GRAM_MAX_D];
#pragma unroll
  for (int u = 0; u < GRAM_MAX_D; ++u) ar[u] = ai[u] = 0.0;
  for (long long e = threadIdx.x; e < K; e += blockDim.x) {
    const long long x = e / ((long long)d * Mr);
    const int t = (int)((e / Mr) % d);
    const int c = (int)(e % Mr);
    const cplx vv = V[(((long long)v * Ml + x) * D + (long long)s * d + t) * Mr + c];
    const cplx* up = U + (((long long)w * Ml + x) * D + t) * Mr + c;
#pragma unroll
    for (int u = 0; u < GRAM_MAX_D; ++u) {
      if (u < d) {
        const cplx uu = up[(long long)u * d * Mr];
        ar[u] = fma(uu.x, vv.x, fma(-uu.y, vv.y, ar[u]));
        ai[u] = fma(uu.x, vv.y, fma(uu.y, vv.x, ai[u]));
      }
    }
  }
  const int lane = threadIdx.x & 31, wv = threadIdx.x >> 5;
#pragma unroll
  for (int u = 0; u < GRAM_MAX_D; ++u) {
    if (u < d) {
      double x = ar[u], y = ai[u];
      for (int o = 16; o > 0; o >>= 1) {
        x += __shfl_xor_sync(0xffffffffu, x, o);
        y += __shfl_xor_sync(0xffffffffu, y, o);
      }
      if (lane == 0) {
        red[2 * u][wv] = x;
        red[2 * u + 1][wv] = y;
      }
    }
  }
  __syncthreads();
  if ((int)threadIdx.x < d) {
    const int u = threadIdx.x;
    double x = 0.0, y = 0.0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) {
      x += red[2 * u][q];
      y += red[2 * u + 1][q];
    }
    cplx& g = G[(((long long)w * Dr + v) * d + s) * d + u];
    g = make_double2(g.x + k.x * x - k.y * y, g.y + k.x * y + k.y * x);
  }
}

cudaError_t param_gram(int Dl, int Dr, int Ml, int d, int Mr, const cplx* U, const cplx* V,
                       cplx k, cplx* G, cudaStream_t s) {
  if (d > GRAM_MAX_D || d < 1) return cudaErrorInvalidValue;
  count_launch();
  param_gram_kernel<<<Dl * Dr * d, 256, 0, s>>>(Dl, Dr, Ml, d, Mr, U, V, k, G);
  return cudaGetLastError();
}

}  // namespace tdmrg
