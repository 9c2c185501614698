// Blocked gauge QR: the same factorisation and completion as the column-by-column kernel
// (Gram-Schmidt with skipped columns, deterministic completion), processed 16 columns at a
// time so that the cooperative grid synchronises ~5 times per block instead of once or more
// per column.
//
// Per block of columns [j0, j0 + b):
//  1. projection against the accepted columns < j0 (classical Gram-Schmidt as a small FP64
//     product per CTA; the cross-CTA sums are reduced slice-wise: every CTA sums a slice of
//     the coefficients over all CTAs, then all read the result); a second projection pass is
//     made when a column lost more than half its norm (sum|h|^2 > 0.75 ||v||^2);
//  2. the block Gram matrix of the projected columns, reduced the same way;
//  3. Gram-Schmidt with skips inside the block in Gram form (right-looking, one warp), with a
//     guard: if a column's residual^2 falls below 1/4 of its projected norm^2 (cancellation),
//     the block stops before it and the next block starts at that column, where its residual
//     is formed from the vectors themselves;
//  4. the accepted columns are formed locally (q_t = (v_t - sum_s q_s R_st) / R_tt).
// Skipped positions are completed afterwards by the column-wise routine of kernels_f64.cu.
#include "tdmrg_internal.cuh"

namespace tdmrg {

namespace {

constexpr int QB = 16;                 // columns per block
constexpr int QB_THREADS = 256;
static_assert(QB * QB == QB_THREADS, "the in-block update gives one Gram entry to each thread");


__device__ __forceinline__ double wsum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Grid barrier on one monotonic counter: barrier number e is passed once the counter reaches
// e * nblocks (one atomic per CTA; the launcher clears the counter).  Bounded: gives up after
// ~2 s, sets *status = 1, and every CTA then leaves.
__device__ bool qb_barrier(unsigned* bar, unsigned nblocks, int* status, unsigned& epoch,
                           long long limit) {
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

struct QbArgs {
  int m, n;
  QrRef Y;
  cplx* Q;
  cplx* R;
  cplx* part;        // [G][PS] per-CTA partial sums
  cplx* fin;         // [PS] reduced sums
  int PS;            // n*QB + QB + QB*QB
  unsigned* bar;
  int* status;
  long long wait;           // grid-barrier wait limit (clock cycles)
  unsigned char* acc_out;   // [n] accepted flags (for the completion pass)
  double rank_tol;
};

__device__ __forceinline__ cplx qb_load(const QrRef& Y, long long r, long long c) {
  const long long off = r * Y.rs + (c % Y.cb) * Y.cs + (c / Y.cb) * Y.cbs;
  const cplx v = Y.p[off];
  return Y.conj ? make_double2(v.x, -v.y) : v;
}

// Reduce `cnt` partial entries (offset `off` in each CTA's partial block) over all CTAs into
// fin[off..off+cnt): CTA g sums the slice it owns -- one warp per entry, every lane loading its
// share of the G partials at once -- then a barrier, then everyone may read fin.
__device__ bool qb_reduce(const QbArgs& A, int off, int cnt, unsigned G, unsigned& ep) {
  if (!qb_barrier(A.bar, G, A.status, ep, A.wait)) return false;
  const int per = (cnt + (int)G - 1) / (int)G;
  const int lo = blockIdx.x * per, hi = min(cnt, lo + per);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int e = lo + warp; e < hi; e += nw) {
    double ax = 0.0, ay = 0.0;
    for (unsigned g = lane; g < G; g += 32) {
      const cplx u = __ldcg(&A.part[(long long)g * A.PS + off + e]);   // other CTAs' data
      ax += u.x;
      ay += u.y;
    }
    ax = wsum(ax);
    ay = wsum(ay);
    if (lane == 0) A.fin[off + e] = make_double2(ax, ay);
  }
  return qb_barrier(A.bar, G, A.status, ep, A.wait);
}

}  // namespace

__global__ void __launch_bounds__(QB_THREADS) gauge_qr_blocked_kernel(QbArgs A) {
  extern __shared__ unsigned char smem[];
  const int m = A.m, n = A.n;
  const unsigned G = gridDim.x;
  const int rows = (m + G - 1) / G;
  const int r0 = blockIdx.x * rows;
  const int nr = max(0, min(m, r0 + rows) - r0);
  const int T = blockDim.x;
  cplx* vb = reinterpret_cast<cplx*>(smem);                 // [QB][rows]
  cplx* H = vb + QB * rows;                                   // [n][QB] projection coefficients
  cplx* Gb = H + n * QB;                                      // [QB][QB] Gram, then R of the block
  double* dvec = reinterpret_cast<double*>(Gb + QB * QB);     // vv[QB], hh[QB], diag0[QB], misc
  unsigned char* acc = reinterpret_cast<unsigned char*>(dvec + 4 * QB + 8);   // [n]
  unsigned char* accb = acc + n;                              // [QB]
  int* sint = reinterpret_cast<int*>(((reinterpret_cast<uintptr_t>(accb + QB) + 15) & ~(uintptr_t)15));
  cplx* mypart = A.part + (long long)blockIdx.x * A.PS;
  unsigned ep = 0;                                            // grid barriers passed

  for (long long e = threadIdx.x; e < (long long)nr * n; e += T)
    A.Q[(long long)r0 * n + e] = make_double2(0.0, 0.0);
  if (blockIdx.x == 0)
    for (long long e = threadIdx.x; e < (long long)n * n; e += T) A.R[e] = make_double2(0.0, 0.0);
  for (int i = threadIdx.x; i < n; i += T) acc[i] = 0;
  // ||Y||_F: partial in mypart[0]
  {
    double s = 0.0;
    for (long long e = threadIdx.x; e < (long long)nr * n; e += T) {
      const cplx y = qb_load(A.Y, r0 + e / n, e % n);
      s += y.x * y.x + y.y * y.y;
    }
    s = wsum(s);
    __shared__ double red[32];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int w = 0; w < T / 32; ++w) t += red[w];
      mypart[0] = make_double2(t, 0.0);
    }
  }
  if (!qb_reduce(A, 0, 1, G, ep)) return;
  const double thr = A.rank_tol * sqrt(__ldcg(&A.fin[0]).x);

  int j0 = 0;
  while (j0 < n) {
    const int bsz = min(QB, n - j0);
    for (int e = threadIdx.x; e < bsz * nr; e += T) {
      const int t = e / nr, r = e % nr;
      vb[t * rows + r] = qb_load(A.Y, r0 + r, j0 + t);
    }
    // the block's coefficients accumulate over the passes straight into R (CTA 0 only, each
    // entry by the same thread; a block that stopped early leaves partial sums in the columns it
    // did not finish, which the next block clears here)
    if (blockIdx.x == 0)
      for (int e = threadIdx.x; e < j0 * bsz; e += T)
        A.R[(long long)(e / bsz) * n + j0 + e % bsz] = make_double2(0.0, 0.0);
    __syncthreads();
    // ---- projection passes against the accepted columns < j0
    for (int pass = 0; pass < 2 && j0 > 0; ++pass) {
      // partial dots P[i][t] = sum_r conj(Q[r][i]) v_t[r]; partial ||v_t||^2 after them
      for (int e = threadIdx.x; e < j0 * bsz; e += T) {
        const int i = e / bsz, t = e % bsz;
        double ax = 0.0, bx = 0.0, ay = 0.0, by = 0.0;
        if (acc[i]) {
          const cplx* vt = vb + t * rows;
          for (int r = 0; r < nr; ++r) {
            const cplx q = A.Q[(long long)(r0 + r) * n + i];
            const cplx x = vt[r];
            ax = fma(q.x, x.x, ax);
            bx = fma(q.y, x.y, bx);
            ay = fma(q.x, x.y, ay);
            by = fma(-q.y, x.x, by);
          }
        }
        mypart[i * QB + t] = make_double2(ax + bx, ay + by);
      }
      for (int t = threadIdx.x >> 5; t < bsz; t += T >> 5) {
        double s = 0.0;
        for (int r = threadIdx.x & 31; r < nr; r += 32) {
          const cplx x = vb[t * rows + r];
          s += x.x * x.x + x.y * x.y;
        }
        s = wsum(s);
        if ((threadIdx.x & 31) == 0) mypart[j0 * QB + t] = make_double2(s, 0.0);
      }
      // reduce the j0*QB coefficients and, right after them, the QB norms
      if (!qb_reduce(A, 0, j0 * QB + QB, G, ep)) return;
      for (int e = threadIdx.x; e < j0 * bsz; e += T) {
        const int i = e / bsz, t = e % bsz;
        const cplx h = acc[i] ? __ldcg(&A.fin[i * QB + t]) : make_double2(0.0, 0.0);
        H[i * QB + t] = h;
        if (blockIdx.x == 0) {
          cplx& r = A.R[(long long)i * n + j0 + t];
          r = make_double2(r.x + h.x, r.y + h.y);
        }
      }
      __syncthreads();
      // hh[t] = sum_i |h_it|^2 (one warp per column), vv[t] from fin
      for (int t = threadIdx.x >> 5; t < bsz; t += T >> 5) {
        double s = 0.0;
        for (int i = threadIdx.x & 31; i < j0; i += 32) {
          const cplx h = H[i * QB + t];
          s += h.x * h.x + h.y * h.y;
        }
        s = wsum(s);
        if ((threadIdx.x & 31) == 0) {
          dvec[QB + t] = s;
          dvec[t] = __ldcg(&A.fin[j0 * QB + t]).x;
        }
      }
      // v_t[r] -= sum_i Q[r][i] h_it: thread per (r, t, part of the i range).  With few
      // (r, t) pairs the i range is split over up to 8 threads (partials summed in order through
      // shared memory): FP64 instructions cost the same whatever the number of active lanes, so
      // the work is spread over every warp.
      {
        const int pairs = nr * bsz;
        int split = 1;
        while (split < 8 && pairs * split * 2 <= T) split *= 2;
        cplx* hpart = Gb;      // QB*QB = T entries, free until the block Gram matrix
        for (int e0 = 0; e0 < pairs; e0 += T / split) {
          const int e = e0 + threadIdx.x / split, part = threadIdx.x % split;
          double ax = 0.0, bx = 0.0, ay = 0.0, by = 0.0;
          if (e < pairs) {
            const int r = e / bsz, t = e % bsz;
            for (int i = part; i < j0; i += split) {
              const cplx q = A.Q[(long long)(r0 + r) * n + i];
              const cplx h = H[i * QB + t];
              ax = fma(q.x, h.x, ax);
              bx = fma(-q.y, h.y, bx);
              ay = fma(q.x, h.y, ay);
              by = fma(q.y, h.x, by);
            }
          }
          if (split == 1) {
            if (e < pairs) {
              const int r = e / bsz, t = e % bsz;
              cplx& v = vb[t * rows + r];
              v = make_double2(v.x - (ax + bx), v.y - (ay + by));
            }
          } else {
            hpart[threadIdx.x] = make_double2(ax + bx, ay + by);
            __syncthreads();
            if (part == 0 && e < pairs) {
              const int r = e / bsz, t = e % bsz;
              double sx = 0.0, sy = 0.0;
              for (int k = 0; k < split; ++k) {
                sx += hpart[threadIdx.x + k].x;
                sy += hpart[threadIdx.x + k].y;
              }
              cplx& v = vb[t * rows + r];
              v = make_double2(v.x - sx, v.y - sy);
            }
            __syncthreads();
          }
        }
      }
      __syncthreads();
      bool again = false;
      for (int t = 0; t < bsz; ++t) again = again || (dvec[QB + t] > 0.75 * dvec[t]);
      if (!again) break;
    }
    // ---- block Gram matrix (upper triangle, s <= t)
    for (int e = threadIdx.x; e < QB * QB; e += T) {
      const int s = e / QB, t = e % QB;
      double ax = 0.0, bx = 0.0, ay = 0.0, by = 0.0;
      if (s <= t && t < bsz) {
        const cplx* vs = vb + s * rows;
        const cplx* vt = vb + t * rows;
        for (int r = 0; r < nr; ++r) {
          const cplx a = vs[r], b = vt[r];
          ax = fma(a.x, b.x, ax);
          bx = fma(a.y, b.y, bx);
          ay = fma(a.x, b.y, ay);
          by = fma(-a.y, b.x, by);
        }
      }
      mypart[e] = make_double2(ax + bx, ay + by);
    }
    if (!qb_reduce(A, 0, QB * QB, G, ep)) return;
    for (int e = threadIdx.x; e < QB * QB; e += T) Gb[e] = __ldcg(&A.fin[e]);
    __syncthreads();
    // ---- Gram-Schmidt with skips inside the block (Gram form, right-looking).  Thread 0 takes
    // the pivot (cancellation guard, acceptance, one reciprocal); the row scaling and the
    // trailing update use every thread, one entry each (QB * QB = T).
    if (threadIdx.x < QB)
      dvec[2 * QB + threadIdx.x] = threadIdx.x < bsz ? Gb[threadIdx.x * QB + threadIdx.x].x : 0.0;
    if (threadIdx.x == 0) {
      sint[0] = bsz;
      sint[1] = 0;
    }
    __syncthreads();
    for (int s = 0; s < bsz; ++s) {
      if (threadIdx.x == 0) {
        const double rho = Gb[s * QB + s].x;
        if (s > 0 && rho < 0.25 * dvec[2 * QB + s]) {
          sint[0] = s;          // the next block starts at this column
          sint[1] = 1;
        } else {
          // one reciprocal square root gives both R_ss and 1 / R_ss
          const double rp = fmax(rho, 0.0);
          const double rin = rp > 0.0 ? rsqrt(rp) : 0.0;
          const double nrm = rp * rin;
          const bool take = nrm > thr;
          accb[s] = take ? 1 : 0;
          Gb[s * QB + s] = make_double2(take ? nrm : 0.0, 0.0);
          dvec[3 * QB + s] = take ? rin : 0.0;
        }
      }
      __syncthreads();
      if (sint[1]) break;
      const bool take = accb[s] != 0;
      const double inv = dvec[3 * QB + s];
      // row s of R: R_st = G'_st / R_ss (t > s); rows of skipped columns are zero
      if ((int)threadIdx.x > s && (int)threadIdx.x < bsz) {
        const cplx g = Gb[s * QB + threadIdx.x];
        Gb[s * QB + threadIdx.x] = take ? make_double2(g.x * inv, g.y * inv) : make_double2(0.0, 0.0);
      }
      __syncthreads();
      // trailing update G'_tu -= conj(R_st) R_su for s < t <= u
      if (take) {
        const int t = threadIdx.x / QB, u = threadIdx.x % QB;
        if (t > s && u >= t && u < bsz) {
          const cplx a = Gb[s * QB + t], b = Gb[s * QB + u];
          Gb[t * QB + u] = make_double2(Gb[t * QB + u].x - (a.x * b.x + a.y * b.y),
                                        Gb[t * QB + u].y - (a.x * b.y - a.y * b.x));
        }
      }
      __syncthreads();
    }
    const int done = sint[0];
    // ---- form the accepted columns locally: q_t = (v_t - sum_{s<t} q_s R_st) / R_tt
    for (int r = threadIdx.x; r < nr; r += T) {
      for (int t = 0; t < done; ++t) {
        if (!accb[t]) continue;
        double x = vb[t * rows + r].x, y = vb[t * rows + r].y;
        for (int s = 0; s < t; ++s) {
          if (!accb[s]) continue;
          const cplx q = vb[s * rows + r], c = Gb[s * QB + t];
          x -= q.x * c.x - q.y * c.y;
          y -= q.x * c.y + q.y * c.x;
        }
        const double inv = dvec[3 * QB + t];
        const cplx qt = make_double2(x * inv, y * inv);
        vb[t * rows + r] = qt;
        A.Q[(long long)(r0 + r) * n + j0 + t] = qt;
      }
    }
    if (blockIdx.x == 0) {
      for (int e = threadIdx.x; e < done * done; e += T) {
        const int s = e / done, t = e % done;
        if (s <= t) A.R[(long long)(j0 + s) * n + j0 + t] = Gb[s * QB + t];
      }
    }
    __syncthreads();
    for (int t = threadIdx.x; t < done; t += T) acc[j0 + t] = accb[t];
    __syncthreads();
    j0 += done;
  }
  if (blockIdx.x == 0)
    for (int i = threadIdx.x; i < n; i += T) A.acc_out[i] = acc[i];
}

static bool g_qb_attr = false;

int gauge_qr_blocked_grid(int m) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int g = (m + 3) / 4;
  if (g > sms) g = sms;
  if (g < 1) g = 1;
  return g;
}

long long gauge_qr_blocked_scratch(int n, int gmax) {
  const long long PS = (long long)n * QB + QB + QB * QB;
  return (long long)gmax * PS + PS;      // complex entries (partials of every CTA + reduced)
}

cudaError_t gauge_qr_blocked(int m, int n, QrRef Y, int p, QrRef E, cplx* Q, cplx* R,
                             cplx* scratch, long long scratch_len, unsigned char* acc,
                             const QrScratch& W, int* status, cudaStream_t s, int gcap,
                             double rank_tol, int* src) {
  int G = gauge_qr_blocked_grid(m);
  if (gcap > 0 && G > gcap) G = gcap;
  const long long PS = (long long)n * QB + QB + QB * QB;
  if ((long long)G * PS + PS > scratch_len) return cudaErrorInvalidValue;
  const int rows = (m + G - 1) / G;
  const size_t smem = (size_t)QB * rows * sizeof(cplx) + (size_t)n * QB * sizeof(cplx) +
                      QB * QB * sizeof(cplx) + (4 * QB + 8) * sizeof(double) + (size_t)n + QB +
                      64;
  if (smem > 200 * 1024)
    return gauge_qr(m, n, Y, p, E, Q, R, W, status, s, gcap, rank_tol, src);
  if (!g_qb_attr) {
    cudaError_t e = cudaFuncSetAttribute(gauge_qr_blocked_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (e != cudaSuccess) return e;
    g_qb_attr = true;
  }
  cudaError_t e = cudaMemsetAsync(W.bar, 0, 2 * sizeof(unsigned), s);
  if (e != cudaSuccess) return e;
  QbArgs a;
  a.m = m; a.n = n; a.Y = Y; a.Q = Q; a.R = R;
  a.part = scratch; a.fin = scratch + (long long)G * PS; a.PS = (int)PS;
  a.bar = W.bar; a.status = status; a.acc_out = acc; a.rank_tol = rank_tol;
  a.wait = W.wait > 0 ? W.wait : kBarrierWaitCycles;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(G);
  cfg.blockDim = dim3(QB_THREADS);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  count_launch();
  e = cudaLaunchKernelEx(&cfg, gauge_qr_blocked_kernel, a);
  if (e != cudaSuccess) return e;
  // completion of skipped positions (only when some column was skipped: decided on device)
  return gauge_qr_complete(m, n, p, p > 0 ? E : Y, Q, acc, W, status, s, gcap, src);
}

}  // namespace tdmrg
