// One orthogonalisation step of the host-driven Lanczos exponential (the site update of the
// projector-splitting step, Eq. S1) in one cooperative launch.  Given w = H_eff q_j (stored
// as Krylov vector j+1), the launch takes the three-term pass against q_{j-1}, q_j, the full
// re-orthogonalisation pass against q_0 .. q_j, the norm, the tridiagonal bookkeeping with the
// small exponential and the stopping test, and scales w into q_{j+1} -- work that took seven
// launches (dots, projection, dots, projection, norm, small exponential, scaling).  Every
// quantity is FP64.  CTA g owns a contiguous slice of the vectors; three bounded grid barriers
// separate the two passes and the norm; every CTA evaluates the same reductions in the same
// order, and CTA 0 records the results in the Lanczos state (the layout the host-driven
// kernels use, so the final combination and the host's stop-flag poll are unchanged).
#include "lanczos_coop.cuh"

namespace tdmrg {

namespace {

constexpr int LT = 512;                 // 16 warps per SM to cover FP64 load latency
using lzc::NV;

struct LzStepArgs {
  long long n;
  int j, G, S, kcap, fixed;
  cplx* V;           // q_0 .. q_j, and w = H q_j as vector j+1
  LzState* st;
  cplx* part;        // 2 * G * NV
  double* partn;     // G
  unsigned* bar;
  int* status;
  long long wait;    // grid-barrier wait limit (clock cycles)
  int* noconv;       // sticky flag of unconverged runs (may be NULL)
  double tr, ti, tol;
};

__global__ void __launch_bounds__(LT) lz_step_kernel(LzStepArgs A) {
  LzState* S = A.st;
  // converged in an earlier launch (the host queues one step ahead of its poll)
  if (*reinterpret_cast<volatile int*>(&S->done)) return;
  __shared__ cplx h1[NV], h2[NV];
  __shared__ double red[8 * (LT / 32)];
  __shared__ double alpha[KMAX], beta[KMAX + 1];
  __shared__ double s_nrm, s_inv;
  __shared__ int s_done, s_second;
  const long long n = A.n;
  const int j = A.j;
  const long long e0 = (long long)blockIdx.x * A.S;
  const int len = (int)(e0 < n ? (n - e0 < A.S ? n - e0 : A.S) : 0);
  cplx* w = A.V + (size_t)(j + 1) * n + e0;
  cplx* part1 = A.part;
  cplx* part2 = A.part + (size_t)A.G * NV;
  unsigned epoch = 0;
  for (int i = threadIdx.x; i < j; i += blockDim.x) alpha[i] = __ldcg(&S->alpha[i]);
  for (int i = threadIdx.x; i <= j; i += blockDim.x) beta[i] = i > 0 ? __ldcg(&S->beta[i]) : 0.0;

  const int lo = j > 0 ? j - 1 : 0;
  lzc::slice_dots_block(A.V, n, w, e0, len, lo, j + 1, part1, red);
  lzc::slice_norm(w, len, red, A.partn + A.G);      // ||w||^2 before the projection
  if (!lzc::barrier(A.bar, A.G, epoch, A.status, A.wait)) return;
  lzc::reduce_dots(part1, A.G, lo, j + 1, h1);
  lzc::reduce_norm(A.partn + A.G, A.G, &s_nrm);
  lzc::slice_project(A.V, n, w, e0, len, lo, j + 1, h1);
  // Re-orthogonalisation against every Krylov vector only when the three-term projection
  // removed more than half of ||w||^2 (the criterion of Daniel, Gragg, Kaufman and Stewart):
  // without such cancellation w stays orthogonal to the basis to rounding.  The decision is
  // taken from grid-wide reduced values, so every CTA takes the same branch.
  if (threadIdx.x == 0) {
    double rem = s_nrm;
    for (int i = lo; i <= j; ++i) rem -= h1[i].x * h1[i].x + h1[i].y * h1[i].y;
    s_second = (rem < 0.5 * s_nrm) ? 1 : 0;
  }
  __syncthreads();
  if (s_second) {
    lzc::slice_dots_block(A.V, n, w, e0, len, 0, j + 1, part2, red);
    if (!lzc::barrier(A.bar, A.G, epoch, A.status, A.wait)) return;
    lzc::reduce_dots(part2, A.G, 0, j + 1, h2);
    lzc::slice_project(A.V, n, w, e0, len, 0, j + 1, h2);
  } else {
    for (int i = threadIdx.x; i <= j; i += blockDim.x) h2[i] = make_double2(0.0, 0.0);
    __syncthreads();
  }
  lzc::slice_norm(w, len, red, A.partn);
  if (!lzc::barrier(A.bar, A.G, epoch, A.status, A.wait)) return;
  lzc::reduce_norm(A.partn, A.G, &s_nrm);
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    const double aj = h1[j].x + h2[j].x;          // alpha_j = Re <q_j, H q_j>
    double yr, yi, err;
    bool done, bd;
    lzc::tridiag_step(j, aj, s_nrm, A.tr, A.ti, A.tol, A.kcap, A.fixed, alpha, beta, false, yr,
                      yi, done, err, bd);
    const double nb = sqrt(s_nrm);
    if (blockIdx.x == 0) {
      if (lane == 0) {
        S->h1[j] = h1[j];
        S->h2[j] = h2[j];
        S->alpha[j] = aj;
        S->beta[j + 1] = nb;
        S->nrm2 = s_nrm;
      }
      if (done) {
        const double b0 = __ldcg(&S->b0);
        if (lane <= j) S->c[lane] = make_double2(b0 * yr, b0 * yi);
        if (lane == 0) {
          S->k = j + 1;
          S->err = err;
          S->noconv = (!bd && !A.fixed && err > 1e3 * A.tol) ? 1 : 0;
          if (S->noconv && A.noconv) atomicExch(A.noconv, 1);
          __threadfence();
          S->done = 1;
        }
      } else if (lane == 0) {
        S->inv = 1.0 / nb;
      }
    }
    if (lane == 0) {
      s_done = done ? 1 : 0;
      s_inv = done ? 0.0 : 1.0 / nb;
    }
  }
  __syncthreads();
  if (!s_done) {
    const double f = s_inv;
    for (int e = threadIdx.x; e < len; e += blockDim.x) w[e] = make_double2(w[e].x * f, w[e].y * f);
  }
}

}  // namespace

cudaError_t lz_step(long long n, int j, cplx* V, LzState* S, const BondScratch& W, int* status,
                    double tr, double ti, double tol, int kcap, int fixed, int gcap,
                    cudaStream_t s) {
  if (n < 1 || j < 0 || j >= KMAX || kcap < 1 || kcap > KMAX || !W.part || !W.bar)
    return cudaErrorInvalidValue;
  long long g = (n + 255) / 256;           // every SM's FP64 pipe once n >= 256 per SM
  int cap = W.gmax;
  if (gcap > 0 && gcap < cap) cap = gcap;
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  cudaError_t e = cudaMemsetAsync(W.bar, 0, 2 * sizeof(unsigned), s);
  if (e != cudaSuccess) return e;
  LzStepArgs a;
  a.n = n; a.j = j; a.G = (int)g;
  a.S = (int)((n + g - 1) / g);
  a.kcap = kcap; a.fixed = fixed;
  a.V = V; a.st = S; a.part = W.part; a.partn = W.partn; a.bar = W.bar; a.status = status;
  a.wait = W.wait > 0 ? W.wait : kBarrierWaitCycles;
  a.noconv = W.noconv;
  a.tr = tr; a.ti = ti; a.tol = tol;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)g);
  cfg.blockDim = dim3(LT);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  count_launch();
  return cudaLaunchKernelEx(&cfg, lz_step_kernel, a);
}

}  // namespace tdmrg
