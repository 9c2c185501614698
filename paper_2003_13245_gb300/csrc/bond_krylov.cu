// Fused bond exponential of the mixed-precision path: out = exp(tau K) C for the bond
// operator K C = sum_w L_w C R_w^T (the zero-site term of the projector-splitting step,
// Eq. S1), the whole Lanczos run in one cooperative launch.
//
// Why one launch: a bond matrix holds M^2 elements (16384 at M = 128), so each step of the
// host-driven Lanczos -- two contractions, four Gram-Schmidt kernels, a norm, the small
// exponential and the host's poll of the stop flag -- lasts a few microseconds and the
// chain of launches sets the pace.  Here the grid synchronises through a bounded barrier
// five times per Krylov vector and never returns to the host.
//
// Per Krylov vector j (CTA g owns the contiguous slice [g*S, g*S + S) of every vector):
//  A.  T_w = L_w q_j for every channel w: complex FP32 FMA on 32 x 32 output tiles with the
//      whole K = M extent staged in shared memory (M <= 256; the contraction is 2 Dw M^3
//      complex MACs, too small to keep a tensor-core pipeline busy);
//  B.  P_w = T_w R_w^T, one partial per channel (the channel sum is taken in C1, in order);
//  C1. w = sum_w P_w in FP64 on the own slice; partial dots against q_{j-1}, q_j;
//  C2. first projection; partial dots against q_0 .. q_j (second, full pass);
//  C3. second projection; partial ||w||^2;
//  C4. every CTA sums the same partials in the same order and runs the same small
//      exponential on one warp, so all reach the same result and the same stop decision
//      without a broadcast; otherwise q_{j+1} = w / beta_{j+1} on the own slice.
// Precision follows the mixed path: the contractions in complex FP32 (FMA, 24-bit
// significands: no coarser than the 3xTF32 tensor-core products), every Lanczos quantity,
// the small exponential and all norms in FP64.  All reductions have a fixed order: the
// result does not depend on timing.
#include "lanczos_coop.cuh"

namespace tdmrg {

namespace {

constexpr int BT = 256;                 // threads per CTA
constexpr int TL = 32;                  // output tile edge and k chunk
constexpr int TP = TL + 2;              // padded row (16-byte aligned float2 pairs)
using lzc::NV;

struct BondArgs {
  int M, Dw, G, S, kcap, fixed;
  long long n;
  const cplx* L;       // [Dw][M][M]
  const cplx* R;       // [Dw][M][M]
  const cplx* v;       // [M][M]
  cplx* out;           // [M][M]
  cplx* V;             // kcap vectors of n
  cplx* W;             // n: the projected, unnormalised new vector
  float2* T;           // [Dw][n]
  float2* P;           // [Dw][n]
  cplx* part;          // 2 * G * NV
  double* partn;       // G
  unsigned* bar;
  int* status;
  long long wait;      // grid-barrier wait limit (clock cycles)
  unsigned long long* mv;
  double tr, ti, tol;
};

__device__ __forceinline__ void cfma32(float2& acc, float2 a, float2 b) {
  acc.x = fmaf(a.x, b.x, acc.x);
  acc.x = fmaf(-a.y, b.y, acc.x);
  acc.y = fmaf(a.x, b.y, acc.y);
  acc.y = fmaf(a.y, b.x, acc.y);
}

constexpr int KT = BOND_EXP_MAX_M;      // largest K staged at once (bond dimension)
constexpr size_t TILE_SMEM = 2 * (size_t)KT * TP * sizeof(float2);

// acc[i][j] += sum_{k < K} A(r0 + i, k) B(k, c0 + j) for the thread's 2 x 2 outputs
// (r0 = 2 (tid / 16), c0 = 2 (tid % 16)) of a 32 x 32 tile.  The whole K extent (<= KT,
// zero-padded to a multiple of 32) is staged in shared memory at once -- at[k][row] (A
// transposed) and b[k][col] -- so that one round of loads is in flight per tile.  ldA(r, k)
// / ldB(k, c) return the operand (zero outside the matrices); kfastB selects the load order
// of B that is contiguous in global memory.
template <bool kfastB, class FA, class FB>
__device__ __forceinline__ void tile_cgemm(int K, FA ldA, FB ldB, float2* at, float2* bt,
                                           float2 acc[2][2]) {
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int nk = (K + TL - 1) / TL;
  for (int c0 = 0; c0 < nk; c0 += 2) {
    float2 ra[2][4], rb[2][4];
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int e = tid + u * BT;
        const int r = e >> 5, kk = e & 31, k0 = (c0 + c) * TL;
        const bool live = c0 + c < nk;
        ra[c][u] = live ? ldA(r, k0 + kk) : make_float2(0.f, 0.f);
        rb[c][u] = live ? (kfastB ? ldB(k0 + kk, r) : ldB(k0 + r, kk)) : make_float2(0.f, 0.f);
      }
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int e = tid + u * BT;
        const int r = e >> 5, kk = e & 31, k0 = (c0 + c) * TL;
        if (c0 + c < nk) {
          at[(k0 + kk) * TP + r] = ra[c][u];
          if (kfastB)
            bt[(k0 + kk) * TP + r] = rb[c][u];      // (k fast, c = e / 32)
          else
            bt[(k0 + r) * TP + kk] = rb[c][u];      // (c fast, k = e / 32)
        }
      }
  }
  __syncthreads();
  const int kend = nk * TL;
#pragma unroll 8
  for (int kk = 0; kk < kend; ++kk) {
    const float4 a = *reinterpret_cast<const float4*>(&at[kk * TP + 2 * ty]);
    const float4 b = *reinterpret_cast<const float4*>(&bt[kk * TP + 2 * tx]);
    const float2 a0 = make_float2(a.x, a.y), a1 = make_float2(a.z, a.w);
    const float2 b0 = make_float2(b.x, b.y), b1 = make_float2(b.z, b.w);
    cfma32(acc[0][0], a0, b0);
    cfma32(acc[0][1], a0, b1);
    cfma32(acc[1][0], a1, b0);
    cfma32(acc[1][1], a1, b1);
  }
  __syncthreads();
}

__device__ __forceinline__ float2 to_f2(cplx z) {
  return make_float2(__double2float_rn(z.x), __double2float_rn(z.y));
}

__global__ void __launch_bounds__(BT, 1) bond_exp_kernel(BondArgs A) {
  extern __shared__ __align__(16) unsigned char dyn[];
  float2* at = reinterpret_cast<float2*>(dyn);        // [KT][TP]
  float2* bt = at + (size_t)KT * TP;                  // [KT][TP]
  cplx* ws = reinterpret_cast<cplx*>(dyn + TILE_SMEM);   // own slice of w, S entries
  unsigned epoch = 0;
  __shared__ cplx h1[NV], h2[NV], cc[KMAX];
  __shared__ double alpha[KMAX], beta[KMAX + 1], red[BT / 32];
  __shared__ double s_nrm, s_b0, s_scale;
  __shared__ int s_done, s_k, s_second;

  const int M = A.M, Dw = A.Dw;
  const long long n = A.n;
  const long long e0 = (long long)blockIdx.x * A.S;
  const int len = (int)(e0 < n ? (n - e0 < A.S ? n - e0 : A.S) : 0);
  const int nt = (M + TL - 1) / TL;
  const int items = Dw * nt * nt;
  cplx* part1 = A.part;
  cplx* part2 = A.part + (size_t)A.G * NV;

  // ||v||: q_0 = v / ||v||
  for (int e = threadIdx.x; e < len; e += BT) ws[e] = A.v[e0 + e];
  __syncthreads();
  lzc::slice_norm(ws, len, red, A.partn);
  if (!lzc::barrier(A.bar, A.G, epoch, A.status, A.wait)) return;
  lzc::reduce_norm(A.partn, A.G, &s_nrm);
  const double b0 = sqrt(s_nrm);
  if (threadIdx.x == 0) {
    s_b0 = b0;
    s_done = 0;
    s_k = 0;
  }
  if (b0 == 0.0) {
    for (int e = threadIdx.x; e < len; e += BT) A.out[e0 + e] = make_double2(0.0, 0.0);
    return;
  }
  double inv = 1.0 / b0;
  for (int e = threadIdx.x; e < len; e += BT)
    A.V[e0 + e] = make_double2(ws[e].x * inv, ws[e].y * inv);
  const cplx* src = A.v;        // q_j = src * inv (src is read by every CTA)

  int k = 0;
  for (int j = 0; j < A.kcap; ++j) {
    // ---- A: T_w = L_w q_j
    for (int it = blockIdx.x; it < items; it += A.G) {
      const int w = it / (nt * nt), rem = it - w * nt * nt;
      const int ra = (rem / nt) * TL, cb = (rem % nt) * TL;
      const cplx* Lw = A.L + (size_t)w * M * M;
      const double sc = inv;
      float2 acc[2][2] = {};
      tile_cgemm<false>(
          M,
          [&](int r, int kk) {
            const int a = ra + r;
            return (a < M && kk < M) ? to_f2(__ldg(&Lw[(size_t)a * M + kk]))
                                     : make_float2(0.f, 0.f);
          },
          [&](int kk, int c) {
            const int b = cb + c;
            if (kk >= M || b >= M) return make_float2(0.f, 0.f);
            const cplx z = __ldcg(&src[(size_t)kk * M + b]);
            return make_float2(__double2float_rn(z.x * sc), __double2float_rn(z.y * sc));
          },
          at, bt, acc);
      const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
      float2* Tw = A.T + (size_t)w * n;
#pragma unroll
      for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int jj = 0; jj < 2; ++jj) {
          const int a = ra + 2 * ty + i, b = cb + 2 * tx + jj;
          if (a < M && b < M) Tw[(size_t)a * M + b] = acc[i][jj];
        }
    }
    if (!lzc::barrier(A.bar, A.G, epoch, A.status, A.wait)) return;
    // ---- B: P_w = T_w R_w^T
    for (int it = blockIdx.x; it < items; it += A.G) {
      const int w = it / (nt * nt), rem = it - w * nt * nt;
      const int ra = (rem / nt) * TL, cb = (rem % nt) * TL;
      const float2* Tw = A.T + (size_t)w * n;
      const cplx* Rw = A.R + (size_t)w * M * M;
      float2 acc[2][2] = {};
      tile_cgemm<true>(
          M,
          [&](int r, int kk) {
            const int a = ra + r;
            return (a < M && kk < M) ? __ldcg(&Tw[(size_t)a * M + kk]) : make_float2(0.f, 0.f);
          },
          [&](int kk, int c) {
            const int b = cb + c;
            return (kk < M && b < M) ? to_f2(__ldg(&Rw[(size_t)b * M + kk]))
                                     : make_float2(0.f, 0.f);
          },
          at, bt, acc);
      const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
      float2* Pw = A.P + (size_t)w * n;
#pragma unroll
      for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int jj = 0; jj < 2; ++jj) {
          const int a = ra + 2 * ty + i, b = cb + 2 * tx + jj;
          if (a < M && b < M) Pw[(size_t)a * M + b] = acc[i][jj];
        }
    }
    if (!lzc::barrier(A.bar, A.G, epoch, A.status, A.wait)) return;
    // ---- C1: w = sum_w P_w (FP64, channel order); dots against q_lo .. q_j
    for (int e = threadIdx.x; e < len; e += BT) {
      double x = 0.0, y = 0.0;
      for (int w = 0; w < Dw; ++w) {
        const float2 p = __ldcg(&A.P[(size_t)w * n + e0 + e]);
        x += (double)p.x;
        y += (double)p.y;
      }
      ws[e] = make_double2(x, y);
    }
    __syncthreads();
    const int lo = j > 0 ? j - 1 : 0;
    lzc::slice_dots(A.V, n, ws, e0, len, lo, j + 1, part1);
    lzc::slice_norm(ws, len, red, A.partn + A.G);     // ||w||^2 before the projection
    if (!lzc::barrier(A.bar, A.G, epoch, A.status, A.wait)) return;
    // ---- C2: first projection; then, only if it cancelled more than half of ||w||^2
    // (the criterion of Daniel, Gragg, Kaufman and Stewart), the second one against q_0 .. q_j
    lzc::reduce_dots(part1, A.G, lo, j + 1, h1);
    lzc::reduce_norm(A.partn + A.G, A.G, &s_nrm);
    lzc::slice_project(A.V, n, ws, e0, len, lo, j + 1, h1);
    if (threadIdx.x == 0) {
      double rem = s_nrm;
      for (int i = lo; i <= j; ++i) rem -= h1[i].x * h1[i].x + h1[i].y * h1[i].y;
      s_second = (rem < 0.5 * s_nrm) ? 1 : 0;
    }
    __syncthreads();
    if (s_second) {
      lzc::slice_dots(A.V, n, ws, e0, len, 0, j + 1, part2);
      if (!lzc::barrier(A.bar, A.G, epoch, A.status, A.wait)) return;
      // ---- C3: second projection
      lzc::reduce_dots(part2, A.G, 0, j + 1, h2);
      lzc::slice_project(A.V, n, ws, e0, len, 0, j + 1, h2);
    } else {
      for (int i = threadIdx.x; i <= j; i += blockDim.x) h2[i] = make_double2(0.0, 0.0);
      __syncthreads();
    }
    // ---- ||w||^2
    for (int e = threadIdx.x; e < len; e += BT) A.W[e0 + e] = ws[e];
    lzc::slice_norm(ws, len, red, A.partn);
    if (!lzc::barrier(A.bar, A.G, epoch, A.status, A.wait)) return;
    // ---- C4: tridiagonal bookkeeping and the small exponential (warp 0 of every CTA)
    lzc::reduce_norm(A.partn, A.G, &s_nrm);
    if (threadIdx.x < 32) {
      const int lane = threadIdx.x;
      double yr, yi, err;
      bool done, bd;
      lzc::tridiag_step(j, h1[j].x + h2[j].x, s_nrm, A.tr, A.ti, A.tol, A.kcap, A.fixed, alpha,
                        beta, true, yr, yi, done, err, bd);
      if (done && lane <= j) cc[lane] = make_double2(s_b0 * yr, s_b0 * yi);
      if (lane == 0) {
        s_done = done ? 1 : 0;
        s_k = j + 1;
        s_scale = sqrt(s_nrm);
      }
    }
    __syncthreads();
    k = s_k;
    if (s_done) break;
    inv = 1.0 / s_scale;
    for (int e = threadIdx.x; e < len; e += BT)
      A.V[(size_t)(j + 1) * n + e0 + e] = make_double2(ws[e].x * inv, ws[e].y * inv);
    src = A.W;
  }
  // out = sum_{i < k} c_i q_i on the own slice
  for (int e = threadIdx.x; e < len; e += BT) {
    double x = 0.0, y = 0.0;
    for (int i = 0; i < k; ++i) {
      const cplx q = A.V[(size_t)i * n + e0 + e], c = cc[i];
      x = fma(c.x, q.x, x);
      x = fma(-c.y, q.y, x);
      y = fma(c.x, q.y, y);
      y = fma(c.y, q.x, y);
    }
    A.out[e0 + e] = make_double2(x, y);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0 && A.mv) atomicAdd(A.mv, (unsigned long long)k);
}

}  // namespace

int bond_exp_grid(int M, int Dw, int gcap, int sms) {
  const int nt = (M + TL - 1) / TL;
  const long long n = (long long)M * M;
  long long g = (long long)Dw * nt * nt;
  const long long gn = (n + BT - 1) / BT;
  if (gn > g) g = gn;
  int cap = sms;
  if (gcap > 0 && gcap < cap) cap = gcap;
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  return (int)g;
}

size_t bond_exp_smem(int M, int G) {
  const long long n = (long long)M * M;
  const long long S = (n + G - 1) / G;
  return TILE_SMEM + (size_t)S * sizeof(cplx);
}

cudaError_t bond_exp_fused(int M, int Dw, const cplx* L, const cplx* R, const cplx* C, cplx* out,
                           cplx* V, const BondScratch& W, int* status, double tr, double ti,
                           double tol, int kcap, int fixed, int gcap, cudaStream_t s) {
  if (M < 1 || M > KT || Dw < 1 || Dw > W.maxDw || (long long)M * M > W.maxn || kcap < 1 ||
      kcap > KMAX)
    return cudaErrorInvalidValue;
  const int G = bond_exp_grid(M, Dw, gcap, W.gmax);
  const size_t smem = bond_exp_smem(M, G);
  if (smem > BOND_EXP_MAX_SMEM) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(bond_exp_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)BOND_EXP_MAX_SMEM);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(W.bar, 0, 2 * sizeof(unsigned), s);
  if (e != cudaSuccess) return e;
  BondArgs a;
  a.M = M; a.Dw = Dw; a.G = G;
  a.n = (long long)M * M;
  a.S = (int)((a.n + G - 1) / G);
  a.kcap = kcap; a.fixed = fixed;
  a.L = L; a.R = R; a.v = C; a.out = out; a.V = V;
  a.W = W.W; a.T = W.T; a.P = W.P; a.part = W.part; a.partn = W.partn; a.bar = W.bar;
  a.status = status; a.mv = W.mv;
  a.wait = W.wait > 0 ? W.wait : kBarrierWaitCycles;
  a.tr = tr; a.ti = ti; a.tol = tol;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(G);
  cfg.blockDim = dim3(BT);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  count_launch();
  return cudaLaunchKernelEx(&cfg, bond_exp_kernel, a);
}

}  // namespace tdmrg
