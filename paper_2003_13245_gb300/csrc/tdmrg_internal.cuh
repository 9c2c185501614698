// Internal declarations shared by the CUDA translation units of libtdmrg.
// Complex numbers are double2 {re, im} (FP64 path); every tensor is row-major.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>

namespace tdmrg {

typedef double2 cplx;

constexpr int KMAX = 32;            // largest Krylov dimension

// message returned by tdmrg_last_global_error() (set by entry points that have no handle)
void set_global_error(const char* msg);

// number of kernels this library has launched (host-side counter)
long long launch_count();
void count_launch(int n = 1);

// Strided view of a matrix operand: element (i, j) = p[i * rs + j * cs] (conjugated if conj),
// batch b / reduction term r shift the pointer by b * sb + r * sr.
struct MatRef {
  const cplx* p;
  long long rs, cs, sb, sr;
  int conj;
};

// C_b = alpha * sum_{r < nred} op(A_{b,r}) op(B_{b,r}) + beta * C_b, b < nbatch.
// C row-major with leading dimension ldc and batch stride sc.
cudaError_t zgemm(int m, int n, int k, int nbatch, int nred, cplx alpha, MatRef A, MatRef B,
                  cplx beta, cplx* C, long long ldc, long long sc, const int* skip,
                  cudaStream_t s);

// Sparse MPO mixing over the channel and the physical (P) level of a site:
// Y[wo][a][s][t][b] = sum_{blocks of wo} sum_u op[s][u] X[wi][a][u][t][b].
struct MixTable {
  int Dout;
  const int* start;      // Dout + 1
  const int* chan;       // input channel of each block
  const cplx* ops;       // d x d per block
  const float2* ops32;   // the same operators rounded to FP32 (mixed-precision path)
  int nblk;
};
cudaError_t mpo_mix(const MixTable& T, int Ma, int d, int Mb, const cplx* X, long long xs,
                    cplx* Y, long long ys, const int* skip, cudaStream_t s);

// Lanczos scalars living on the device.
struct LzState {
  cplx h1[KMAX + 1];
  cplx h2[KMAX + 1];
  double alpha[KMAX];
  double beta[KMAX + 1];
  cplx c[KMAX];
  double nrm2;
  double b0;
  double inv;
  double err;
  int k;
  int done;
  int noconv;
  int pad;
};

// *out = sum |x|^2 (one launch; partial: 304 entries, counter: one zero-initialised ticket)
cudaError_t znorm2(long long n, const cplx* x, double* out, double* partial, unsigned* counter,
                   const int* skip, cudaStream_t s);
cudaError_t zscale_by(long long n, cplx* x, const double* factor, const int* skip,
                      cudaStream_t s);
// x /= sqrt(*nrm2) and *logacc += log(*nrm2) (no host round trip)
cudaError_t znormalize_log(long long n, cplx* x, const double* nrm2, double* logacc,
                           cudaStream_t s);
cudaError_t lz_start(LzState* S, const double* nrm2, cudaStream_t s);
cudaError_t zcombine(long long n, const LzState* S, const cplx* V, long long ldv, cplx* out,
                     cudaStream_t s);

// Gauge QR (cooperative kernel). Y(r, c) and E(r, c) are read through the refs; E columns are
// split in blocks: E(r, c) = p[r*rs + (c % cb) * cs + (c / cb) * cbs].
struct QrRef {
  const cplx* p;
  long long rs, cs, cb, cbs;
  int conj;
};
// Fused bond exponential (bond_krylov.cu): out = exp(tau K) C, K C = sum_w L_w C R_w^T, the
// whole Lanczos run in one cooperative launch (complex FP32 contractions, FP64 Lanczos).
struct BondScratch {
  cplx* W = nullptr;                 // maxn
  float2* T = nullptr;               // maxDw * maxn
  float2* P = nullptr;               // maxDw * maxn
  cplx* part = nullptr;              // 2 * gmax * (KMAX + 1)
  double* partn = nullptr;           // 2 * gmax (lz_step: the norms before and after)
  unsigned* bar = nullptr;           // 2 (barrier counter, generation)
  unsigned long long* mv = nullptr;  // Krylov vectors used, accumulated over launches
  long long maxn = 0;
  int maxDw = 0, gmax = 0;
  long long wait = 0;                // grid-barrier wait limit in clock cycles (0: ~2 s)
  int* noconv = nullptr;             // lz_step: set to 1 when a Krylov run stops unconverged
};
// One orthogonalisation step of the host-driven Lanczos (lanczos_step.cu): w = V[j+1] holds
// H q_j; both Gram-Schmidt passes, the norm, the small exponential, the stop test and the
// scaling into q_{j+1} in one cooperative launch (part, partn, bar of W are used).
cudaError_t lz_step(long long n, int j, cplx* V, LzState* S, const BondScratch& W, int* status,
                    double tr, double ti, double tol, int kcap, int fixed, int gcap,
                    cudaStream_t s);
constexpr int BOND_EXP_MAX_M = 256;
constexpr size_t BOND_EXP_MAX_SMEM = 200 * 1024;
int bond_exp_grid(int M, int Dw, int gcap, int sms);
size_t bond_exp_smem(int M, int G);
cudaError_t bond_exp_fused(int M, int Dw, const cplx* L, const cplx* R, const cplx* C, cplx* out,
                           cplx* V, const BondScratch& W, int* status, double tr, double ti,
                           double tol, int kcap, int fixed, int gcap, cudaStream_t s);

struct QrScratch {
  cplx* part = nullptr;       // 2 * gmax * (nmax + 1)
  double* partn = nullptr;    // 2 * gmax
  unsigned* bar = nullptr;    // 2
  int gmax = 0;
  int nmax = 0;
  long long wait = 0;         // grid-barrier wait limit in clock cycles (0: ~2 s)
};
// the default limit of every bounded grid-barrier wait: about 2 s at 2 GHz
constexpr long long kBarrierWaitCycles = 4000000000LL;
// gcap > 0 caps the cooperative grid (several QRs of concurrent instances can then co-reside)
cudaError_t gauge_qr(int m, int n, QrRef Y, int p, QrRef E, cplx* Q, cplx* R,
                     const QrScratch& W, int* status, cudaStream_t s, int gcap = 0,
                     double rank_tol = 1e-12, int* src = nullptr);
int gauge_qr_grid(int m);
// dynamic shared memory of the column-wise QR on a grid of G blocks (each block stages its
// ceil(m / G) rows); launches above kQrMaxSmem are refused
constexpr size_t kQrMaxSmem = 200 * 1024;
size_t gauge_qr_smem(int m, int n, int G);
// completion pass only (skipped positions of a factorisation whose accepted flags are `acc`);
// if src is not NULL, src[j] receives the candidate that filled completed position j (i < p:
// column i of E, p + i: unit vector e_i; other entries untouched)
cudaError_t gauge_qr_complete(int m, int n, int p, QrRef E, cplx* Q, const unsigned char* acc,
                              const QrScratch& W, int* status, cudaStream_t s, int gcap = 0,
                              int* src = nullptr);
// blocked variant (16 columns per block); scratch: gauge_qr_blocked_scratch(n, gmax) complex
// entries and n accepted flags; W supplies the barrier and the completion pass' scratch.  When a
// block's row slice and coefficients do not fit its shared memory (very tall or wide factors on
// a capped grid) the column-wise kernel does the factorisation instead.
long long gauge_qr_blocked_scratch(int n, int gmax);
cudaError_t gauge_qr_blocked(int m, int n, QrRef Y, int p, QrRef E, cplx* Q, cplx* R,
                             cplx* scratch, long long scratch_len, unsigned char* acc,
                             const QrScratch& W, int* status, cudaStream_t s, int gcap = 0,
                             double rank_tol = 1e-12, int* src = nullptr);

// dst[j][i] = conj?(src[i][j]) for an m x n source.
cudaError_t ztranspose(int m, int n, const cplx* src, cplx* dst, int conj, cudaStream_t s);
// FP64 FMA throughput probe: blocks x 256 threads x 8 chains x iters FMAs, results to sink
// (blocks * 256 doubles)
cudaError_t dfma_loop(int blocks, long long iters, double* sink, cudaStream_t s);
// hopping-limit mobility of Eq. 7 for P parameter sets (device arrays omega[P K], g[P K],
// V[P], kT[P] -> mu[P]); K <= 64 (fgr.cu)
cudaError_t fgr_mobility(int P, int K, const double* omega, const double* g, const double* V,
                         const double* kT, double dt, int nt, double* mu, cudaStream_t s);
// G[w][v][s][u] += k sum_{x,t,c} U[w][x][u][t][c] V[v][x][s][t][c] (Dl x Dr x d x d, d <= 16):
// the parameter cotangent of a site operator from U = L b and V = conj(a) R (kernels_f64.cu)
cudaError_t param_gram(int Dl, int Dr, int Ml, int d, int Mr, const cplx* U, const cplx* V,
                       cplx k, cplx* G, cudaStream_t s);
// *out = trace of the M x M matrix E (one launch)
cudaError_t ztrace(const cplx* E, int M, cplx* out, cudaStream_t s);
// x <- conj(x)
cudaError_t zconj(long long n, cplx* x, cudaStream_t s);
// y <- y + alpha x
cudaError_t zaxpy(long long n, cplx alpha, const cplx* x, cplx* y, cudaStream_t s);
// QR VJP helpers: S = Hermitian fold of the strictly lower triangle of M with Re diag;
// X R^H = B row by row (R upper triangular); zero the strictly lower triangle in place
cudaError_t herm_lower(int n, const cplx* M, cplx* S, cudaStream_t s);
cudaError_t solve_rh(int m, int n, const cplx* R, const cplx* B, cplx* X, cudaStream_t s);
cudaError_t triu_inplace(int n, cplx* A, cudaStream_t s);
cudaError_t zfill_identity_mps(cplx* A, int Ml, int D, int Mr, const int* entries, int nent,
                               cudaStream_t s);

}  // namespace tdmrg
