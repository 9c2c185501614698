// Reverse of one second-order projector-splitting step (Eq. S1) in complex FP64.
//
// The step is run again with every intermediate kept on the device (a tape): per site and
// half-sweep the site tensor before and after its exponential, the gauge-QR factors with the
// accepted flags and the source of every completed column, the bond matrix before and after
// its exponential and the neighbour before absorption, plus the three environment sets in use
// (right environments of the input, the new left ones, the new right ones).  The tape is then
// reversed site by site with the kernel-level VJP entry points (site and bond exponentials,
// environment updates, completion candidates, gauge QR with completed columns, absorptions as
// GEMMs).  Parameter cotangents enter through the derivative MPO sites dW/dtheta as directional
// contractions.  The step is the one the oracle takes: no renormalisation in imaginary time.
#include <algorithm>
#include <cmath>
#include <vector>

#include "../../include/tdmrg.h"
#include "engine.h"
#include "small_exp.h"

namespace tdmrg {

namespace {
constexpr long long kNoSplit = 1LL << 60;
const cplx kOne = {1.0, 0.0};
const cplx kZero = {0.0, 0.0};

MatRef mr(const cplx* p, long long rs, long long cs, int conj = 0) {
  MatRef r;
  r.p = p;
  r.rs = rs;
  r.cs = cs;
  r.sb = 0;
  r.sr = 0;
  r.conj = conj;
  return r;
}

MatRef mrb(const cplx* p, long long rs, long long cs, long long sb, int conj = 0) {
  MatRef r = mr(p, rs, cs, conj);
  r.sb = sb;
  return r;
}

QrRef qr(const cplx* p, long long rs, long long cs, long long cb, long long cbs, int conj) {
  QrRef r;
  r.p = p;
  r.rs = rs;
  r.cs = cs;
  r.cb = cb;
  r.cbs = cbs;
  r.conj = conj;
  return r;
}

// device allocations of one call, freed on return
struct Tape {
  std::vector<void*> p;
  cplx* get(long long n) {
    void* q = nullptr;
    CK(cudaMalloc(&q, sizeof(cplx) * (size_t)(n > 0 ? n : 1)));
    p.push_back(q);
    return (cplx*)q;
  }
  int* geti(long long n) {
    void* q = nullptr;
    CK(cudaMalloc(&q, sizeof(int) * (size_t)(n > 0 ? n : 1)));
    p.push_back(q);
    return (int*)q;
  }
  ~Tape() {
    for (void* q : p) cudaFree(q);
  }
};

// dense site [Dl][Dr][d][d], complex interleaved
std::vector<double> dense_site(int Dl, int Dr, int d, const std::vector<MpoBlock>& blocks) {
  const size_t dd = (size_t)d * d;
  std::vector<double> out(2 * (size_t)Dl * Dr * dd, 0.0);
  for (const auto& b : blocks)
    for (size_t e = 0; e < dd; ++e) {
      const size_t off = 2 * (((size_t)b.wl * Dr + b.wr) * dd + e);
      out[off] += b.op[e].real();
      out[off + 1] += b.op[e].imag();
    }
  return out;
}

void call(int rc) {
  if (rc != TDMRG_OK) throw Failure{rc, tdmrg_last_global_error()};
}

// <g, x> = sum conj(g_i) x_i: 256 chunk sums by one batched GEMM plus the tail, added on the
// host in a fixed order (part: 257 device entries); synchronises st
Cx dot(const cplx* g, const cplx* x, long long n, cplx* part, cudaStream_t st) {
  const int B = 256;
  const long long kc = n / B, rem = n - kc * B;
  if (kc > 0) {
    MatRef a = mr(g, 0, 1, 1), b = mr(x, 1, 0);
    a.sb = kc;
    b.sb = kc;
    CK(zgemm(1, 1, (int)kc, B, 1, kOne, a, b, kZero, part, 1, 1, nullptr, st));
  }
  if (rem > 0)
    CK(zgemm(1, 1, (int)rem, 1, 1, kOne, mr(g + kc * B, 0, 1, 1), mr(x + kc * B, 1, 0), kZero,
             part + B, 1, 0, nullptr, st));
  std::vector<cplx> h(B + 1);
  CK(cudaMemcpyAsync(h.data(), part, sizeof(cplx) * (B + 1), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  Cx acc(0.0, 0.0);
  if (kc > 0)
    for (int b = 0; b < B; ++b) acc += Cx(h[b].x, h[b].y);
  if (rem > 0) acc += Cx(h[B].x, h[B].y);
  return acc;
}
// scratch of the gauge-shift reverses below (each at least site-sized, Xfullb and cand at
// least max(Dl, Dr) times site-sized)
struct ShiftScratch {
  cplx *Qb2, *Yb2, *b3, *Xsel, *Xselb, *Xfullb, *cand, *e1, *s1;
};

std::vector<int> completed_positions(const std::vector<unsigned char>& acc, std::vector<int>& accv) {
  std::vector<int> K;
  accv.assign(acc.size(), 0);
  for (size_t j = 0; j < acc.size(); ++j) {
    accv[j] = acc[j] ? 1 : 0;
    if (!acc[j]) K.push_back((int)j);
  }
  return K;
}

// Reverse of a right-to-left gauge shift: Y = a^H (m = d^2 Mr rows, Ml columns) = Q2 R2 with
// completions from X = P^H, P = right_partial(R, W, c).  Qs_bar: cotangent of the site Q2^H;
// Cm_bar: cotangent of C = R2^H (NULL: none).  Writes abar (cotangent of a); adds the
// candidates' cotangents to R (Rbar), c (cbar) and theta.
void qr_left_reverse(const Ctx& ctx, const ShiftScratch& w, cplx* X, cplx* Y,
                     const DevMpoSite& W, const double* Wd, int np, const double* dWd, int Ml,
                     int Mr, int d, const cplx* R, const cplx* c, const cplx* Q2, const cplx* R2,
                     const std::vector<unsigned char>& acc, const std::vector<int>& src,
                     const cplx* Qs_bar, const cplx* Cm_bar, cplx* abar, cplx* Rbar, cplx* cbar,
                     double* theta, std::vector<double>& tht) {
  cudaStream_t st = ctx.st;
  const int D = d * d;
  const long long m = (long long)D * Mr, n = (long long)Ml * m;
  const long long nr = (long long)W.Dr * Mr * Mr;
  CK(ztranspose(Ml, (int)m, Qs_bar, w.Qb2, 1, st));
  if (Cm_bar)
    CK(ztranspose(Ml, Ml, Cm_bar, w.b3, 1, st));
  else
    CK(cudaMemsetAsync(w.b3, 0, sizeof(cplx) * (size_t)Ml * Ml, st));
  std::vector<int> accv;
  const std::vector<int> K = completed_positions(acc, accv);
  const int p = W.Dl * Ml, nk = (int)K.size();
  if (nk > 0) {
    right_partial_f64(ctx, W, Ml, D, d, Mr, Mr, R, c, w.cand, nullptr);
    CK(cudaMemsetAsync(w.Xsel, 0, sizeof(cplx) * (size_t)(m * nk), st));
    for (int i = 0; i < nk; ++i) {
      const int s = src[K[i]];
      if (s < 0) throw Failure{TDMRG_ERR_CUDA, "gauge shift reverse: completion source not recorded"};
      if (s < p) {
        CK(cudaMemcpy2DAsync(w.Xsel + i, sizeof(cplx) * nk, w.cand + (long long)s * m,
                             sizeof(cplx), sizeof(cplx), (size_t)m, cudaMemcpyDeviceToDevice, st));
      } else {
        const cplx one = kOne;
        CK(cudaMemcpyAsync(w.Xsel + (long long)(s - p) * nk + i, &one, sizeof(cplx),
                           cudaMemcpyHostToDevice, st));
        CK(cudaStreamSynchronize(st));
      }
    }
    CK(zconj(m * nk, w.Xsel, st));
  }
  call(tdmrg_kernel_qr_vjp_completed((int)m, Ml, accv.data(), Q2, R2, nk ? w.Xsel : nullptr,
                                     w.Qb2, w.b3, w.Yb2, nk ? w.Xselb : nullptr, (void*)st));
  CK(ztranspose((int)m, Ml, w.Yb2, abar, 1, st));
  if (nk > 0) {
    CK(cudaMemsetAsync(w.Xfullb, 0, sizeof(cplx) * (size_t)(m * p), st));
    for (int i = 0; i < nk; ++i) {
      const int s = src[K[i]];
      if (s < p)
        CK(cudaMemcpy2DAsync(w.Xfullb + s, sizeof(cplx) * p, w.Xselb + i, sizeof(cplx) * nk,
                             sizeof(cplx), (size_t)m, cudaMemcpyDeviceToDevice, st));
    }
    call(tdmrg_kernel_expansion_vjp(1, Ml, Mr, d, W.Dl, W.Dr, Wd, np, dWd, R, c, w.Xfullb, w.e1,
                                    w.s1, tht.data(), X, Y, (void*)st));
    for (int q = 0; q < np; ++q) theta[q] += tht[q];
    CK(zaxpy(nr, kOne, w.e1, Rbar, st));
    CK(zaxpy(n, kOne, w.s1, cbar, st));
  }
}

// Reverse of a left-to-right gauge shift: a (Ml d^2 x Mr) = Q R with completions from the
// columns of left_partial(L, W, c).  Q_bar, R_bar (NULL: none) -> abar (written); adds the
// candidates' cotangents to L (Lbar), c (cbar) and theta.
void qr_right_reverse(const Ctx& ctx, const ShiftScratch& w, cplx* X, cplx* Y,
                      const DevMpoSite& W, const double* Wd, int np, const double* dWd, int Ml,
                      int Mr, int d, const cplx* L, const cplx* c, const cplx* Q, const cplx* R,
                      const std::vector<unsigned char>& acc, const std::vector<int>& src,
                      const cplx* Q_bar, const cplx* R_bar, cplx* abar, cplx* Lbar, cplx* cbar,
                      double* theta, std::vector<double>& tht) {
  cudaStream_t st = ctx.st;
  const int D = d * d;
  const long long m = (long long)Ml * D, n = m * Mr;
  const long long nl = (long long)W.Dl * Ml * Ml;
  if (R_bar)
    CK(cudaMemcpyAsync(w.b3, R_bar, sizeof(cplx) * (size_t)Mr * Mr, cudaMemcpyDeviceToDevice, st));
  else
    CK(cudaMemsetAsync(w.b3, 0, sizeof(cplx) * (size_t)Mr * Mr, st));
  std::vector<int> accv;
  const std::vector<int> K = completed_positions(acc, accv);
  const int p = W.Dr * Mr, nk = (int)K.size();
  if (nk > 0) {
    left_partial_f64(ctx, W, Ml, Ml, D, d, Mr, L, c, w.cand, nullptr);
    CK(cudaMemsetAsync(w.Xsel, 0, sizeof(cplx) * (size_t)(m * nk), st));
    for (int i = 0; i < nk; ++i) {
      const int s = src[K[i]];
      if (s < 0) throw Failure{TDMRG_ERR_CUDA, "gauge shift reverse: completion source not recorded"};
      if (s < p) {
        const long long v = s / Mr, cc = s % Mr;
        CK(cudaMemcpy2DAsync(w.Xsel + i, sizeof(cplx) * nk, w.cand + v * n + cc,
                             sizeof(cplx) * Mr, sizeof(cplx), (size_t)m, cudaMemcpyDeviceToDevice,
                             st));
      } else {
        const cplx one = kOne;
        CK(cudaMemcpyAsync(w.Xsel + (long long)(s - p) * nk + i, &one, sizeof(cplx),
                           cudaMemcpyHostToDevice, st));
        CK(cudaStreamSynchronize(st));
      }
    }
  }
  call(tdmrg_kernel_qr_vjp_completed((int)m, Mr, accv.data(), Q, R, nk ? w.Xsel : nullptr, Q_bar,
                                     w.b3, abar, nk ? w.Xselb : nullptr, (void*)st));
  if (nk > 0) {
    CK(cudaMemsetAsync(w.Xfullb, 0, sizeof(cplx) * (size_t)(m * p), st));
    for (int i = 0; i < nk; ++i) {
      const int s = src[K[i]];
      if (s < p)
        CK(cudaMemcpy2DAsync(w.Xfullb + s, sizeof(cplx) * p, w.Xselb + i, sizeof(cplx) * nk,
                             sizeof(cplx), (size_t)m, cudaMemcpyDeviceToDevice, st));
    }
    call(tdmrg_kernel_expansion_vjp(0, Ml, Mr, d, W.Dl, W.Dr, Wd, np, dWd, L, c, w.Xfullb, w.e1,
                                    w.s1, tht.data(), X, Y, (void*)st));
    for (int q = 0; q < np; ++q) theta[q] += tht[q];
    CK(zaxpy(nl, kOne, w.e1, Lbar, st));
    CK(zaxpy(n, kOne, w.s1, cbar, st));
  }
}
}  // namespace

template <class F>
void Engine::exp_vjp_nodes(long long n, const cplx* v, const cplx* ybar, double tr, double ti,
                           int nodes, cplx* vbar, cplx* Aq, cplx* Bq, cplx* basis,
                           std::vector<Cx>& kq, F&& matvec) {
  auto read_state = [&](int& k, double& b0, std::vector<double>& al, std::vector<double>& be) {
    LzState h;
    CK(cudaMemcpyAsync(&h, lz_, sizeof(LzState), cudaMemcpyDeviceToHost, st_));
    CK(cudaStreamSynchronize(st_));
    k = h.k;
    b0 = h.b0;
    al.assign(h.alpha, h.alpha + (k > 0 ? k : 0));
    be.assign(k > 1 ? h.beta + 1 : h.beta, k > 1 ? h.beta + k : h.beta);   // beta_1 .. beta_{k-1}
  };
  // forward Lanczos of v: its basis is kept for the b_q
  int k1 = 0, k2 = 0;
  double b1 = 0.0, b2 = 0.0;
  std::vector<double> a1, e1, a2, e2;
  krylov(n, v, Kout_, tr, ti, matvec);
  read_state(k1, b1, a1, e1);
  if (k1 > 0)
    CK(cudaMemcpyAsync(basis, V_, sizeof(cplx) * (size_t)k1 * n, cudaMemcpyDeviceToDevice, st_));
  // Lanczos of ybar with conj(tau): vbar, and its basis (left in V_) for the a_q
  krylov(n, ybar, vbar, tr, -ti, matvec);
  read_state(k2, b2, a2, e2);
  // node count: at most `nodes`, the fewest for which the Gauss-Legendre error bound of the
  // Frechet integrand s -> e^{s tau T1} (.) e^{(1-s) tau T2} stays below 1e-15 of its scale
  // (r = |tau| (|T1| + |T2|), infinity norms of the two Lanczos matrices)
  auto tnorm = [](const std::vector<double>& al, const std::vector<double>& be) {
    double m = 0.0;
    for (size_t i = 0; i < al.size(); ++i) {
      double r = std::fabs(al[i]);
      if (i > 0) r += std::fabs(be[i - 1]);
      if (i < be.size()) r += std::fabs(be[i]);
      m = std::max(m, r);
    }
    return m;
  };
  const double r = std::hypot(tr, ti) * (tnorm(a1, e1) + tnorm(a2, e2));
  nodes = gauss_legendre_nodes_for(r, nodes, 1e-15);
  std::vector<double> sq, wq;
  gauss_legendre01(nodes, sq, wq);
  kq.resize(nodes);
  for (int q = 0; q < nodes; ++q) kq[q] = wq[q] * std::conj(Cx(tr, ti));
  std::vector<Cx> zb(nodes), za(nodes), cb((size_t)nodes * std::max(k1, 1)),
      ca((size_t)nodes * std::max(k2, 1));
  for (int q = 0; q < nodes; ++q) {
    zb[q] = sq[q] * Cx(tr, ti);
    za[q] = (1.0 - sq[q]) * Cx(tr, -ti);
  }
  Tape tp;
  if (k1 > 0 && b1 > 0.0) {
    tridiag_exp_e1(k1, a1.data(), e1.data(), nodes, zb.data(), cb.data());
    std::vector<cplx> h((size_t)nodes * k1);
    for (size_t i = 0; i < h.size(); ++i) h[i] = {b1 * cb[i].real(), b1 * cb[i].imag()};
    cplx* d = tp.get((long long)h.size());
    CK(cudaMemcpyAsync(d, h.data(), sizeof(cplx) * h.size(), cudaMemcpyHostToDevice, st_));
    CK(zgemm(nodes, (int)n, k1, 1, 1, kOne, mr(d, k1, 1), mr(basis, n, 1), kZero, Bq, n, 0,
             nullptr, st_));
    CK(cudaStreamSynchronize(st_));
  } else {
    CK(cudaMemsetAsync(Bq, 0, sizeof(cplx) * (size_t)nodes * n, st_));
  }
  if (k2 > 0 && b2 > 0.0) {
    tridiag_exp_e1(k2, a2.data(), e2.data(), nodes, za.data(), ca.data());
    std::vector<cplx> h((size_t)nodes * k2);
    for (size_t i = 0; i < h.size(); ++i) h[i] = {b2 * ca[i].real(), b2 * ca[i].imag()};
    cplx* d = tp.get((long long)h.size());
    CK(cudaMemcpyAsync(d, h.data(), sizeof(cplx) * h.size(), cudaMemcpyHostToDevice, st_));
    CK(zgemm(nodes, (int)n, k2, 1, 1, kOne, mr(d, k2, 1), mr(V_, n, 1), kZero, Aq, n, 0,
             nullptr, st_));
    CK(cudaStreamSynchronize(st_));
  } else {
    CK(cudaMemsetAsync(Aq, 0, sizeof(cplx) * (size_t)nodes * n, st_));
  }
}

void Engine::step_vjp(int M, const cplx* const* A_in, double tr, double ti,
                      const cplx* const* Abar_out, cplx* const* A_out, cplx* const* Abar_in,
                      double* theta_bar, int nodes, bool normalize, double logn_bar,
                      double* log_norm) {
  if (mixed()) throw Failure{TDMRG_ERR_ARG, "step_vjp: the reverse pass runs in FP64 precision"};
  const int L = (int)sites_.size();
  const std::vector<int> Mb = bond_dimensions(sites_, M);
  std::vector<int> D(L), dd(L);
  std::vector<long long> n(L), nL(L), nR(L);
  long long maxsite = 1, maxxy = 1, maxenv = 1;
  int maxbond = 1;
  const int Dmax = std::max(H_.maxD, J_.maxD);
  for (int k = 0; k < L; ++k) {
    dd[k] = sites_[k].d;
    D[k] = dd[k] * dd[k];
    n[k] = (long long)Mb[k] * D[k] * Mb[k + 1];
    nL[k] = (long long)H_.s[k].Dl * Mb[k] * Mb[k];
    nR[k] = (long long)H_.s[k].Dr * Mb[k + 1] * Mb[k + 1];
    maxsite = std::max(maxsite, n[k]);
    maxxy = std::max(maxxy, (long long)Dmax * n[k]);
    maxenv = std::max(maxenv, std::max(nL[k], nR[k]));
    maxbond = std::max(maxbond, Mb[k + 1]);
  }
  maxxy = std::max(maxxy, (long long)Dmax * maxbond * maxbond);
  ensure_workspace(maxsite, maxxy, maxbond, maxbond);
  const double hr = 0.5 * tr, hi = 0.5 * ti;
  const int np = parameter_count(P);
  std::vector<std::vector<double>> Wd(L), dWd(L);
  for (int k = 0; k < L; ++k) {
    const DevMpoSite& W = H_.s[k];
    Wd[k] = dense_site(W.Dl, W.Dr, W.d, W.host);
    for (int p = 0; p < np; ++p) {
      const MpoSite dW = mpo_site_derivative(P, 0, p, k);
      const std::vector<double> x = dense_site(W.Dl, W.Dr, W.d, dW.blocks);
      dWd[k].insert(dWd[k].end(), x.begin(), x.end());
    }
  }
  auto dWp = [&](int k) { return np > 0 ? dWd[k].data() : nullptr; };
  const cudaMemcpyKind d2d = cudaMemcpyDeviceToDevice;
  auto copy = [&](cplx* dst, const cplx* src, long long cnt) {
    CK(cudaMemcpyAsync(dst, src, sizeof(cplx) * (size_t)cnt, d2d, st_));
  };
  Ctx c = ctx();
  Tape tp;

  // ---- forward with the tape ----
  std::vector<cplx*> A(L), Lenv(L), Rin(L), Rnew(L);
  std::vector<cplx*> ain_lr(L), a1_lr(L), Q_lr(L), R_lr(L), c_lr(L), nxt_lr(L);
  std::vector<cplx*> ain_rl(L), a1_rl(L), Q2_rl(L), R2_rl(L), Qs_rl(L), Cm_rl(L), c_rl(L),
      nxt_rl(L);
  std::vector<std::vector<unsigned char>> acc_lr(L), acc_rl(L);
  std::vector<std::vector<int>> src_lr(L), src_rl(L);
  for (int k = 0; k < L; ++k) {
    A[k] = tp.get(n[k]);
    Lenv[k] = tp.get(nL[k]);
    Rin[k] = tp.get(nR[k]);
    Rnew[k] = tp.get(nR[k]);
    copy(A[k], A_in[k], n[k]);
  }
  int* src_dev = tp.geti(maxbond);
  set_ones(Lenv[0]);
  set_ones(Rin[L - 1]);
  set_ones(Rnew[L - 1]);
  for (int k = L - 1; k > 0; --k)
    env_right_f64(c, H_.s[k], Mb[k], Mb[k + 1], Mb[k], Mb[k + 1], D[k], dd[k], Rin[k], A[k], A[k],
                  Rin[k - 1]);
  auto flags = [&](int cols, std::vector<unsigned char>& acc, std::vector<int>& src) {
    acc.resize(cols);
    src.resize(cols);
    CK(cudaMemcpyAsync(acc.data(), qb_acc_, (size_t)cols, cudaMemcpyDeviceToHost, st_));
    CK(cudaMemcpyAsync(src.data(), src_dev, sizeof(int) * (size_t)cols, cudaMemcpyDeviceToHost,
                       st_));
    CK(cudaStreamSynchronize(st_));
  };
  // left to right
  for (int k = 0; k < L; ++k) {
    const DevMpoSite& W = H_.s[k];
    const int Ml = Mb[k], Mr = Mb[k + 1];
    const cplx* Le = Lenv[k];
    const cplx* Re = Rin[k];
    ain_lr[k] = tp.get(n[k]);
    a1_lr[k] = tp.get(n[k]);
    copy(ain_lr[k], A[k], n[k]);
    krylov(n[k], ain_lr[k], a1_lr[k], hr, hi, [&](const cplx* in, cplx* out, const int* skip) {
      heff_f64(c, W, Ml, Mr, D[k], dd[k], Le, Re, in, out, skip);
    });
    if (k == L - 1) {
      copy(A[k], a1_lr[k], n[k]);
      continue;
    }
    Q_lr[k] = tp.get(n[k]);
    R_lr[k] = tp.get((long long)Mr * Mr);
    c_lr[k] = tp.get((long long)Mr * Mr);
    nxt_lr[k] = tp.get(n[k + 1]);
    left_partial_f64(c, W, Ml, Ml, D[k], dd[k], Mr, Le, a1_lr[k], Y_, nullptr);
    CK(cudaMemsetAsync(src_dev, 0xff, sizeof(int) * (size_t)Mr, st_));
    gauge_qr_dev(Ml * D[k], Mr, qr(a1_lr[k], Mr, 1, kNoSplit, 0, 0), W.Dr * Mr,
                 qr(Y_, Mr, 1, Mr, n[k], 0), Q_lr[k], R_lr[k], src_dev);
    flags(Mr, acc_lr[k], src_lr[k]);
    env_left_f64(c, W, Ml, Mr, Ml, Mr, D[k], dd[k], Le, Q_lr[k], Q_lr[k], Lenv[k + 1]);
    const int Dw = W.Dr;
    const cplx* Le1 = Lenv[k + 1];
    krylov((long long)Mr * Mr, R_lr[k], c_lr[k], -hr, -hi,
           [&](const cplx* in, cplx* out, const int* sk) {
             bond_f64(c, Mr, Dw, Le1, Re, in, out, sk);
           });
    copy(nxt_lr[k], A[k + 1], n[k + 1]);
    const long long ncols = (long long)D[k + 1] * Mb[k + 2];
    CK(zgemm(Mr, (int)ncols, Mr, 1, 1, kOne, mr(c_lr[k], Mr, 1), mr(nxt_lr[k], ncols, 1), kZero,
             A[k + 1], ncols, 0, nullptr, st_));
    copy(A[k], Q_lr[k], n[k]);
  }
  // right to left
  for (int k = L - 1; k >= 0; --k) {
    const DevMpoSite& W = H_.s[k];
    const int Ml = Mb[k], Mr = Mb[k + 1];
    const cplx* Le = Lenv[k];
    const cplx* Re = Rnew[k];
    ain_rl[k] = tp.get(n[k]);
    a1_rl[k] = tp.get(n[k]);
    copy(ain_rl[k], A[k], n[k]);
    krylov(n[k], ain_rl[k], a1_rl[k], hr, hi, [&](const cplx* in, cplx* out, const int* skip) {
      heff_f64(c, W, Ml, Mr, D[k], dd[k], Le, Re, in, out, skip);
    });
    if (k == 0) {
      copy(A[0], a1_rl[0], n[0]);
      continue;
    }
    const long long m = (long long)D[k] * Mr;
    Q2_rl[k] = tp.get(n[k]);
    R2_rl[k] = tp.get((long long)Ml * Ml);
    Qs_rl[k] = tp.get(n[k]);
    Cm_rl[k] = tp.get((long long)Ml * Ml);
    c_rl[k] = tp.get((long long)Ml * Ml);
    nxt_rl[k] = tp.get(n[k - 1]);
    right_partial_f64(c, W, Ml, D[k], dd[k], Mr, Mr, Re, a1_rl[k], Y_, nullptr);
    CK(cudaMemsetAsync(src_dev, 0xff, sizeof(int) * (size_t)Ml, st_));
    gauge_qr_dev((int)m, Ml, qr(a1_rl[k], 1, m, kNoSplit, 0, 1), W.Dl * Ml,
                 qr(Y_, 1, m, kNoSplit, 0, 1), Q2_rl[k], R2_rl[k], src_dev);
    flags(Ml, acc_rl[k], src_rl[k]);
    CK(ztranspose((int)m, Ml, Q2_rl[k], Qs_rl[k], 1, st_));     // the site: Q2^H
    CK(ztranspose(Ml, Ml, R2_rl[k], Cm_rl[k], 1, st_));          // the bond matrix: R2^H
    env_right_f64(c, W, Ml, Mr, Ml, Mr, D[k], dd[k], Re, Qs_rl[k], Qs_rl[k], Rnew[k - 1]);
    const int Dw = W.Dl;
    const cplx* Re1 = Rnew[k - 1];
    krylov((long long)Ml * Ml, Cm_rl[k], c_rl[k], -hr, -hi,
           [&](const cplx* in, cplx* out, const int* sk) {
             bond_f64(c, Ml, Dw, Le, Re1, in, out, sk);
           });
    copy(nxt_rl[k], A[k - 1], n[k - 1]);
    const long long nrows = (long long)Mb[k - 1] * D[k - 1];
    CK(zgemm((int)nrows, Ml, Ml, 1, 1, kOne, mr(nxt_rl[k], Ml, 1), mr(c_rl[k], Ml, 1), kZero,
             A[k - 1], Ml, 0, nullptr, st_));
    copy(A[k], Qs_rl[k], n[k]);
  }
  // optional normalisation of the output center: A0 <- A0 / ||A0||, log ||A0||^2 reported
  cplx* part = tp.get(257);
  double nrm = 1.0;
  cplx* A0raw = nullptr;
  if (normalize) {
    nrm = std::sqrt(dot(A[0], A[0], n[0], part, st_).real());
    if (!std::isfinite(nrm) || nrm <= 0.0)
      throw Failure{TDMRG_ERR_NONFINITE, "step_vjp: non-finite norm of the output center"};
    A0raw = tp.get(n[0]);
    copy(A0raw, A[0], n[0]);
    scale_dev(A[0], n[0], 1.0 / nrm);
    if (log_norm) *log_norm = 2.0 * std::log(nrm);
  }
  if (A_out)
    for (int k = 0; k < L; ++k) copy(A_out[k], A[k], n[k]);
  check_status();
  if (!Abar_out) {                       // forward only
    CK(cudaStreamSynchronize(st_));
    return;
  }

  // ---- reverse ----
  std::vector<cplx*> ab(L), Lb(L), Rib(L), Rnb(L);
  for (int k = 0; k < L; ++k) {
    ab[k] = tp.get(n[k]);
    copy(ab[k], Abar_out[k], n[k]);
  }
  if (normalize) {
    // A0n = A0 / n:  abar0 <- (g - Re<A0n, g> A0n) / n  (+ logn_bar * 2 A0 / n^2 for log n^2)
    const double re = dot(A[0], ab[0], n[0], part, st_).real();
    const cplx f = {-re, 0.0};
    CK(zaxpy(n[0], f, A[0], ab[0], st_));
    scale_dev(ab[0], n[0], 1.0 / nrm);
    if (logn_bar != 0.0) {
      const cplx lf = {2.0 * logn_bar / (nrm * nrm), 0.0};
      CK(zaxpy(n[0], lf, A0raw, ab[0], st_));
    }
  }
  for (int k = 0; k < L; ++k) {
    Lb[k] = tp.get(nL[k]);
    Rib[k] = tp.get(nR[k]);
    Rnb[k] = tp.get(nR[k]);
    CK(cudaMemsetAsync(Lb[k], 0, sizeof(cplx) * (size_t)nL[k], st_));
    CK(cudaMemsetAsync(Rib[k], 0, sizeof(cplx) * (size_t)nR[k], st_));
    CK(cudaMemsetAsync(Rnb[k], 0, sizeof(cplx) * (size_t)nR[k], st_));
  }
  cplx* a1b = tp.get(maxsite);
  cplx* s1 = tp.get(maxsite);
  cplx* s2 = tp.get(maxsite);
  cplx* s3 = tp.get(maxsite);
  cplx* Qb2 = tp.get(maxsite);
  cplx* Yb2 = tp.get(maxsite);
  cplx* Xsel = tp.get(maxsite);
  cplx* Xselb = tp.get(maxsite);
  cplx* Xfullb = tp.get(maxxy);
  cplx* cand = tp.get(maxxy);
  cplx* e1 = tp.get(maxenv);
  cplx* e2 = tp.get(maxenv);
  cplx* b1 = tp.get((long long)maxbond * maxbond);
  cplx* b2 = tp.get((long long)maxbond * maxbond);
  cplx* b3 = tp.get((long long)maxbond * maxbond);
  std::vector<double> th(np, 0.0), tht(np > 0 ? np : 1, 0.0);
  const double tol = ktol_;
  void* sv = (void*)st_;
  // exponential VJPs: the entry points (fresh Lanczos exponentials at every node) or the
  // Krylov-basis quadrature on this engine (node vectors from the bases of v and vbar)
  cplx *Aq = nullptr, *Bq = nullptr, *basis = nullptr, *tq = nullptr, *El = nullptr;
  cplx* Gacc = nullptr;      // parameter cotangent of one site operator, Dl x Dr x d x d
  std::vector<std::vector<DevMpo>> dWdev;
  struct FreeDev {
    std::vector<std::vector<DevMpo>>& m;
    ~FreeDev() {
      for (auto& row : m)
        for (auto& x : row) Engine::free_mpo(x);
    }
  } free_dev{dWdev};
  if (adjoint_basis_) {
    Aq = tp.get((long long)nodes * maxsite);
    Bq = tp.get((long long)nodes * maxsite);
    basis = tp.get((long long)KMAX * maxsite);
    tq = tp.get(maxsite);
    El = tp.get(maxenv);
    Gacc = tp.get((long long)Dmax * Dmax * 256);
    dWdev.assign(L, std::vector<DevMpo>(np));
    for (int k = 0; k < L; ++k)
      for (int p = 0; p < np; ++p) {
        const MpoSite dW = mpo_site_derivative(P, 0, p, k);
        if (!dW.blocks.empty()) upload_mpo({dW}, dWdev[k][p]);
      }
  }
  auto site_vjp = [&](int k, const cplx* Le, const cplx* Re, const cplx* ain, const cplx* ybar,
                      cplx* Abar, cplx* Lbar, cplx* Rbar) {
    const DevMpoSite& W = H_.s[k];
    const int Ml = Mb[k], Mr = Mb[k + 1];
    if (!adjoint_basis_) {
      call(tdmrg_kernel_site_exp_vjp_theta(Ml, Mr, dd[k], W.Dl, W.Dr, Wd[k].data(), Le, Re, ain,
                                           ybar, hr, hi, nodes, tol, np, dWp(k), Abar, Lbar, Rbar,
                                           tht.data(), sv));
      return;
    }
    std::vector<Cx> kq;
    exp_vjp_nodes(n[k], ain, ybar, hr, hi, nodes, Abar, Aq, Bq, basis, kq,
                  [&](const cplx* in, cplx* out, const int* skip) {
                    heff_f64(c, W, Ml, Mr, D[k], dd[k], Le, Re, in, out, skip);
                  });
    CK(cudaMemsetAsync(Lbar, 0, sizeof(cplx) * (size_t)nL[k], st_));
    CK(cudaMemsetAsync(Rbar, 0, sizeof(cplx) * (size_t)nR[k], st_));
    for (int p = 0; p < np; ++p) tht[p] = 0.0;
    const int gsz = W.Dl * W.Dr * D[k];
    const bool gram = np > 0 && dd[k] <= 16;
    if (gram) CK(cudaMemsetAsync(Gacc, 0, sizeof(cplx) * (size_t)gsz, st_));
    for (int q = 0; q < (int)kq.size(); ++q) {
      const cplx* a = Aq + (size_t)q * n[k];
      const cplx* b = Bq + (size_t)q * n[k];
      const Cx kc = std::conj(kq[q]);                 // w_q tau
      const cplx kcc = {kc.real(), kc.imag()};
      // Lbar = conj(sum_q conj(k_q) env_right(R, a_q, W, b_q)), Rbar likewise with env_left
      env_right_f64(c, W, Ml, Mr, Ml, Mr, D[k], dd[k], Re, a, b, El);
      CK(zaxpy(nL[k], kcc, El, Lbar, st_));
      env_left_f64(c, W, Ml, Mr, Ml, Mr, D[k], dd[k], Le, a, b, El);
      CK(zaxpy(nR[k], kcc, El, Rbar, st_));
      if (gram) {
        // theta_p = Re sum_q k_q <a_q, H_eff(dW_p) b_q> = Re sum dW_p . G, G accumulated over
        // the nodes: U = L b_q, V = conj(a_q) R, then one contraction over (x, t, c)
        CK(zgemm(W.Dl * Ml, D[k] * Mr, Ml, 1, 1, kOne, mr(Le, Ml, 1), mr(b, (long long)D[k] * Mr, 1),
                 kZero, X_, (long long)D[k] * Mr, 0, nullptr, st_));
        CK(zgemm(Ml * D[k], Mr, Mr, W.Dr, 1, kOne, mr(a, Mr, 1, 1),
                 mrb(Re, Mr, 1, (long long)Mr * Mr), kZero, Y_, Mr, (long long)Ml * D[k] * Mr,
                 nullptr, st_));
        CK(param_gram(W.Dl, W.Dr, Ml, dd[k], Mr, X_, Y_, kcc, Gacc, st_));
      } else {
        for (int p = 0; p < np; ++p) {
          if (dWdev[k][p].s.empty()) continue;
          heff_f64(c, dWdev[k][p].s[0], Ml, Mr, D[k], dd[k], Le, Re, b, tq, nullptr);
          tht[p] += (kc * dot(a, tq, n[k], part, st_)).real();
        }
      }
    }
    if (gram) {
      std::vector<cplx> gh(gsz);
      CK(cudaMemcpyAsync(gh.data(), Gacc, sizeof(cplx) * (size_t)gsz, cudaMemcpyDeviceToHost,
                         st_));
      CK(cudaStreamSynchronize(st_));
      for (int p = 0; p < np; ++p) {
        const double* dw = dWd[k].data() + 2 * (size_t)gsz * p;
        double acc = 0.0;
        for (int e = 0; e < gsz; ++e) acc += dw[2 * e] * gh[e].x - dw[2 * e + 1] * gh[e].y;
        tht[p] = acc;
      }
    }
    CK(zconj(nL[k], Lbar, st_));
    CK(zconj(nR[k], Rbar, st_));
  };
  auto bond_vjp = [&](int M, int Dw, const cplx* Le, const cplx* Re, const cplx* C0,
                      const cplx* ybar, cplx* Cbar, cplx* Lbar, cplx* Rbar) {
    if (!adjoint_basis_) {
      call(tdmrg_kernel_bond_exp_vjp(M, Dw, Le, Re, C0, ybar, -hr, -hi, nodes, tol, Cbar, Lbar,
                                     Rbar, sv));
      return;
    }
    const long long mm = (long long)M * M;
    std::vector<Cx> kq;
    exp_vjp_nodes(mm, C0, ybar, -hr, -hi, nodes, Cbar, Aq, Bq, basis, kq,
                  [&](const cplx* in, cplx* out, const int* skip) {
                    bond_f64(c, M, Dw, Le, Re, in, out, skip);
                  });
    CK(cudaMemsetAsync(Lbar, 0, sizeof(cplx) * (size_t)(Dw * mm), st_));
    CK(cudaMemsetAsync(Rbar, 0, sizeof(cplx) * (size_t)(Dw * mm), st_));
    for (int q = 0; q < (int)kq.size(); ++q) {
      const cplx* a = Aq + (size_t)q * mm;
      const cplx* b = Bq + (size_t)q * mm;
      const cplx kk = {kq[q].real(), kq[q].imag()};  // w_q conj(tau)
      // Lbar_w += k a conj(R_w) b^H;  Rbar_w += k a^T conj(L_w) conj(b)
      CK(zgemm(M, M, M, Dw, 1, kOne, mrb(Re, M, 1, mm, 1), mr(b, 1, M, 1), kZero, El, M, mm,
               nullptr, st_));
      CK(zgemm(M, M, M, Dw, 1, kk, mr(a, M, 1), mrb(El, M, 1, mm), kOne, Lbar, M, mm, nullptr,
               st_));
      CK(zgemm(M, M, M, Dw, 1, kOne, mrb(Le, M, 1, mm, 1), mr(b, M, 1, 1), kZero, El, M, mm,
               nullptr, st_));
      CK(zgemm(M, M, M, Dw, 1, kk, mr(a, 1, M), mrb(El, M, 1, mm), kOne, Rbar, M, mm, nullptr,
               st_));
    }
    CK(cudaStreamSynchronize(st_));
  };
  auto add = [&](cplx* dst, const cplx* src, long long cnt) {
    CK(zaxpy(cnt, kOne, src, dst, st_));
  };
  auto take_theta = [&]() {
    for (int p = 0; p < np; ++p) th[p] += tht[p];
  };
  // the vectors that completed a QR: column i of Xsel from candidate src (i < p: a column of
  // the candidate matrix, read by `column`; otherwise the unit vector e_{src - p})
  auto gather = [&](long long m, int p, const std::vector<int>& K, const std::vector<int>& src,
                    auto&& column) {
    const int nk = (int)K.size();
    CK(cudaMemsetAsync(Xsel, 0, sizeof(cplx) * (size_t)(m * nk), st_));
    for (int i = 0; i < nk; ++i) {
      const int s = src[K[i]];
      if (s < 0) throw Failure{TDMRG_ERR_CUDA, "step_vjp: completion source not recorded"};
      if (s < p) {
        column(i, s);
      } else {
        const cplx one = kOne;
        CK(cudaMemcpyAsync(Xsel + (long long)(s - p) * nk + i, &one, sizeof(cplx),
                           cudaMemcpyHostToDevice, st_));
        CK(cudaStreamSynchronize(st_));
      }
    }
  };
  auto scatter = [&](long long m, int p, const std::vector<int>& K, const std::vector<int>& src) {
    const int nk = (int)K.size();
    CK(cudaMemsetAsync(Xfullb, 0, sizeof(cplx) * (size_t)(m * p), st_));
    for (int i = 0; i < nk; ++i) {
      const int s = src[K[i]];
      if (s < p)
        CK(cudaMemcpy2DAsync(Xfullb + s, sizeof(cplx) * p, Xselb + i, sizeof(cplx) * nk,
                             sizeof(cplx), (size_t)m, d2d, st_));
    }
  };
  auto completed = [](const std::vector<unsigned char>& acc, std::vector<int>& accv) {
    std::vector<int> K;
    accv.assign(acc.size(), 0);
    for (size_t j = 0; j < acc.size(); ++j) {
      accv[j] = acc[j] ? 1 : 0;
      if (!acc[j]) K.push_back((int)j);
    }
    return K;
  };

  // right-to-left half, last site update first
  for (int k = 0; k < L; ++k) {
    const DevMpoSite& W = H_.s[k];
    const int Ml = Mb[k], Mr = Mb[k + 1], Dl = W.Dl, Dr = W.Dr;
    if (k > 0) {
      const long long m = (long long)D[k] * Mr;
      const long long nrows = (long long)Mb[k - 1] * D[k - 1];
      // A[k-1] = nxt c:  cbar = nxt^H abar,  abar <- abar c^H
      CK(zgemm(Ml, Ml, (int)nrows, 1, 1, kOne, mr(nxt_rl[k], 1, Ml, 1), mr(ab[k - 1], Ml, 1),
               kZero, b1, Ml, 0, nullptr, st_));
      CK(zgemm((int)nrows, Ml, Ml, 1, 1, kOne, mr(ab[k - 1], Ml, 1), mr(c_rl[k], 1, Ml, 1), kZero,
               s1, Ml, 0, nullptr, st_));
      copy(ab[k - 1], s1, n[k - 1]);
      // c = exp(-h K(Lenv[k], Rnew[k-1])) Cm
      bond_vjp(Ml, Dl, Lenv[k], Rnew[k - 1], Cm_rl[k], b1, b2, e1, e2);
      add(Lb[k], e1, nL[k]);
      add(Rnb[k - 1], e2, nR[k - 1]);
      // Rnew[k-1] = env_right(Rnew[k], Qs, W, Qs)
      call(tdmrg_kernel_env_vjp(1, Ml, Mr, dd[k], Dl, Dr, Wd[k].data(), np, dWp(k), Rnew[k],
                                Qs_rl[k], Qs_rl[k], Rnb[k - 1], e1, s1, s2, tht.data(), X_, Y_,
                                sv));
      take_theta();
      add(Rnb[k], e1, nR[k]);
      copy(s3, ab[k], n[k]);
      add(s3, s1, n[k]);
      add(s3, s2, n[k]);
      // QR of Y = a1^H (m x Ml): outputs Qs = Q2^H and Cm = R2^H
      CK(ztranspose(Ml, (int)m, s3, Qb2, 1, st_));
      CK(ztranspose(Ml, Ml, b2, b3, 1, st_));
      std::vector<int> accv;
      const std::vector<int> K = completed(acc_rl[k], accv);
      const int p = Dl * Ml;
      const int nk = (int)K.size();
      if (nk > 0) {
        // candidates X = P^H, P = right_partial(Rnew[k], W, a1) (p x m): column s = conj row s
        right_partial_f64(c, W, Ml, D[k], dd[k], Mr, Mr, Rnew[k], a1_rl[k], cand, nullptr);
        gather(m, p, K, src_rl[k], [&](int i, int s) {
          CK(cudaMemcpy2DAsync(Xsel + i, sizeof(cplx) * nk, cand + (long long)s * m,
                               sizeof(cplx), sizeof(cplx), (size_t)m, d2d, st_));
        });
        CK(zconj(m * nk, Xsel, st_));
      }
      call(tdmrg_kernel_qr_vjp_completed((int)m, Ml, accv.data(), Q2_rl[k], R2_rl[k],
                                         nk ? Xsel : nullptr, Qb2, b3, Yb2,
                                         nk ? Xselb : nullptr, sv));
      CK(ztranspose((int)m, Ml, Yb2, a1b, 1, st_));
      if (nk > 0) {
        scatter(m, p, K, src_rl[k]);
        call(tdmrg_kernel_expansion_vjp(1, Ml, Mr, dd[k], Dl, Dr, Wd[k].data(), np, dWp(k),
                                        Rnew[k], a1_rl[k], Xfullb, e1, s1, tht.data(), X_, Y_,
                                        sv));
        take_theta();
        add(Rnb[k], e1, nR[k]);
        add(a1b, s1, n[k]);
      }
    } else {
      copy(a1b, ab[0], n[0]);
    }
    // a1 = exp(h H_eff(Lenv[k], W, Rnew[k])) ain
    site_vjp(k, Lenv[k], Rnew[k], ain_rl[k], a1b, ab[k], e1, e2);
    take_theta();
    add(Lb[k], e1, nL[k]);
    add(Rnb[k], e2, nR[k]);
  }
  // left-to-right half, last site update first
  for (int k = L - 1; k >= 0; --k) {
    const DevMpoSite& W = H_.s[k];
    const int Ml = Mb[k], Mr = Mb[k + 1], Dl = W.Dl, Dr = W.Dr;
    if (k < L - 1) {
      const long long m = (long long)Ml * D[k];
      const long long ncols = (long long)D[k + 1] * Mb[k + 2];
      // A[k+1] = c nxt:  cbar = abar nxt^H,  abar <- c^H abar
      CK(zgemm(Mr, Mr, (int)ncols, 1, 1, kOne, mr(ab[k + 1], ncols, 1), mr(nxt_lr[k], 1, ncols, 1),
               kZero, b1, Mr, 0, nullptr, st_));
      CK(zgemm(Mr, (int)ncols, Mr, 1, 1, kOne, mr(c_lr[k], 1, Mr, 1), mr(ab[k + 1], ncols, 1),
               kZero, s1, ncols, 0, nullptr, st_));
      copy(ab[k + 1], s1, n[k + 1]);
      // c = exp(-h K(Lenv[k+1], Rin[k])) R
      bond_vjp(Mr, Dr, Lenv[k + 1], Rin[k], R_lr[k], b1, b2, e1, e2);
      add(Lb[k + 1], e1, nL[k + 1]);
      add(Rib[k], e2, nR[k]);
      // Lenv[k+1] = env_left(Lenv[k], Q, W, Q)
      call(tdmrg_kernel_env_vjp(0, Ml, Mr, dd[k], Dl, Dr, Wd[k].data(), np, dWp(k), Lenv[k],
                                Q_lr[k], Q_lr[k], Lb[k + 1], e1, s1, s2, tht.data(), X_, Y_, sv));
      take_theta();
      add(Lb[k], e1, nL[k]);
      copy(s3, ab[k], n[k]);
      add(s3, s1, n[k]);
      add(s3, s2, n[k]);
      std::vector<int> accv;
      const std::vector<int> K = completed(acc_lr[k], accv);
      const int p = Dr * Mr;
      const int nk = (int)K.size();
      if (nk > 0) {
        // candidates: column (v, c) of left_partial(Lenv[k], W, a1) = Y[v][.][c]
        left_partial_f64(c, W, Ml, Ml, D[k], dd[k], Mr, Lenv[k], a1_lr[k], cand, nullptr);
        gather(m, p, K, src_lr[k], [&](int i, int s) {
          const long long v = s / Mr, cc = s % Mr;
          CK(cudaMemcpy2DAsync(Xsel + i, sizeof(cplx) * nk, cand + v * n[k] + cc,
                               sizeof(cplx) * Mr, sizeof(cplx), (size_t)m, d2d, st_));
        });
      }
      call(tdmrg_kernel_qr_vjp_completed((int)m, Mr, accv.data(), Q_lr[k], R_lr[k],
                                         nk ? Xsel : nullptr, s3, b2, a1b, nk ? Xselb : nullptr,
                                         sv));
      if (nk > 0) {
        scatter(m, p, K, src_lr[k]);
        call(tdmrg_kernel_expansion_vjp(0, Ml, Mr, dd[k], Dl, Dr, Wd[k].data(), np, dWp(k),
                                        Lenv[k], a1_lr[k], Xfullb, e1, s1, tht.data(), X_, Y_,
                                        sv));
        take_theta();
        add(Lb[k], e1, nL[k]);
        add(a1b, s1, n[k]);
      }
    } else {
      copy(a1b, ab[L - 1], n[L - 1]);
    }
    // a1 = exp(h H_eff(Lenv[k], W, Rin[k])) ain
    site_vjp(k, Lenv[k], Rin[k], ain_lr[k], a1b, ab[k], e1, e2);
    take_theta();
    add(Lb[k], e1, nL[k]);
    add(Rib[k], e2, nR[k]);
  }
  // right environments of the input: Rin[k-1] = env_right(Rin[k], A_in[k], W, A_in[k])
  for (int k = 1; k < L; ++k) {
    const DevMpoSite& W = H_.s[k];
    call(tdmrg_kernel_env_vjp(1, Mb[k], Mb[k + 1], dd[k], W.Dl, W.Dr, Wd[k].data(), np, dWp(k),
                              Rin[k], A_in[k], A_in[k], Rib[k - 1], e1, s1, s2, tht.data(), X_,
                              Y_, sv));
    take_theta();
    add(Rib[k], e1, nR[k]);
    add(ab[k], s1, n[k]);
    add(ab[k], s2, n[k]);
  }
  for (int k = 0; k < L; ++k) copy(Abar_in[k], ab[k], n[k]);
  for (int p = 0; p < np; ++p) theta_bar[p] = th[p];
  CK(cudaStreamSynchronize(st_));
  check_status();
}

void Engine::overlap_vjp(const std::vector<cplx*>& bra, const std::vector<cplx*>& ket,
                         const std::vector<int>& Mb, Cx cbar, const std::vector<cplx*>& gbra,
                         const std::vector<cplx*>& gket, std::vector<double>& theta) {
  const int L = (int)sites_.size();
  const int np = parameter_count(P);
  std::vector<long long> n(L), ne(L + 1);
  long long maxenv = 1, maxsite = 1;
  for (int k = 0; k < L; ++k) {
    n[k] = (long long)Mb[k] * sites_[k].d * sites_[k].d * Mb[k + 1];
    ne[k] = (long long)J_.s[k].Dl * Mb[k] * Mb[k];
    maxenv = std::max(maxenv, ne[k]);
    maxsite = std::max(maxsite, n[k]);
  }
  ne[L] = 1;
  Tape tp;
  std::vector<cplx*> e(L + 1);
  for (int k = 0; k <= L; ++k) e[k] = tp.get(ne[k]);
  Ctx c = ctx();
  // forward chain e_{k+1} = env_left(e_k, bra_k, j_k, ket_k)
  set_ones(e[0]);
  for (int k = 0; k < L; ++k) {
    const int d = sites_[k].d;
    env_left_f64(c, J_.s[k], Mb[k], Mb[k + 1], Mb[k], Mb[k + 1], d * d, d, e[k], bra[k], ket[k],
                 e[k + 1]);
  }
  // reverse: the cotangent of the 1 x 1 x 1 final environment is cbar
  cplx* G[2] = {tp.get(maxenv), tp.get(maxenv)};
  cplx* bb = tp.get(maxsite);
  cplx* kb = tp.get(maxsite);
  const cplx cb = {cbar.real(), cbar.imag()};
  CK(cudaMemcpyAsync(G[L & 1], &cb, sizeof(cplx), cudaMemcpyHostToDevice, st_));
  CK(cudaStreamSynchronize(st_));
  std::vector<double> tht(np > 0 ? np : 1, 0.0);
  for (int k = L - 1; k >= 0; --k) {
    const DevMpoSite& W = J_.s[k];
    const int d = sites_[k].d;
    const std::vector<double> Wd = dense_site(W.Dl, W.Dr, d, W.host);
    std::vector<double> dWd;
    for (int p = 0; p < np; ++p) {
      const std::vector<double> x = dense_site(W.Dl, W.Dr, d, mpo_site_derivative(P, 1, p, k).blocks);
      dWd.insert(dWd.end(), x.begin(), x.end());
    }
    call(tdmrg_kernel_env_vjp(0, Mb[k], Mb[k + 1], d, W.Dl, W.Dr, Wd.data(), np,
                              np > 0 ? dWd.data() : nullptr, e[k], bra[k], ket[k], G[(k + 1) & 1],
                              G[k & 1], bb, kb, tht.data(), X_, Y_, (void*)st_));
    for (int p = 0; p < np; ++p) theta[p] += tht[p];
    CK(zaxpy(n[k], kOne, bb, gbra[k], st_));
    CK(zaxpy(n[k], kOne, kb, gket[k], st_));
  }
  CK(cudaStreamSynchronize(st_));
}

void Engine::correlation_states_vjp(int M, const cplx* const* psi1, const cplx* const* psi2,
                                    double dt, int nsteps, int every, const double* cbar,
                                    double* C, cplx* const* g1_out, cplx* const* g2_out,
                                    double* theta_bar, int nodes) {
  if (mixed())
    throw Failure{TDMRG_ERR_ARG, "correlation_states_vjp: the reverse pass runs in FP64 precision"};
  if (nsteps < 0 || every < 1) throw Failure{TDMRG_ERR_ARG, "correlation_states_vjp: bad counts"};
  const int L = (int)sites_.size();
  const int np = parameter_count(P);
  DevMps s1, s2;
  struct Free {
    Engine& e;
    DevMps& a;
    DevMps& b;
    ~Free() {
      e.free_mps(a);
      e.free_mps(b);
    }
  } fr{*this, s1, s2};
  alloc_mps(s1, M);
  alloc_mps(s2, M);
  const std::vector<int>& Mb = s1.Mb;
  std::vector<long long> n(L);
  for (int k = 0; k < L; ++k) n[k] = s1.size(k);
  Tape tp;
  auto snapshot = [&](const DevMps& s) {
    std::vector<cplx*> out(L);
    for (int k = 0; k < L; ++k) {
      out[k] = tp.get(n[k]);
      CK(cudaMemcpyAsync(out[k], s.A[k], sizeof(cplx) * (size_t)n[k], cudaMemcpyDeviceToDevice,
                         st_));
    }
    return out;
  };
  auto load = [&](DevMps& s, const std::vector<cplx*>& a) {
    for (int k = 0; k < L; ++k)
      CK(cudaMemcpyAsync(s.A[k], a[k], sizeof(cplx) * (size_t)n[k], cudaMemcpyDeviceToDevice,
                         st_));
    build_right_envs(s);
  };
  auto step = [&](DevMps& s) {
    tdvp_step_body(s, 0.0, -dt);
    check_status();
  };
  // forward: C_n and the stored states
  std::vector<cplx*> p1(L), p2(L);     // read only
  for (int k = 0; k < L; ++k) {
    p1[k] = const_cast<cplx*>(psi1[k]);
    p2[k] = const_cast<cplx*>(psi2[k]);
  }
  struct Ckpt {
    int n;
    std::vector<cplx*> a, b;
  };
  std::vector<Ckpt> ck;
  load(s1, p1);
  load(s2, p2);
  ck.push_back({0, snapshot(s1), snapshot(s2)});
  for (int t = 0; t <= nsteps; ++t) {
    if (t > 0) {
      step(s1);
      step(s2);
      if (t % every == 0 && t < nsteps) ck.push_back({t, snapshot(s1), snapshot(s2)});
    }
    const Cx v = overlap(s1, J_, s2);
    C[2 * t] = v.real();
    C[2 * t + 1] = v.imag();
  }
  // reverse over the stretches between stored states, latest first
  std::vector<cplx*> g1(L), g2(L), h1(L), h2(L);
  for (int k = 0; k < L; ++k) {
    g1[k] = tp.get(n[k]);
    g2[k] = tp.get(n[k]);
    h1[k] = tp.get(n[k]);
    h2[k] = tp.get(n[k]);
    CK(cudaMemsetAsync(g1[k], 0, sizeof(cplx) * (size_t)n[k], st_));
    CK(cudaMemsetAsync(g2[k], 0, sizeof(cplx) * (size_t)n[k], st_));
  }
  std::vector<double> th(np, 0.0), ths(np > 0 ? np : 1, 0.0);
  auto cb = [&](int t) { return Cx(cbar[2 * t], cbar[2 * t + 1]); };
  for (int i = (int)ck.size() - 1; i >= 0; --i) {
    const int s0 = ck[i].n;
    const int e0 = (i + 1 < (int)ck.size()) ? ck[i + 1].n : nsteps;
    if (e0 <= s0) continue;
    std::vector<std::vector<cplx*>> st1{ck[i].a}, st2{ck[i].b};
    Tape seg;
    load(s1, ck[i].a);
    load(s2, ck[i].b);
    for (int t = s0 + 1; t <= e0; ++t) {
      step(s1);
      step(s2);
      std::vector<cplx*> a(L), b(L);
      for (int k = 0; k < L; ++k) {
        a[k] = seg.get(n[k]);
        b[k] = seg.get(n[k]);
        CK(cudaMemcpyAsync(a[k], s1.A[k], sizeof(cplx) * (size_t)n[k], cudaMemcpyDeviceToDevice,
                           st_));
        CK(cudaMemcpyAsync(b[k], s2.A[k], sizeof(cplx) * (size_t)n[k], cudaMemcpyDeviceToDevice,
                           st_));
      }
      st1.push_back(a);
      st2.push_back(b);
    }
    for (int t = e0; t > s0; --t) {
      overlap_vjp(st1[t - s0], st2[t - s0], Mb, cb(t), g1, g2, th);
      step_vjp(M, st1[t - s0 - 1].data(), 0.0, -dt, g1.data(), nullptr, h1.data(), ths.data(),
               nodes, false, 0.0, nullptr);
      for (int p = 0; p < np; ++p) th[p] += ths[p];
      step_vjp(M, st2[t - s0 - 1].data(), 0.0, -dt, g2.data(), nullptr, h2.data(), ths.data(),
               nodes, false, 0.0, nullptr);
      for (int p = 0; p < np; ++p) th[p] += ths[p];
      std::swap(g1, h1);
      std::swap(g2, h2);
    }
  }
  overlap_vjp(ck[0].a, ck[0].b, Mb, cb(0), g1, g2, th);
  for (int k = 0; k < L; ++k) {
    CK(cudaMemcpyAsync(g1_out[k], g1[k], sizeof(cplx) * (size_t)n[k], cudaMemcpyDeviceToDevice,
                       st_));
    CK(cudaMemcpyAsync(g2_out[k], g2[k], sizeof(cplx) * (size_t)n[k], cudaMemcpyDeviceToDevice,
                       st_));
  }
  for (int p = 0; p < np; ++p) theta_bar[p] = th[p];
  CK(cudaStreamSynchronize(st_));
}

namespace {
// sizes of one call's MPS: bond dimensions, local dimensions, site sizes
struct Dims {
  std::vector<int> Mb, D, d;
  std::vector<long long> n;
  long long maxsite = 1, maxxy = 1, maxenv = 1;
  int maxbond = 1;
};
}  // namespace

static Dims make_dims(const std::vector<SiteInfo>& sites, int M, int Dmax) {
  Dims z;
  const int L = (int)sites.size();
  z.Mb = bond_dimensions(sites, M);
  z.D.resize(L);
  z.d.resize(L);
  z.n.resize(L);
  for (int k = 0; k < L; ++k) {
    z.d[k] = sites[k].d;
    z.D[k] = z.d[k] * z.d[k];
    z.n[k] = (long long)z.Mb[k] * z.D[k] * z.Mb[k + 1];
    z.maxsite = std::max(z.maxsite, z.n[k]);
    z.maxxy = std::max(z.maxxy, (long long)Dmax * z.n[k]);
    z.maxenv = std::max(z.maxenv, (long long)Dmax * z.Mb[k] * z.Mb[k]);
    z.maxenv = std::max(z.maxenv, (long long)Dmax * z.Mb[k + 1] * z.Mb[k + 1]);
    z.maxbond = std::max(z.maxbond, z.Mb[k + 1]);
  }
  z.maxxy = std::max(z.maxxy, (long long)Dmax * z.maxbond * z.maxbond);
  return z;
}

void Engine::canonicalize_vjp(int M, cplx* const* psi0, const cplx* const* gbar, double logn_bar,
                              double* theta, double* log_norm) {
  const int L = (int)sites_.size();
  const Dims z = make_dims(sites_, M, std::max(H_.maxD, J_.maxD));
  ensure_workspace(z.maxsite, z.maxxy, z.maxbond, z.maxbond);
  const int np = parameter_count(P);
  std::vector<std::vector<double>> Wd(L), dWd(L);
  for (int k = 0; k < L; ++k) {
    const DevMpoSite& W = H_.s[k];
    Wd[k] = dense_site(W.Dl, W.Dr, W.d, W.host);
    for (int p = 0; p < np; ++p) {
      const auto x = dense_site(W.Dl, W.Dr, W.d, mpo_site_derivative(P, 0, p, k).blocks);
      dWd[k].insert(dWd[k].end(), x.begin(), x.end());
    }
  }
  auto copy = [&](cplx* dst, const cplx* src, long long cnt) {
    CK(cudaMemcpyAsync(dst, src, sizeof(cplx) * (size_t)cnt, cudaMemcpyDeviceToDevice, st_));
  };
  Ctx c = ctx();
  Tape tp;
  std::vector<cplx*> A(L), Renv(L), ain(L), Q2(L), R2(L), Qs(L), Cm(L), nxt(L);
  std::vector<std::vector<unsigned char>> acc(L);
  std::vector<std::vector<int>> src(L);
  std::vector<long long> nR(L);
  // |I> on the one-carrier sector
  const auto ent = identity_state_entries(P);
  size_t maxe = 1;
  for (auto& e : ent) maxe = std::max(maxe, e.size());
  int* d_ent = tp.geti((long long)maxe);
  for (int k = 0; k < L; ++k) {
    A[k] = tp.get(z.n[k]);
    nR[k] = (long long)H_.s[k].Dr * z.Mb[k + 1] * z.Mb[k + 1];
    Renv[k] = tp.get(nR[k]);
    CK(cudaMemcpy(d_ent, ent[k].data(), sizeof(int) * ent[k].size(), cudaMemcpyHostToDevice));
    CK(zfill_identity_mps(A[k], z.Mb[k], z.D[k], z.Mb[k + 1], d_ent, (int)ent[k].size() / 3, st_));
    CK(cudaStreamSynchronize(st_));
  }
  int* src_dev = tp.geti(z.maxbond);
  set_ones(Renv[L - 1]);
  for (int k = L - 1; k > 0; --k) {
    const DevMpoSite& W = H_.s[k];
    const int Ml = z.Mb[k], Mr = z.Mb[k + 1];
    const long long m = (long long)z.D[k] * Mr;
    ain[k] = tp.get(z.n[k]);
    copy(ain[k], A[k], z.n[k]);
    right_partial_f64(c, W, Ml, z.D[k], z.d[k], Mr, Mr, Renv[k], A[k], Y_, nullptr);
    CK(cudaMemsetAsync(src_dev, 0xff, sizeof(int) * (size_t)Ml, st_));
    Q2[k] = tp.get(z.n[k]);
    R2[k] = tp.get((long long)Ml * Ml);
    gauge_qr_dev((int)m, Ml, qr(A[k], 1, m, kNoSplit, 0, 1), W.Dl * Ml, qr(Y_, 1, m, kNoSplit, 0, 1),
                 Q2[k], R2[k], src_dev);
    acc[k].resize(Ml);
    src[k].resize(Ml);
    CK(cudaMemcpyAsync(acc[k].data(), qb_acc_, (size_t)Ml, cudaMemcpyDeviceToHost, st_));
    CK(cudaMemcpyAsync(src[k].data(), src_dev, sizeof(int) * (size_t)Ml, cudaMemcpyDeviceToHost,
                       st_));
    CK(cudaStreamSynchronize(st_));
    Qs[k] = tp.get(z.n[k]);
    Cm[k] = tp.get((long long)Ml * Ml);
    CK(ztranspose((int)m, Ml, Q2[k], Qs[k], 1, st_));
    CK(ztranspose(Ml, Ml, R2[k], Cm[k], 1, st_));
    env_right_f64(c, W, Ml, Mr, Ml, Mr, z.D[k], z.d[k], Renv[k], Qs[k], Qs[k], Renv[k - 1]);
    nxt[k] = tp.get(z.n[k - 1]);
    copy(nxt[k], A[k - 1], z.n[k - 1]);
    const long long nrows = (long long)z.Mb[k - 1] * z.D[k - 1];
    CK(zgemm((int)nrows, Ml, Ml, 1, 1, kOne, mr(nxt[k], Ml, 1), mr(Cm[k], Ml, 1), kZero, A[k - 1],
             Ml, 0, nullptr, st_));
    copy(A[k], Qs[k], z.n[k]);
  }
  cplx* part = tp.get(257);
  const double nrm = std::sqrt(dot(A[0], A[0], z.n[0], part, st_).real());
  if (!std::isfinite(nrm) || nrm <= 0.0)
    throw Failure{TDMRG_ERR_NONFINITE, "canonicalize_vjp: non-finite norm"};
  cplx* A0raw = tp.get(z.n[0]);
  copy(A0raw, A[0], z.n[0]);
  scale_dev(A[0], z.n[0], 1.0 / nrm);
  if (log_norm) *log_norm = 2.0 * std::log(nrm);
  for (int k = 0; k < L; ++k) copy(psi0[k], A[k], z.n[k]);
  check_status();
  if (!gbar) {
    CK(cudaStreamSynchronize(st_));
    return;
  }
  // ---- reverse ----
  std::vector<cplx*> ab(L), Rb(L);
  for (int k = 0; k < L; ++k) {
    ab[k] = tp.get(z.n[k]);
    copy(ab[k], gbar[k], z.n[k]);
    Rb[k] = tp.get(nR[k]);
    CK(cudaMemsetAsync(Rb[k], 0, sizeof(cplx) * (size_t)nR[k], st_));
  }
  {
    const double re = dot(A[0], ab[0], z.n[0], part, st_).real();
    const cplx f = {-re, 0.0};
    CK(zaxpy(z.n[0], f, A[0], ab[0], st_));
    scale_dev(ab[0], z.n[0], 1.0 / nrm);
    if (logn_bar != 0.0) {
      const cplx lf = {2.0 * logn_bar / (nrm * nrm), 0.0};
      CK(zaxpy(z.n[0], lf, A0raw, ab[0], st_));
    }
  }
  ShiftScratch w{tp.get(z.maxsite), tp.get(z.maxsite), tp.get((long long)z.maxbond * z.maxbond),
                 tp.get(z.maxsite), tp.get(z.maxsite), tp.get(z.maxxy), tp.get(z.maxxy),
                 tp.get(z.maxenv), tp.get(z.maxsite)};
  cplx* bb = tp.get(z.maxsite);
  cplx* kb = tp.get(z.maxsite);
  cplx* qsb = tp.get(z.maxsite);
  cplx* t1 = tp.get(z.maxsite);
  cplx* a1b = tp.get(z.maxsite);
  cplx* e1 = tp.get(z.maxenv);
  cplx* cmb = tp.get((long long)z.maxbond * z.maxbond);
  std::vector<double> tht(np > 0 ? np : 1, 0.0);
  for (int k = 1; k < L; ++k) {
    const DevMpoSite& W = H_.s[k];
    const int Ml = z.Mb[k], Mr = z.Mb[k + 1];
    const long long nrows = (long long)z.Mb[k - 1] * z.D[k - 1];
    // A[k-1] = nxt Cm:  Cmbar = nxt^H abar,  abar <- abar Cm^H
    CK(zgemm(Ml, Ml, (int)nrows, 1, 1, kOne, mr(nxt[k], 1, Ml, 1), mr(ab[k - 1], Ml, 1), kZero,
             cmb, Ml, 0, nullptr, st_));
    CK(zgemm((int)nrows, Ml, Ml, 1, 1, kOne, mr(ab[k - 1], Ml, 1), mr(Cm[k], 1, Ml, 1), kZero, t1,
             Ml, 0, nullptr, st_));
    copy(ab[k - 1], t1, z.n[k - 1]);
    // Renv[k-1] = env_right(Renv[k], Qs, W, Qs)
    call(tdmrg_kernel_env_vjp(1, Ml, Mr, z.d[k], W.Dl, W.Dr, Wd[k].data(), np,
                              np > 0 ? dWd[k].data() : nullptr, Renv[k], Qs[k], Qs[k], Rb[k - 1],
                              e1, bb, kb, tht.data(), X_, Y_, (void*)st_));
    for (int q = 0; q < np; ++q) theta[q] += tht[q];
    CK(zaxpy(nR[k], kOne, e1, Rb[k], st_));
    copy(qsb, ab[k], z.n[k]);
    CK(zaxpy(z.n[k], kOne, bb, qsb, st_));
    CK(zaxpy(z.n[k], kOne, kb, qsb, st_));
    // LQ of ain with completions from right_partial(Renv[k], W, ain)
    qr_left_reverse(c, w, X_, Y_, W, Wd[k].data(), np, np > 0 ? dWd[k].data() : nullptr, Ml, Mr,
                    z.d[k], Renv[k], ain[k], Q2[k], R2[k], acc[k], src[k], qsb, cmb, a1b, Rb[k],
                    a1b, theta, tht);
    copy(ab[k], a1b, z.n[k]);
  }
  CK(cudaStreamSynchronize(st_));
  check_status();
}

void Engine::fit_vjp(int M, const cplx* const* psi, cplx* const* phi, const cplx* const* gphi,
                     cplx* const* gpsi, double* theta) {
  const int L = (int)sites_.size();
  const Dims z = make_dims(sites_, M, std::max(H_.maxD, J_.maxD));
  ensure_workspace(z.maxsite, z.maxxy, z.maxbond, z.maxbond);
  const int np = parameter_count(P);
  constexpr int S = 2;   // sweeps, as in realtime_init
  std::vector<std::vector<double>> Jd(L), dJd(L);
  for (int k = 0; k < L; ++k) {
    const DevMpoSite& W = J_.s[k];
    Jd[k] = dense_site(W.Dl, W.Dr, W.d, W.host);
    for (int p = 0; p < np; ++p) {
      const auto x = dense_site(W.Dl, W.Dr, W.d, mpo_site_derivative(P, 1, p, k).blocks);
      dJd[k].insert(dJd[k].end(), x.begin(), x.end());
    }
  }
  auto dJ = [&](int k) { return np > 0 ? dJd[k].data() : nullptr; };
  auto copy = [&](cplx* dst, const cplx* src, long long cnt) {
    CK(cudaMemcpyAsync(dst, src, sizeof(cplx) * (size_t)cnt, cudaMemcpyDeviceToDevice, st_));
  };
  std::vector<long long> nLj(L), nRj(L);
  for (int k = 0; k < L; ++k) {
    nLj[k] = (long long)J_.s[k].Dl * z.Mb[k] * z.Mb[k];
    nRj[k] = (long long)J_.s[k].Dr * z.Mb[k + 1] * z.Mb[k + 1];
  }
  Ctx c = ctx();
  Tape tp;
  int* src_dev = tp.geti(z.maxbond);
  auto flags = [&](int cols, std::vector<unsigned char>& acc, std::vector<int>& src) {
    acc.resize(cols);
    src.resize(cols);
    CK(cudaMemcpyAsync(acc.data(), qb_acc_, (size_t)cols, cudaMemcpyDeviceToHost, st_));
    CK(cudaMemcpyAsync(src.data(), src_dev, sizeof(int) * (size_t)cols, cudaMemcpyDeviceToHost,
                       st_));
    CK(cudaStreamSynchronize(st_));
  };
  // initial right environments, phi = psi: Rf0[k-1] = env_right(Rf0[k], psi, j, psi)
  std::vector<cplx*> Rf0(L);
  for (int k = 0; k < L; ++k) Rf0[k] = tp.get(nRj[k]);
  set_ones(Rf0[L - 1]);
  for (int k = L - 1; k > 0; --k)
    env_right_f64(c, J_.s[k], z.Mb[k], z.Mb[k + 1], z.Mb[k], z.Mb[k + 1], z.D[k], z.d[k], Rf0[k],
                  psi[k], psi[k], Rf0[k - 1]);
  struct Sweep {
    std::vector<cplx*> Lf, Rn, a_lr, Q_lr, R_lr, a_rl, Q2_rl, R2_rl, Qs_rl;
    std::vector<std::vector<unsigned char>> acc_lr, acc_rl;
    std::vector<std::vector<int>> src_lr, src_rl;
  };
  std::vector<Sweep> sw(S);
  std::vector<cplx*> ph(L);
  for (int s = 0; s < S; ++s) {
    Sweep& q = sw[s];
    for (auto* v : {&q.Lf, &q.Rn, &q.a_lr, &q.Q_lr, &q.R_lr, &q.a_rl, &q.Q2_rl, &q.R2_rl, &q.Qs_rl})
      v->assign(L, nullptr);
    q.acc_lr.resize(L);
    q.acc_rl.resize(L);
    q.src_lr.resize(L);
    q.src_rl.resize(L);
    const std::vector<cplx*>& Rin = s == 0 ? Rf0 : sw[s - 1].Rn;
    for (int k = 0; k < L; ++k) q.Lf[k] = tp.get(nLj[k]);
    set_ones(q.Lf[0]);
    for (int k = 0; k < L; ++k) {
      const DevMpoSite& W = J_.s[k];
      const int Ml = z.Mb[k], Mr = z.Mb[k + 1];
      q.a_lr[k] = tp.get(z.n[k]);
      heff_f64(c, W, Ml, Mr, z.D[k], z.d[k], q.Lf[k], Rin[k], psi[k], q.a_lr[k], nullptr);
      if (k == L - 1) {
        ph[k] = q.a_lr[k];
        continue;
      }
      left_partial_f64(c, W, Ml, Ml, z.D[k], z.d[k], Mr, q.Lf[k], psi[k], Y_, nullptr);
      CK(cudaMemsetAsync(src_dev, 0xff, sizeof(int) * (size_t)Mr, st_));
      q.Q_lr[k] = tp.get(z.n[k]);
      q.R_lr[k] = tp.get((long long)Mr * Mr);
      gauge_qr_dev(Ml * z.D[k], Mr, qr(q.a_lr[k], Mr, 1, kNoSplit, 0, 0), W.Dr * Mr,
                   qr(Y_, Mr, 1, Mr, z.n[k], 0), q.Q_lr[k], q.R_lr[k], src_dev);
      flags(Mr, q.acc_lr[k], q.src_lr[k]);
      env_left_f64(c, W, Ml, Mr, Ml, Mr, z.D[k], z.d[k], q.Lf[k], q.Q_lr[k], psi[k], q.Lf[k + 1]);
      ph[k] = q.Q_lr[k];
    }
    for (int k = 0; k < L; ++k) q.Rn[k] = tp.get(nRj[k]);
    set_ones(q.Rn[L - 1]);
    for (int k = L - 1; k >= 0; --k) {
      const DevMpoSite& W = J_.s[k];
      const int Ml = z.Mb[k], Mr = z.Mb[k + 1];
      const long long m = (long long)z.D[k] * Mr;
      q.a_rl[k] = tp.get(z.n[k]);
      heff_f64(c, W, Ml, Mr, z.D[k], z.d[k], q.Lf[k], q.Rn[k], psi[k], q.a_rl[k], nullptr);
      if (k == 0) {
        ph[0] = q.a_rl[0];
        continue;
      }
      right_partial_f64(c, W, Ml, z.D[k], z.d[k], Mr, Mr, q.Rn[k], psi[k], Y_, nullptr);
      CK(cudaMemsetAsync(src_dev, 0xff, sizeof(int) * (size_t)Ml, st_));
      q.Q2_rl[k] = tp.get(z.n[k]);
      q.R2_rl[k] = tp.get((long long)Ml * Ml);
      gauge_qr_dev((int)m, Ml, qr(q.a_rl[k], 1, m, kNoSplit, 0, 1), W.Dl * Ml,
                   qr(Y_, 1, m, kNoSplit, 0, 1), q.Q2_rl[k], q.R2_rl[k], src_dev);
      flags(Ml, q.acc_rl[k], q.src_rl[k]);
      q.Qs_rl[k] = tp.get(z.n[k]);
      CK(ztranspose((int)m, Ml, q.Q2_rl[k], q.Qs_rl[k], 1, st_));
      env_right_f64(c, W, Ml, Mr, Ml, Mr, z.D[k], z.d[k], q.Rn[k], q.Qs_rl[k], psi[k],
                    q.Rn[k - 1]);
      ph[k] = q.Qs_rl[k];
    }
  }
  for (int k = 0; k < L; ++k) copy(phi[k], ph[k], z.n[k]);
  check_status();
  if (!gphi) {
    CK(cudaStreamSynchronize(st_));
    return;
  }
  // ---- reverse ----
  std::vector<std::vector<cplx*>> Lb(S, std::vector<cplx*>(L)), Rnb(S, std::vector<cplx*>(L));
  std::vector<cplx*> R0b(L);
  for (int k = 0; k < L; ++k) {
    R0b[k] = tp.get(nRj[k]);
    CK(cudaMemsetAsync(R0b[k], 0, sizeof(cplx) * (size_t)nRj[k], st_));
    for (int s = 0; s < S; ++s) {
      Lb[s][k] = tp.get(nLj[k]);
      Rnb[s][k] = tp.get(nRj[k]);
      CK(cudaMemsetAsync(Lb[s][k], 0, sizeof(cplx) * (size_t)nLj[k], st_));
      CK(cudaMemsetAsync(Rnb[s][k], 0, sizeof(cplx) * (size_t)nRj[k], st_));
    }
  }
  ShiftScratch w{tp.get(z.maxsite), tp.get(z.maxsite), tp.get((long long)z.maxbond * z.maxbond),
                 tp.get(z.maxsite), tp.get(z.maxsite), tp.get(z.maxxy), tp.get(z.maxxy),
                 tp.get(z.maxenv), tp.get(z.maxsite)};
  cplx* phib = tp.get(z.maxsite);
  cplx* ab = tp.get(z.maxsite);
  cplx* bb = tp.get(z.maxsite);
  cplx* kb = tp.get(z.maxsite);
  cplx* tA = tp.get(z.maxsite);
  cplx* e1 = tp.get(z.maxenv);
  cplx* tL = tp.get(z.maxenv);
  cplx* tR = tp.get(z.maxenv);
  cplx* part = tp.get(257);
  std::vector<double> tht(np > 0 ? np : 1, 0.0);
  // a = H_eff(L, j, R) psi with cotangent abar: psi, L, R cotangents and the parameters
  auto heff_reverse = [&](int k, const cplx* Le, const cplx* Re, const cplx* abar, cplx* Lbar,
                          cplx* Rbar) {
    const DevMpoSite& W = J_.s[k];
    const int Ml = z.Mb[k], Mr = z.Mb[k + 1];
    call(tdmrg_kernel_heff_vjp(Ml, Mr, z.d[k], W.Dl, W.Dr, Jd[k].data(), Le, Re, psi[k], abar, tA,
                               tL, tR, X_, Y_, (void*)st_));
    CK(zaxpy(z.n[k], kOne, tA, gpsi[k], st_));
    CK(zaxpy(nLj[k], kOne, tL, Lbar, st_));
    CK(zaxpy(nRj[k], kOne, tR, Rbar, st_));
    for (int p = 0; p < np; ++p) {
      const MpoSite dW = mpo_site_derivative(P, 1, p, k);
      if (dW.blocks.empty()) continue;
      DevMpo dm;
      upload_mpo({dW}, dm);
      struct FreeMpo {
        DevMpo& m;
        ~FreeMpo() { free_mpo(m); }
      } fm{dm};
      heff_f64(c, dm.s[0], Ml, Mr, z.D[k], z.d[k], Le, Re, psi[k], bb, nullptr);
      theta[p] += dot(abar, bb, z.n[k], part, st_).real();
    }
  };
  for (int s = S - 1; s >= 0; --s) {
    Sweep& q = sw[s];
    std::vector<cplx*>& Rinb = s == 0 ? R0b : Rnb[s - 1];
    const std::vector<cplx*>& Rin = s == 0 ? Rf0 : sw[s - 1].Rn;
    // right-to-left half, last update first; the output phi is this half's last sweep
    for (int k = 0; k < L; ++k) {
      const DevMpoSite& W = J_.s[k];
      const int Ml = z.Mb[k], Mr = z.Mb[k + 1];
      if (s == S - 1)
        copy(phib, gphi[k], z.n[k]);
      else
        CK(cudaMemsetAsync(phib, 0, sizeof(cplx) * (size_t)z.n[k], st_));
      if (k > 0) {
        // Rn[k-1] = env_right(Rn[k], Qs (bra), j, psi (ket))
        call(tdmrg_kernel_env_vjp(1, Ml, Mr, z.d[k], W.Dl, W.Dr, Jd[k].data(), np, dJ(k),
                                  q.Rn[k], q.Qs_rl[k], psi[k], Rnb[s][k - 1], e1, bb, kb,
                                  tht.data(), X_, Y_, (void*)st_));
        for (int p = 0; p < np; ++p) theta[p] += tht[p];
        CK(zaxpy(nRj[k], kOne, e1, Rnb[s][k], st_));
        CK(zaxpy(z.n[k], kOne, bb, phib, st_));
        CK(zaxpy(z.n[k], kOne, kb, gpsi[k], st_));
        qr_left_reverse(c, w, X_, Y_, W, Jd[k].data(), np, dJ(k), Ml, Mr, z.d[k], q.Rn[k], psi[k],
                        q.Q2_rl[k], q.R2_rl[k], q.acc_rl[k], q.src_rl[k], phib, nullptr, ab,
                        Rnb[s][k], gpsi[k], theta, tht);
      } else {
        copy(ab, phib, z.n[0]);
      }
      heff_reverse(k, q.Lf[k], q.Rn[k], ab, Lb[s][k], Rnb[s][k]);
    }
    // left-to-right half, last update first (its last site is overwritten unread)
    for (int k = L - 2; k >= 0; --k) {
      const DevMpoSite& W = J_.s[k];
      const int Ml = z.Mb[k], Mr = z.Mb[k + 1];
      // Lf[k+1] = env_left(Lf[k], Q (bra), j, psi (ket))
      call(tdmrg_kernel_env_vjp(0, Ml, Mr, z.d[k], W.Dl, W.Dr, Jd[k].data(), np, dJ(k), q.Lf[k],
                                q.Q_lr[k], psi[k], Lb[s][k + 1], e1, phib, kb, tht.data(), X_, Y_,
                                (void*)st_));
      for (int p = 0; p < np; ++p) theta[p] += tht[p];
      CK(zaxpy(nLj[k], kOne, e1, Lb[s][k], st_));
      CK(zaxpy(z.n[k], kOne, kb, gpsi[k], st_));
      qr_right_reverse(c, w, X_, Y_, W, Jd[k].data(), np, dJ(k), Ml, Mr, z.d[k], q.Lf[k], psi[k],
                       q.Q_lr[k], q.R_lr[k], q.acc_lr[k], q.src_lr[k], phib, nullptr, ab,
                       Lb[s][k], gpsi[k], theta, tht);
      heff_reverse(k, q.Lf[k], Rin[k], ab, Lb[s][k], Rinb[k]);
    }
  }
  // the initial right environments (bra and ket both psi)
  for (int k = 1; k < L; ++k) {
    const DevMpoSite& W = J_.s[k];
    call(tdmrg_kernel_env_vjp(1, z.Mb[k], z.Mb[k + 1], z.d[k], W.Dl, W.Dr, Jd[k].data(), np,
                              dJ(k), Rf0[k], psi[k], psi[k], R0b[k - 1], e1, bb, kb, tht.data(),
                              X_, Y_, (void*)st_));
    for (int p = 0; p < np; ++p) theta[p] += tht[p];
    CK(zaxpy(nRj[k], kOne, e1, R0b[k], st_));
    CK(zaxpy(z.n[k], kOne, bb, gpsi[k], st_));
    CK(zaxpy(z.n[k], kOne, kb, gpsi[k], st_));
  }
  CK(cudaStreamSynchronize(st_));
  check_status();
}

void Engine::correlation_vjp(double beta, double dtau, int M, double dt, int nsteps, int every,
                             const double* cbar, double* C, double* theta_bar, double* logz,
                             int nodes) {
  if (mixed()) throw Failure{TDMRG_ERR_ARG, "correlation_vjp: the reverse pass runs in FP64 precision"};
  if (!(beta > 0.0) || !(dtau > 0.0) || M < 2 || !(dt > 0.0) || nsteps < 0 || every < 1)
    throw Failure{TDMRG_ERR_ARG, "correlation_vjp: bad arguments"};
  const long long ntau = std::llround(beta / (2.0 * dtau));
  if (ntau < 1 || std::fabs(ntau * 2.0 * dtau - beta) > 1e-9 * std::max(1.0, beta))
    throw Failure{TDMRG_ERR_ARG, "correlation_vjp: beta must be an even multiple of dtau"};
  const int L = (int)sites_.size();
  const int np = parameter_count(P);
  const Dims z = make_dims(sites_, M, std::max(H_.maxD, J_.maxD));
  Tape tp;
  auto state = [&]() {
    std::vector<cplx*> a(L);
    for (int k = 0; k < L; ++k) a[k] = tp.get(z.n[k]);
    return a;
  };
  std::vector<double> th(np, 0.0), ths(np > 0 ? np : 1, 0.0);
  // forward: |I> canonicalised and normalised, imaginary-time steps each normalised, the fit
  std::vector<std::vector<cplx*>> psi(ntau + 1);
  psi[0] = state();
  double lz = 0.0, ln = 0.0;
  canonicalize_vjp(M, psi[0].data(), nullptr, 0.0, nullptr, &ln);
  lz += ln;
  for (long long i = 1; i <= ntau; ++i) {
    psi[i] = state();
    step_vjp(M, psi[i - 1].data(), -dtau, 0.0, nullptr, psi[i].data(), nullptr, ths.data(), nodes,
             true, 0.0, &ln);
    lz += ln;
  }
  if (logz) *logz = lz;
  std::vector<cplx*> phi = state(), g1 = state(), g2 = state(), h = state();
  fit_vjp(M, psi[ntau].data(), phi.data(), nullptr, nullptr, nullptr);
  // real time with its reverse
  correlation_states_vjp(M, psi[ntau].data(), phi.data(), dt, nsteps, every, cbar, C, g1.data(),
                         g2.data(), ths.data(), nodes);
  for (int p = 0; p < np; ++p) th[p] += ths[p];
  // the fit: psi_beta receives the cotangent through phi
  fit_vjp(M, psi[ntau].data(), h.data(), g2.data(), g1.data(), th.data());
  // the preparation, last step first
  for (long long i = ntau; i >= 1; --i) {
    step_vjp(M, psi[i - 1].data(), -dtau, 0.0, g1.data(), nullptr, h.data(), ths.data(), nodes,
             true, 0.0, nullptr);
    for (int p = 0; p < np; ++p) th[p] += ths[p];
    std::swap(g1, h);
  }
  canonicalize_vjp(M, h.data(), g1.data(), 0.0, th.data(), nullptr);
  for (int p = 0; p < np; ++p) theta_bar[p] = th[p];
  CK(cudaStreamSynchronize(st_));
}

}  // namespace tdmrg
