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
#include <vector>

#include "../../include/tdmrg.h"
#include "engine.h"

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
}  // namespace

void Engine::step_vjp(int M, const cplx* const* A_in, double tr, double ti,
                      const cplx* const* Abar_out, cplx* const* A_out, cplx* const* Abar_in,
                      double* theta_bar, int nodes) {
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
  if (A_out)
    for (int k = 0; k < L; ++k) copy(A_out[k], A[k], n[k]);
  check_status();

  // ---- reverse ----
  std::vector<cplx*> ab(L), Lb(L), Rib(L), Rnb(L);
  for (int k = 0; k < L; ++k) {
    ab[k] = tp.get(n[k]);
    copy(ab[k], Abar_out[k], n[k]);
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
      call(tdmrg_kernel_bond_exp_vjp(Ml, Dl, Lenv[k], Rnew[k - 1], Cm_rl[k], b1, -hr, -hi, nodes,
                                     tol, b2, e1, e2, sv));
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
    call(tdmrg_kernel_site_exp_vjp_theta(Ml, Mr, dd[k], Dl, Dr, Wd[k].data(), Lenv[k], Rnew[k],
                                         ain_rl[k], a1b, hr, hi, nodes, tol, np, dWp(k), ab[k],
                                         e1, e2, tht.data(), sv));
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
      call(tdmrg_kernel_bond_exp_vjp(Mr, Dr, Lenv[k + 1], Rin[k], R_lr[k], b1, -hr, -hi, nodes,
                                     tol, b2, e1, e2, sv));
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
    call(tdmrg_kernel_site_exp_vjp_theta(Ml, Mr, dd[k], Dl, Dr, Wd[k].data(), Lenv[k], Rin[k],
                                         ain_lr[k], a1b, hr, hi, nodes, tol, np, dWp(k), ab[k],
                                         e1, e2, tht.data(), sv));
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
               nodes);
      for (int p = 0; p < np; ++p) th[p] += ths[p];
      step_vjp(M, st2[t - s0 - 1].data(), 0.0, -dt, g2.data(), nullptr, h2.data(), ths.data(),
               nodes);
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

}  // namespace tdmrg
