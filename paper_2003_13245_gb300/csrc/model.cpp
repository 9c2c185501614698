// Host-side model: site list and sparse MPOs of the Holstein(-Peierls) Hamiltonian (Eq. 1,
// Eq. 10) and of the current operator (Eq. 3).  Pure C++, no CUDA.
#include "model.h"

#include <cmath>
#include <stdexcept>

namespace tdmrg {

std::vector<SiteInfo> chain_sites(const ModelParams& P) {
  std::vector<SiteInfo> out;
  for (int n = 0; n < P.N; ++n) {
    out.push_back({SiteInfo::ELEC, n, -1, 2});
    for (int m = 0; m < (int)P.omega.size(); ++m) out.push_back({SiteInfo::MODE, n, m, P.nmax[m]});
    if (P.peierls) out.push_back({SiteInfo::BOND, n, -1, P.nmax_p});
  }
  return out;
}

namespace {

// dense d x d operators, row = output level, column = input level
std::vector<Cx> identity(int d) {
  std::vector<Cx> o(d * d, Cx(0, 0));
  for (int i = 0; i < d; ++i) o[i * d + i] = Cx(1, 0);
  return o;
}
std::vector<Cx> number(int d) {
  std::vector<Cx> o(d * d, Cx(0, 0));
  for (int i = 0; i < d; ++i) o[i * d + i] = Cx(i, 0);
  return o;
}
std::vector<Cx> displacement(int d) {      // b + b^+
  std::vector<Cx> o(d * d, Cx(0, 0));
  for (int v = 1; v < d; ++v) {
    o[(v - 1) * d + v] = Cx(std::sqrt((double)v), 0);
    o[v * d + (v - 1)] = Cx(std::sqrt((double)v), 0);
  }
  return o;
}
std::vector<Cx> raise_e() { return {Cx(0, 0), Cx(0, 0), Cx(1, 0), Cx(0, 0)}; }   // |1><0|
std::vector<Cx> lower_e() { return {Cx(0, 0), Cx(1, 0), Cx(0, 0), Cx(0, 0)}; }   // |0><1|
std::vector<Cx> occ_e() { return {Cx(0, 0), Cx(0, 0), Cx(0, 0), Cx(1, 0)}; }

std::vector<Cx> scaled(std::vector<Cx> o, Cx c) {
  for (auto& x : o) x *= c;
  return o;
}
std::vector<Cx> affine(const std::vector<Cx>& I, const std::vector<Cx>& X, Cx a, Cx b) {
  std::vector<Cx> o(I.size());
  for (size_t i = 0; i < I.size(); ++i) o[i] = a * I[i] + b * X[i];
  return o;
}

void add(MpoSite& s, int wl, int wr, std::vector<Cx> op) { s.blocks.push_back({wl, wr, std::move(op)}); }

// Restrict the first site to its "nothing placed" row and the last to the "closed" column.
void cut_boundaries(std::vector<MpoSite>& W, int open, int closed) {
  std::vector<MpoBlock> first;
  for (auto& b : W.front().blocks)
    if (b.wl == open) first.push_back({0, b.wr, b.op});
  W.front().blocks = first;
  W.front().Dl = 1;
  std::vector<MpoBlock> last;
  for (auto& b : W.back().blocks)
    if (b.wr == closed) last.push_back({b.wl, 0, b.op});
  W.back().blocks = last;
  W.back().Dr = 1;
}

}  // namespace

// Finite-state automaton of H.  Channel meaning (between two sites):
//   OPEN   only identities so far            DONE   one complete term placed
//   UP     c+_n placed, c_{n+1} to come      DN     c_n placed, c+_{n+1} to come
//   DENS   n_e(n) placed, one of molecule n's modes to come
//   RUP    c+_0 placed, c_{N-1} to come      RDN    c_0 placed, c+_{N-1} to come
// With a bond mode the transfer integral V (1 + alpha x) is attached on p_n instead of e_n.
std::vector<MpoSite> hamiltonian_mpo(const ModelParams& P) {
  enum { OPEN = 0, UP, DN, DENS, RUP, RDN, DONE, NCH };
  const auto sites = chain_sites(P);
  std::vector<MpoSite> W;
  const int N = P.N;
  for (const auto& st : sites) {
    MpoSite s;
    s.Dl = s.Dr = NCH;
    s.d = st.d;
    const auto I = identity(st.d);
    add(s, OPEN, OPEN, I);
    add(s, DONE, DONE, I);
    if (st.kind == SiteInfo::ELEC) {
      const Cx hop = P.peierls ? Cx(1, 0) : Cx(P.V, 0);
      const int n = st.mol;
      if (n + 1 < N) {
        add(s, OPEN, UP, scaled(raise_e(), hop));
        add(s, OPEN, DN, scaled(lower_e(), hop));
      }
      if (n > 0) {
        add(s, UP, DONE, lower_e());
        add(s, DN, DONE, raise_e());
      }
      if (n == 0) {
        add(s, OPEN, RUP, scaled(raise_e(), hop));
        add(s, OPEN, RDN, scaled(lower_e(), hop));
      } else if (n == N - 1) {
        const int tgt_up = P.peierls ? RUP : DONE;
        const int tgt_dn = P.peierls ? RDN : DONE;
        add(s, RUP, tgt_up, lower_e());
        add(s, RDN, tgt_dn, raise_e());
      } else {
        add(s, RUP, RUP, I);
        add(s, RDN, RDN, I);
      }
      add(s, OPEN, DENS, occ_e());
    } else if (st.kind == SiteInfo::MODE) {
      const double w = P.omega[st.mode], gm = P.g[st.mode];
      for (int ch : {UP, DN, RUP, RDN, DENS}) add(s, ch, ch, I);
      add(s, OPEN, DONE, scaled(number(st.d), Cx(w, 0)));
      add(s, DENS, DONE, scaled(displacement(st.d), Cx(gm * w, 0)));
    } else {
      const auto Vn = affine(I, displacement(st.d), Cx(P.V, 0), Cx(P.V * P.alpha, 0));
      add(s, OPEN, DONE, scaled(number(st.d), Cx(P.omega_p, 0)));
      if (st.mol + 1 < N) {
        add(s, UP, UP, Vn);
        add(s, DN, DN, Vn);
        add(s, RUP, RUP, I);
        add(s, RDN, RDN, I);
      } else {
        add(s, RUP, DONE, Vn);
        add(s, RDN, DONE, Vn);
      }
    }
    W.push_back(std::move(s));
  }
  cut_boundaries(W, OPEN, DONE);
  return W;
}

// Automaton of j = (V/i) sum_n (c+_{n+1} c_n - c+_n c_{n+1}) on the ring (Eq. 3):
// -iV on every c+_{n+1} c_n, +iV on every c+_n c_{n+1}; the ring bond is n = N-1 -> 0.
std::vector<MpoSite> current_mpo(const ModelParams& P) {
  enum { OPEN = 0, UP, DN, RUP, RDN, DONE, NCH };
  const auto sites = chain_sites(P);
  std::vector<MpoSite> W;
  const int N = P.N;
  const Cx iv = P.peierls ? Cx(0, 1) : Cx(0, P.V);     // i V (V sits on p_n with a bond mode)
  for (const auto& st : sites) {
    MpoSite s;
    s.Dl = s.Dr = NCH;
    s.d = st.d;
    const auto I = identity(st.d);
    add(s, OPEN, OPEN, I);
    add(s, DONE, DONE, I);
    if (st.kind == SiteInfo::ELEC) {
      const int n = st.mol;
      if (n + 1 < N) {
        add(s, OPEN, UP, scaled(raise_e(), iv));       // +iV c+_n c_{n+1}
        add(s, OPEN, DN, scaled(lower_e(), -iv));      // -iV c+_{n+1} c_n
      }
      if (n > 0) {
        add(s, UP, DONE, lower_e());
        add(s, DN, DONE, raise_e());
      }
      if (n == 0) {
        add(s, OPEN, RUP, scaled(raise_e(), -iv));     // -iV c+_0 c_{N-1}
        add(s, OPEN, RDN, scaled(lower_e(), iv));      // +iV c+_{N-1} c_0
      } else if (n == N - 1) {
        add(s, RUP, P.peierls ? RUP : DONE, lower_e());
        add(s, RDN, P.peierls ? RDN : DONE, raise_e());
      } else {
        add(s, RUP, RUP, I);
        add(s, RDN, RDN, I);
      }
    } else if (st.kind == SiteInfo::MODE) {
      for (int ch : {UP, DN, RUP, RDN}) add(s, ch, ch, I);
    } else {
      const auto Vn = affine(I, displacement(st.d), Cx(P.V, 0), Cx(P.V * P.alpha, 0));
      if (st.mol + 1 < N) {
        add(s, UP, UP, Vn);
        add(s, DN, DN, Vn);
        add(s, RUP, RUP, I);
        add(s, RDN, RDN, I);
      } else {
        add(s, RUP, DONE, Vn);
        add(s, RDN, DONE, Vn);
      }
    }
    W.push_back(std::move(s));
  }
  cut_boundaries(W, OPEN, DONE);
  return W;
}

std::vector<MpoSite> identity_mpo(const ModelParams& P) {
  std::vector<MpoSite> W;
  for (const auto& st : chain_sites(P)) {
    MpoSite s;
    s.Dl = s.Dr = 1;
    s.d = st.d;
    add(s, 0, 0, identity(st.d));
    W.push_back(std::move(s));
  }
  return W;
}

// |I> restricted to one carrier: bond channel 0 = carrier not placed yet, 1 = placed.
// Returns, per site, the unit entries (a, s, b) of the bond-2 tensor embedded in the
// padded bond dimensions (the first site only has a = 0, the last only b = 0 <-> channel 1).
std::vector<std::vector<int>> identity_state_entries(const ModelParams& P) {
  const auto sites = chain_sites(P);
  const int L = (int)sites.size();
  std::vector<std::vector<int>> out(L);
  for (int k = 0; k < L; ++k) {
    const int d = sites[k].d;
    auto emit = [&](int ca, int s, int cb) {
      if (k == 0 && ca != 0) return;
      if (k == L - 1 && cb != 1) return;
      const int a = (k == 0) ? 0 : ca;
      const int b = (k == L - 1) ? 0 : cb;
      out[k].push_back(a);
      out[k].push_back(s);
      out[k].push_back(b);
    };
    if (sites[k].kind == SiteInfo::ELEC) {
      emit(0, 0, 0);              // molecule empty, carrier still to come
      emit(0, 1 * d + 1, 1);      // carrier here, in P and in Q
      emit(1, 0, 1);              // molecule empty, carrier already placed
    } else {
      for (int c = 0; c < 2; ++c)
        for (int v = 0; v < d; ++v) emit(c, v * d + v, c);
    }
  }
  return out;
}

std::vector<int> bond_dimensions(const std::vector<SiteInfo>& sites, int M) {
  const int L = (int)sites.size();
  std::vector<int> out(L + 1);
  for (int k = 0; k <= L; ++k) {
    double left = 1.0, right = 1.0;
    for (int i = 0; i < k; ++i) left *= (double)sites[i].d * sites[i].d;
    for (int i = k; i < L; ++i) right *= (double)sites[i].d * sites[i].d;
    double v = (double)M;
    if (left < v) v = left;
    if (right < v) v = right;
    out[k] = (int)v;
  }
  return out;
}

std::vector<MpoSite> build_mpo(const ModelParams& P, int which) {
  if (which == 0) return hamiltonian_mpo(P);
  if (which == 1) return current_mpo(P);
  if (which == 2) return identity_mpo(P);
  throw std::invalid_argument("build_mpo: which must be 0 (H), 1 (j) or 2 (identity)");
}

int parameter_count(const ModelParams& P) {
  return 2 * (int)P.omega.size() + 1 + (P.peierls ? 2 : 0);
}

ModelParams shifted(const ModelParams& P, int param, double delta) {
  const int K = (int)P.omega.size();
  if (param < 0 || param >= parameter_count(P))
    throw std::invalid_argument("shifted: parameter index out of range");
  ModelParams Q = P;
  if (param < K)
    Q.omega[param] += delta;
  else if (param < 2 * K)
    Q.g[param - K] += delta;
  else if (param == 2 * K)
    Q.V += delta;
  else if (param == 2 * K + 1)
    Q.alpha += delta;
  else
    Q.omega_p += delta;
  return Q;
}

MpoSite mpo_site_derivative(const ModelParams& P, int which, int param, int k) {
  const auto W0 = build_mpo(P, which);
  const auto W1 = build_mpo(shifted(P, param, 1.0), which);
  if (k < 0 || k >= (int)W0.size()) throw std::invalid_argument("mpo_site_derivative: bad site");
  const MpoSite& a = W0[k];
  const MpoSite& b = W1[k];
  // the automata add their blocks in an order that does not depend on the parameter values
  if (a.blocks.size() != b.blocks.size())
    throw std::logic_error("mpo_site_derivative: block structure depends on the parameter");
  MpoSite out;
  out.Dl = a.Dl;
  out.Dr = a.Dr;
  out.d = a.d;
  for (size_t i = 0; i < a.blocks.size(); ++i) {
    const MpoBlock& x = a.blocks[i];
    const MpoBlock& y = b.blocks[i];
    if (x.wl != y.wl || x.wr != y.wr)
      throw std::logic_error("mpo_site_derivative: block structure depends on the parameter");
    std::vector<Cx> op(x.op.size());
    bool nz = false;
    for (size_t e = 0; e < op.size(); ++e) {
      op[e] = y.op[e] - x.op[e];
      nz = nz || op[e] != Cx(0, 0);
    }
    if (nz) out.blocks.push_back({x.wl, x.wr, std::move(op)});
  }
  return out;
}

}  // namespace tdmrg
