// Host-side model description: chain sites and sparse MPOs (no CUDA).
#pragma once
#include <complex>
#include <vector>

namespace tdmrg {

typedef std::complex<double> Cx;

struct ModelParams {
  int N = 0;
  std::vector<double> omega, g;
  std::vector<int> nmax;
  double V = 0.0;
  bool peierls = false;
  double alpha = 0.0, omega_p = 0.2;
  int nmax_p = 8;
};

struct SiteInfo {
  enum Kind { ELEC, MODE, BOND } kind;
  int mol, mode, d;
};

// one nonzero operator block W[wl, wr, :, :] (d x d, row = output level)
struct MpoBlock {
  int wl, wr;
  std::vector<Cx> op;
};
struct MpoSite {
  int Dl = 0, Dr = 0, d = 0;
  std::vector<MpoBlock> blocks;
};

std::vector<SiteInfo> chain_sites(const ModelParams& P);
std::vector<MpoSite> hamiltonian_mpo(const ModelParams& P);
std::vector<MpoSite> current_mpo(const ModelParams& P);
std::vector<MpoSite> identity_mpo(const ModelParams& P);
std::vector<std::vector<int>> identity_state_entries(const ModelParams& P);
std::vector<int> bond_dimensions(const std::vector<SiteInfo>& sites, int M);

// The MPOs by kind: 0 = H (Eq. 1 / Eq. 10), 1 = j (Eq. 3), 2 = identity.
std::vector<MpoSite> build_mpo(const ModelParams& P, int which);

// Parameters theta_p the MPOs depend on: p < K: omega_p; K <= p < 2K: g_{p-K}; p = 2K: V; with
// a bond mode also p = 2K+1: alpha and p = 2K+2: omega_p (K modes per molecule).
int parameter_count(const ModelParams& P);
ModelParams shifted(const ModelParams& P, int param, double delta);

// dW_k/dtheta_param of site k of MPO `which`.  Every block is affine in each parameter on its
// own (g_m omega_m and V alpha are bilinear), so W(theta + 1) - W(theta) is exact; blocks that
// do not depend on theta are dropped.
MpoSite mpo_site_derivative(const ModelParams& P, int which, int param, int k);

}  // namespace tdmrg
