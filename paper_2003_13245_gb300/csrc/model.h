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

}  // namespace tdmrg
