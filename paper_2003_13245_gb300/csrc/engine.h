// TDVP engine: device MPS/MPO storage and the one-site projector-splitting sweep.
#pragma once
#include <memory>
#include <string>
#include <vector>

#include "model.h"
#include "tdmrg_internal.cuh"

namespace tdmrg {

constexpr int NBLK = 1024;   // partial sums of the one-launch FP64 norm (>= its 304 blocks)

struct Failure {
  int code;
  std::string msg;
};

// device copy of one site of an MPO: mixing tables for both contraction directions
struct DevMpoSite {
  int Dl = 0, Dr = 0, d = 0, nblk = 0;
  MixTable lr{}, rl{};               // lr: in = wl, out = wr;  rl: in = wr, out = wl
  void* mem = nullptr;               // one allocation holding all tables
  std::vector<MpoBlock> host;
};

struct DevMpo {
  std::vector<DevMpoSite> s;
  int maxD = 1;
};

struct DevMps {
  std::vector<int> Mb;               // bond dims, L + 1 entries
  std::vector<int> D;                // local (fused P,Q) dims d^2
  std::vector<int> d;
  std::vector<cplx*> A;              // site tensors [Ml][D][Mr]
  std::vector<cplx*> Lenv, Renv;     // environments for the Hamiltonian MPO
  int L() const { return (int)A.size(); }
  long long size(int k) const { return (long long)Mb[k] * D[k] * Mb[k + 1]; }
};

// Contraction building blocks, FP64.  X and Y are workspaces of at least
// max(Dl, Dr) * (left dim) * D * (right dim) entries.  All enqueue on `st`.
struct Ctx {
  cudaStream_t st;
  cplx* X;
  cplx* Y;
};
// out[a,s,t,b] = sum L[w,a,y] W[w,v,s,u] in[y,u,t,c] R[v,b,c]  (bra dims = ket dims)
void heff_f64(const Ctx& c, const DevMpoSite& W, int Ml, int Mr, int D, int d, const cplx* Lenv,
              const cplx* Renv, const cplx* in, cplx* out, const int* skip);
// Y[v][a][s][t][c] = sum L[w,a,y] W[w,v,s,u] ket[y,u,t,c]   (a < Ml1, y < Ml2, c < Mr2)
void left_partial_f64(const Ctx& c, const DevMpoSite& W, int Ml1, int Ml2, int D, int d,
                      int Mr2, const cplx* Lenv, const cplx* ket, cplx* Y, const int* skip);
// Y[w][y][s][t][b] = sum W[w,v,s,u] ket[y,u,t,c] R[v,b,c]     (y < Ml2, b < Mr1, c < Mr2)
void right_partial_f64(const Ctx& c, const DevMpoSite& W, int Ml2, int D, int d, int Mr1,
                       int Mr2, const cplx* Renv, const cplx* ket, cplx* Y, const int* skip);
void env_left_f64(const Ctx& c, const DevMpoSite& W, int Ml1, int Mr1, int Ml2, int Mr2, int D,
                  int d, const cplx* Lenv, const cplx* bra, const cplx* ket, cplx* Lout);
void env_right_f64(const Ctx& c, const DevMpoSite& W, int Ml1, int Mr1, int Ml2, int Mr2, int D,
                   int d, const cplx* Renv, const cplx* bra, const cplx* ket, cplx* Rout);
// out = sum_w L_w in R_w^T (zero-site effective Hamiltonian of a bond of dimension M)
void bond_f64(const Ctx& c, int M, int Dw, const cplx* Lenv, const cplx* Renv, const cplx* in,
              cplx* out, const int* skip);

// Mixed-precision (3xTF32 tensor-core) H_eff: split planes of the environments are made once
// per site update (heff_tc_envs), the matvec splits its FP64 input, runs the two contractions
// on tcgen05 and writes FP64.
struct TcWork {
  float* Lp = nullptr;     // 4 * Dl*Ml * pad4(Ml)
  float* Rp = nullptr;     // 4 * Dr*Mr * pad4(Mr)
  float* Bt = nullptr;     // 4 * D*Mr * pad4(Ml)
  float* X = nullptr;      // 2 * Dl*Ml*D*Mr
  float* Yp = nullptr;     // 4 * Dr*Ml*D * pad4(Mr)
  int* status = nullptr;
};
// Buffers of the mixed-precision contractions (float counts are set by the engine)
struct TcBufs {
  float* envA = nullptr;   // split planes of a left environment
  float* envB = nullptr;   // split planes of a right environment
  float* siteA = nullptr;  // split planes of a site-sized operand
  float* siteB = nullptr;
  float* x32 = nullptr;    // FP32 planar intermediate (MPO channel x site)
  float* mix = nullptr;    // split planes of an MPO-channel x site operand
  float* kpart = nullptr;  // split-K partial sums
  long long kpart_len = 0;
  int* status = nullptr;
};
void heff_tc_prepare(cudaStream_t st, const TcBufs& b, int Ml, int Mr, int Dl, int Dr,
                     const cplx* Lenv, const cplx* Renv);
void heff_tc_apply(cudaStream_t st, const TcBufs& b, const DevMpoSite& W, int Ml, int Mr, int D,
                   int d, const cplx* in, cplx* out);
void left_partial_tc(cudaStream_t st, const TcBufs& b, const DevMpoSite& W, int Ml1, int Ml2, int D,
                     int d, int Mr2, const cplx* Lenv, const cplx* ket, cplx* Yout);
void right_partial_tc(cudaStream_t st, const TcBufs& b, const DevMpoSite& W, int Ml2, int D, int d,
                      int Mr1, int Mr2, const cplx* Renv, const cplx* ket, cplx* Yout);
void env_left_tc(cudaStream_t st, const TcBufs& b, const DevMpoSite& W, int Ml1, int Mr1, int Ml2,
                 int Mr2, int D, int d, const cplx* Lenv, const cplx* bra, const cplx* ket,
                 cplx* Lout);
void env_right_tc(cudaStream_t st, const TcBufs& b, const DevMpoSite& W, int Ml1, int Mr1, int Ml2,
                  int Mr2, int D, int d, const cplx* Renv, const cplx* bra, const cplx* ket,
                  cplx* Rout);
void bond_tc_prepare(cudaStream_t st, const TcBufs& b, int M, int Dw, const cplx* Lenv,
                     const cplx* Renv);
void bond_tc_apply(cudaStream_t st, const TcBufs& b, int M, int Dw, const cplx* in, cplx* out);

long long heff_tc_floats(int Ml, int Mr, int D, int Dl, int Dr);
TcWork heff_tc_carve(float* base, int Ml, int Mr, int D, int Dl, int Dr, int* status);
void heff_tc_envs(cudaStream_t st, const TcWork& w, int Ml, int Mr, int Dl, int Dr,
                  const cplx* Lenv, const cplx* Renv);
void heff_tc(cudaStream_t st, const TcWork& w, const DevMpoSite& W, int Ml, int Mr, int D, int d,
             const cplx* in, cplx* out);

void throw_cuda(cudaError_t e, const char* what, int line);
#define CK(x)                                                 \
  do {                                                        \
    cudaError_t e__ = (x);                                    \
    if (e__ != cudaSuccess) ::tdmrg::throw_cuda(e__, #x, __LINE__); \
  } while (0)

struct Stats {
  double site_updates = 0, matvecs = 0, heff_flops = 0, krylov_vectors = 0, bond_matvecs = 0,
         qrs = 0, completions = 0, env_updates = 0;
  double heff_ms = 0;                 // event-timed duration of the site H_eff matvecs
  double qr_ms = 0, qr_flops = 0;     // event-timed gauge QRs and their algorithmic flops
  double qr_bulk_ms = 0, qr_bulk_flops = 0, qr_bulk_n = 0;   // the same for QRs of m >= 4096
  double lz_ms = 0;                   // event-timed Lanczos orthogonalisation steps
  // host wall time per phase (filled only when profiling is on; the phase ends synchronise)
  double t_site = 0, t_qr = 0, t_env = 0, t_bond = 0, t_absorb = 0, t_observe = 0;
  double h2d_bytes = 0, d2h_bytes = 0;
  double launches_at_reset = 0;
  double replayed_launches = 0;       // kernels launched through graph replays
};

// Mixed path: bond exponentials up to this bond dimension run as one fused cooperative launch
// (FP32 FMA contractions, 2 Dw M^3 complex MACs per Krylov vector); larger bonds use the
// host-driven Lanczos with the tensor-core contraction.
constexpr int kFusedBondMaxM = BOND_EXP_MAX_M;

class Engine {
 public:
  explicit Engine(const ModelParams& P);
  ~Engine();

  void set_precision(int p);
  void set_krylov(double tol, int kmax, int fixed_k);
  void set_stream(cudaStream_t s) { st_ = s; }
  void set_rank_tol(double t) {
    rank_tol_ = t;
    rank_tol_user_ = true;
    clear_graphs();
  }
  // Graph mode: with a fixed Krylov dimension every half-sweep pair of a state is captured
  // once into a CUDA graph and replayed.  qr_cap > 0 caps the QR grid (batched instances).
  void set_graphs(bool on, int qr_cap = 0);
  bool graphs() const { return graphs_; }
  void sync_and_check();
  // Records one half-step (half 1: left-to-right, 2: right-to-left) of both real-time states
  // into the stream capture the caller has started and joined this engine's stream to (one
  // graph over several instances); returns the counters one replay adds.  Graph mode only.
  Stats capture_realtime_half(double dt, int half);
  void add_stats(const Stats& d);
  void reset_stats();   // reads pending QR timings first, then zeroes the counters
  // Real-time propagation of the two states side by side: j Psi_b is stepped by a twin engine
  // (own workspaces, stream and host thread) while this engine steps Psi_b; cooperative grids
  // of both are capped to half of the SMs meanwhile so that the two lanes co-reside.  Off in
  // graph mode (batched instances already run side by side).  On by default.
  void set_concurrent(bool on) { concurrent_ = on; }
  bool concurrent() const { return concurrent_; }
  // counters of this engine plus those of its twin
  Stats total_stats() const;
  void set_profiling(bool on) { prof_ = on; }
  // limit of every bounded grid-barrier wait in clock cycles (0: the default, ~2 s); lowering
  // it makes the barriers give up, which is how the timeout path is tested
  void set_wait_cycles(long long c) {
    qr_.wait = c;
    bs_.wait = c;
    clear_graphs();
  }
  void rebuild_mpos();
  void thermal_prepare(double beta, double dtau, int M);
  void realtime_init();
  void realtime_step(int nsteps, double dt);
  void realtime_observe(double* C, double* obs);
  // sigma = Tr_ph rho_beta of the prepared thermal state (Eq. 9): sigma_ij = <c+_j c_i>,
  // written to sigma[2 (i N + j)] (interleaved re, im; host)
  void reduced_density(double* sigma);
  double logz() const { return logZ_; }
  bool prepared() const { return prepared_; }
  bool rt_ready() const { return rt_ready_; }
  Stats stats;
  ModelParams P;

  void ensure_workspace(long long maxsite, long long maxxy, int maxbond, int maxm);
  static void upload_mpo(const std::vector<MpoSite>& W, DevMpo& out);
  static void free_mpo(DevMpo& m);
  cudaStream_t stream() const { return st_; }
  cplx* X() { return X_; }
  cplx* Y() { return Y_; }

  // Lanczos exponential exp(tau M) v for a matvec callback (device pointers); returns the
  // number of matvecs that ran
  template <class F>
  int krylov(long long n, const cplx* v, cplx* out, double tr, double ti, F&& matvec);
  void gauge_qr_dev(int m, int n, QrRef Y, int p, QrRef E, cplx* Q, cplx* R,
                    int* src = nullptr);
  // Reverse of one FP64 projector-splitting step exp(tau H) (Eq. S1) of an MPS with bond
  // dimensions bond_dimensions(sites, M): A_in (device, sites 1.. right-orthonormal), the
  // cotangents Abar_out of the output sites -> the output A_out (may be NULL), Abar_in and
  // theta_bar[parameter_count(P)] (host).  The step is run again with its intermediates kept
  // (step_adjoint.cu).
  // With normalize, the output center is divided by its norm n (log n^2 to *log_norm) and the
  // cotangent Abar_out refers to the normalised output, plus logn_bar for log n^2.  With
  // Abar_out NULL only the forward step runs (A_out written).
  void step_vjp(int M, const cplx* const* A_in, double tr, double ti, const cplx* const* Abar_out,
                cplx* const* A_out, cplx* const* Abar_in, double* theta_bar, int nodes,
                bool normalize = false, double logn_bar = 0.0, double* log_norm = nullptr);
  // C_n = <psi1(n dt)| j |psi2(n dt)>, n = 0..nsteps, of two FP64 states stepped in real time,
  // and the reverse pass for the loss Re sum_n conj(cbar_n) C_n: states stored every `every`
  // steps, each stretch recomputed and reversed step by step (step_vjp) with the overlap VJPs;
  // writes C (2 (nsteps+1) host), the cotangents g1, g2 of the initial states (device) and
  // theta_bar (host, through H and j).
  void correlation_states_vjp(int M, const cplx* const* psi1, const cplx* const* psi2, double dt,
                              int nsteps, int every, const double* cbar, double* C,
                              cplx* const* g1, cplx* const* g2, double* theta_bar, int nodes);
  // |I> right-canonicalised (completions from the H coupling) with its center normalised ->
  // psi0 (device); with gbar (the cotangent of psi0, plus logn_bar for log n^2) the reverse
  // adds the parameter cotangents to theta (pipeline_adjoint.cu)
  void canonicalize_vjp(int M, cplx* const* psi0, const cplx* const* gbar, double logn_bar,
                        double* theta, double* log_norm);
  // phi ~ j|psi> by two one-site fitting sweeps (completions from the j coupling of psi) ->
  // phi (device); with gphi the reverse adds the cotangent of psi to gpsi and the parameter
  // cotangents to theta
  void fit_vjp(int M, const cplx* const* psi, cplx* const* phi, const cplx* const* gphi,
               cplx* const* gpsi, double* theta);
  // the whole C(t) pipeline in FP64 (preparation, fit, real-time steps, overlaps) and the
  // parameter cotangents of Re sum_n conj(cbar_n) C_n
  void correlation_vjp(double beta, double dtau, int M, double dt, int nsteps, int every,
                       const double* cbar, double* C, double* theta_bar, double* logz,
                       int nodes);
  // Quadrature of the exponential VJPs in the reverse passes: from fresh Lanczos
  // exponentials at every node (false, the default) or from the two Krylov bases of v and
  // vbar (true: the node vectors as basis combinations, small exponentials on the host).
  void set_adjoint_krylov_basis(bool on) { adjoint_basis_ = on; }
  // Krylov-basis reverse of y = exp(tau H) v: vbar = exp(conj(tau) H) ybar, and the node
  // vectors a_q (rows of Aq) and b_q (rows of Bq), q < kq.size() <= nodes, with
  // Hbar = sum_q k_q a_q b_q^H, k_q = w_q conj(tau) returned in kq; the node count is the
  // fewest whose Gauss-Legendre error bound meets 1e-15 for the two Lanczos matrices' norms
  // (step_adjoint.cu)
  template <class F>
  void exp_vjp_nodes(long long n, const cplx* v, const cplx* ybar, double tr, double ti,
                     int nodes, cplx* vbar, cplx* Aq, cplx* Bq, cplx* basis,
                     std::vector<Cx>& kq, F&& matvec);

 private:
  void alloc_mps(DevMps& s, int M);
  void free_mps(DevMps& s);
  void copy_mps(const DevMps& src, DevMps& dst);
  void right_canonicalize(DevMps& s);
  void build_right_envs(DevMps& s);
  void tdvp_step(DevMps& s, double tr, double ti);
  void site_update(DevMps& s, int k, double hr, double hi);
  void shift_right(DevMps& s, int k, const cplx* center, cplx* Cbond);
  void shift_left(DevMps& s, int k, const cplx* center, cplx* Cbond);
  Ctx ctx() const { return Ctx{st_, X_, Y_}; }
  bool mixed() const { return precision_ != 0; }
  double tic();
  void toc(double& acc, double t0);
  void env_left_any(const DevMpoSite& W, int Ml1, int Mr1, int Ml2, int Mr2, int D, int d,
                    const cplx* Lenv, const cplx* bra, const cplx* ket, cplx* Lout);
  void env_right_any(const DevMpoSite& W, int Ml1, int Mr1, int Ml2, int Mr2, int D, int d,
                     const cplx* Renv, const cplx* bra, const cplx* ket, cplx* Rout);
  void alloc_tc(const DevMps& s);
  void absorb_left(const cplx* C, int M, cplx* A, long long ncols);
  void absorb_right(cplx* A, long long nrows, const cplx* C, int M);
  void set_ones(cplx* p);
  void renormalize(cplx* A, long long n);
  double norm2_dev(const cplx* x, long long n);
  void scale_dev(cplx* x, long long n, double f);
  Cx overlap(const DevMps& bra, const DevMpo& W, const DevMps& ket);
  // adds the cotangents of <bra| j |ket> for the cotangent cbar of the overlap (step_adjoint.cu)
  void overlap_vjp(const std::vector<cplx*>& bra, const std::vector<cplx*>& ket, const std::vector<int>& Mb,
                   Cx cbar, const std::vector<cplx*>& gbra, const std::vector<cplx*>& gket,
                   std::vector<double>& theta);
  void fit_apply(const DevMpo& W, const DevMps& psi, DevMps& phi, int sweeps);
  void check_status();
  void harvest_qr_events();
  void ensure_bond_scratch(int maxbond);
  void bond_exp(int M, int Dw, const cplx* Le, const cplx* Re, double tr, double ti);
  long long env_size(const DevMps& s, int k, int Dw, bool left) const;

  cudaStream_t st_ = 0;
  int precision_ = 0;
  double ktol_ = 1e-13;
  bool ktol_user_ = false;
  double rank_tol_ = 1e-12;
  bool rank_tol_user_ = false;
  bool prof_ = false;
  bool graphs_ = false, capturing_ = false;
  int qr_gcap_ = 0;
  cudaStream_t own_stream_ = nullptr;
  struct StepGraph {
    const DevMps* state;
    double tr, ti;
    int half;             // 0: the whole step, 1: left-to-right half, 2: right-to-left half
    cudaGraphExec_t exec;
    Stats delta;
  };
  std::vector<StepGraph> step_graphs_;
  void clear_graphs();
  void tdvp_step_body(DevMps& s, double tr, double ti, int half = 0);
  const StepGraph& step_graph(DevMps& s, double tr, double ti, int half = 0);
  int kmax_ = 32, fixed_k_ = 0;
  bool adjoint_basis_ = false;
  bool concurrent_ = true;
  int dev_ = 0;
  std::unique_ptr<Engine> twin_;     // steps the second real-time state when concurrent
  bool twin_on_ = false;             // the twin holds the current second state
  void sync_twin_settings();
  void adopt_state(const DevMps& src, cudaStream_t src_stream);
  bool prepared_ = false, rt_ready_ = false;
  double logZ_ = 0.0;
  std::vector<SiteInfo> sites_;
  DevMpo H_, J_, I_;
  DevMps psi_b_, psi1_, psi2_;

  // workspace
  long long ws_site_ = 0, ws_xy_ = 0;
  int ws_bond_ = 0, ws_m_ = 0;
  cplx *X_ = nullptr, *Y_ = nullptr, *V_ = nullptr, *Kout_ = nullptr, *T1_ = nullptr;
  cplx *Cb_ = nullptr, *Rb_ = nullptr, *Ex_ = nullptr;
  double* part_d_ = nullptr;
  unsigned* red_cnt_ = nullptr;     // reduction tickets (KMAX + 2), zero between launches
  double* scal_ = nullptr;          // device scalars
  LzState* lz_ = nullptr;
  QrScratch qr_{};
  cplx* qb_scratch_ = nullptr;
  long long qb_len_ = 0;
  unsigned char* qb_acc_ = nullptr;
  int* status_ = nullptr;
  int* h_pinned_ = nullptr;
  double* h_pinned_d_ = nullptr;
  cplx* env_tmp_[2] = {nullptr, nullptr};
  cudaEvent_t ev_[2 * KMAX + 2] = {};
  static constexpr int QR_EV = 256;   // gauge-QR event pairs held before they are read
  cudaEvent_t qr_ev_[2 * QR_EV] = {};
  int qr_ev_n_ = 0;
  unsigned char qr_ev_bulk_[QR_EV] = {};   // the QR of event pair i has m >= 4096
  cudaEvent_t lz_ev_[2 * QR_EV] = {};
  int lz_ev_n_ = 0;
  TcBufs tcb_{};
  BondScratch bs_{};
  unsigned long long* h_mv_ = nullptr;   // pinned copy of the device Krylov-vector counter
  unsigned long long mv_seen_ = 0;
  long long tc_site_ = 0, tc_env_ = 0, tc_x_ = 0;
  long long env_tmp_size_ = 0;
};

// Lanczos with full re-orthogonalisation in FP64: the three-term step against q_j and
// q_{j-1}, then one classical Gram-Schmidt pass against every Krylov vector, the norm, the
// small exponential and the stopping test -- one cooperative launch per Krylov vector.  The host polls the stop flag of
// iteration j-1 while iteration j is already queued (its kernels skip once the flag is set),
// so the device never waits for the host between iterations.
template <class F>
inline int Engine::krylov(long long n, const cplx* v, cplx* out, double tr, double ti, F&& matvec) {
  const int cap0 = fixed_k_ > 0 ? fixed_k_ : kmax_;
  const int kcap = (int)std::min<long long>(cap0, n);
  LzState* S = lz_;
  const int* done = &S->done;
  CK(znorm2(n, v, scal_, part_d_, red_cnt_ + KMAX + 1, nullptr, st_));
  CK(lz_start(S, scal_, st_));
  CK(cudaMemcpyAsync(V_, v, sizeof(cplx) * (size_t)n, cudaMemcpyDeviceToDevice, st_));
  CK(zscale_by(n, V_, &S->inv, done, st_));
  int launched = 0;
  bool stop = false;
  for (int j = 0; j < kcap && !stop; ++j) {
    cplx* q = V_ + (size_t)j * n;
    cplx* w = V_ + (size_t)(j + 1) * n;
    matvec(q, w, done);
    // both Gram-Schmidt passes, norm, small exponential, stop test and scaling: one launch
    const bool timed = !capturing_;
    if (timed) {
      if (lz_ev_n_ == QR_EV) harvest_qr_events();
      CK(cudaEventRecord(lz_ev_[2 * lz_ev_n_], st_));
    }
    CK(lz_step(n, j, V_, S, bs_, status_ + 1, tr, ti, ktol_, kcap, fixed_k_ > 0 ? 1 : 0,
               qr_gcap_, st_));
    if (timed) CK(cudaEventRecord(lz_ev_[2 * lz_ev_n_++ + 1], st_));
    CK(cudaMemcpyAsync(h_pinned_ + 4 + (j & 1) * 2, done, sizeof(int), cudaMemcpyDeviceToHost,
                       st_));
    CK(cudaEventRecord(ev_[2 * KMAX + (j & 1)], st_));
    stats.d2h_bytes += sizeof(int);
    launched = j + 1;
    if (capturing_) continue;   // a captured Krylov loop runs its fixed number of vectors
    if (j >= 1) {
      // the flag of iteration j-1 (iteration j is queued behind it)
      CK(cudaEventSynchronize(ev_[2 * KMAX + ((j - 1) & 1)]));
      if (h_pinned_[4 + ((j - 1) & 1) * 2]) stop = true;
    }
  }
  if (!stop && !capturing_) {
    CK(cudaEventSynchronize(ev_[2 * KMAX + ((launched - 1) & 1)]));
  }
  // when the stop flag of iteration j-1 was seen, iteration j was queued but skipped
  const int used = stop ? launched - 1 : launched;
  stats.krylov_vectors += used;
  CK(zcombine(n, S, V_, n, out, st_));
  return used;
}
}  // namespace tdmrg
