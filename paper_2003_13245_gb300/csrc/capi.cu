// extern "C" boundary of libtdmrg: argument checks, exception-to-status translation and
// the kernel-level entry points.  Every computation runs in the CUDA kernels of the engine.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <memory>
#include <string>
#include <vector>

#include "../../include/tdmrg.h"
#include "engine.h"
#include "small_exp.h"
#include "tc.cuh"

using tdmrg::Engine;
using tdmrg::Failure;

struct tdmrg_model {
  std::unique_ptr<Engine> eng;
  std::string err;
};

struct tdmrg_batch {
  std::vector<tdmrg_model*> models;
  int phase = 0;   // 1 after a left-to-right half-step (the step is completed by the next one)
  // one CUDA graph per half-step over every instance (each instance a branch on its own
  // stream), captured at the first use of a time step dt
  cudaStream_t s0 = nullptr;
  cudaEvent_t fork = nullptr;
  std::vector<cudaEvent_t> join;
  cudaGraphExec_t exec[2] = {nullptr, nullptr};
  double dt[2] = {0.0, 0.0};
  std::vector<tdmrg::Stats> delta[2];
  ~tdmrg_batch() {
    for (auto& e : exec)
      if (e) cudaGraphExecDestroy(e);
    for (auto& e : join)
      if (e) cudaEventDestroy(e);
    if (fork) cudaEventDestroy(fork);
    if (s0) {
      cudaStreamSynchronize(s0);
      cudaStreamDestroy(s0);
    }
  }
};

static thread_local std::string g_err;

namespace tdmrg {
void set_global_error(const char* msg) { g_err = msg; }
}  // namespace tdmrg

namespace {

template <class F>
int guarded(tdmrg_model* h, F&& f) {
  try {
    f();
    return TDMRG_OK;
  } catch (const Failure& e) {
    if (h) h->err = e.msg;
    g_err = e.msg;
    return e.code;
  } catch (const std::bad_alloc&) {
    if (h) h->err = "host allocation failed";
    g_err = "host allocation failed";
    return TDMRG_ERR_OOM;
  } catch (const std::exception& e) {
    if (h) h->err = e.what();
    g_err = e.what();
    return TDMRG_ERR_ARG;
  }
}

int fail(tdmrg_model* h, int code, const char* msg) {
  if (h) h->err = msg;
  g_err = msg;
  return code;
}

// a dense host W[Dl][Dr][d][d] (complex interleaved) as a one-site device MPO
struct TempMpo {
  tdmrg::DevMpo m;
  TempMpo(int Dl, int Dr, int d, const double* W) {
    tdmrg::MpoSite s;
    s.Dl = Dl;
    s.Dr = Dr;
    s.d = d;
    for (int wl = 0; wl < Dl; ++wl)
      for (int wr = 0; wr < Dr; ++wr) {
        std::vector<tdmrg::Cx> op(d * d);
        bool nz = false;
        for (int e = 0; e < d * d; ++e) {
          const size_t off = 2 * (((size_t)wl * Dr + wr) * d * d + e);
          op[e] = tdmrg::Cx(W[off], W[off + 1]);
          nz = nz || op[e] != tdmrg::Cx(0, 0);
        }
        if (nz) s.blocks.push_back({wl, wr, op});
      }
    Engine::upload_mpo({s}, m);
  }
  ~TempMpo() { Engine::free_mpo(m); }
};

using tdmrg::cplx;

tdmrg::MatRef mat(const void* p, long long rs, long long cs, long long sb = 0, long long sr = 0,
                  int conj = 0) {
  return tdmrg::MatRef{(const cplx*)p, rs, cs, sb, sr, conj};
}

// device temporaries of one entry point, freed when it returns
struct DevBufs {
  std::vector<void*> p;
  cplx* get(long long n) {
    void* q = nullptr;
    CK(cudaMalloc(&q, sizeof(cplx) * (size_t)(n > 0 ? n : 1)));
    p.push_back(q);
    return (cplx*)q;
  }
  ~DevBufs() {
    for (void* q : p) cudaFree(q);
  }
};

// op'[s][u] = conj(op[u][s]) for every channel pair of a dense site [Dl][Dr][d][d]
std::vector<double> transpose_conj_ops(const double* W, int Dl, int Dr, int d) {
  const int D = d * d;
  std::vector<double> out((size_t)2 * Dl * Dr * D);
  for (int b = 0; b < Dl * Dr; ++b)
    for (int si = 0; si < d; ++si)
      for (int ui = 0; ui < d; ++ui) {
        const size_t dst = 2 * ((size_t)b * D + si * d + ui);
        const size_t src = 2 * ((size_t)b * D + ui * d + si);
        out[dst] = W[src];
        out[dst + 1] = -W[src + 1];
      }
  return out;
}

bool any_nonzero(const double* x, size_t n) {
  for (size_t i = 0; i < n; ++i)
    if (x[i] != 0.0) return true;
  return false;
}

// <g, x> = sum conj(g_i) x_i: 256 chunk sums by one batched GEMM plus the tail, added on the
// host in a fixed order.  part: 257 device entries.  Synchronises s.
cplx dot_c(const cplx* g, const cplx* x, long long n, cplx* part, cudaStream_t s) {
  const int B = 256;
  const long long kc = n / B, rem = n - kc * B;
  const cplx one = {1.0, 0.0}, zero = {0.0, 0.0};
  if (kc > 0)
    CK(tdmrg::zgemm(1, 1, (int)kc, B, 1, one, mat(g, 0, 1, kc, 0, 1), mat(x, 1, 0, kc), zero,
                    part, 1, 1, nullptr, s));
  if (rem > 0)
    CK(tdmrg::zgemm(1, 1, (int)rem, 1, 1, one, mat(g + kc * B, 0, 1, 0, 0, 1),
                    mat(x + kc * B, 1, 0), zero, part + B, 1, 0, nullptr, s));
  std::vector<cplx> h(B + 1);
  CK(cudaMemcpyAsync(h.data(), part, sizeof(cplx) * (B + 1), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  cplx acc = {0.0, 0.0};
  if (kc > 0)
    for (int b = 0; b < B; ++b) {
      acc.x += h[b].x;
      acc.y += h[b].y;
    }
  if (rem > 0) {
    acc.x += h[B].x;
    acc.y += h[B].y;
  }
  return acc;
}

double dot_re(const cplx* g, const cplx* x, long long n, cplx* part, cudaStream_t s) {
  return dot_c(g, x, n, part, s).x;
}

// the chain of Eq. 1 from the arguments of tdmrg_model_create; nullptr or the failed check
const char* fill_params(int N, int modes, const double* omega, const double* g, double V,
                        const int* nmax, tdmrg::ModelParams& P) {
  if (N < 3) return "N must be >= 3 (periodic chain)";
  if (modes < 0 || modes > 64) return "modes out of range";
  if (modes > 0 && (!omega || !g || !nmax)) return "NULL mode arrays";
  P.N = N;
  P.V = V;
  for (int m = 0; m < modes; ++m) {
    if (nmax[m] < 2 || nmax[m] > 32) return "nmax must be in [2, 32]";
    if (!std::isfinite(omega[m]) || !std::isfinite(g[m])) return "non-finite mode parameter";
    P.omega.push_back(omega[m]);
    P.g.push_back(g[m]);
    P.nmax.push_back(nmax[m]);
  }
  if (!std::isfinite(V)) return "non-finite V";
  return nullptr;
}

}  // namespace

extern "C" {

int tdmrg_model_create(int N, int modes, const double* omega, const double* g, double V,
                       const int* nmax, tdmrg_model** out) {
  if (!out) return fail(nullptr, TDMRG_ERR_ARG, "out is NULL");
  *out = nullptr;
  tdmrg::ModelParams P;
  if (const char* msg = fill_params(N, modes, omega, g, V, nmax, P))
    return fail(nullptr, TDMRG_ERR_ARG, msg);
  auto* h = new (std::nothrow) tdmrg_model;
  if (!h) return fail(nullptr, TDMRG_ERR_OOM, "host allocation failed");
  const int rc = guarded(h, [&] { h->eng.reset(new Engine(P)); });
  if (rc != TDMRG_OK) {
    g_err = h->err;
    delete h;
    return rc;
  }
  *out = h;
  return TDMRG_OK;
}

int tdmrg_model_set_peierls(tdmrg_model* h, double alpha, double omega_p, int nmax_p) {
  if (!h) return fail(nullptr, TDMRG_ERR_ARG, "NULL handle");
  if (nmax_p < 2 || nmax_p > 32 || !std::isfinite(alpha) || !std::isfinite(omega_p))
    return fail(h, TDMRG_ERR_ARG, "peierls: nmax_p in [2, 32], finite alpha and omega_p");
  return guarded(h, [&] {
    h->eng->P.peierls = true;
    h->eng->P.alpha = alpha;
    h->eng->P.omega_p = omega_p;
    h->eng->P.nmax_p = nmax_p;
    h->eng->rebuild_mpos();
  });
}

int tdmrg_model_set_precision(tdmrg_model* h, int precision) {
  if (!h) return fail(nullptr, TDMRG_ERR_ARG, "NULL handle");
  return guarded(h, [&] { h->eng->set_precision(precision); });
}

int tdmrg_model_set_krylov(tdmrg_model* h, double tol, int kmax, int fixed_k) {
  if (!h) return fail(nullptr, TDMRG_ERR_ARG, "NULL handle");
  return guarded(h, [&] { h->eng->set_krylov(tol, kmax, fixed_k); });
}

int tdmrg_model_set_stream(tdmrg_model* h, void* stream) {
  if (!h) return fail(nullptr, TDMRG_ERR_ARG, "NULL handle");
  h->eng->set_stream((cudaStream_t)stream);
  return TDMRG_OK;
}

int tdmrg_model_set_wait_cycles(tdmrg_model* h, long long cycles) {
  if (!h) return fail(nullptr, TDMRG_ERR_ARG, "NULL handle");
  if (cycles < 0) return fail(h, TDMRG_ERR_ARG, "wait_cycles: need cycles >= 0");
  return guarded(h, [&] { h->eng->set_wait_cycles(cycles); });
}

int tdmrg_model_set_profiling(tdmrg_model* h, int on) {
  if (!h) return fail(nullptr, TDMRG_ERR_ARG, "NULL handle");
  h->eng->set_profiling(on != 0);
  return TDMRG_OK;
}

int tdmrg_model_set_rank_tol(tdmrg_model* h, double rank_tol) {
  if (!h) return fail(nullptr, TDMRG_ERR_ARG, "NULL handle");
  if (!(rank_tol > 0.0) || rank_tol > 1e-2) return fail(h, TDMRG_ERR_ARG, "rank_tol in (0, 1e-2]");
  h->eng->set_rank_tol(rank_tol);
  return TDMRG_OK;
}

int tdmrg_model_set_adjoint_krylov_basis(tdmrg_model* h, int on) {
  if (!h) return fail(nullptr, TDMRG_ERR_ARG, "NULL handle");
  h->eng->set_adjoint_krylov_basis(on != 0);
  return TDMRG_OK;
}

int tdmrg_model_set_graphs(tdmrg_model* h, int on) {
  if (!h) return fail(nullptr, TDMRG_ERR_ARG, "NULL handle");
  return guarded(h, [&] { h->eng->set_graphs(on != 0, 0); });
}

int tdmrg_batch_create(tdmrg_model* const* models, int n, tdmrg_batch** out) {
  if (!models || n < 1 || !out) return fail(nullptr, TDMRG_ERR_ARG, "batch: need n >= 1 models");
  *out = nullptr;
  for (int i = 0; i < n; ++i) {
    if (!models[i]) return fail(nullptr, TDMRG_ERR_ARG, "batch: NULL model");
    for (int j = 0; j < i; ++j)
      if (models[j] == models[i]) return fail(nullptr, TDMRG_ERR_ARG, "batch: model listed twice");
    if (!models[i]->eng->rt_ready())
      return fail(nullptr, TDMRG_ERR_STATE, "batch: every model needs tdmrg_realtime_init first");
  }
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return fail(nullptr, TDMRG_ERR_CUDA, "batch: no device");
  // concurrent instances share the SMs: cap each QR grid so that four fit side by side
  const int cap = sms / 4 > 8 ? sms / 4 : 8;
  for (int i = 0; i < n; ++i) {
    tdmrg_model* h = models[i];
    const int rc = guarded(h, [&] {
      h->eng->set_graphs(true, cap);
    });
    if (rc != TDMRG_OK) {
      g_err = h->err;
      return rc;
    }
  }
  auto* b = new (std::nothrow) tdmrg_batch;
  if (!b) return fail(nullptr, TDMRG_ERR_OOM, "host allocation failed");
  b->models.assign(models, models + n);
  *out = b;
  return TDMRG_OK;
}

namespace {
// the grid of tdmrg_correlation: t_grid[0] = 0, ascending integer multiples of dt -> step counts
const char* grid_steps(const double* t_grid, int nt, double dt, std::vector<long long>& steps) {
  if (!t_grid || nt < 1 || !(dt > 0.0)) return "bad grid arguments";
  if (t_grid[0] != 0.0) return "t_grid[0] must be 0";
  steps.assign(nt, 0);
  for (int i = 0; i < nt; ++i) {
    const double q = t_grid[i] / dt;
    const long long r = std::llround(q);
    if (std::fabs(q - r) > 1e-9 * std::max(1.0, std::fabs(q)))
      return "t_grid points must be integer multiples of dt";
    if (i > 0 && r <= steps[i - 1]) return "t_grid must be ascending";
    steps[i] = r;
  }
  return nullptr;
}

// the graph of one half-step of every instance: captured from a fork on the batch stream, each
// instance's engine recording its work on its own stream, joined back before the capture ends
void batch_capture(tdmrg_batch* b, double dt, int half) {
  const int n = (int)b->models.size();
  if (!b->s0) CK(cudaStreamCreateWithFlags(&b->s0, cudaStreamNonBlocking));
  if (!b->fork) CK(cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming));
  while ((int)b->join.size() < n) {
    cudaEvent_t e = nullptr;
    CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    b->join.push_back(e);
  }
  cudaGraphExec_t& ex = b->exec[half - 1];
  if (ex) {
    cudaGraphExecDestroy(ex);
    ex = nullptr;
  }
  std::vector<tdmrg::Stats> delta(n);
  CK(cudaStreamBeginCapture(b->s0, cudaStreamCaptureModeThreadLocal));
  cudaGraph_t graph = nullptr;
  try {
    CK(cudaEventRecord(b->fork, b->s0));
    for (int i = 0; i < n; ++i) {
      Engine& e = *b->models[i]->eng;
      CK(cudaStreamWaitEvent(e.stream(), b->fork, 0));
      delta[i] = e.capture_realtime_half(dt, half);
      CK(cudaEventRecord(b->join[i], e.stream()));
      CK(cudaStreamWaitEvent(b->s0, b->join[i], 0));
    }
  } catch (...) {
    cudaStreamEndCapture(b->s0, &graph);
    if (graph) cudaGraphDestroy(graph);
    throw;
  }
  CK(cudaStreamEndCapture(b->s0, &graph));
  const cudaError_t e = cudaGraphInstantiate(&ex, graph, 0);
  cudaGraphDestroy(graph);
  CK(e);
  b->dt[half - 1] = dt;
  b->delta[half - 1] = delta;
}

// one half-step (half 1 or 2) of every instance: a single graph launch, then each instance's
// status words are read
int batch_half(tdmrg_batch* b, double dt, int half) {
  const int rc0 = guarded(nullptr, [&] {
    if (!b->exec[half - 1] || b->dt[half - 1] != dt) batch_capture(b, dt, half);
    CK(cudaGraphLaunch(b->exec[half - 1], b->s0));
    for (size_t i = 0; i < b->models.size(); ++i)
      b->models[i]->eng->add_stats(b->delta[half - 1][i]);
    CK(cudaStreamSynchronize(b->s0));
  });
  if (rc0 != TDMRG_OK) return rc0;
  for (tdmrg_model* h : b->models) {
    const int rc = guarded(h, [&] { h->eng->sync_and_check(); });
    if (rc != TDMRG_OK) {
      g_err = h->err;
      return rc;
    }
  }
  return TDMRG_OK;
}
}  // namespace

int tdmrg_batch_step_half(tdmrg_batch* b, double dt) {
  if (!b || !(dt > 0.0)) return fail(nullptr, TDMRG_ERR_ARG, "batch half-step: bad arguments");
  const int rc = batch_half(b, dt, b->phase == 0 ? 1 : 2);
  if (rc == TDMRG_OK) b->phase ^= 1;
  return rc;
}

int tdmrg_batch_correlation(tdmrg_batch* b, const double* t_grid, int nt, double dt,
                            double* C_out) {
  if (!b || !C_out) return fail(nullptr, TDMRG_ERR_ARG, "batch correlation: bad arguments");
  std::vector<long long> steps;
  if (const char* msg = grid_steps(t_grid, nt, dt, steps))
    return fail(nullptr, TDMRG_ERR_ARG, msg);
  const int n = (int)b->models.size();
  for (tdmrg_model* h : b->models) {
    const int rc = guarded(h, [&] { h->eng->realtime_init(); });
    if (rc != TDMRG_OK) {
      g_err = h->err;
      return rc;
    }
  }
  b->phase = 0;
  long long at = 0;
  for (int i = 0; i < nt; ++i) {
    for (; at < steps[i]; ++at) {
      int rc = batch_half(b, dt, 1);
      if (rc == TDMRG_OK) rc = batch_half(b, dt, 2);
      if (rc != TDMRG_OK) return rc;
    }
    for (int j = 0; j < n; ++j) {
      tdmrg_model* h = b->models[j];
      const int rc = guarded(h, [&] {
        h->eng->realtime_observe(C_out + 2 * ((size_t)j * nt + i), nullptr);
      });
      if (rc != TDMRG_OK) {
        g_err = h->err;
        return rc;
      }
    }
  }
  return TDMRG_OK;
}

int tdmrg_batch_realtime_step(tdmrg_batch* b, int nsteps, double dt) {
  if (!b || nsteps < 0 || !(dt > 0.0)) return fail(nullptr, TDMRG_ERR_ARG, "batch step: bad arguments");
  if (b->phase != 0)
    return fail(nullptr, TDMRG_ERR_STATE, "batch step: a half-step is pending (call tdmrg_batch_step_half)");
  for (int st = 0; st < nsteps; ++st) {
    int rc = batch_half(b, dt, 1);
    if (rc == TDMRG_OK) rc = batch_half(b, dt, 2);
    if (rc != TDMRG_OK) return rc;
  }
  return TDMRG_OK;
}

int tdmrg_batch_destroy(tdmrg_batch* b) {
  delete b;
  return TDMRG_OK;
}

int tdmrg_model_destroy(tdmrg_model* h) {
  if (!h) return TDMRG_OK;
  if (h->eng) cudaStreamSynchronize(h->eng->stream());
  delete h;
  return TDMRG_OK;
}

int tdmrg_thermal_prepare(tdmrg_model* h, double beta, double dtau, int M) {
  if (!h) return fail(nullptr, TDMRG_ERR_ARG, "NULL handle");
  return guarded(h, [&] { h->eng->thermal_prepare(beta, dtau, M); });
}

int tdmrg_realtime_init(tdmrg_model* h) {
  if (!h) return fail(nullptr, TDMRG_ERR_ARG, "NULL handle");
  return guarded(h, [&] { h->eng->realtime_init(); });
}

int tdmrg_realtime_step(tdmrg_model* h, int nsteps, double dt) {
  if (!h) return fail(nullptr, TDMRG_ERR_ARG, "NULL handle");
  return guarded(h, [&] { h->eng->realtime_step(nsteps, dt); });
}

int tdmrg_realtime_observe(tdmrg_model* h, double* C_out, double* obs) {
  if (!h || !C_out) return fail(h, TDMRG_ERR_ARG, "NULL argument");
  return guarded(h, [&] { h->eng->realtime_observe(C_out, obs); });
}

int tdmrg_correlation(tdmrg_model* h, const double* t_grid, int nt, double dt, double* C_out) {
  if (!h) return fail(nullptr, TDMRG_ERR_ARG, "NULL handle");
  if (!C_out) return fail(h, TDMRG_ERR_ARG, "bad grid arguments");
  std::vector<long long> steps;
  if (const char* msg = grid_steps(t_grid, nt, dt, steps)) return fail(h, TDMRG_ERR_ARG, msg);
  return guarded(h, [&] {
    h->eng->realtime_init();
    long long at = 0;
    for (int i = 0; i < nt; ++i) {
      h->eng->realtime_step((int)(steps[i] - at), dt);
      at = steps[i];
      h->eng->realtime_observe(C_out + 2 * i, nullptr);
    }
  });
}

int tdmrg_mobility(const double* t_grid, const double* C, int nt, double kT, double* mu_out) {
  if (!t_grid || !C || !mu_out || nt < 2 || !(kT > 0.0))
    return fail(nullptr, TDMRG_ERR_ARG, "mobility: need nt >= 2, kT > 0, non-NULL arrays");
  if (t_grid[0] != 0.0) return fail(nullptr, TDMRG_ERR_ARG, "mobility: t_grid[0] must be 0");
  double integral = 0.0;
  for (int i = 0; i + 1 < nt; ++i) {
    const double h = t_grid[i + 1] - t_grid[i];
    if (!(h > 0.0)) return fail(nullptr, TDMRG_ERR_ARG, "mobility: t_grid must be ascending");
    integral += 0.5 * h * (C[2 * i] + C[2 * i + 2]);
  }
  *mu_out = 2.0 * integral / (2.0 * kT);
  return TDMRG_OK;
}

int tdmrg_fgr_mobility_batch(int P, int K, const double* omega, const double* g,
                             const double* V, const double* kT, double dt, int nt, double* mu_out,
                             void* stream) {
  if (P < 1 || K < 1 || K > 64 || !omega || !g || !V || !kT || !mu_out || nt < 2 || !(dt > 0.0))
    return fail(nullptr, TDMRG_ERR_ARG,
                "fgr_mobility_batch: need P >= 1, 1 <= K <= 64, nt >= 2, dt > 0, host arrays");
  for (long long i = 0; i < (long long)P * K; ++i)
    if (!std::isfinite(omega[i]) || !(omega[i] > 0.0) || !std::isfinite(g[i]))
      return fail(nullptr, TDMRG_ERR_ARG, "fgr_mobility_batch: need finite g and omega > 0");
  for (int p = 0; p < P; ++p)
    if (!std::isfinite(V[p]) || !(kT[p] > 0.0) || !std::isfinite(kT[p]))
      return fail(nullptr, TDMRG_ERR_ARG, "fgr_mobility_batch: need finite V and kT > 0");
  return guarded(nullptr, [&] {
    cudaStream_t s = (cudaStream_t)stream;
    const size_t nk = (size_t)P * K;
    double* d = nullptr;
    struct Free {
      double*& p;
      ~Free() {
        if (p) cudaFree(p);
      }
    } fr{d};
    CK(cudaMalloc(&d, sizeof(double) * (2 * nk + 3 * (size_t)P)));
    double *dw = d, *dg = d + nk, *dV = d + 2 * nk, *dT = dV + P, *dmu = dT + P;
    CK(cudaMemcpyAsync(dw, omega, sizeof(double) * nk, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(dg, g, sizeof(double) * nk, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(dV, V, sizeof(double) * P, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(dT, kT, sizeof(double) * P, cudaMemcpyHostToDevice, s));
    CK(tdmrg::fgr_mobility(P, K, dw, dg, dV, dT, dt, nt, dmu, s));
    CK(cudaMemcpyAsync(mu_out, dmu, sizeof(double) * P, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
  });
}

int tdmrg_reduced_density(tdmrg_model* h, double* sigma_out) {
  if (!h) return fail(nullptr, TDMRG_ERR_ARG, "NULL handle");
  if (!sigma_out) return fail(h, TDMRG_ERR_ARG, "reduced_density: sigma_out is NULL");
  return guarded(h, [&] { h->eng->reduced_density(sigma_out); });
}

int tdmrg_coherence_length(int N, const double* sigma, double* L_out) {
  if (N < 1 || !sigma || !L_out)
    return fail(nullptr, TDMRG_ERR_ARG, "coherence_length: need N >= 1 and non-NULL arrays");
  double s1 = 0.0, s2 = 0.0;
  for (long long e = 0; e < (long long)N * N; ++e) {
    const double a = std::hypot(sigma[2 * e], sigma[2 * e + 1]);
    s1 += a;
    s2 += a * a;
  }
  if (!(s2 > 0.0) || !std::isfinite(s1))
    return fail(nullptr, TDMRG_ERR_ARG, "coherence_length: sigma is zero or not finite");
  *L_out = s1 * s1 / (N * s2);
  return TDMRG_OK;
}

int tdmrg_mean_free_path(const double* t_grid, const double* C, int nt, double* vtl_out) {
  if (!t_grid || !C || !vtl_out || nt < 2)
    return fail(nullptr, TDMRG_ERR_ARG, "mean_free_path: need nt >= 2 and non-NULL arrays");
  if (t_grid[0] != 0.0) return fail(nullptr, TDMRG_ERR_ARG, "mean_free_path: t_grid[0] must be 0");
  const double c0 = C[0];
  if (!(c0 > 0.0) || !std::isfinite(c0))
    return fail(nullptr, TDMRG_ERR_ARG, "mean_free_path: Re C(0) = <j j> must be positive");
  double area = 0.0;
  for (int i = 0; i + 1 < nt; ++i) {
    const double h = t_grid[i + 1] - t_grid[i];
    if (!(h > 0.0)) return fail(nullptr, TDMRG_ERR_ARG, "mean_free_path: t_grid must be ascending");
    area += 0.5 * h * (std::fabs(C[2 * i]) + std::fabs(C[2 * i + 2]));
  }
  const double v = std::sqrt(c0), tau = area / c0;
  vtl_out[0] = v;
  vtl_out[1] = tau;
  vtl_out[2] = v * tau;
  return TDMRG_OK;
}

int tdmrg_host_mpo_site(int N, int modes, const double* omega, const double* g, double V,
                        const int* nmax, double alpha, double omega_p, int nmax_p, int which,
                        int param, int site, int* dims, double* W_out) {
  if (!dims) return fail(nullptr, TDMRG_ERR_ARG, "host_mpo_site: dims is NULL");
  tdmrg::ModelParams P;
  if (const char* msg = fill_params(N, modes, omega, g, V, nmax, P))
    return fail(nullptr, TDMRG_ERR_ARG, msg);
  if (nmax_p != 0) {
    if (nmax_p < 2 || nmax_p > 32 || !std::isfinite(alpha) || !std::isfinite(omega_p))
      return fail(nullptr, TDMRG_ERR_ARG, "host_mpo_site: nmax_p in [2, 32], finite alpha and omega_p");
    P.peierls = true;
    P.alpha = alpha;
    P.omega_p = omega_p;
    P.nmax_p = nmax_p;
  }
  if (which < TDMRG_MPO_H || which > TDMRG_MPO_IDENTITY)
    return fail(nullptr, TDMRG_ERR_ARG, "host_mpo_site: unknown operator");
  if (param < -1 || param >= tdmrg::parameter_count(P))
    return fail(nullptr, TDMRG_ERR_ARG, "host_mpo_site: parameter index out of range");
  if (site < 0 || site >= (int)tdmrg::chain_sites(P).size())
    return fail(nullptr, TDMRG_ERR_ARG, "host_mpo_site: site out of range");
  return guarded(nullptr, [&] {
    const tdmrg::MpoSite W = param < 0 ? tdmrg::build_mpo(P, which)[site]
                                       : tdmrg::mpo_site_derivative(P, which, param, site);
    dims[0] = W.Dl;
    dims[1] = W.Dr;
    dims[2] = W.d;
    if (!W_out) return;
    const size_t dd = (size_t)W.d * W.d;
    std::memset(W_out, 0, sizeof(double) * 2 * (size_t)W.Dl * W.Dr * dd);
    for (const auto& b : W.blocks)
      for (size_t e = 0; e < dd; ++e) {
        const size_t off = 2 * (((size_t)b.wl * W.Dr + b.wr) * dd + e);
        W_out[off] += b.op[e].real();
        W_out[off + 1] += b.op[e].imag();
      }
  });
}

int tdmrg_parameter_count(const tdmrg_model* h, int* count) {
  if (!h || !count) return fail(nullptr, TDMRG_ERR_ARG, "parameter_count: NULL argument");
  *count = tdmrg::parameter_count(h->eng->P);
  return TDMRG_OK;
}

int tdmrg_step_vjp(tdmrg_model* h, int M, const void* const* A_in, double tau_re, double tau_im,
                   const void* const* Abar_out, void* const* A_out, void* const* Abar_in,
                   double* theta_bar, int nodes) {
  if (!h) return fail(nullptr, TDMRG_ERR_ARG, "NULL handle");
  if (M < 1 || !A_in || !Abar_out || !Abar_in || !theta_bar || nodes < 1 || nodes > 64)
    return fail(h, TDMRG_ERR_ARG, "step_vjp: bad arguments");
  return guarded(h, [&] {
    h->eng->step_vjp(M, (const tdmrg::cplx* const*)A_in, tau_re, tau_im,
                     (const tdmrg::cplx* const*)Abar_out, (tdmrg::cplx* const*)A_out,
                     (tdmrg::cplx* const*)Abar_in, theta_bar, nodes);
  });
}

int tdmrg_correlation_states_vjp(tdmrg_model* h, int M, const void* const* psi1,
                                 const void* const* psi2, double dt, int nsteps, int every,
                                 const double* Cbar, double* C_out, void* const* g1,
                                 void* const* g2, double* theta_bar, int nodes) {
  if (!h) return fail(nullptr, TDMRG_ERR_ARG, "NULL handle");
  if (M < 1 || !psi1 || !psi2 || !(dt > 0.0) || nsteps < 0 || every < 1 || !Cbar || !C_out ||
      !g1 || !g2 || !theta_bar || nodes < 1 || nodes > 64)
    return fail(h, TDMRG_ERR_ARG, "correlation_states_vjp: bad arguments");
  return guarded(h, [&] {
    h->eng->correlation_states_vjp(M, (const tdmrg::cplx* const*)psi1,
                                   (const tdmrg::cplx* const*)psi2, dt, nsteps, every, Cbar,
                                   C_out, (tdmrg::cplx* const*)g1, (tdmrg::cplx* const*)g2,
                                   theta_bar, nodes);
  });
}

int tdmrg_correlation_vjp(tdmrg_model* h, double beta, double dtau, int M, double dt,
                          int nsteps, int every, const double* Cbar, double* C_out,
                          double* theta_bar, double* logz_out, int nodes) {
  if (!h) return fail(nullptr, TDMRG_ERR_ARG, "NULL handle");
  if (!Cbar || !C_out || !theta_bar || nodes < 1 || nodes > 64)
    return fail(h, TDMRG_ERR_ARG, "correlation_vjp: bad arguments");
  return guarded(h, [&] {
    h->eng->correlation_vjp(beta, dtau, M, dt, nsteps, every, Cbar, C_out, theta_bar, logz_out,
                            nodes);
  });
}

int tdmrg_host_quadrature_nodes(double r, int nmax, double eps, int* n_out) {
  if (!(r >= 0.0) || !std::isfinite(r) || nmax < 1 || nmax > 64 || !(eps > 0.0) || !n_out)
    return fail(nullptr, TDMRG_ERR_ARG, "host_quadrature_nodes: need r >= 0, 1 <= nmax <= 64, eps > 0");
  return guarded(nullptr, [&] { *n_out = tdmrg::gauss_legendre_nodes_for(r, nmax, eps); });
}

int tdmrg_host_gauss_legendre(int n, double* s, double* w) {
  if (n < 1 || n > 64 || !s || !w)
    return fail(nullptr, TDMRG_ERR_ARG, "host_gauss_legendre: need 1 <= n <= 64");
  return guarded(nullptr, [&] {
    std::vector<double> sv, wv;
    tdmrg::gauss_legendre01(n, sv, wv);
    for (int i = 0; i < n; ++i) {
      s[i] = sv[i];
      w[i] = wv[i];
    }
  });
}

int tdmrg_host_tridiag_exp(int k, const double* alpha, const double* beta, int nz,
                           const double* z, double* out) {
  if (k < 1 || k > 64 || nz < 0 || !alpha || (k > 1 && !beta) || (nz > 0 && (!z || !out)))
    return fail(nullptr, TDMRG_ERR_ARG, "host_tridiag_exp: need 1 <= k <= 64 and non-NULL arrays");
  for (int i = 0; i < k; ++i)
    if (!std::isfinite(alpha[i]) || (i + 1 < k && !std::isfinite(beta[i])))
      return fail(nullptr, TDMRG_ERR_ARG, "host_tridiag_exp: non-finite entry");
  return guarded(nullptr, [&] {
    std::vector<tdmrg::Cx> zz(nz), o((size_t)nz * k);
    for (int s = 0; s < nz; ++s) zz[s] = tdmrg::Cx(z[2 * s], z[2 * s + 1]);
    tdmrg::tridiag_exp_e1(k, alpha, beta, nz, zz.data(), o.data());
    for (size_t i = 0; i < o.size(); ++i) {
      out[2 * i] = o[i].real();
      out[2 * i + 1] = o[i].imag();
    }
  });
}

int tdmrg_get_logz(const tdmrg_model* h, double* logz) {
  if (!h || !logz) return fail(nullptr, TDMRG_ERR_ARG, "NULL argument");
  if (!h->eng->prepared()) return fail(const_cast<tdmrg_model*>(h), TDMRG_ERR_STATE, "not prepared");
  *logz = h->eng->logz();
  return TDMRG_OK;
}

int tdmrg_get_stats(const tdmrg_model* h, double* stats, int n) {
  if (!h || !stats || n < 0) return fail(nullptr, TDMRG_ERR_ARG, "NULL argument");
  const tdmrg::Stats s = h->eng->total_stats();
  const double v[24] = {s.site_updates, s.matvecs, s.heff_flops, s.krylov_vectors,
                        s.bond_matvecs, s.qrs, s.completions, s.env_updates, s.heff_ms,
                        s.h2d_bytes, s.d2h_bytes,
                        (double)tdmrg::launch_count() - s.launches_at_reset + s.replayed_launches,
                        s.t_site, s.t_qr, s.t_env, s.t_bond, s.t_absorb, s.t_observe,
                        s.qr_ms, s.qr_flops, s.lz_ms, s.qr_bulk_ms, s.qr_bulk_flops, s.qr_bulk_n};
  for (int i = 0; i < n && i < 24; ++i) stats[i] = v[i];
  return TDMRG_OK;
}

int tdmrg_reset_stats(tdmrg_model* h) {
  if (!h) return fail(nullptr, TDMRG_ERR_ARG, "NULL handle");
  return guarded(h, [&] { h->eng->reset_stats(); });
}

const char* tdmrg_last_error(const tdmrg_model* h) { return h ? h->err.c_str() : g_err.c_str(); }
const char* tdmrg_last_global_error(void) { return g_err.c_str(); }

// ---------------------------------------------------------------------------------------
// kernel-level entry points
// ---------------------------------------------------------------------------------------
long long tdmrg_heff_workspace_floats(int Ml, int Mr, int d, int Dl, int Dr) {
  if (Ml < 1 || Mr < 1 || d < 1 || Dl < 1 || Dr < 1) return -1;
  return tdmrg::heff_tc_floats(Ml, Mr, d * d, Dl, Dr);
}

int tdmrg_kernel_heff(int Ml, int Mr, int d, int Dl, int Dr, const double* W_host, const void* L,
                      const void* R, const void* A, void* out, void* X, void* Y, void* ws32,
                      int precision, void* stream) {
  if (Ml < 1 || Mr < 1 || d < 1 || Dl < 1 || Dr < 1 || !W_host || !L || !R || !A || !out)
    return fail(nullptr, TDMRG_ERR_ARG, "heff: bad arguments");
  if (precision == TDMRG_PREC_C128 && (!X || !Y))
    return fail(nullptr, TDMRG_ERR_ARG, "heff: C128 needs the X and Y workspaces");
  if (precision == TDMRG_PREC_C64_3XTF32 && !ws32)
    return fail(nullptr, TDMRG_ERR_ARG, "heff: 3xTF32 needs the ws32 workspace");
  if (precision != TDMRG_PREC_C128 && precision != TDMRG_PREC_C64_3XTF32)
    return fail(nullptr, TDMRG_ERR_ARG, "heff: unknown precision");
  return guarded(nullptr, [&] {
    TempMpo W(Dl, Dr, d, W_host);
    cudaStream_t s = (cudaStream_t)stream;
    if (precision == TDMRG_PREC_C128) {
      tdmrg::Ctx c{s, (tdmrg::cplx*)X, (tdmrg::cplx*)Y};
      tdmrg::heff_f64(c, W.m.s[0], Ml, Mr, d * d, d, (const tdmrg::cplx*)L,
                      (const tdmrg::cplx*)R, (const tdmrg::cplx*)A, (tdmrg::cplx*)out, nullptr);
    } else {
      int* st = nullptr;
      CK(cudaMalloc(&st, sizeof(int)));
      CK(cudaMemsetAsync(st, 0, sizeof(int), s));
      tdmrg::TcWork w = tdmrg::heff_tc_carve((float*)ws32, Ml, Mr, d * d, Dl, Dr, st);
      tdmrg::heff_tc_envs(s, w, Ml, Mr, Dl, Dr, (const tdmrg::cplx*)L, (const tdmrg::cplx*)R);
      tdmrg::heff_tc(s, w, W.m.s[0], Ml, Mr, d * d, d, (const tdmrg::cplx*)A, (tdmrg::cplx*)out);
      int hs = 0;
      CK(cudaMemcpyAsync(&hs, st, sizeof(int), cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      cudaFree(st);
      if (hs) throw Failure{TDMRG_ERR_TIMEOUT, "tensor-core pipeline wait timed out"};
    }
    CK(cudaStreamSynchronize(s));
  });
}

int tdmrg_kernel_heff_timed(int Ml, int Mr, int d, int Dl, int Dr, const double* W_host,
                            const void* L, const void* R, const void* A, void* out, int precision,
                            int reps, double* ms_per_matvec, void* stream) {
  if (Ml < 1 || Mr < 1 || d < 1 || Dl < 1 || Dr < 1 || !W_host || !L || !R || !A || !out ||
      reps < 1 || !ms_per_matvec)
    return fail(nullptr, TDMRG_ERR_ARG, "heff_timed: bad arguments");
  if (precision != TDMRG_PREC_C128 && precision != TDMRG_PREC_C64_3XTF32)
    return fail(nullptr, TDMRG_ERR_ARG, "heff_timed: unknown precision");
  return guarded(nullptr, [&] {
    using tdmrg::cplx;
    using tdmrg::pad4;
    TempMpo W(Dl, Dr, d, W_host);
    cudaStream_t s = (cudaStream_t)stream;
    const int D = d * d;
    const long long site = (long long)Ml * D * Mr;
    std::vector<void*> mem;
    struct Free {
      std::vector<void*>& m;
      ~Free() {
        for (void* p : m) cudaFree(p);
      }
    } fr{mem};
    auto get = [&](size_t bytes) {
      void* p = nullptr;
      CK(cudaMalloc(&p, bytes > 0 ? bytes : 16));
      mem.push_back(p);
      return p;
    };
    int* st = (int*)get(sizeof(int));
    CK(cudaMemsetAsync(st, 0, sizeof(int), s));
    const int Dm = Dl > Dr ? Dl : Dr;
    tdmrg::TcBufs b{};
    cplx *X = nullptr, *Y = nullptr;
    if (precision == TDMRG_PREC_C64_3XTF32) {
      b.envA = (float*)get(sizeof(float) * 4 * (size_t)Dl * Ml * pad4(Ml));
      b.envB = (float*)get(sizeof(float) * 4 * (size_t)Dr * Mr * pad4(Mr));
      b.siteA = (float*)get(sizeof(float) * 4 * (size_t)D * Mr * pad4(Ml));
      b.x32 = (float*)get(sizeof(float) * 2 * (size_t)Dm * site);
      b.mix = (float*)get(sizeof(float) * 4 * (size_t)Dr * Ml * D * pad4(Mr));
      b.kpart_len = 4LL << 20;
      b.kpart = (float*)get(sizeof(float) * (size_t)b.kpart_len);
      b.status = st;
      tdmrg::heff_tc_prepare(s, b, Ml, Mr, Dl, Dr, (const cplx*)L, (const cplx*)R);
    } else {
      X = (cplx*)get(sizeof(cplx) * (size_t)Dm * site);
      Y = (cplx*)get(sizeof(cplx) * (size_t)Dm * site);
    }
    auto once = [&] {
      if (precision == TDMRG_PREC_C64_3XTF32)
        tdmrg::heff_tc_apply(s, b, W.m.s[0], Ml, Mr, D, d, (const cplx*)A, (cplx*)out);
      else
        tdmrg::heff_f64(tdmrg::Ctx{s, X, Y}, W.m.s[0], Ml, Mr, D, d, (const cplx*)L,
                        (const cplx*)R, (const cplx*)A, (cplx*)out, nullptr);
    };
    once();   // warm-up
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    CK(cudaEventRecord(e0, s));
    for (int r = 0; r < reps; ++r) once();
    CK(cudaEventRecord(e1, s));
    CK(cudaEventSynchronize(e1));
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    int hs = 0;
    CK(cudaMemcpyAsync(&hs, st, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (hs) throw Failure{TDMRG_ERR_TIMEOUT, "tensor-core pipeline wait timed out"};
    *ms_per_matvec = ms / reps;
  });
}

int tdmrg_model_set_concurrent(tdmrg_model* h, int on) {
  if (!h) return fail(nullptr, TDMRG_ERR_ARG, "NULL handle");
  return guarded(h, [&] { h->eng->set_concurrent(on != 0); });
}

int tdmrg_tune_record_shapes(int on) {
  tdmrg::tc_record_shapes(on != 0);
  return TDMRG_OK;
}

int tdmrg_tune_recorded_shapes(int* shapes, int capacity, int* count) {
  if (!count || capacity < 0 || (capacity > 0 && !shapes))
    return fail(nullptr, TDMRG_ERR_ARG, "recorded_shapes: bad arguments");
  const auto v = tdmrg::tc_recorded_shapes();
  *count = (int)v.size();
  for (int i = 0; i < (int)v.size() && i < capacity; ++i)
    for (int j = 0; j < 5; ++j) shapes[5 * i + j] = v[i][j];
  return TDMRG_OK;
}

int tdmrg_tune_reload_table(void) {
  tdmrg::tc_reload_table();
  return TDMRG_OK;
}

int tdmrg_tune_table_lookup(int M, int N, int K, int nred, int nbatch, int* ksplit, int* tile_n) {
  if (!ksplit || !tile_n) return fail(nullptr, TDMRG_ERR_ARG, "tune_table_lookup: NULL output");
  return guarded(nullptr, [&] {
    int ks = 0, bn = 0;
    if (!tdmrg::tc_table_lookup(M, N, K, nred, nbatch, &ks, &bn)) ks = bn = 0;
    *ksplit = ks;
    *tile_n = bn;
  });
}

int tdmrg_kernel_tc_gemm_timed(int M, int N, int K, int nred, int nbatch, int ksplit, int tile_n,
                               int reps, double* ms_out, void* stream) {
  if (M < 1 || N < 1 || K < 1 || nred < 1 || nbatch < 1 || ksplit < 0 || reps < 1 || !ms_out ||
      (tile_n != 0 && tile_n != 64 && tile_n != 128))
    return fail(nullptr, TDMRG_ERR_ARG, "tc_gemm_timed: bad arguments");
  return guarded(nullptr, [&] {
    using tdmrg::pad4;
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<void*> mem;
    struct Free {
      std::vector<void*>& m;
      ~Free() {
        for (void* p : m) cudaFree(p);
      }
    } fr{mem};
    auto get = [&](size_t bytes) {
      void* p = nullptr;
      CK(cudaMalloc(&p, bytes));
      mem.push_back(p);
      return p;
    };
    tdmrg::TcOperand A{nullptr, M, K, pad4(K), nred};
    tdmrg::TcOperand B{nullptr, N, K, pad4(K), nred * nbatch};
    A.p = (float*)get(sizeof(float) * (size_t)A.floats());
    B.p = (float*)get(sizeof(float) * (size_t)B.floats());
    CK(cudaMemsetAsync(A.p, 0, sizeof(float) * (size_t)A.floats(), s));
    CK(cudaMemsetAsync(B.p, 0, sizeof(float) * (size_t)B.floats(), s));
    const long long mn = (long long)nbatch * M * N;
    float* C = (float*)get(sizeof(float) * 2 * (size_t)mn);
    int* st = (int*)get(sizeof(int));
    CK(cudaMemsetAsync(st, 0, sizeof(int), s));
    tdmrg::TcGemm g{};
    g.M = M; g.N = N; g.K = K; g.nred = nred; g.nbatch = nbatch;
    g.a_red = nred > 1 ? 1 : 0; g.b_red = nred > 1 ? 1 : 0; g.b_bat = nbatch > 1 ? nred : 0;
    g.out_mode = 1; g.C = C; g.ldc = N; g.sbc = (long long)M * N; g.plane = mn;
    g.status = st; g.ksplit = ksplit; g.bn = tile_n;
    g.part_len = 4LL << 20;           // the engine's split-K scratch
    g.part = (float*)get(sizeof(float) * (size_t)g.part_len);
    CK(tdmrg::tc_gemm(A, B, g, s));   // warm-up
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    CK(cudaEventRecord(e0, s));
    for (int r = 0; r < reps; ++r) CK(tdmrg::tc_gemm(A, B, g, s));
    CK(cudaEventRecord(e1, s));
    CK(cudaEventSynchronize(e1));
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    int hs = 0;
    CK(cudaMemcpyAsync(&hs, st, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (hs) throw Failure{TDMRG_ERR_TIMEOUT, "tensor-core pipeline wait timed out"};
    *ms_out = ms / reps;
  });
}

int tdmrg_kernel_heff_vjp(int Ml, int Mr, int d, int Dl, int Dr, const double* W_host,
                          const void* L, const void* R, const void* A, const void* ybar,
                          void* Abar, void* Lbar, void* Rbar, void* X, void* Y, void* stream) {
  if (Ml < 1 || Mr < 1 || d < 1 || Dl < 1 || Dr < 1 || !W_host || !L || !R || !A || !ybar ||
      !Abar || !Lbar || !Rbar || !X || !Y)
    return fail(nullptr, TDMRG_ERR_ARG, "heff_vjp: bad arguments");
  return guarded(nullptr, [&] {
    cudaStream_t s = (cudaStream_t)stream;
    using tdmrg::cplx;
    const int D = d * d;
    // W^T conj: op'[s][u] = conj(op[u][s]) for every channel pair
    std::vector<double> Wt((size_t)2 * Dl * Dr * D);
    for (int b = 0; b < Dl * Dr; ++b)
      for (int si = 0; si < d; ++si)
        for (int ui = 0; ui < d; ++ui) {
          const size_t dst = 2 * ((size_t)b * D + si * d + ui);
          const size_t src = 2 * ((size_t)b * D + ui * d + si);
          Wt[dst] = W_host[src];
          Wt[dst + 1] = -W_host[src + 1];
        }
    TempMpo W(Dl, Dr, d, W_host);
    TempMpo Wc(Dl, Dr, d, Wt.data());
    cplx* Lh = nullptr;
    cplx* Rh = nullptr;
    struct Free {
      cplx*& a;
      cplx*& b;
      ~Free() {
        if (a) cudaFree(a);
        if (b) cudaFree(b);
      }
    } fr{Lh, Rh};
    CK(cudaMalloc(&Lh, sizeof(cplx) * (size_t)Dl * Ml * Ml));
    CK(cudaMalloc(&Rh, sizeof(cplx) * (size_t)Dr * Mr * Mr));
    // per-channel Hermitian conjugates of the environments
    for (int w = 0; w < Dl; ++w)
      CK(tdmrg::ztranspose(Ml, Ml, (const cplx*)L + (size_t)w * Ml * Ml, Lh + (size_t)w * Ml * Ml,
                           1, s));
    for (int w = 0; w < Dr; ++w)
      CK(tdmrg::ztranspose(Mr, Mr, (const cplx*)R + (size_t)w * Mr * Mr, Rh + (size_t)w * Mr * Mr,
                           1, s));
    tdmrg::Ctx c{s, (cplx*)X, (cplx*)Y};
    // Abar = H_eff(L^dagger, W^T conj, R^dagger) ybar
    tdmrg::heff_f64(c, Wc.m.s[0], Ml, Mr, D, d, Lh, Rh, (const cplx*)ybar, (cplx*)Abar, nullptr);
    // Lbar = conj(env_right(R, bra = ybar, W, ket = A)); Rbar = conj(env_left(L, ybar, W, A))
    tdmrg::env_right_f64(c, W.m.s[0], Ml, Mr, Ml, Mr, D, d, (const cplx*)R, (const cplx*)ybar,
                         (const cplx*)A, (cplx*)Lbar);
    CK(tdmrg::zconj((long long)Dl * Ml * Ml, (cplx*)Lbar, s));
    tdmrg::env_left_f64(c, W.m.s[0], Ml, Mr, Ml, Mr, D, d, (const cplx*)L, (const cplx*)ybar,
                        (const cplx*)A, (cplx*)Rbar);
    CK(tdmrg::zconj((long long)Dr * Mr * Mr, (cplx*)Rbar, s));
    CK(cudaStreamSynchronize(s));
  });
}

int tdmrg_kernel_zgemm_tc(int M, int N, int K, const void* A, const void* B, int conjA, int conjB,
                          void* C, void* stream) {
  if (M < 1 || N < 1 || K < 1 || !A || !B || !C) return fail(nullptr, TDMRG_ERR_ARG, "zgemm_tc: bad arguments");
  return guarded(nullptr, [&] {
    cudaStream_t s = (cudaStream_t)stream;
    tdmrg::TcOperand a{nullptr, M, K, tdmrg::pad4(K), 1}, b{nullptr, N, K, tdmrg::pad4(K), 1};
    int* st = nullptr;
    float* part = nullptr;
    const long long part_len = 2LL * M * N * 64;      // room for a split-K of up to 64
    CK(cudaMalloc(&a.p, sizeof(float) * a.floats()));
    CK(cudaMalloc(&b.p, sizeof(float) * b.floats()));
    CK(cudaMalloc(&st, sizeof(int)));
    CK(cudaMalloc(&part, sizeof(float) * part_len));
    struct F {
      void* x[4];
      ~F() {
        for (void* p : x)
          if (p) cudaFree(p);
      }
    } f{{a.p, b.p, st, part}};
    CK(cudaMemsetAsync(st, 0, sizeof(int), s));
    CK(tdmrg::split_f64((const tdmrg::cplx*)A, 0, K, 1, 0, a, s));
    CK(tdmrg::split_f64((const tdmrg::cplx*)B, 0, K, 1, 0, b, s));
    tdmrg::TcGemm g{};
    g.M = M; g.N = N; g.K = K; g.nred = 1; g.nbatch = 1; g.conjA = conjA; g.conjB = conjB;
    g.out_mode = 0; g.C = C; g.ldc = N; g.status = st;
    g.part = part; g.part_len = part_len;
    CK(tdmrg::tc_gemm(a, b, g, s));
    int hs = 0;
    CK(cudaMemcpyAsync(&hs, st, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (hs) throw Failure{TDMRG_ERR_TIMEOUT, "tensor-core pipeline wait timed out"};
  });
}

int tdmrg_kernel_env_left(int Ml1, int Mr1, int Ml2, int Mr2, int d, int Dl, int Dr,
                          const double* W_host, const void* L, const void* bra, const void* ket,
                          void* Lout, void* X, void* Y, void* stream) {
  if (Ml1 < 1 || Mr1 < 1 || Ml2 < 1 || Mr2 < 1 || d < 1 || Dl < 1 || Dr < 1 || !W_host || !L ||
      !bra || !ket || !Lout || !X || !Y)
    return fail(nullptr, TDMRG_ERR_ARG, "env_left: bad arguments");
  return guarded(nullptr, [&] {
    TempMpo W(Dl, Dr, d, W_host);
    tdmrg::Ctx c{(cudaStream_t)stream, (tdmrg::cplx*)X, (tdmrg::cplx*)Y};
    tdmrg::env_left_f64(c, W.m.s[0], Ml1, Mr1, Ml2, Mr2, d * d, d, (const tdmrg::cplx*)L,
                        (const tdmrg::cplx*)bra, (const tdmrg::cplx*)ket, (tdmrg::cplx*)Lout);
    CK(cudaStreamSynchronize((cudaStream_t)stream));
  });
}

int tdmrg_kernel_gauge_qr(int m, int n, const void* Y, int p, const void* E, void* Q, void* R,
                          int* status, void* stream) {
  if (m < 1 || n < 1 || m < n || !Y || !Q || !R || p < 0 || (p > 0 && !E))
    return fail(nullptr, TDMRG_ERR_ARG, "gauge_qr: need m >= n >= 1 and non-NULL buffers");
  return guarded(nullptr, [&] {
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0, sms = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    tdmrg::QrScratch W{};
    W.gmax = sms;
    W.nmax = n;
    int* st = status;
    struct Free {
      tdmrg::QrScratch& w;
      int*& st;
      bool own;
      ~Free() {
        if (w.part) cudaFree(w.part);
        if (w.partn) cudaFree(w.partn);
        if (w.bar) cudaFree(w.bar);
        if (own && st) cudaFree(st);
      }
    } fr{W, st, status == nullptr};
    CK(cudaMalloc(&W.part, sizeof(tdmrg::cplx) * 2 * (size_t)sms * (n + 1)));
    CK(cudaMalloc(&W.partn, sizeof(double) * 2 * (size_t)sms));
    CK(cudaMalloc(&W.bar, sizeof(unsigned) * 2));
    if (!st) {
      CK(cudaMalloc(&st, sizeof(int)));
      CK(cudaMemsetAsync(st, 0, sizeof(int), s));
    }
    tdmrg::QrRef y{(const tdmrg::cplx*)Y, n, 1, 1LL << 60, 0, 0};
    tdmrg::QrRef e{(const tdmrg::cplx*)(p > 0 ? E : Y), p > 0 ? p : n, 1, 1LL << 60, 0, 0};
    CK(tdmrg::gauge_qr(m, n, y, p, e, (tdmrg::cplx*)Q, (tdmrg::cplx*)R, W, st, s));
    int hs = 0;
    CK(cudaMemcpyAsync(&hs, st, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (hs == 1) throw Failure{TDMRG_ERR_TIMEOUT, "gauge QR grid barrier timed out"};
    if (hs == 2) throw Failure{TDMRG_ERR_CUDA, "gauge QR ran out of completion vectors"};
  });
}

int tdmrg_kernel_dfma_loop(int blocks, long long iters, double* sink, double* flops_out,
                           void* stream) {
  if (blocks < 1 || iters < 1 || !sink)
    return fail(nullptr, TDMRG_ERR_ARG, "dfma_loop: need blocks >= 1, iters >= 1, a sink");
  return guarded(nullptr, [&] {
    CK(tdmrg::dfma_loop(blocks, iters, sink, (cudaStream_t)stream));
    if (flops_out) *flops_out = 2.0 * 8.0 * 256.0 * (double)blocks * (double)iters;
  });
}

int tdmrg_kernel_gauge_qr_blocked(int m, int n, const void* Y, int p, const void* E, void* Q,
                                  void* R, int* status, void* stream) {
  if (m < 1 || n < 1 || m < n || !Y || !Q || !R || p < 0 || (p > 0 && !E))
    return fail(nullptr, TDMRG_ERR_ARG, "gauge_qr_blocked: need m >= n >= 1 and non-NULL buffers");
  return guarded(nullptr, [&] {
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0, sms = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    tdmrg::QrScratch W{};
    W.gmax = sms;
    W.nmax = n;
    tdmrg::cplx* qb = nullptr;
    unsigned char* acc = nullptr;
    int* st = status;
    const long long qlen = tdmrg::gauge_qr_blocked_scratch(n, sms);
    struct Free {
      tdmrg::QrScratch& w;
      tdmrg::cplx*& qb;
      unsigned char*& acc;
      int*& st;
      bool own;
      ~Free() {
        if (w.part) cudaFree(w.part);
        if (w.partn) cudaFree(w.partn);
        if (w.bar) cudaFree(w.bar);
        if (qb) cudaFree(qb);
        if (acc) cudaFree(acc);
        if (own && st) cudaFree(st);
      }
    } fr{W, qb, acc, st, status == nullptr};
    CK(cudaMalloc(&W.part, sizeof(tdmrg::cplx) * 2 * (size_t)sms * (n + 1)));
    CK(cudaMalloc(&W.partn, sizeof(double) * 2 * (size_t)sms));
    CK(cudaMalloc(&W.bar, sizeof(unsigned) * 2));
    CK(cudaMalloc(&qb, sizeof(tdmrg::cplx) * (size_t)qlen));
    CK(cudaMalloc(&acc, (size_t)n + 16));
    if (!st) {
      CK(cudaMalloc(&st, sizeof(int)));
      CK(cudaMemsetAsync(st, 0, sizeof(int), s));
    }
    tdmrg::QrRef y{(const tdmrg::cplx*)Y, n, 1, 1LL << 60, 0, 0};
    tdmrg::QrRef e{(const tdmrg::cplx*)(p > 0 ? E : Y), p > 0 ? p : n, 1, 1LL << 60, 0, 0};
    CK(tdmrg::gauge_qr_blocked(m, n, y, p, e, (tdmrg::cplx*)Q, (tdmrg::cplx*)R, qb, qlen, acc, W,
                               st, s));
    int hs = 0;
    CK(cudaMemcpyAsync(&hs, st, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (hs == 1) throw Failure{TDMRG_ERR_TIMEOUT, "gauge QR grid barrier timed out"};
    if (hs == 2) throw Failure{TDMRG_ERR_CUDA, "gauge QR ran out of completion vectors"};
  });
}

int tdmrg_kernel_bond_exp(int M, int Dw, const void* L, const void* R, const void* C, void* out,
                          double tau_re, double tau_im, double tol, int kmax, int* kused,
                          void* stream) {
  if (M < 1 || M > tdmrg::BOND_EXP_MAX_M || Dw < 1 || !L || !R || !C || !out || kmax < 1 ||
      kmax > tdmrg::KMAX || !(tol > 0.0))
    return fail(nullptr, TDMRG_ERR_ARG,
                "bond_exp: need 1 <= M <= 256, Dw >= 1, 1 <= kmax <= 32, tol > 0");
  return guarded(nullptr, [&] {
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0, sms = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const long long n = (long long)M * M;
    if (tdmrg::bond_exp_smem(M, tdmrg::bond_exp_grid(M, Dw, 0, sms)) > tdmrg::BOND_EXP_MAX_SMEM)
      throw Failure{TDMRG_ERR_ARG, "bond_exp: bond dimension too large for one cooperative grid"};
    const int kcap = (int)std::min<long long>(kmax, n);
    tdmrg::BondScratch W{};
    W.maxn = n;
    W.maxDw = Dw;
    W.gmax = sms;
    tdmrg::cplx* V = nullptr;
    int* st = nullptr;
    struct Free {
      tdmrg::BondScratch& w;
      tdmrg::cplx*& V;
      int*& st;
      ~Free() {
        for (void* p : {(void*)w.W, (void*)w.T, (void*)w.P, (void*)w.part, (void*)w.partn,
                        (void*)w.bar, (void*)w.mv, (void*)V, (void*)st})
          if (p) cudaFree(p);
      }
    } fr{W, V, st};
    CK(cudaMalloc(&W.W, sizeof(tdmrg::cplx) * (size_t)n));
    CK(cudaMalloc(&W.T, sizeof(float2) * (size_t)Dw * n));
    CK(cudaMalloc(&W.P, sizeof(float2) * (size_t)Dw * n));
    CK(cudaMalloc(&W.part, sizeof(tdmrg::cplx) * 2 * (size_t)sms * (tdmrg::KMAX + 1)));
    CK(cudaMalloc(&W.partn, sizeof(double) * 2 * (size_t)sms));   // 2 * gmax
    CK(cudaMalloc(&W.bar, sizeof(unsigned) * 2));
    CK(cudaMalloc(&W.mv, sizeof(unsigned long long)));
    CK(cudaMalloc(&V, sizeof(tdmrg::cplx) * (size_t)kcap * n));
    CK(cudaMalloc(&st, sizeof(int)));
    CK(cudaMemsetAsync(W.mv, 0, sizeof(unsigned long long), s));
    CK(cudaMemsetAsync(st, 0, sizeof(int), s));
    CK(tdmrg::bond_exp_fused(M, Dw, (const tdmrg::cplx*)L, (const tdmrg::cplx*)R,
                             (const tdmrg::cplx*)C, (tdmrg::cplx*)out, V, W, st, tau_re, tau_im,
                             tol, kcap, 0, 0, s));
    int hs = 0;
    unsigned long long used = 0;
    CK(cudaMemcpyAsync(&hs, st, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(&used, W.mv, sizeof(used), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (hs == 1) throw Failure{TDMRG_ERR_TIMEOUT, "bond exponential grid barrier timed out"};
    if (kused) *kused = (int)used;
  });
}


}  // extern "C"

namespace {
// exp(tau H_eff) VJP with, for nparam derivative sites, theta_bar[p] = Re<Hbar, H_eff(dW_p)>
int site_exp_vjp_impl(int Ml, int Mr, int d, int Dl, int Dr, const double* W_host, const void* L,
                      const void* R, const void* A, const void* ybar, double tau_re,
                      double tau_im, int nodes, double tol, int nparam, const double* dW_host,
                      void* Abar, void* Lbar, void* Rbar, double* theta_bar, void* stream) {
  if (Ml < 1 || Mr < 1 || d < 1 || Dl < 1 || Dr < 1 || !W_host || !L || !R || !A || !ybar ||
      !Abar || !Lbar || !Rbar || nodes < 1 || nodes > 64 || !(tol > 0.0) || nparam < 0 ||
      (nparam > 0 && (!dW_host || !theta_bar)))
    return fail(nullptr, TDMRG_ERR_ARG, "site_exp_vjp: bad arguments");
  return guarded(nullptr, [&] {
    cudaStream_t s = (cudaStream_t)stream;
    const int D = d * d;
    const size_t site = (size_t)Dl * Dr * D;
    const long long n = (long long)Ml * D * Mr;
    const long long nl = (long long)Dl * Ml * Ml, nr = (long long)Dr * Mr * Mr;
    TempMpo W(Dl, Dr, d, W_host);
    std::vector<std::unique_ptr<TempMpo>> dWs(nparam);
    for (int p = 0; p < nparam; ++p) {
      theta_bar[p] = 0.0;
      if (any_nonzero(dW_host + 2 * site * p, 2 * site))
        dWs[p].reset(new TempMpo(Dl, Dr, d, dW_host + 2 * site * p));
    }
    tdmrg::ModelParams P;
    P.N = 3;
    Engine eng(P);
    eng.set_stream(s);
    eng.set_krylov(tol, tdmrg::KMAX, 0);
    eng.ensure_workspace(n, n, 1, 1);
    const long long xy = (long long)std::max(Dl, Dr) * n;
    DevBufs buf;
    cplx* X = buf.get(xy);
    cplx* Y = buf.get(xy);
    cplx* a = buf.get(n);
    cplx* b = buf.get(n);
    cplx* El = buf.get(nl);
    cplx* Er = buf.get(nr);
    cplx* t = nparam > 0 ? buf.get(n) : nullptr;
    cplx* part = nparam > 0 ? buf.get(257) : nullptr;
    tdmrg::Ctx c{s, X, Y};
    const cplx* Ld = (const cplx*)L;
    const cplx* Rd = (const cplx*)R;
    auto heff = [&](const cplx* in, cplx* out, const int* skip) {
      tdmrg::heff_f64(c, W.m.s[0], Ml, Mr, D, d, Ld, Rd, in, out, skip);
    };
    // Abar = exp(conj(tau) H) ybar  (H Hermitian)
    eng.krylov(n, (const cplx*)ybar, (cplx*)Abar, tau_re, -tau_im, heff);
    // Hbar = conj(tau) int_0^1 a(s) b(s)^H ds, a(s) = e^{(1-s) conj(tau) H} ybar,
    // b(s) = e^{s tau H} A; its L and R parts are conjugated environment updates with a(s)
    // as bra and b(s) as ket: Lbar = conj(sum_s conj(k_s) env_right(R, a_s, W, b_s)),
    // k_s = w_s conj(tau), and the same for Rbar with env_left.  A parameter enters through
    // W only: theta_bar = sum_s Re(conj(k_s) <a_s, H_eff(dW) b_s>).
    CK(cudaMemsetAsync(Lbar, 0, sizeof(cplx) * (size_t)nl, s));
    CK(cudaMemsetAsync(Rbar, 0, sizeof(cplx) * (size_t)nr, s));
    std::vector<double> sn, wn;
    tdmrg::gauss_legendre01(nodes, sn, wn);
    for (int q = 0; q < nodes; ++q) {
      eng.krylov(n, (const cplx*)A, b, sn[q] * tau_re, sn[q] * tau_im, heff);
      eng.krylov(n, (const cplx*)ybar, a, (1.0 - sn[q]) * tau_re, -(1.0 - sn[q]) * tau_im, heff);
      const cplx kc = {wn[q] * tau_re, wn[q] * tau_im};     // conj(w_s conj(tau)) = w_s tau
      tdmrg::env_right_f64(c, W.m.s[0], Ml, Mr, Ml, Mr, D, d, Rd, a, b, El);
      CK(tdmrg::zaxpy(nl, kc, El, (cplx*)Lbar, s));
      tdmrg::env_left_f64(c, W.m.s[0], Ml, Mr, Ml, Mr, D, d, Ld, a, b, Er);
      CK(tdmrg::zaxpy(nr, kc, Er, (cplx*)Rbar, s));
      for (int p = 0; p < nparam; ++p) {
        if (!dWs[p]) continue;
        tdmrg::heff_f64(c, dWs[p]->m.s[0], Ml, Mr, D, d, Ld, Rd, b, t, nullptr);
        const cplx z = dot_c(a, t, n, part, s);
        theta_bar[p] += kc.x * z.x - kc.y * z.y;
      }
    }
    CK(tdmrg::zconj(nl, (cplx*)Lbar, s));
    CK(tdmrg::zconj(nr, (cplx*)Rbar, s));
    eng.sync_and_check();
  });
}
}  // namespace

extern "C" {

int tdmrg_kernel_site_exp_vjp(int Ml, int Mr, int d, int Dl, int Dr, const double* W_host,
                              const void* L, const void* R, const void* A, const void* ybar,
                              double tau_re, double tau_im, int nodes, double tol, void* Abar,
                              void* Lbar, void* Rbar, void* stream) {
  return site_exp_vjp_impl(Ml, Mr, d, Dl, Dr, W_host, L, R, A, ybar, tau_re, tau_im, nodes, tol,
                           0, nullptr, Abar, Lbar, Rbar, nullptr, stream);
}

int tdmrg_kernel_site_exp_vjp_theta(int Ml, int Mr, int d, int Dl, int Dr, const double* W_host,
                                    const void* L, const void* R, const void* A,
                                    const void* ybar, double tau_re, double tau_im, int nodes,
                                    double tol, int nparam, const double* dW_host, void* Abar,
                                    void* Lbar, void* Rbar, double* theta_bar, void* stream) {
  return site_exp_vjp_impl(Ml, Mr, d, Dl, Dr, W_host, L, R, A, ybar, tau_re, tau_im, nodes, tol,
                           nparam, dW_host, Abar, Lbar, Rbar, theta_bar, stream);
}

int tdmrg_kernel_bond_exp_vjp(int M, int Dw, const void* L, const void* R, const void* C,
                              const void* ybar, double tau_re, double tau_im, int nodes,
                              double tol, void* Cbar, void* Lbar, void* Rbar, void* stream) {
  if (M < 1 || Dw < 1 || !L || !R || !C || !ybar || !Cbar || !Lbar || !Rbar || nodes < 1 ||
      nodes > 64 || !(tol > 0.0))
    return fail(nullptr, TDMRG_ERR_ARG, "bond_exp_vjp: bad arguments");
  return guarded(nullptr, [&] {
    using tdmrg::cplx;
    using tdmrg::MatRef;
    cudaStream_t s = (cudaStream_t)stream;
    const long long mm = (long long)M * M;
    tdmrg::ModelParams P;
    P.N = 3;
    Engine eng(P);
    eng.set_stream(s);
    eng.set_krylov(tol, tdmrg::KMAX, 0);
    eng.ensure_workspace(mm, mm, 1, 1);
    cplx *X = nullptr, *a = nullptr, *b = nullptr, *T = nullptr;
    struct Free {
      cplx** p[4];
      ~Free() {
        for (auto q : p)
          if (*q) cudaFree(*q);
      }
    } fr{{&X, &a, &b, &T}};
    CK(cudaMalloc(&X, sizeof(cplx) * (size_t)Dw * mm));
    CK(cudaMalloc(&a, sizeof(cplx) * (size_t)mm));
    CK(cudaMalloc(&b, sizeof(cplx) * (size_t)mm));
    CK(cudaMalloc(&T, sizeof(cplx) * (size_t)Dw * mm));
    tdmrg::Ctx c{s, X, nullptr};
    const cplx* Ld = (const cplx*)L;
    const cplx* Rd = (const cplx*)R;
    auto kmv = [&](const cplx* in, cplx* out, const int* skip) {
      tdmrg::bond_f64(c, M, Dw, Ld, Rd, in, out, skip);
    };
    // Cbar = exp(conj(tau) K) ybar
    eng.krylov(mm, (const cplx*)ybar, (cplx*)Cbar, tau_re, -tau_im, kmv);
    // cotangent of K: sum_s k_s a_s b_s^H with k_s = w_s conj(tau); for K C = sum_w L_w C R_w^T
    //   Lbar_w = sum_s k_s a_s conj(R_w) b_s^H,   Rbar_w = sum_s k_s a_s^T conj(L_w) conj(b_s)
    CK(cudaMemsetAsync(Lbar, 0, sizeof(cplx) * (size_t)Dw * mm, s));
    CK(cudaMemsetAsync(Rbar, 0, sizeof(cplx) * (size_t)Dw * mm, s));
    std::vector<double> sn, wn;
    tdmrg::gauss_legendre01(nodes, sn, wn);
    const cplx one = {1.0, 0.0}, zero = {0.0, 0.0};
    for (int q = 0; q < nodes; ++q) {
      eng.krylov(mm, (const cplx*)C, b, sn[q] * tau_re, sn[q] * tau_im, kmv);
      eng.krylov(mm, (const cplx*)ybar, a, (1.0 - sn[q]) * tau_re, -(1.0 - sn[q]) * tau_im, kmv);
      const cplx k = {wn[q] * tau_re, -wn[q] * tau_im};
      // T_w = conj(R_w) b^H;  Lbar_w += k a T_w
      CK(tdmrg::zgemm(M, M, M, Dw, 1, one, MatRef{Rd, M, 1, mm, 0, 1}, MatRef{b, 1, M, 0, 0, 1},
                      zero, T, M, mm, nullptr, s));
      CK(tdmrg::zgemm(M, M, M, Dw, 1, k, MatRef{a, M, 1, 0, 0, 0}, MatRef{T, M, 1, mm, 0, 0}, one,
                      (cplx*)Lbar, M, mm, nullptr, s));
      // T_w = conj(L_w) conj(b);  Rbar_w += k a^T T_w
      CK(tdmrg::zgemm(M, M, M, Dw, 1, one, MatRef{Ld, M, 1, mm, 0, 1}, MatRef{b, M, 1, 0, 0, 1},
                      zero, T, M, mm, nullptr, s));
      CK(tdmrg::zgemm(M, M, M, Dw, 1, k, MatRef{a, 1, M, 0, 0, 0}, MatRef{T, M, 1, mm, 0, 0}, one,
                      (cplx*)Rbar, M, mm, nullptr, s));
    }
    eng.sync_and_check();
  });
}

int tdmrg_kernel_qr_vjp(int m, int n, const void* Q, const void* R, const void* Qbar,
                        const void* Rbar, void* Ybar, void* stream) {
  if (m < 1 || n < 1 || m < n || !Q || !R || !Qbar || !Rbar || !Ybar)
    return fail(nullptr, TDMRG_ERR_ARG, "qr_vjp: need m >= n >= 1 and non-NULL buffers");
  return guarded(nullptr, [&] {
    using tdmrg::cplx;
    using tdmrg::MatRef;
    cudaStream_t s = (cudaStream_t)stream;
    cplx *Ru = nullptr, *M = nullptr, *S = nullptr, *rhs = nullptr;
    struct Free {
      cplx** p[4];
      ~Free() {
        for (auto q : p)
          if (*q) cudaFree(*q);
      }
    } fr{{&Ru, &M, &S, &rhs}};
    CK(cudaMalloc(&Ru, sizeof(cplx) * (size_t)n * n));
    CK(cudaMalloc(&M, sizeof(cplx) * (size_t)n * n));
    CK(cudaMalloc(&S, sizeof(cplx) * (size_t)n * n));
    CK(cudaMalloc(&rhs, sizeof(cplx) * (size_t)m * n));
    const cplx one = {1.0, 0.0}, mone = {-1.0, 0.0}, zero = {0.0, 0.0};
    // entries of Rbar below the diagonal are structural zeros of R
    CK(cudaMemcpyAsync(Ru, Rbar, sizeof(cplx) * (size_t)n * n, cudaMemcpyDeviceToDevice, s));
    CK(tdmrg::triu_inplace(n, Ru, s));
    // M = R Rbar^H - Qbar^H Q
    CK(tdmrg::zgemm(n, n, n, 1, 1, one, MatRef{(const cplx*)R, n, 1, 0, 0, 0},
                    MatRef{Ru, 1, n, 0, 0, 1}, zero, M, n, 0, nullptr, s));
    CK(tdmrg::zgemm(n, n, m, 1, 1, mone, MatRef{(const cplx*)Qbar, 1, n, 0, 0, 1},
                    MatRef{(const cplx*)Q, n, 1, 0, 0, 0}, one, M, n, 0, nullptr, s));
    CK(tdmrg::herm_lower(n, M, S, s));
    // rhs = Qbar + Q S;  Ybar R^H = rhs
    CK(cudaMemcpyAsync(rhs, Qbar, sizeof(cplx) * (size_t)m * n, cudaMemcpyDeviceToDevice, s));
    CK(tdmrg::zgemm(m, n, n, 1, 1, one, MatRef{(const cplx*)Q, n, 1, 0, 0, 0},
                    MatRef{S, n, 1, 0, 0, 0}, one, rhs, n, 0, nullptr, s));
    CK(tdmrg::solve_rh(m, n, (const cplx*)R, rhs, (cplx*)Ybar, s));
    CK(cudaStreamSynchronize(s));
  });
}

int tdmrg_kernel_env_vjp(int side, int Ml, int Mr, int d, int Dl, int Dr, const double* W_host,
                         int nparam, const double* dW_host, const void* E, const void* bra,
                         const void* ket, const void* G, void* Ebar, void* brabar, void* ketbar,
                         double* theta_bar, void* X, void* Y, void* stream) {
  if ((side != 0 && side != 1) || Ml < 1 || Mr < 1 || d < 1 || Dl < 1 || Dr < 1 || !W_host ||
      nparam < 0 || (nparam > 0 && (!dW_host || !theta_bar)) || !E || !bra || !ket || !G ||
      !Ebar || !brabar || !ketbar || !X || !Y)
    return fail(nullptr, TDMRG_ERR_ARG, "env_vjp: bad arguments");
  return guarded(nullptr, [&] {
    cudaStream_t s = (cudaStream_t)stream;
    const int D = d * d;
    const size_t site = (size_t)Dl * Dr * D;
    TempMpo W(Dl, Dr, d, W_host);
    const std::vector<double> Wt = transpose_conj_ops(W_host, Dl, Dr, d);
    TempMpo Wc(Dl, Dr, d, Wt.data());
    const int Me = side == 0 ? Ml : Mr, De = side == 0 ? Dl : Dr;   // E (environment in)
    const int Mg = side == 0 ? Mr : Ml, Dg = side == 0 ? Dr : Dl;   // G (environment out)
    const long long ne = (long long)De * Me * Me, ng = (long long)Dg * Mg * Mg;
    DevBufs buf;
    cplx* Eh = buf.get(ne);     // E^dagger per channel
    cplx* Gt = buf.get(ng);     // G^T per channel
    cplx* Gc = buf.get(ng);     // conj G
    cplx* tmp = buf.get(ng);
    cplx* part = buf.get(257);
    for (int w = 0; w < De; ++w)
      CK(tdmrg::ztranspose(Me, Me, (const cplx*)E + (size_t)w * Me * Me, Eh + (size_t)w * Me * Me,
                           1, s));
    for (int w = 0; w < Dg; ++w)
      CK(tdmrg::ztranspose(Mg, Mg, (const cplx*)G + (size_t)w * Mg * Mg, Gt + (size_t)w * Mg * Mg,
                           0, s));
    CK(cudaMemcpyAsync(Gc, G, sizeof(cplx) * (size_t)ng, cudaMemcpyDeviceToDevice, s));
    CK(tdmrg::zconj(ng, Gc, s));
    tdmrg::Ctx c{s, (cplx*)X, (cplx*)Y};
    const cplx* Ed = (const cplx*)E;
    const cplx* Bd = (const cplx*)bra;
    const cplx* Kd = (const cplx*)ket;
    if (side == 0) {
      // ketbar = H_eff(E^dagger, W^T conj, G^T) bra,  brabar = H_eff(E, W, conj G) ket,
      // Ebar = conj(env_right(conj G, bra, W, ket))
      tdmrg::heff_f64(c, Wc.m.s[0], Ml, Mr, D, d, Eh, Gt, Bd, (cplx*)ketbar, nullptr);
      tdmrg::heff_f64(c, W.m.s[0], Ml, Mr, D, d, Ed, Gc, Kd, (cplx*)brabar, nullptr);
      tdmrg::env_right_f64(c, W.m.s[0], Ml, Mr, Ml, Mr, D, d, Gc, Bd, Kd, (cplx*)Ebar);
    } else {
      // ketbar = H_eff(G^T, W^T conj, E^dagger) bra,  brabar = H_eff(conj G, W, E) ket,
      // Ebar = conj(env_left(conj G, bra, W, ket))
      tdmrg::heff_f64(c, Wc.m.s[0], Ml, Mr, D, d, Gt, Eh, Bd, (cplx*)ketbar, nullptr);
      tdmrg::heff_f64(c, W.m.s[0], Ml, Mr, D, d, Gc, Ed, Kd, (cplx*)brabar, nullptr);
      tdmrg::env_left_f64(c, W.m.s[0], Ml, Mr, Ml, Mr, D, d, Gc, Bd, Kd, (cplx*)Ebar);
    }
    CK(tdmrg::zconj(ne, (cplx*)Ebar, s));
    // theta_bar[p] = Re <G, update(E, bra, dW_p, ket)>  (the update is linear in W)
    for (int p = 0; p < nparam; ++p) {
      const double* dW = dW_host + 2 * site * p;
      if (!any_nonzero(dW, 2 * site)) {
        theta_bar[p] = 0.0;
        continue;
      }
      TempMpo dWp(Dl, Dr, d, dW);
      if (side == 0)
        tdmrg::env_left_f64(c, dWp.m.s[0], Ml, Mr, Ml, Mr, D, d, Ed, Bd, Kd, tmp);
      else
        tdmrg::env_right_f64(c, dWp.m.s[0], Ml, Mr, Ml, Mr, D, d, Ed, Bd, Kd, tmp);
      theta_bar[p] = dot_re((const cplx*)G, tmp, ng, part, s);
    }
    CK(cudaStreamSynchronize(s));
  });
}

int tdmrg_kernel_expansion_vjp(int side, int Ml, int Mr, int d, int Dl, int Dr,
                               const double* W_host, int nparam, const double* dW_host,
                               const void* E, const void* A, const void* Xbar, void* Ebar,
                               void* Abar, double* theta_bar, void* X, void* Y, void* stream) {
  if ((side != 0 && side != 1) || Ml < 1 || Mr < 1 || d < 1 || Dl < 1 || Dr < 1 || !W_host ||
      nparam < 0 || (nparam > 0 && (!dW_host || !theta_bar)) || !E || !A || !Xbar || !Ebar ||
      !Abar || !X || !Y)
    return fail(nullptr, TDMRG_ERR_ARG, "expansion_vjp: bad arguments");
  return guarded(nullptr, [&] {
    cudaStream_t s = (cudaStream_t)stream;
    const int D = d * d;
    const size_t site = (size_t)Dl * Dr * D;
    const long long per = (long long)Ml * D * Mr;
    const int Dmax = Dl > Dr ? Dl : Dr;
    const std::vector<double> Wt = transpose_conj_ops(W_host, Dl, Dr, d);
    TempMpo Wc(Dl, Dr, d, Wt.data());
    DevBufs buf;
    cplx* Pb = buf.get((long long)Dmax * per);    // Xbar in the channel-major partial layout
    cplx* Z = buf.get((long long)Dmax * per);
    cplx* tmp = buf.get((long long)Dmax * per);
    cplx* part = buf.get(257);
    tdmrg::Ctx c{s, (cplx*)X, (cplx*)Y};
    const cplx one = {1.0, 0.0}, zero = {0.0, 0.0};
    const cplx* Ed = (const cplx*)E;
    const cplx* Ad = (const cplx*)A;
    const int np = side == 0 ? Dr : Dl;           // channels of the partial contraction
    if (side == 0) {
      // Pb[v][(x,s,t)][c] = Xbar[(x,s,t)][(v,c)]
      for (int v = 0; v < Dr; ++v)
        CK(cudaMemcpy2DAsync(Pb + (size_t)v * per, sizeof(cplx) * Mr,
                             (const cplx*)Xbar + (size_t)v * Mr, sizeof(cplx) * (size_t)Dr * Mr,
                             sizeof(cplx) * Mr, (size_t)Ml * D, cudaMemcpyDeviceToDevice, s));
      // Z[w][x][u][t][c] = sum_{v,s} conj(W[w,v,s,u]) Pb[v][x][s][t][c]
      CK(tdmrg::mpo_mix(Wc.m.s[0].rl, Ml, d, Mr, Pb, per, Z, per, nullptr, s));
      // Abar[y][(u,t,c)] = sum_{w,x} conj(L[w,x,y]) Z[w][x][(u,t,c)]
      CK(tdmrg::zgemm(Ml, D * Mr, Ml, 1, Dl, one, mat(Ed, 1, Ml, 0, (long long)Ml * Ml, 1),
                      mat(Z, (long long)D * Mr, 1, 0, per), zero, (cplx*)Abar, (long long)D * Mr,
                      0, nullptr, s));
      // Lbar[w][x][y] = sum_k Z[w][x][k] conj(A[y][k])
      CK(tdmrg::zgemm(Ml, Ml, D * Mr, Dl, 1, one, mat(Z, (long long)D * Mr, 1, per),
                      mat(Ad, 1, (long long)D * Mr, 0, 0, 1), zero, (cplx*)Ebar, Ml,
                      (long long)Ml * Ml, nullptr, s));
    } else {
      // Pb[(w,y)][(s,t,b)] = conj(Xbar[(s,t,b)][(w,y)])   (X = P^H)
      CK(tdmrg::ztranspose(D * Mr, Dl * Ml, (const cplx*)Xbar, Pb, 1, s));
      // Z[v][y][u][t][b] = sum_{w,s} conj(W[w,v,s,u]) Pb[w][y][s][t][b]
      CK(tdmrg::mpo_mix(Wc.m.s[0].lr, Ml, d, Mr, Pb, per, Z, per, nullptr, s));
      // Abar[(y,u,t)][c] = sum_{v,b} Z[v][(y,u,t)][b] conj(R[v][b][c])
      CK(tdmrg::zgemm(Ml * D, Mr, Mr, 1, Dr, one, mat(Z, Mr, 1, 0, per),
                      mat(Ed, Mr, 1, 0, (long long)Mr * Mr, 1), zero, (cplx*)Abar, Mr, 0,
                      nullptr, s));
      // Rbar[v][b][c] = sum_k Z[v][k][b] conj(A[k][c])
      CK(tdmrg::zgemm(Mr, Mr, Ml * D, Dr, 1, one, mat(Z, 1, Mr, per), mat(Ad, Mr, 1, 0, 0, 1),
                      zero, (cplx*)Ebar, Mr, (long long)Mr * Mr, nullptr, s));
    }
    // theta_bar[p] = Re <Pb, partial(E, dW_p, A)>  (the candidates are linear in W)
    for (int p = 0; p < nparam; ++p) {
      const double* dW = dW_host + 2 * site * p;
      if (!any_nonzero(dW, 2 * site)) {
        theta_bar[p] = 0.0;
        continue;
      }
      TempMpo dWp(Dl, Dr, d, dW);
      if (side == 0)
        tdmrg::left_partial_f64(c, dWp.m.s[0], Ml, Ml, D, d, Mr, Ed, Ad, tmp, nullptr);
      else
        tdmrg::right_partial_f64(c, dWp.m.s[0], Ml, D, d, Mr, Mr, Ed, Ad, tmp, nullptr);
      theta_bar[p] = dot_re(Pb, tmp, (long long)np * per, part, s);
    }
    CK(cudaStreamSynchronize(s));
  });
}

int tdmrg_kernel_qr_vjp_completed(int m, int n, const int* accepted, const void* Q, const void* R,
                                  const void* Xsel, const void* Qbar, const void* Rbar,
                                  void* Ybar, void* Xselbar, void* stream) {
  if (m < 1 || n < 1 || m < n || !accepted || !Q || !R || !Qbar || !Rbar || !Ybar)
    return fail(nullptr, TDMRG_ERR_ARG, "qr_vjp_completed: need m >= n >= 1 and non-NULL buffers");
  std::vector<int> S, K;
  for (int j = 0; j < n; ++j) (accepted[j] ? S : K).push_back(j);
  const int ns = (int)S.size(), nk = (int)K.size();
  if (nk > 0 && (!Xsel || !Xselbar))
    return fail(nullptr, TDMRG_ERR_ARG, "qr_vjp_completed: completed columns need Xsel, Xselbar");
  return guarded(nullptr, [&] {
    cudaStream_t s = (cudaStream_t)stream;
    const cplx one = {1.0, 0.0}, mone = {-1.0, 0.0}, zero = {0.0, 0.0};
    const size_t cb = sizeof(cplx);
    const cudaMemcpyKind dd = cudaMemcpyDeviceToDevice;
    std::vector<int> order(S);
    order.insert(order.end(), K.begin(), K.end());
    const long long mn = (long long)m * n, nn = (long long)n * n;
    DevBufs buf;
    cplx* Qp = buf.get(mn);
    cplx* Z = buf.get(mn);
    cplx* Yr = buf.get(mn);
    cplx* Qbp = buf.get(mn);
    cplx* rhs = buf.get(mn);
    cplx* Zb = buf.get(mn);
    cplx* T = buf.get(mn);
    cplx* Rp = buf.get(nn);
    cplx* Rb = buf.get(nn);
    cplx* Mt = buf.get(nn);
    cplx* Sh = buf.get(nn);
    cplx* RS = buf.get((long long)(ns > 0 ? ns : 1) * n);
    cplx* RbS = buf.get((long long)(ns > 0 ? ns : 1) * n);
    // column scol of a row-major matrix with leading dimension sld -> column dcol of dst
    auto col = [&](cplx* dst, long long dld, int dcol, const void* src, long long sld, int scol) {
      CK(cudaMemcpy2DAsync(dst + dcol, cb * dld, (const cplx*)src + scol, cb * sld, cb, (size_t)m,
                           dd, s));
    };
    // processing order: accepted columns S, then completed columns K
    for (int i = 0; i < n; ++i) col(Qp, n, i, Q, n, order[i]);
    for (int i = 0; i < n; ++i) col(Qbp, n, i, Qbar, n, order[i]);
    CK(cudaMemcpyAsync(Rb, Rbar, cb * (size_t)nn, dd, s));
    CK(tdmrg::triu_inplace(n, Rb, s));
    for (int i = 0; i < ns; ++i) {
      CK(cudaMemcpyAsync(RS + (size_t)i * n, (const cplx*)R + (size_t)S[i] * n, cb * n, dd, s));
      CK(cudaMemcpyAsync(RbS + (size_t)i * n, Rb + (size_t)S[i] * n, cb * n, dd, s));
    }
    // the factorised matrix Y = Q_S R_S, and Z = [Y_S | Xsel]
    CK(tdmrg::zgemm(m, n, ns, 1, 1, one, mat(Qp, n, 1), mat(RS, n, 1), zero, Yr, n, 0, nullptr, s));
    for (int i = 0; i < ns; ++i) col(Z, n, i, Yr, n, S[i]);
    for (int i = 0; i < nk; ++i) col(Z, n, ns + i, Xsel, nk, i);
    // R_Z = triu(Qp^H Z) with its accepted block taken from R
    CK(tdmrg::zgemm(n, n, m, 1, 1, one, mat(Qp, 1, n, 0, 0, 1), mat(Z, n, 1), zero, Rp, n, 0,
                    nullptr, s));
    CK(tdmrg::triu_inplace(n, Rp, s));
    for (int j = 0; j < ns; ++j)
      CK(cudaMemcpy2DAsync(Rp + j, cb * n, RS + S[j], cb * n, cb, (size_t)ns, dd, s));
    // Qbar_S += Y Rbar_S^H  (the R_S = Q_S^H Y term)
    if (ns > 0)
      CK(tdmrg::zgemm(m, ns, n, 1, 1, one, mat(Yr, n, 1), mat(RbS, 1, n, 0, 0, 1), one, Qbp, n, 0,
                      nullptr, s));
    // Zbar = full-rank QR VJP of Z = Qp R_Z with Rbar_Z = 0:
    //   M = -Qbp^H Qp, S = Hermitian fold of M, Zbar R_Z^H = Qbp + Qp S
    CK(tdmrg::zgemm(n, n, m, 1, 1, mone, mat(Qbp, 1, n, 0, 0, 1), mat(Qp, n, 1), zero, Mt, n, 0,
                    nullptr, s));
    CK(tdmrg::herm_lower(n, Mt, Sh, s));
    CK(cudaMemcpyAsync(rhs, Qbp, cb * (size_t)mn, dd, s));
    CK(tdmrg::zgemm(m, n, n, 1, 1, one, mat(Qp, n, 1), mat(Sh, n, 1), one, rhs, n, 0, nullptr, s));
    CK(tdmrg::solve_rh(m, n, Rp, rhs, Zb, s));
    // Ybar = Q_S Rbar_S + Zbar_S scattered to the positions S;  Xselbar = Zbar_K
    CK(tdmrg::zgemm(m, n, ns, 1, 1, one, mat(Qp, n, 1), mat(RbS, n, 1), zero, (cplx*)Ybar, n, 0,
                    nullptr, s));
    CK(cudaMemsetAsync(T, 0, cb * (size_t)mn, s));
    for (int i = 0; i < ns; ++i) col(T, n, S[i], Zb, n, i);
    CK(tdmrg::zaxpy(mn, one, T, (cplx*)Ybar, s));
    for (int i = 0; i < nk; ++i) col((cplx*)Xselbar, nk, i, Zb, n, ns + i);
    CK(cudaStreamSynchronize(s));
  });
}

int tdmrg_kernel_krylov_dense(int n, const void* H, const void* v, void* out, double tau_re,
                              double tau_im, double tol, int kmax, int* kused, void* stream) {
  if (n < 1 || !H || !v || !out || kmax < 1 || kmax > tdmrg::KMAX || !(tol > 0.0))
    return fail(nullptr, TDMRG_ERR_ARG, "krylov_dense: bad arguments");
  return guarded(nullptr, [&] {
    // a minimal engine-free Lanczos: reuse the engine's Krylov driver on a 3-site dummy model
    tdmrg::ModelParams P;
    P.N = 3;
    Engine eng(P);
    eng.set_stream((cudaStream_t)stream);
    eng.set_krylov(tol, kmax, 0);
    eng.ensure_workspace(n, n, 1, 1);
    const tdmrg::cplx one = {1.0, 0.0}, zero = {0.0, 0.0};
    const tdmrg::cplx* Hd = (const tdmrg::cplx*)H;
    const int used = eng.krylov(n, (const tdmrg::cplx*)v, (tdmrg::cplx*)out, tau_re, tau_im,
                                [&](const tdmrg::cplx* in, tdmrg::cplx* o, const int* skip) {
                                  tdmrg::MatRef a{Hd, n, 1, 0, 0, 0}, b{in, 1, 1, 0, 0, 0};
                                  CK(tdmrg::zgemm(n, 1, n, 1, 1, one, a, b, zero, o, 1, 0, skip,
                                                  (cudaStream_t)stream));
                                });
    eng.sync_and_check();
    if (kused) *kused = used;
  });
}

}  // extern "C"
