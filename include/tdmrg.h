/*
 * tdmrg.h -- C ABI of the GB300 finite-temperature TD-DMRG library (libtdmrg.so).
 *
 * The library computes the current-current correlation function of a periodic
 * multi-mode Holstein(-Peierls) chain with one carrier and the Kubo mobility from it
 * (Li, Ren & Shuai, "Finite temperature TD-DMRG for the carrier mobility of organic
 * semiconductors"):
 *
 *   H     = V sum_n (c+_{n+1} c_n + h.c.) + sum_{n,m} w_m b+_{nm} b_{nm}
 *           + sum_{n,m} g_m w_m (b+_{nm} + b_{nm}) c+_n c_n                      (Eq. 1)
 *   j     = (V / i) sum_n (c+_{n+1} c_n - c+_n c_{n+1})            (Eq. 3, e0 = R = 1)
 *   Psi_b = exp(-beta H / 2) |I>,  |I> = sum_i |i>_P |i>_Q            (Eq. 4-5)
 *   C(t)  = <Psi_b| e^{iHt} j e^{-iHt} j |Psi_b> / Z                     (Eq. 6)
 *   mu    = 1/(2 kT) int C(t) dt                                          (Eq. 2)
 *
 * Both propagations use the one-site TDVP projector-splitting integrator on a purified
 * MPS (Eq. S1), every step of it in CUDA kernels for sm_103a.  Units: hbar = kB = e0 = R = 1.
 *
 * Conventions for every function:
 *  - return TDMRG_OK (0) on success, a negative TDMRG_ERR_* code otherwise; the message of
 *    the last failure is available from tdmrg_last_error(h) (a string owned by the handle,
 *    valid until the next call on it) or tdmrg_last_global_error() when no handle exists;
 *  - host pointers are owned by the caller and only read/written during the call;
 *  - the handle owns all device memory it allocates (cudaMalloc on the current device);
 *    tdmrg_model_destroy frees it;
 *  - all work is issued on the handle's stream (default: the legacy default stream);
 *    functions that return results to host memory synchronise that stream;
 *  - no exception crosses the ABI; a handle is not thread safe.
 */
#ifndef TDMRG_H
#define TDMRG_H

#ifdef __cplusplus
extern "C" {
#endif

#define TDMRG_OK             0
#define TDMRG_ERR_ARG       -1   /* invalid argument (sizes, grids, order of calls)      */
#define TDMRG_ERR_CUDA      -2   /* a CUDA runtime call failed                           */
#define TDMRG_ERR_OOM       -3   /* device allocation failed                             */
#define TDMRG_ERR_NONFINITE -4   /* NaN/Inf detected in a norm after a half-sweep        */
#define TDMRG_ERR_NOCONV    -5   /* a site Krylov exponential stopped at kmax with its
                                    a-posteriori error estimate above 1e3 tol (not in
                                    fixed-k mode); the step's result is kept, the handle
                                    stays usable                                          */
#define TDMRG_ERR_TIMEOUT   -6   /* a bounded device-side wait (grid barrier) gave up    */
#define TDMRG_ERR_STATE     -7   /* call out of order (e.g. correlation before prepare)  */

#define TDMRG_PREC_C128        0 /* every contraction in complex FP64                    */
#define TDMRG_PREC_C64_3XTF32  1 /* H_eff / environment contractions as complex FP32 via
                                    3xTF32 split products on the tensor cores, bond
                                    contractions (M <= 256) as complex FP32 FMA; Lanczos
                                    orthogonalisation, small exponential, QR and all norms
                                    and traces stay FP64                                   */

typedef struct tdmrg_model tdmrg_model;

/* Build the chain of Eq. 1: N >= 3 molecules on a ring, `modes` intramolecular modes per
 * molecule with frequencies omega[modes], dimensionless couplings g[modes] and nmax[modes]
 * harmonic-oscillator levels (2 <= nmax <= 32), transfer integral V.  Builds the MPOs of
 * H (bond dimension 7) and j (bond dimension 6) on the host and uploads them.
 * Site order along the MPS: e_1, v_{1,1..modes}, e_2, ... (plus p_n with a Peierls mode). */
int tdmrg_model_create(int N, int modes, const double* omega, const double* g, double V,
                       const int* nmax, tdmrg_model** out);

/* Holstein-Peierls extension (Eq. 10): one bond mode p_n (frequency omega_p, nmax_p levels)
 * per bond, modulating the transfer integral as V (1 + alpha (b_p + b_p^+)); the current
 * operator becomes j = i[H, P] (Eq. 3 with V -> V (1 + alpha x_p)).  Call before
 * tdmrg_thermal_prepare. */
int tdmrg_model_set_peierls(tdmrg_model* h, double alpha, double omega_p, int nmax_p);

/* TDMRG_PREC_C128 (default) or TDMRG_PREC_C64_3XTF32. */
int tdmrg_model_set_precision(tdmrg_model* h, int precision);

/* Krylov exponential control: stop when beta_k |(exp(tau T_k) e_1)_k| < tol (default 1e-13
 * for C128, 1e-7 for 3xTF32), at most kmax (<= 32) vectors; fixed_k > 0 forces exactly that
 * many vectors (smooth map for finite differences). */
int tdmrg_model_set_krylov(tdmrg_model* h, double tol, int kmax, int fixed_k);

/* Rank threshold of the gauge QR: a column whose Gram-Schmidt residual is <= rank_tol ||Y||_F
 * is skipped and its position completed deterministically (default 1e-12 for both
 * precisions). */
int tdmrg_model_set_rank_tol(tdmrg_model* h, double rank_tol);

/* Quadrature of the exponential VJPs in the reverse passes (tdmrg_step_vjp and the calls built
 * on it): 0 (default) evaluates exp(s tau H) v and exp((1-s) conj(tau) H) ybar by a fresh
 * Lanczos exponential at every Gauss-Legendre node; 1 builds every node vector from the two
 * Krylov bases of v and ybar (small exponentials on the host, one GEMM with each basis), which
 * keeps the Krylov tolerance and needs two Lanczos runs instead of 1 + 2 nodes. */
int tdmrg_model_set_adjoint_krylov_basis(tdmrg_model* h, int on);

/* Work stream (a cudaStream_t passed as void*; NULL = legacy default stream). */
int tdmrg_model_set_stream(tdmrg_model* h, void* stream);

/* Graph mode (needs a fixed Krylov dimension, tdmrg_model_set_krylov(h, tol, kmax, k)): each
 * state's full second-order step is captured once into a CUDA graph and replayed, so a step
 * is one graph launch (the thermal preparation and both real-time states each keep one graph).
 * If no stream was set, the handle creates its own non-blocking stream. */
int tdmrg_model_set_graphs(tdmrg_model* h, int on);

/* Batched real-time stepping of several independent instances (the (V, T, N) parameter sweep):
 * every model must have been prepared and passed tdmrg_realtime_init with a fixed Krylov
 * dimension.  tdmrg_batch_create puts each model in graph mode on its own stream (with its
 * cooperative grids capped to a quarter of the SMs so that instances run side by side; the
 * models keep their own data).  A half-step of the whole batch is ONE CUDA graph launch: the
 * graph, captured at the first use of a time step, holds every instance's half-sweeps of both
 * states as independent branches.  tdmrg_batch_realtime_step runs whole steps (two half-step
 * graphs each).  Results are those of the individual models (tdmrg_realtime_observe on each).
 * The batch does not own the models; destroy it before them. */
typedef struct tdmrg_batch tdmrg_batch;
int tdmrg_batch_create(tdmrg_model* const* models, int n, tdmrg_batch** out);
int tdmrg_batch_realtime_step(tdmrg_batch* b, int nsteps, double dt);

/* One half of the second-order projector-splitting step (Eq. S1) of both real-time states of
 * every instance: the first call runs the left-to-right half-sweeps (half a step dt/2 on every
 * site with the backward bond steps), the next call the right-to-left ones, which completes the
 * step; calls alternate.  All instances' half-step graphs are launched before any is waited
 * for.  tdmrg_batch_realtime_step returns TDMRG_ERR_STATE while a second half is pending. */
int tdmrg_batch_step_half(tdmrg_batch* b, double dt);

/* C(t) of Eq. 6 for every instance of the batch on one grid (t_grid[nt] host, ascending,
 * t_grid[0] = 0, integer multiples of dt, as tdmrg_correlation): re-forms Psi_1 = Psi_b and
 * Psi_2 = j Psi_b of every instance (each must be prepared), advances all of them together by
 * half-steps and writes C_out[n][2 nt] (host, instance-major, interleaved re, im) in the
 * order the models were given to tdmrg_batch_create. */
int tdmrg_batch_correlation(tdmrg_batch* b, const double* t_grid, int nt, double dt,
                            double* C_out);
int tdmrg_batch_destroy(tdmrg_batch* b);

/* Limit of every bounded grid-barrier wait of the handle's cooperative kernels (gauge QRs,
 * Lanczos steps, fused bond exponentials) in SM clock cycles; 0 (default) is about 2 s.  A
 * barrier that gives up sets a status word, every block of the launch leaves at its next
 * barrier, and the call returns TDMRG_ERR_TIMEOUT with the status cleared (the handle stays
 * usable; the interrupted state is not: prepare again).  Lowering the limit is how the timeout
 * path is tested without a stuck GPU. */
int tdmrg_model_set_wait_cycles(tdmrg_model* h, long long cycles);

/* Real-time propagation of the two states of Eq. 6 side by side (on by default): Psi_2 = j Psi_b
 * is stepped by a second set of workspaces on its own stream and host thread while Psi_1 is
 * stepped on the handle's stream; the cooperative grids of both are capped to half of the SMs
 * meanwhile.  Results equal the one-after-the-other order up to rounding (the capped grids sum
 * in other partitions).  Takes effect at the next tdmrg_realtime_init; not used in graph mode.
 * The second set of workspaces roughly doubles the device memory of the real-time phase. */
int tdmrg_model_set_concurrent(tdmrg_model* h, int on);

/* Phase timers: when on, the library synchronises its stream at every phase boundary and
 * accumulates host wall time per phase into the stats (slightly slower; off by default). */
int tdmrg_model_set_profiling(tdmrg_model* h, int on);

int tdmrg_model_destroy(tdmrg_model* h);

/* Imaginary-time preparation of Psi_beta (Eq. 5): |I> restricted to the one-carrier sector,
 * bond dimensions M_k = min(M, prod of local dims on either side), right-canonicalised, then
 * round(beta / (2 dtau)) symmetric projector-splitting steps of exp(-dtau H), normalised
 * after each step.  beta must be an even multiple of dtau.  Stores log Z. */
int tdmrg_thermal_prepare(tdmrg_model* h, double beta, double dtau, int M);

/* C(t) of Eq. 6 on t_grid[nt] (host, ascending, t_grid[0] = 0, every point an integer
 * multiple of dt).  Forms j|Psi_b> (MPO applied by one-site variational fitting at the
 * bond dimensions of Psi_b) and propagates both states with steps dt.  Writes C_out[2*nt]
 * (host, interleaved re, im).  Requires tdmrg_thermal_prepare. */
int tdmrg_correlation(tdmrg_model* h, const double* t_grid, int nt, double dt, double* C_out);

/* Stepping interface under tdmrg_correlation: realtime_init forms Psi_1 = Psi_b and
 * Psi_2 = j Psi_b; realtime_step advances both by nsteps steps dt; realtime_observe writes
 * the current C (C_out[2] host) and, if obs is not NULL, obs[3] = {<Psi1|Psi1>, <Psi2|Psi2>,
 * <Psi1|H|Psi1>}. */
int tdmrg_realtime_init(tdmrg_model* h);
int tdmrg_realtime_step(tdmrg_model* h, int nsteps, double dt);
int tdmrg_realtime_observe(tdmrg_model* h, double* C_out, double* obs);

/* Kubo mobility of Eq. 2 with the cut-off t_max = t_grid[nt-1]:
 * mu = (1 / (2 kT)) * 2 int_0^{t_max} Re C dt by the trapezoid rule (C(-t) = C(t)^*).
 * t_grid[nt], C[2*nt] host; pure host arithmetic, no handle needed. */
int tdmrg_mobility(const double* t_grid, const double* C, int nt, double kT, double* mu_out);

/* Hopping-limit mobility from the Fermi-golden-rule correlation function of Eq. 7 for a batch
 * of P parameter sets (the frequency-scaling isotope scan and other sweeps): for the current
 * of Eq. 3 on the ring and one carrier, to second order in V,
 *   C(t) = 2 V^2 exp{-sum_m 2 g_m^2 [(2 n_m + 1) - n_m e^{i w_m t} - (n_m + 1) e^{-i w_m t}]},
 * n_m = 1 / (e^{w_m / kT} - 1) (the printed Eq. 7 differs by these conventions: two molecules'
 * modes relax per hop, two neighbours, opposite time phase), and mu = (1 / kT) int_0^{t_max}
 * Re C dt by the trapezoid rule on t_i = i dt, i < nt (Eq. 2 cut off at t_max = (nt-1) dt).
 * omega[P K], g[P K] (row p = parameter set, K <= 64 modes), V[P], kT[P], mu_out[P]: host.
 * One GPU block per parameter set, fixed summation order.  Allocates its device copies (freed
 * before return); synchronises `stream`. */
int tdmrg_fgr_mobility_batch(int P, int K, const double* omega, const double* g,
                             const double* V, const double* kT, double dt, int nt, double* mu_out,
                             void* stream);

/* Reduced electronic density matrix of the prepared thermal state (Eq. 9): sigma = Tr_ph
 * rho_beta, rho_beta = Tr_Q |Psi_b><Psi_b| / Z, so sigma_ij = Tr[rho_beta c+_j c_i] on the
 * one-carrier sector (Tr sigma = 1).  All N^2 entries come from one left-to-right pass of
 * transfer contractions over Psi_b (right-orthonormal beyond its center, so every right
 * environment is the identity), in the model's precision.  Writes sigma_out[2 N N] (host,
 * row-major sigma_ij at 2 (i N + j), interleaved re, im).  Requires tdmrg_thermal_prepare;
 * allocates its environments (freed before return); synchronises the handle's stream. */
int tdmrg_reduced_density(tdmrg_model* h, double* sigma_out);

/* Coherence length of Eq. 9, L = (sum_ij |sigma_ij|)^2 / (N sum_ij |sigma_ij|^2): 1 for a
 * fully localised state (sigma = I / N), N for a fully delocalised one (|sigma_ij| = 1 / N).
 * sigma[2 N N] as tdmrg_reduced_density writes it (host).  Pure host arithmetic. */
int tdmrg_coherence_length(int N, const double* sigma, double* L_out);

/* Mean free path of Eq. 8 from a computed C(t): group velocity v = sqrt(<j(0) j(0)>) =
 * sqrt(Re C(0)), relaxation time tau = 1/2 int |Re C(t) / Re C(0)| dt over (-t_max, t_max) =
 * int_0^{t_max} |Re C| dt / Re C(0) (Re C is even), trapezoid rule on the grid values of |Re C|,
 * cut off at t_max = t_grid[nt-1]; l = v tau (in units of the lattice spacing R = 1).
 * t_grid[nt] (ascending, t_grid[0] = 0), C[2*nt] interleaved (host); writes vtl_out[3] =
 * {v, tau, l}.  TDMRG_ERR_ARG unless nt >= 2 and Re C(0) > 0.  Pure host arithmetic. */
int tdmrg_mean_free_path(const double* t_grid, const double* C, int nt, double* vtl_out);

/* Number of model parameters theta (omega_m, g_m, V, then alpha, omega_p with a bond mode), the
 * numbering of tdmrg_host_mpo_site and of the parameter cotangents below. */
int tdmrg_parameter_count(const tdmrg_model* h, int* count);

/* Reverse of one second-order projector-splitting step exp(tau H) (Eq. S1) in complex FP64
 * (needs TDMRG_PREC_C128; no counterpart in the paper: a building block of the adjoint).
 * The MPS has the bond dimensions tdmrg_thermal_prepare uses for M; A_in[L] are device pointers
 * to its site tensors (Ml x d*d x Mr, sites 1.. right-orthonormal, the center at site 0, as the
 * library's states are between steps).  The step is run again with its intermediates kept on
 * the device, then reversed: with Abar_out[L] (device) the cotangents of the output sites it
 * writes Abar_in[L] (device) and theta_bar[count] (host, tdmrg_parameter_count numbering) such
 * that Re sum_k <Abar_out_k, dA_out_k> = Re sum_k <Abar_in_k, dA_in_k> + sum_p theta_bar_p
 * dtheta_p, and the output sites to A_out[L] if A_out is not NULL.  The step is the one without
 * renormalisation (imaginary time included); completed gauge columns follow their coupling
 * candidates.  nodes: Gauss-Legendre nodes of the exponential VJPs (16 is rounding-accurate
 * for |tau| times the spectral spread <= 5).  Allocates its tape (freed before return);
 * synchronises the handle's stream. */
int tdmrg_step_vjp(tdmrg_model* h, int M, const void* const* A_in, double tau_re, double tau_im,
                   const void* const* Abar_out, void* const* A_out, void* const* Abar_in,
                   double* theta_bar, int nodes);

/* Real-time correlation of two given states and its reverse pass, complex FP64 (needs
 * TDMRG_PREC_C128; no counterpart in the paper: the adjoint of Eq. 6 for fixed initial
 * states).  psi1[L], psi2[L]: device site tensors as for tdmrg_step_vjp.  Both are stepped by
 * nsteps steps exp(-i dt H) and C_n = <psi1(n dt)| j |psi2(n dt)> is written to
 * C_out[2 (nsteps+1)] (host, interleaved).  For the loss Re sum_n conj(Cbar_n) C_n
 * (Cbar[2 (nsteps+1)] host) it writes the cotangents g1[L], g2[L] of the initial states (device)
 * and theta_bar[count] (host, through H and j).  The states are stored every `every` steps;
 * each stretch is recomputed from its stored state and reversed step by step as
 * tdmrg_step_vjp does (memory: nsteps / every stored pairs plus one stretch and one step's
 * tape).  Allocates its storage (freed before return); synchronises the handle's stream. */
int tdmrg_correlation_states_vjp(tdmrg_model* h, int M, const void* const* psi1,
                                 const void* const* psi2, double dt, int nsteps, int every,
                                 const double* Cbar, double* C_out, void* const* g1,
                                 void* const* g2, double* theta_bar, int nodes);

/* Gradient of the whole C(t) computation of Eq. 6 (the adjoint; no counterpart in the paper),
 * complex FP64 (needs TDMRG_PREC_C128).  Runs, as tdmrg_thermal_prepare and tdmrg_correlation
 * do, the right-canonicalised |I>, round(beta / (2 dtau)) imaginary-time steps (center
 * normalised after each), the fit of j Psi_b and nsteps real-time steps dt, writing
 * C_out[2 (nsteps+1)] (host, C_n at t = n dt) and *logz_out (if not NULL); then reverses all
 * of it for the loss Re sum_n conj(Cbar_n) C_n (Cbar[2 (nsteps+1)] host) and writes
 * theta_bar[count] = dloss/dtheta (host, tdmrg_parameter_count numbering: omega_m, g_m, V,
 * ...).  For dmu/dtheta pass the trapezoid weights of tdmrg_mobility as Cbar.  The real-time
 * states are stored every `every` steps and each stretch recomputed; the imaginary-time states
 * are all kept.  Completed gauge columns follow their coupling candidates; a rank threshold
 * above rounding (tdmrg_model_set_rank_tol, e.g. 1e-8) keeps the reverse pass conditioned
 * when bonds are wider than the state's rank.  Allocates its storage (freed before return);
 * synchronises the handle's stream. */
int tdmrg_correlation_vjp(tdmrg_model* h, double beta, double dtau, int M, double dt,
                          int nsteps, int every, const double* Cbar, double* C_out,
                          double* theta_bar, double* logz_out, int nodes);

/* One site of an MPO of the chain, dense, built on the host (no handle, no GPU): the chain of
 * tdmrg_model_create (same arguments and checks) with, when nmax_p != 0, the bond mode of
 * tdmrg_model_set_peierls (alpha, omega_p, nmax_p in [2, 32]).  which: TDMRG_MPO_H (Eq. 1 /
 * Eq. 10), TDMRG_MPO_J (Eq. 3) or TDMRG_MPO_IDENTITY.  param = -1 gives the site itself;
 * param >= 0 its derivative with respect to the parameter theta_param, numbered omega_0 ..
 * omega_{modes-1}, g_0 .. g_{modes-1}, V, then (bond mode only) alpha, omega_p.  Every block
 * is affine in each parameter on its own, so the derivative is W(theta + 1) - W(theta) exactly;
 * H = sum_k (site k replaced by its derivative) gives dH/dtheta, as the adjoint needs it.
 * dims[3] (host) receives (Dl, Dr, d); W_out (host, may be NULL to query dims) receives
 * Dl*Dr*d*d complex entries, interleaved re/im, layout [wl][wr][s][u] (row s = output level),
 * zero outside the automaton's blocks.  TDMRG_ERR_ARG on a bad argument. */
#define TDMRG_MPO_H        0
#define TDMRG_MPO_J        1
#define TDMRG_MPO_IDENTITY 2
int tdmrg_host_mpo_site(int N, int modes, const double* omega, const double* g, double V,
                        const int* nmax, double alpha, double omega_p, int nmax_p, int which,
                        int param, int site, int* dims, double* W_out);

/* Gauss-Legendre nodes s[n] (ascending) and weights w[n] on [0, 1] (1 <= n <= 64), on the host:
 * the quadrature of the exponential VJPs' Frechet integrals. */
int tdmrg_host_gauss_legendre(int n, double* s, double* w);

/* The node count the Krylov-basis quadrature of the exponential VJPs uses (host only): the
 * smallest n in [min(2, nmax), nmax] whose n-point Gauss-Legendre error bound on [0, 1],
 * (n!)^4 / ((2n + 1) ((2n)!)^3) r^(2n) e^r, is at most eps, for the Frechet integrand
 * s -> e^{sA} E e^{(1-s)A} with r = 2 |A| (its 2n-th derivative is at most r^(2n) e^r |E|);
 * nmax when no smaller count meets it.  r >= 0, 1 <= nmax <= 64, eps > 0, else TDMRG_ERR_ARG.
 * The count is written to *n_out. */
int tdmrg_host_quadrature_nodes(double r, int nmax, double eps, int* n_out);

/* exp(z_s T) e_1, s < nz, for the real symmetric tridiagonal Lanczos matrix T = tridiag(beta,
 * alpha, beta) (alpha[k] diagonal, beta[k-1] off-diagonal, 1 <= k <= 64), from one cyclic
 * Jacobi eigendecomposition of T on the host (no handle, no GPU): z[2 nz] interleaved complex,
 * out[2 k nz] interleaved, layout [s][k].  The small exponentials a reverse pass needs at many
 * points of [0, tau] from one Krylov basis. */
int tdmrg_host_tridiag_exp(int k, const double* alpha, const double* beta, int nz,
                           const double* z, double* out);

/* log Z = log Tr[exp(-beta H) P_1] accumulated by tdmrg_thermal_prepare. */
int tdmrg_get_logz(const tdmrg_model* h, double* logz);

/* Counters since the last reset: stats[0] site updates, [1] H_eff matvecs, [2] algorithmic
 * H_eff flops (8 real flops per complex multiply-add of the two dense contractions),
 * [3] Krylov vectors, [4] bond matvecs, [5] gauge QRs, [6] completions, [7] environment
 * updates, [8] event-timed milliseconds of the site H_eff matvecs, [9] host-to-device and
 * [10] device-to-host bytes copied by the library, [11] kernels launched by the library
 * (process-wide counter, relative to this handle's last reset), and with profiling on the
 * host wall seconds of [12] site exponentials, [13] gauge QRs (included in [14]),
 * [14] gauge shifts with environment updates, [15] bond back-steps, [16] bond absorption,
 * [17] C(t) overlaps; [18] event-timed milliseconds of the gauge QRs run outside graph
 * captures and [19] their algorithmic FP64 flops (one Gram-Schmidt pass, 8 m n^2 per QR of an
 * m x n matrix), [20] event-timed milliseconds of the Lanczos orthogonalisation steps of the
 * host-driven Krylov exponentials (site updates; also bond steps of the FP64 path), [21] event-timed
 * milliseconds, [22] algorithmic flops and [23] number of the gauge QRs with m >= 4096 rows.
 * n = entries wanted (<= 24). */
int tdmrg_get_stats(const tdmrg_model* h, double* stats, int n);
int tdmrg_reset_stats(tdmrg_model* h);

const char* tdmrg_last_error(const tdmrg_model* h);
const char* tdmrg_last_global_error(void);

/* ----------------------------------------------------------------------------------
 * Kernel-level entry points (device pointers, complex FP64 interleaved re/im, row-major).
 * They run one hot-path operation in isolation, for parity tests and measurement.
 * Arguments are sizes and device pointers owned by the caller; nothing is allocated
 * except where noted; each entry states whether it synchronises `stream`.
 * ---------------------------------------------------------------------------------- */

/* Effective Hamiltonian of one site (the site step of Eq. S1):
 *   out[a,s,t,b] = sum L[w,a,y] W[w,v,s,u] A[y,u,t,c] R[v,b,c]
 * L: Dl x Ml x Ml, R: Dr x Mr x Mr, A/out: Ml x (d*d) x Mr (complex FP64), W: Dl x Dr x d x d
 * (dense, host pointer, complex interleaved).  TDMRG_PREC_C128: X, Y are device workspaces of
 * max(Dl, Dr) * Ml * d*d * Mr complex entries each (ws32 unused).  TDMRG_PREC_C64_3XTF32:
 * both contractions run on the tensor cores with 3xTF32 split operands; ws32 is a device
 * workspace of tdmrg_heff_workspace_floats(...) floats (X, Y unused).  Allocates the device
 * tables of the MPO site (and, for 3xTF32, a status word), freed before return; synchronises
 * `stream`; ERR_TIMEOUT if a bounded pipeline wait gave up. */
int tdmrg_kernel_heff(int Ml, int Mr, int d, int Dl, int Dr, const double* W_host,
                      const void* L, const void* R, const void* A, void* out,
                      void* X, void* Y, void* ws32, int precision, void* stream);

/* The H_eff product of tdmrg_kernel_heff as the engine runs it in the sweep (same definition
 * and layouts), timed: the environments are prepared once, one warm-up product, then `reps`
 * products between two CUDA events on `stream`; *ms_per_matvec (host) receives the average.
 * TDMRG_PREC_C64_3XTF32 uses the engine's tensor-core path (split, L.A contraction with
 * split-K, MPO mixing into split planes, contraction with R); TDMRG_PREC_C128 the FP64 path.
 * Allocates its workspaces (freed before return); synchronises `stream`. */
int tdmrg_kernel_heff_timed(int Ml, int Mr, int d, int Dl, int Dr, const double* W_host,
                            const void* L, const void* R, const void* A, void* out, int precision,
                            int reps, double* ms_per_matvec, void* stream);

/* Vector-Jacobian product of the H_eff product of the one-site step (Eq. S1) -- the building
 * block an adjoint of the step needs (the adjoint itself has no counterpart in the paper).
 * For y = H_eff(L, W, R) A and a cotangent ybar (real loss l with dl = Re<ybar, dy>):
 *   Abar = H_eff(L^dagger, W^T conj, R^dagger) ybar      (per-channel Hermitian conjugates),
 *   Lbar[w,x,y] = sum ybar[x,s,t,b] conj(W[w,v,s,u] A[y,u,t,c] R[v,b,c])
 *               = conj(right environment update with bra = ybar, ket = A),
 *   Rbar[v,b,c] = sum ybar[x,s,t,b] conj(L[w,x,y] W[w,v,s,u] A[y,u,t,c])
 *               = conj(left environment update with bra = ybar, ket = A),
 * so that dl = Re<Abar, dA> + Re<Lbar, dL> + Re<Rbar, dR>.  Layouts as tdmrg_kernel_heff
 * (FP64 complex, device): A, ybar, Abar Ml x d*d x Mr; L, Lbar Dl x Ml x Ml; R, Rbar
 * Dr x Mr x Mr; W_host on the host.  X, Y: workspaces of max(Dl,Dr) * Ml * d*d * Mr complex
 * entries.  Allocates two environment-sized temporaries (freed before return); synchronises
 * `stream`. */
int tdmrg_kernel_heff_vjp(int Ml, int Mr, int d, int Dl, int Dr, const double* W_host,
                          const void* L, const void* R, const void* A, const void* ybar,
                          void* Abar, void* Lbar, void* Rbar, void* X, void* Y, void* stream);

/* Vector-Jacobian product of the site exponential of the one-site step (Eq. S1),
 * y = exp(tau H_eff(L, W, R)) A with H_eff Hermitian (environments of a Hermitian MPO) -- a
 * building block of an adjoint of the step (the adjoint has no counterpart in the paper).
 * For a cotangent ybar (dl = Re<ybar, dy>):
 *   Abar = exp(conj(tau) H_eff) ybar,
 *   Lbar, Rbar from Hbar = conj(tau) int_0^1 a(s) b(s)^H ds, a(s) = exp((1-s) conj(tau) H) ybar,
 *   b(s) = exp(s tau H) A, mapped onto L and R like tdmrg_kernel_heff_vjp's Lbar and Rbar
 *   (conjugated environment updates with a(s) as bra and b(s) as ket),
 * with the integral taken by Gauss-Legendre quadrature on `nodes` (1..64) points and every
 * exponential by the FP64 Lanczos of the sweep at tolerance `tol`.  Layouts as
 * tdmrg_kernel_heff_vjp.  Allocates its scratch (freed before return); synchronises `stream`;
 * TDMRG_ERR_TIMEOUT if a bounded grid barrier gave up. */
int tdmrg_kernel_site_exp_vjp(int Ml, int Mr, int d, int Dl, int Dr, const double* W_host,
                              const void* L, const void* R, const void* A, const void* ybar,
                              double tau_re, double tau_im, int nodes, double tol, void* Abar,
                              void* Lbar, void* Rbar, void* stream);

/* tdmrg_kernel_site_exp_vjp plus parameter cotangents: for nparam derivative sites
 * dW_host[nparam][Dl][Dr][d][d] (host, as tdmrg_host_mpo_site writes them) it also writes
 * theta_bar[p] = Re<Hbar, H_eff(L, dW_p, R)> (host), Hbar the cotangent of the operator from the
 * same quadrature; nparam = 0 is tdmrg_kernel_site_exp_vjp.  Allocates its scratch (freed
 * before return); synchronises `stream`. */
int tdmrg_kernel_site_exp_vjp_theta(int Ml, int Mr, int d, int Dl, int Dr, const double* W_host,
                                    const void* L, const void* R, const void* A,
                                    const void* ybar, double tau_re, double tau_im, int nodes,
                                    double tol, int nparam, const double* dW_host, void* Abar,
                                    void* Lbar, void* Rbar, double* theta_bar, void* stream);

/* Vector-Jacobian product of the bond exponential of the projector-splitting step (Eq. S1,
 * zero-site term), y = exp(tau K) C with (K C)[a][b] = sum_w sum L[w][a][a'] C[a'][b']
 * R[w][b][b'] Hermitian -- a building block of an adjoint of the step (no counterpart in the
 * paper).  For a cotangent ybar: Cbar = exp(conj(tau) K) ybar; with the cotangent of K,
 * conj(tau) int_0^1 a(s) b(s)^H ds (a(s) = exp((1-s) conj(tau) K) ybar, b(s) = exp(s tau K) C,
 * Gauss-Legendre on `nodes` points, FP64 Lanczos at tolerance `tol`):
 *   Lbar_w = sum_s k_s a_s conj(R_w) b_s^H,   Rbar_w = sum_s k_s a_s^T conj(L_w) conj(b_s).
 * L, R, Lbar, Rbar Dw x M x M; C, ybar, Cbar M x M (complex FP64, row-major, device).
 * Allocates its scratch (freed before return); synchronises `stream`. */
int tdmrg_kernel_bond_exp_vjp(int M, int Dw, const void* L, const void* R, const void* C,
                              const void* ybar, double tau_re, double tau_im, int nodes,
                              double tol, void* Cbar, void* Lbar, void* Rbar, void* stream);

/* Vector-Jacobian product of the gauge QR Y = Q R at full column rank, diag(R) real
 * and positive (no completed columns) -- a building block of an adjoint of the step (no
 * counterpart in the paper).  With M = R Rbar^H - Qbar^H Q and S the Hermitian matrix made
 * of the strictly lower triangle of M, its conjugate mirror and Re(M_ii) on the diagonal:
 *   Ybar = (Qbar + Q S) R^{-H},
 * so that dl = Re<Qbar, dQ> + Re<Rbar, dR> = Re<Ybar, dY>.  Q, Qbar, Ybar m x n, R, Rbar
 * n x n (complex FP64, row-major, device; entries of Rbar below the diagonal are ignored).
 * Allocates its scratch (freed before return); synchronises `stream`. */
int tdmrg_kernel_qr_vjp(int m, int n, const void* Q, const void* R, const void* Qbar,
                        const void* Rbar, void* Ybar, void* stream);

/* Vector-Jacobian product of an environment update of the sweep (Eq. S1) -- a building block of
 * an adjoint of the step (no counterpart in the paper).  side 0 (left):
 *   E'[v,b,c] = sum conj(bra[a,s,t,b]) E[w,a,y] W[w,v,s,u] ket[y,u,t,c],
 * E Dl x Ml x Ml, G (the cotangent of E') Dr x Mr x Mr; side 1 (right):
 *   E'[w,a,y] = sum conj(bra[a,s,t,b]) E[v,b,c] W[w,v,s,u] ket[y,u,t,c],
 * E Dr x Mr x Mr, G Dl x Ml x Ml.  bra, ket, brabar, ketbar are Ml x d*d x Mr; W_host is the
 * dense MPO site [Dl][Dr][d][d] (complex interleaved, host).  Writes Ebar (shape of E), brabar,
 * ketbar (device) with Re<G, dE'> = Re<Ebar, dE> + Re<brabar, dbra> + Re<ketbar, dket>; they are
 * forward contractions with transformed operands (side 0: ketbar = H_eff(E^dagger, W^T conj,
 * G^T) bra, brabar = H_eff(E, W, conj G) ket, Ebar = conj(env_right(conj G, bra, W, ket)); side
 * 1 mirrored).  For nparam derivative sites dW_host[nparam][Dl][Dr][d][d] (host, as
 * tdmrg_host_mpo_site writes them) it writes theta_bar[p] = Re<G, E'(W -> dW_p)> (host).
 * X, Y: device workspaces of max(Dl, Dr) * Ml * d*d * Mr complex entries each.  Complex FP64,
 * row-major, device unless stated; allocates its scratch (freed before return); synchronises
 * `stream`. */
int tdmrg_kernel_env_vjp(int side, int Ml, int Mr, int d, int Dl, int Dr, const double* W_host,
                         int nparam, const double* dW_host, const void* E, const void* bra,
                         const void* ket, const void* G, void* Ebar, void* brabar, void* ketbar,
                         double* theta_bar, void* X, void* Y, void* stream);

/* Vector-Jacobian product of the completion candidates of the gauge QR (what H_eff couples a
 * site into, Eq. S1's projector directions).  side 0 (left-to-right shift):
 *   X[(x,s,t), (v,c)] = sum L[w,x,y] W[w,v,s,u] A[y,u,t,c],   Ml d^2 rows, Dr Mr columns,
 * E = L (Dl x Ml x Ml); side 1 (right-to-left shift): X = P^H with
 *   P[(w,y), (s,t,b)] = sum W[w,v,s,u] A[y,u,t,c] R[v,b,c],   d^2 Mr rows, Dl Ml columns,
 * E = R (Dr x Mr x Mr).  Xbar (device, rows x columns, row-major) -> Ebar (shape of E) and Abar
 * (Ml x d*d x Mr) with Re<Xbar, dX> = Re<Ebar, dE> + Re<Abar, dA>, and theta_bar[p] =
 * Re<Xbar, X(W -> dW_p)> for nparam derivative sites as in tdmrg_kernel_env_vjp.  X, Y as
 * there.  Complex FP64; allocates its scratch (freed before return); synchronises `stream`. */
int tdmrg_kernel_expansion_vjp(int side, int Ml, int Mr, int d, int Dl, int Dr,
                               const double* W_host, int nparam, const double* dW_host,
                               const void* E, const void* A, const void* Xbar, void* Ebar,
                               void* Abar, double* theta_bar, void* X, void* Y, void* stream);

/* Vector-Jacobian product of the gauge QR with completed columns (no counterpart in the paper).
 * accepted[n] (host): 1 for a column that Gram-Schmidt took from Y (positions S), 0 for a
 * completed one (positions K, R's row zero there).  The completed columns are residuals of the
 * vectors Xsel (device, m x |K|, in increasing position order) against everything taken before
 * them, so in the order (S, K) the factorisation is the full-rank QR of Z = [Y_S | Xsel] with
 * R_Z = triu(Q^H Z), and R_S = Q_S^H Y.  With Qbar (m x n) and Rbar (n x n, rows K and entries
 * below the diagonal ignored) it writes
 *   Zbar = full-rank QR VJP of Z for Qbar (Qbar_S + Y Rbar_S^H on the columns S), Rbar_Z = 0,
 *   Ybar = Q_S Rbar_S + Zbar_S (scattered to S),   Xselbar = Zbar_K   (device),
 * so that Re<Qbar, dQ> + Re<Rbar_S, dR_S> = Re<Ybar, dY> + Re<Xselbar, dXsel>.  Without
 * completed columns it equals tdmrg_kernel_qr_vjp (Xsel, Xselbar may then be NULL).  Q, R as
 * the gauge QR wrote them; complex FP64, row-major; allocates its scratch (freed before
 * return); synchronises `stream`. */
int tdmrg_kernel_qr_vjp_completed(int m, int n, const int* accepted, const void* Q, const void* R,
                                  const void* Xsel, const void* Qbar, const void* Rbar,
                                  void* Ybar, void* Xselbar, void* stream);

/* Size in floats of the 3xTF32 workspace of tdmrg_kernel_heff (-1 for invalid sizes). */
long long tdmrg_heff_workspace_floats(int Ml, int Mr, int d, int Dl, int Dr);

/* One tensor-core complex contraction C[m][n] = sum_k opA(A[m][k]) opB(B[n][k]) with opX =
 * conjugation when conjX, A: M x K, B: N x K, C: M x N (complex FP64, row-major, device).
 * The operands are split into 3xTF32 planes (allocated and freed inside, with the split-K
 * scratch used when the output has few tiles and K is long); synchronises. */
int tdmrg_kernel_zgemm_tc(int M, int N, int K, const void* A, const void* B, int conjA, int conjB,
                          void* C, void* stream);

/* Left environment update (the gauge shift of Eq. S1 carries it along the sweep):
 *   Lout[v,b,c] = sum conj(bra[a,s,t,b]) L[w,a,y] W[w,v,s,u] ket[y,u,t,c]
 * bra: Ml1 x d*d x Mr1, ket: Ml2 x d*d x Mr2, L: Dl x Ml1 x Ml2, Lout: Dr x Mr1 x Mr2.
 * X, Y: workspace of max(Dl,Dr) * Ml2 * d*d * Mr2 complex entries.  Allocates the device
 * tables of the MPO site (freed before return); synchronises `stream`. */
int tdmrg_kernel_env_left(int Ml1, int Mr1, int Ml2, int Mr2, int d, int Dl, int Dr,
                          const double* W_host, const void* L, const void* bra,
                          const void* ket, void* Lout, void* X, void* Y, void* stream);

/* Gauge QR of the shifts of Eq. S1: Y (m x n row-major, m >= n) = Q R with a deterministic
 * completion: accepted columns are Gram-Schmidt residuals (twice) above
 * 1e-12 ||Y||_F; skipped positions are filled from the columns of E (m x p row-major, may
 * be NULL with p = 0) then unit vectors, each taken when its residual exceeds 1e-2 of its
 * norm.  Q (m x n) and R (n x n) row-major outputs; R rows of completed positions are 0.
 * status (device int, may be NULL): set to 1 if the bounded grid barrier timed out, 2 if the
 * completion ran out of vectors; either way the call returns TDMRG_ERR_TIMEOUT (1) or
 * TDMRG_ERR_CUDA (2).  Each block stages ceil(m / blocks) rows in at most 200 KB of shared
 * memory (blocks = one per SM): about 12,500 rows per block, m ~ 1.9 million on 152 SMs;
 * larger m returns TDMRG_ERR_CUDA.  Allocates its scratch (freed before return);
 * synchronises `stream`. */
int tdmrg_kernel_gauge_qr(int m, int n, const void* Y, int p, const void* E, void* Q,
                          void* R, int* status, void* stream);

/* Blocked gauge QR (the factorisation the engine uses): same definition, arguments, outputs
 * and status handling as tdmrg_kernel_gauge_qr, computed 16 columns at a time (block
 * Gram-Schmidt projections, Gram-form factorisation inside the block with a cancellation
 * guard that restarts the block at any column whose residual lost more than half its norm).
 * Each block stages ceil(m / blocks) rows of 16 columns and 16 n projection coefficients in at
 * most 200 KB of shared memory; a factor that does not fit (e.g. 24576 x 640 on 152 SMs) is
 * factorised by the column-wise kernel of tdmrg_kernel_gauge_qr instead (same result).
 * Allocates and frees its scratch; synchronises `stream`. */
int tdmrg_kernel_gauge_qr_blocked(int m, int n, const void* Y, int p, const void* E, void* Q,
                                  void* R, int* status, void* stream);

/* Gauge QR that allocates nothing.  The paper has no counterpart: this entry point exists for
 * callers that cannot allocate device memory -- programs that hand all device memory to
 * another runtime or pool and may not allocate behind its back, and callers that must not fail
 * for lack of memory (or wait on the synchronisation an allocation can bring) once set up.
 * Same arguments, same result, same layouts and same status handling as tdmrg_kernel_gauge_qr;
 * Y, E, Q, R (and status, if not NULL) are the caller's.  The scratch (cross-block partial
 * sums, barrier counters, status word) is one fixed file-scope device array of about 1.6 MB
 * that every GPU loading the library keeps until exit.
 * Limits: n <= 256, a grid of <= 192 blocks, and m small enough that one block's slice of
 * ceil(m / blocks) rows fits 200 KB of shared memory (about 12,500 rows per block, m ~ 1.9
 * million on 152 SMs); larger sizes return TDMRG_ERR_ARG with a message naming the limit.
 * The first call on each device looks up the array's device address (cudaGetSymbolAddress,
 * with that device current).  All calls share the array and it keeps the last call's contents
 * (the barrier counters and the status word are cleared at the start of every call), so calls
 * that overlap on the GPU race: issue them on one stream or synchronise between them.
 * Synchronises `stream` and reads the status word; TDMRG_ERR_TIMEOUT if the bounded grid
 * barrier gave up, TDMRG_ERR_CUDA if the completion ran out of vectors. */
int tdmrg_kernel_gauge_qr_noalloc(int m, int n, const void* Y, int p, const void* E, void* Q,
                                  void* R, int* status, void* stream);

/* Bond exponential of the projector-splitting step (Eq. S1, the zero-site term):
 * out = exp(tau K) C with (K C)[a][b] = sum_w sum_{a',b'} L[w][a][a'] C[a'][b'] R[w][b][b'],
 * tau = tau_re + i tau_im.  L and R are Dw x M x M left/right environments (device, complex
 * FP64 interleaved, row-major), C and out M x M (device; out may not alias C).  K must be
 * Hermitian (as it is for environments of a Hermitian MPO).  The whole Lanczos run is one
 * cooperative launch: contractions in complex FP32 (the mixed-precision path's bond step),
 * orthogonalisation (two classical Gram-Schmidt passes), small exponential and norms in FP64;
 * stop when beta_{k+1} |c_k| < tol or at kmax (<= 32) vectors.  kused (host, may be NULL)
 * receives the number of Krylov vectors.  Allocates its scratch (freed before return);
 * synchronises `stream`; TDMRG_ERR_TIMEOUT if the bounded grid barrier gave up;
 * TDMRG_ERR_ARG unless 1 <= M <= 256 (the whole contraction depth is staged in shared
 * memory). */
int tdmrg_kernel_bond_exp(int M, int Dw, const void* L, const void* R, const void* C, void* out,
                          double tau_re, double tau_im, double tol, int kmax, int* kused,
                          void* stream);

/* FP64 FMA throughput probe (measurement only; no counterpart in the paper): blocks x 256
 * threads each run 8 independent chains of `iters` fused multiply-adds and write their sum to
 * sink[blocks * 256] (device).  *flops_out (host, may be NULL) receives the flop count
 * 2 * 8 * 256 * blocks * iters.  Asynchronous on `stream` (time it with events there): the
 * measured FP64 rate that the FP64 kernels' roofline fractions are quoted beside. */
int tdmrg_kernel_dfma_loop(int blocks, long long iters, double* sink, double* flops_out,
                           void* stream);

/* Tile tuning of the tensor-core contractions (no counterpart in the paper).  Every
 * contraction of the mixed-precision path is one tcgen05 GEMM of shape (M, N, K) summed over
 * nred operand pairs for nbatch outputs, computed in 128-row tiles of 64 or 128 columns; its K
 * loop may be split over CTAs.  The split and the tile width of each shape are read from
 * tc_splitk_table.txt beside libtdmrg.so (or the file named by the environment variable
 * TDMRG_SPLITK_TABLE), lines "M N K nred nbatch ksplit [tile_n]" (tile_n 64 when absent);
 * shapes not listed use 64-column tiles and an occupancy rule.  The table is written by
 * paper_2003_13245_gb300/tune_splitk.py, which records a workload's shapes and times every
 * candidate split and tile width:
 *   tdmrg_tune_record_shapes(1) starts recording the shapes tc_gemm sees (0 stops);
 *   tdmrg_tune_recorded_shapes writes up to `capacity` shapes as 5 ints each to shapes[] and
 *     their number to *count (host);
 *   tdmrg_tune_reload_table makes the next contraction read the table file again;
 *   tdmrg_tune_table_lookup writes the table's split and tile width for one shape to *ksplit
 *     and *tile_n (host only, no CUDA call; both 0 when the shape is not listed; a line with
 *     a width other than 64 or 128, or a split below 1, is ignored);
 *   tdmrg_kernel_tc_gemm_timed runs one shape with split ksplit and tile width tile_n (64 or
 *     128; 0 for either: the table / rule) on synthetic operands, one warm-up then `reps`
 *     launches between CUDA events on `stream`, and writes the average milliseconds to
 *     *ms_out (allocates and frees its operands); TDMRG_ERR_ARG for another tile_n. */
int tdmrg_tune_record_shapes(int on);
int tdmrg_tune_recorded_shapes(int* shapes, int capacity, int* count);
int tdmrg_tune_reload_table(void);
int tdmrg_tune_table_lookup(int M, int N, int K, int nred, int nbatch, int* ksplit, int* tile_n);
int tdmrg_kernel_tc_gemm_timed(int M, int N, int K, int nred, int nbatch, int ksplit, int tile_n,
                               int reps, double* ms_out, void* stream);

/* Krylov exponential of a dense Hermitian matrix H (n x n, device) -- the site and bond
 * exponentials of Eq. S1 on an explicit matrix:
 * out = exp(tau H) v with tau = tau_re + i tau_im, Lanczos with full re-orthogonalisation
 * in FP64 and the small exponential on the device.  kused (host, may be NULL) receives
 * the number of Krylov vectors.  Allocates its own workspace (freed before return);
 * synchronises `stream`. */
int tdmrg_kernel_krylov_dense(int n, const void* H, const void* v, void* out, double tau_re,
                              double tau_im, double tol, int kmax, int* kused, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* TDMRG_H */
