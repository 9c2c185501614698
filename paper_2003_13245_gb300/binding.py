"""ctypes binding of libtdmrg.so (argument marshalling only).

Every function of ``include/tdmrg.h`` is exposed under the same name; ``Model`` wraps the
handle.  There is no fallback: if the library is missing or cannot be loaded, importing the
binding raises, and every failing call raises ``TdmrgError`` with the library's message.
"""
import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libtdmrg.so")

PREC_C128 = 0
PREC_C64_3XTF32 = 1

ERRORS = {0: "OK", -1: "ERR_ARG", -2: "ERR_CUDA", -3: "ERR_OOM", -4: "ERR_NONFINITE",
          -5: "ERR_NOCONV", -6: "ERR_TIMEOUT", -7: "ERR_STATE"}


class TdmrgError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s (%d): %s" % (ERRORS.get(code, "?"), code, msg))
        self.code = code


_lib = None

_d = ctypes.c_double
_i = ctypes.c_int
_p = ctypes.c_void_p
_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)
_pp = ctypes.POINTER(ctypes.c_void_p)

_SIGS = {
    "tdmrg_model_create": [_i, _i, _dp, _dp, _d, _ip, ctypes.POINTER(_p)],
    "tdmrg_model_set_peierls": [_p, _d, _d, _i],
    "tdmrg_model_set_precision": [_p, _i],
    "tdmrg_model_set_krylov": [_p, _d, _i, _i],
    "tdmrg_model_set_stream": [_p, _p],
    "tdmrg_model_destroy": [_p],
    "tdmrg_model_set_profiling": [_p, _i],
    "tdmrg_model_set_wait_cycles": [_p, ctypes.c_longlong],
    "tdmrg_model_set_concurrent": [_p, _i],
    "tdmrg_kernel_heff_timed": [_i, _i, _i, _i, _i, _dp, _p, _p, _p, _p, _i, _i, _dp, _p],
    "tdmrg_model_set_graphs": [_p, _i],
    "tdmrg_model_set_rank_tol": [_p, _d],
    "tdmrg_batch_create": [ctypes.POINTER(_p), _i, ctypes.POINTER(_p)],
    "tdmrg_batch_realtime_step": [_p, _i, _d],
    "tdmrg_batch_step_half": [_p, _d],
    "tdmrg_batch_correlation": [_p, _dp, _i, _d, _dp],
    "tdmrg_batch_destroy": [_p],
    "tdmrg_mean_free_path": [_dp, _dp, _i, _dp],
    "tdmrg_reduced_density": [_p, _dp],
    "tdmrg_kernel_dfma_loop": [_i, ctypes.c_longlong, _p, _dp, _p],
    "tdmrg_tune_record_shapes": [_i],
    "tdmrg_tune_recorded_shapes": [_ip, _i, _ip],
    "tdmrg_tune_reload_table": [],
    "tdmrg_tune_table_lookup": [_i, _i, _i, _i, _i, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)],
    "tdmrg_kernel_tc_gemm_timed": [_i, _i, _i, _i, _i, _i, _i, _i, _dp, _p],
    "tdmrg_fgr_mobility_batch": [_i, _i, _dp, _dp, _dp, _dp, _d, _i, _dp, _p],
    "tdmrg_coherence_length": [_i, _dp, _dp],
    "tdmrg_thermal_prepare": [_p, _d, _d, _i],
    "tdmrg_correlation": [_p, _dp, _i, _d, _dp],
    "tdmrg_realtime_init": [_p],
    "tdmrg_realtime_step": [_p, _i, _d],
    "tdmrg_realtime_observe": [_p, _dp, _dp],
    "tdmrg_mobility": [_dp, _dp, _i, _d, _dp],
    "tdmrg_get_logz": [_p, _dp],
    "tdmrg_get_stats": [_p, _dp, _i],
    "tdmrg_reset_stats": [_p],
    "tdmrg_kernel_heff": [_i, _i, _i, _i, _i, _dp, _p, _p, _p, _p, _p, _p, _p, _i, _p],
    "tdmrg_kernel_env_left": [_i, _i, _i, _i, _i, _i, _i, _dp, _p, _p, _p, _p, _p, _p, _p],
    "tdmrg_kernel_gauge_qr": [_i, _i, _p, _i, _p, _p, _p, _p, _p],
    "tdmrg_kernel_krylov_dense": [_i, _p, _p, _p, _d, _d, _d, _i, _ip, _p],
    "tdmrg_kernel_bond_exp": [_i, _i, _p, _p, _p, _p, _d, _d, _d, _i, _ip, _p],
    "tdmrg_kernel_heff_vjp": [_i, _i, _i, _i, _i, _dp, _p, _p, _p, _p, _p, _p, _p, _p, _p, _p],
    "tdmrg_kernel_qr_vjp": [_i, _i, _p, _p, _p, _p, _p, _p],
    "tdmrg_kernel_bond_exp_vjp": [_i, _i, _p, _p, _p, _p, _d, _d, _i, _d, _p, _p, _p, _p],
    "tdmrg_kernel_site_exp_vjp": [_i, _i, _i, _i, _i, _dp, _p, _p, _p, _p, _d, _d, _i, _d, _p, _p,
                                  _p, _p],
    "tdmrg_kernel_zgemm_tc": [_i, _i, _i, _p, _p, _i, _i, _p, _p],
    "tdmrg_kernel_gauge_qr_noalloc": [_i, _i, _p, _i, _p, _p, _p, _p, _p],
    "tdmrg_kernel_gauge_qr_blocked": [_i, _i, _p, _i, _p, _p, _p, _p, _p],
    "tdmrg_host_mpo_site": [_i, _i, _dp, _dp, _d, _ip, _d, _d, _i, _i, _i, _i, _ip, _dp],
    "tdmrg_kernel_env_vjp": [_i, _i, _i, _i, _i, _i, _dp, _i, _dp, _p, _p, _p, _p, _p, _p, _p,
                             _dp, _p, _p, _p],
    "tdmrg_kernel_expansion_vjp": [_i, _i, _i, _i, _i, _i, _dp, _i, _dp, _p, _p, _p, _p, _p, _dp,
                                   _p, _p, _p],
    "tdmrg_kernel_qr_vjp_completed": [_i, _i, _ip, _p, _p, _p, _p, _p, _p, _p, _p],
    "tdmrg_kernel_site_exp_vjp_theta": [_i, _i, _i, _i, _i, _dp, _p, _p, _p, _p, _d, _d, _i, _d,
                                        _i, _dp, _p, _p, _p, _dp, _p],
    "tdmrg_parameter_count": [_p, _ip],
    "tdmrg_step_vjp": [_p, _i, _pp, _d, _d, _pp, _pp, _pp, _dp, _i],
    "tdmrg_correlation_states_vjp": [_p, _i, _pp, _pp, _d, _i, _i, _dp, _dp, _pp, _pp, _dp, _i],
    "tdmrg_correlation_vjp": [_p, _d, _d, _i, _d, _i, _i, _dp, _dp, _dp, _dp, _i],
    "tdmrg_host_tridiag_exp": [_i, _dp, _dp, _i, _dp, _dp],
    "tdmrg_model_set_adjoint_krylov_basis": [_p, _i],
    "tdmrg_host_gauss_legendre": [_i, _dp, _dp],
    "tdmrg_host_quadrature_nodes": [_d, _i, _d, ctypes.POINTER(ctypes.c_int)],
}


def load(path: str = LIB_PATH):
    """Load libtdmrg.so (raises OSError if it is missing: build it first)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise OSError("libtdmrg.so not found at %s; run __graft_entry__.build()" % path)
    lib = ctypes.CDLL(path)
    for name, args in _SIGS.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    lib.tdmrg_heff_workspace_floats.argtypes = [_i, _i, _i, _i, _i]
    lib.tdmrg_heff_workspace_floats.restype = ctypes.c_longlong
    lib.tdmrg_last_error.argtypes = [_p]
    lib.tdmrg_last_error.restype = ctypes.c_char_p
    lib.tdmrg_last_global_error.argtypes = []
    lib.tdmrg_last_global_error.restype = ctypes.c_char_p
    _lib = lib
    return lib


def declared_symbols(header: str) -> list:
    """Names of the functions declared in include/tdmrg.h."""
    import re
    text = open(header).read()
    return sorted(set(re.findall(r"\b(tdmrg_[a-z0-9_]+)\s*\(", text)))


def _check(rc, handle=None):
    if rc != 0:
        lib = load()
        msg = lib.tdmrg_last_error(handle) if handle else lib.tdmrg_last_global_error()
        raise TdmrgError(rc, (msg or b"").decode())


def _dptr(a):
    return a.ctypes.data_as(_dp)


def _stream_ptr(stream):
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


class Model:
    """One chain (Eq. 1 / Eq. 10) and its TD-DMRG state, living on the current CUDA device."""

    def __init__(self, N, omega, g, nmax, V, peierls=None, precision=PREC_C128, krylov=None,
                 stream=None):
        lib = load()
        om = np.ascontiguousarray(omega, dtype=np.float64)
        gg = np.ascontiguousarray(g, dtype=np.float64)
        nm = np.ascontiguousarray(nmax, dtype=np.int32)
        h = ctypes.c_void_p()
        _check(lib.tdmrg_model_create(int(N), int(om.size), _dptr(om), _dptr(gg), float(V),
                                      nm.ctypes.data_as(_ip), ctypes.byref(h)))
        self._h = h
        self._lib = lib
        self.N = int(N)
        if peierls is not None:
            alpha, omega_p, nmax_p = peierls
            _check(lib.tdmrg_model_set_peierls(h, float(alpha), float(omega_p), int(nmax_p)), h)
        if precision != PREC_C128:
            _check(lib.tdmrg_model_set_precision(h, int(precision)), h)
        if krylov is not None:
            tol, kmax, fixed = krylov
            _check(lib.tdmrg_model_set_krylov(h, float(tol), int(kmax), int(fixed)), h)
        if stream is not None:
            _check(lib.tdmrg_model_set_stream(h, _stream_ptr(stream)), h)

    def close(self):
        if getattr(self, "_h", None):
            self._lib.tdmrg_model_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def thermal_prepare(self, beta, dtau, M):
        _check(self._lib.tdmrg_thermal_prepare(self._h, float(beta), float(dtau), int(M)), self._h)

    def correlation(self, t_grid, dt):
        t = np.ascontiguousarray(t_grid, dtype=np.float64)
        out = np.zeros(2 * t.size)
        _check(self._lib.tdmrg_correlation(self._h, _dptr(t), int(t.size), float(dt), _dptr(out)),
               self._h)
        return out[0::2] + 1j * out[1::2]

    def realtime_init(self):
        _check(self._lib.tdmrg_realtime_init(self._h), self._h)

    def realtime_step(self, nsteps, dt):
        _check(self._lib.tdmrg_realtime_step(self._h, int(nsteps), float(dt)), self._h)

    def realtime_observe(self, with_obs=False):
        c = np.zeros(2)
        obs = np.zeros(3)
        _check(self._lib.tdmrg_realtime_observe(self._h, _dptr(c),
                                                _dptr(obs) if with_obs else None), self._h)
        return (complex(c[0], c[1]), obs) if with_obs else complex(c[0], c[1])

    def logz(self):
        v = ctypes.c_double()
        _check(self._lib.tdmrg_get_logz(self._h, ctypes.byref(v)), self._h)
        return v.value

    def reduced_density(self):
        """sigma = Tr_ph rho_beta (Eq. 9) of the prepared state: complex N x N, sigma_ij =
        <c+_j c_i>."""
        N = self.N
        out = np.zeros(2 * N * N)
        _check(self._lib.tdmrg_reduced_density(self._h, _dptr(out)), self._h)
        return (out[0::2] + 1j * out[1::2]).reshape(N, N)

    def stats(self):
        s = np.zeros(24)
        _check(self._lib.tdmrg_get_stats(self._h, _dptr(s), 24), self._h)
        keys = ["site_updates", "matvecs", "heff_flops", "krylov_vectors", "bond_matvecs", "qrs",
                "completions", "env_updates", "heff_ms", "h2d_bytes", "d2h_bytes", "launches",
                "t_site", "t_qr", "t_env", "t_bond", "t_absorb", "t_observe", "qr_ms",
                "qr_flops", "lz_ms", "qr_bulk_ms", "qr_bulk_flops", "qr_bulk_n"]
        return dict(zip(keys, s.tolist()))

    def set_rank_tol(self, tol):
        _check(self._lib.tdmrg_model_set_rank_tol(self._h, float(tol)), self._h)

    def set_graphs(self, on=True):
        _check(self._lib.tdmrg_model_set_graphs(self._h, int(bool(on))), self._h)

    def set_profiling(self, on=True):
        _check(self._lib.tdmrg_model_set_profiling(self._h, int(bool(on))), self._h)

    def set_krylov(self, tol, kmax, fixed_k=0):
        """Krylov stopping tolerance, largest dimension and (if > 0) a fixed dimension."""
        _check(self._lib.tdmrg_model_set_krylov(self._h, float(tol), int(kmax), int(fixed_k)),
               self._h)

    def set_concurrent(self, on=True):
        """Step the two real-time states side by side (default) or one after the other."""
        _check(self._lib.tdmrg_model_set_concurrent(self._h, int(bool(on))), self._h)

    def set_wait_cycles(self, cycles):
        """Limit of the bounded grid-barrier waits in clock cycles (0: default, ~2 s)."""
        _check(self._lib.tdmrg_model_set_wait_cycles(self._h, int(cycles)), self._h)

    def set_adjoint_krylov_basis(self, on=True):
        """Node vectors of the exponential VJPs from the Krylov bases (True) or from fresh
        Lanczos exponentials at every node (False, the default)."""
        _check(self._lib.tdmrg_model_set_adjoint_krylov_basis(self._h, int(bool(on))), self._h)

    def parameter_count(self):
        """Number of parameters theta (omega_m, g_m, V, then alpha, omega_p with a bond mode)."""
        n = ctypes.c_int()
        _check(self._lib.tdmrg_parameter_count(self._h, ctypes.byref(n)), self._h)
        return n.value

    def step_vjp(self, M, A_in, tau, Abar_out, nodes=16):
        """Reverse of one FP64 projector-splitting step exp(tau H) through tdmrg_step_vjp: the
        site tensors A_in and the cotangents Abar_out of the output sites (lists of complex128
        CUDA tensors) -> (A_out, Abar_in, theta_bar)."""
        import torch
        L = len(A_in)
        A_out = [torch.empty_like(a) for a in A_in]
        Abar_in = [torch.empty_like(a) for a in A_in]
        arr = lambda ts: (ctypes.c_void_p * L)(*[t.data_ptr() for t in ts])   # noqa: E731
        tb = np.zeros(self.parameter_count())
        _check(self._lib.tdmrg_step_vjp(self._h, int(M), arr(A_in), float(np.real(tau)),
                                        float(np.imag(tau)), arr(Abar_out), arr(A_out),
                                        arr(Abar_in), _dptr(tb), int(nodes)), self._h)
        return A_out, Abar_in, tb

    def correlation_vjp(self, beta, dtau, M, dt, nsteps, cbar, every=2, nodes=16):
        """C_n (t = n dt) of the whole FP64 pipeline and dloss/dtheta for
        loss = Re sum_n conj(cbar_n) C_n through tdmrg_correlation_vjp -> (C, theta_bar, log Z)."""
        cb = np.zeros(2 * (nsteps + 1))
        cb[0::2] = np.real(cbar)
        cb[1::2] = np.imag(cbar)
        C = np.zeros(2 * (nsteps + 1))
        tb = np.zeros(self.parameter_count())
        lz = ctypes.c_double()
        _check(self._lib.tdmrg_correlation_vjp(self._h, float(beta), float(dtau), int(M),
                                               float(dt), int(nsteps), int(every), _dptr(cb),
                                               _dptr(C), _dptr(tb), ctypes.byref(lz), int(nodes)),
               self._h)
        return C[0::2] + 1j * C[1::2], tb, lz.value

    def correlation_states_vjp(self, M, psi1, psi2, dt, nsteps, cbar, every=2, nodes=16):
        """C_n of two given states (lists of complex128 CUDA tensors) stepped in real time and the
        reverse pass for Re sum conj(cbar_n) C_n -> (C, g1, g2, theta_bar)."""
        import torch
        L = len(psi1)
        arr = lambda ts: (ctypes.c_void_p * L)(*[t.data_ptr() for t in ts])   # noqa: E731
        g1 = [torch.empty_like(a) for a in psi1]
        g2 = [torch.empty_like(a) for a in psi2]
        cb = np.zeros(2 * (nsteps + 1))
        cb[0::2] = np.real(cbar)
        cb[1::2] = np.imag(cbar)
        C = np.zeros(2 * (nsteps + 1))
        tb = np.zeros(self.parameter_count())
        _check(self._lib.tdmrg_correlation_states_vjp(self._h, int(M), arr(psi1), arr(psi2),
                                                      float(dt), int(nsteps), int(every),
                                                      _dptr(cb), _dptr(C), arr(g1), arr(g2),
                                                      _dptr(tb), int(nodes)), self._h)
        return C[0::2] + 1j * C[1::2], g1, g2, tb

    def reset_stats(self):
        _check(self._lib.tdmrg_reset_stats(self._h), self._h)


class Batch:
    """Several prepared models (after realtime_init) stepped together (graph mode, one stream
    each, all instances launched before any is waited for)."""

    def __init__(self, models):
        lib = load()
        arr = (_p * len(models))(*[m._h.value for m in models])
        h = ctypes.c_void_p()
        _check(lib.tdmrg_batch_create(arr, len(models), ctypes.byref(h)))
        self._h = h
        self._lib = lib
        self.models = list(models)

    def realtime_step(self, nsteps, dt):
        _check(self._lib.tdmrg_batch_realtime_step(self._h, int(nsteps), float(dt)))

    def step_half(self, dt):
        """One half-step of every instance (left-to-right, then right-to-left on the next call)."""
        _check(self._lib.tdmrg_batch_step_half(self._h, float(dt)))

    def correlation(self, t_grid, dt):
        """C(t) of every instance on one grid: a complex array [instances][len(t_grid)]."""
        t = np.ascontiguousarray(t_grid, dtype=np.float64)
        out = np.zeros(2 * t.size * len(self.models))
        _check(self._lib.tdmrg_batch_correlation(self._h, _dptr(t), int(t.size), float(dt),
                                                 _dptr(out)))
        out = out.reshape(len(self.models), t.size, 2)
        return out[..., 0] + 1j * out[..., 1]

    def close(self):
        if getattr(self, "_h", None):
            self._lib.tdmrg_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def mobility(t_grid, C, kT):
    """Eq. 2 through tdmrg_mobility."""
    lib = load()
    t = np.ascontiguousarray(t_grid, dtype=np.float64)
    c = np.empty(2 * t.size)
    c[0::2] = np.real(C)
    c[1::2] = np.imag(C)
    mu = ctypes.c_double()
    _check(lib.tdmrg_mobility(_dptr(t), _dptr(c), int(t.size), float(kT), ctypes.byref(mu)))
    return mu.value


def kernel_dfma_loop(blocks, iters, sink, stream=None):
    """Launch the FP64 FMA throughput probe on `stream`; returns its flop count."""
    lib = load()
    fl = ctypes.c_double()
    _check(lib.tdmrg_kernel_dfma_loop(int(blocks), int(iters), _ptr(sink), ctypes.byref(fl),
                                      _stream_ptr(stream)))
    return fl.value


def fgr_mobility_batch(omega, g, V, kT, dt, nt, stream=None):
    """Hopping-limit mobilities (Eq. 7 in Eq. 2) of P parameter sets on the GPU:
    omega, g: P x K, V, kT: P; returns mu[P]."""
    lib = load()
    om = np.ascontiguousarray(np.atleast_2d(omega), dtype=np.float64)
    gg = np.ascontiguousarray(np.atleast_2d(g), dtype=np.float64)
    P, K = om.shape
    VV = np.ascontiguousarray(np.broadcast_to(V, (P,)), dtype=np.float64)
    TT = np.ascontiguousarray(np.broadcast_to(kT, (P,)), dtype=np.float64)
    mu = np.zeros(P)
    _check(lib.tdmrg_fgr_mobility_batch(int(P), int(K), _dptr(om), _dptr(gg), _dptr(VV),
                                        _dptr(TT), float(dt), int(nt), _dptr(mu),
                                        _stream_ptr(stream)))
    return mu


def tune_record_shapes(on):
    """Start (True) or stop recording the tensor-core contraction shapes."""
    load().tdmrg_tune_record_shapes(int(bool(on)))


def tune_recorded_shapes():
    """The recorded shapes as a list of (M, N, K, nred, nbatch)."""
    lib = load()
    n = ctypes.c_int()
    _check(lib.tdmrg_tune_recorded_shapes(None, 0, ctypes.byref(n)))
    buf = np.zeros(5 * max(n.value, 1), dtype=np.int32)
    _check(lib.tdmrg_tune_recorded_shapes(buf.ctypes.data_as(_ip), n.value, ctypes.byref(n)))
    return [tuple(int(x) for x in buf[5 * i:5 * i + 5]) for i in range(n.value)]


def tune_reload_table():
    load().tdmrg_tune_reload_table()


def tune_table_lookup(M, N, K, nred, nbatch):
    """(ksplit, tile_n) of the tile table for one contraction shape, (0, 0) when not listed
    (host only)."""
    ks, bn = ctypes.c_int(), ctypes.c_int()
    _check(load().tdmrg_tune_table_lookup(int(M), int(N), int(K), int(nred), int(nbatch),
                                          ctypes.byref(ks), ctypes.byref(bn)))
    return ks.value, bn.value


def kernel_tc_gemm_timed(M, N, K, nred, nbatch, ksplit, reps=10, stream=None, tile_n=0):
    """Average milliseconds of one tensor-core contraction shape with split ksplit and tile
    width tile_n (64 or 128; 0: the table's)."""
    lib = load()
    ms = ctypes.c_double()
    _check(lib.tdmrg_kernel_tc_gemm_timed(int(M), int(N), int(K), int(nred), int(nbatch),
                                          int(ksplit), int(tile_n), int(reps), ctypes.byref(ms),
                                          _stream_ptr(stream)))
    return ms.value


def coherence_length(sigma):
    """Eq. 9 through tdmrg_coherence_length for an N x N complex sigma."""
    lib = load()
    sig = np.ascontiguousarray(sigma, dtype=np.complex128)
    N = sig.shape[0]
    flat = np.empty(2 * N * N)
    flat[0::2] = sig.real.ravel()
    flat[1::2] = sig.imag.ravel()
    out = ctypes.c_double()
    _check(lib.tdmrg_coherence_length(int(N), _dptr(flat), ctypes.byref(out)))
    return out.value


def mean_free_path(t_grid, C):
    """Eq. 8 through tdmrg_mean_free_path: (v, tau, l)."""
    lib = load()
    t = np.ascontiguousarray(t_grid, dtype=np.float64)
    c = np.empty(2 * t.size)
    c[0::2] = np.real(C)
    c[1::2] = np.imag(C)
    out = np.zeros(3)
    _check(lib.tdmrg_mean_free_path(_dptr(t), _dptr(c), int(t.size), _dptr(out)))
    return float(out[0]), float(out[1]), float(out[2])


def host_gauss_legendre(n):
    """Gauss-Legendre nodes and weights on [0, 1] (host only)."""
    sn, wn = np.zeros(int(n)), np.zeros(int(n))
    _check(load().tdmrg_host_gauss_legendre(int(n), _dptr(sn), _dptr(wn)))
    return sn, wn


def host_quadrature_nodes(r, nmax=16, eps=1e-15):
    """Node count of the Krylov-basis quadrature for the integrand bound r (host only)."""
    n = ctypes.c_int()
    _check(load().tdmrg_host_quadrature_nodes(float(r), int(nmax), float(eps), ctypes.byref(n)))
    return n.value


def host_tridiag_exp(alpha, beta, z):
    """exp(z_s T) e_1 for T = tridiag(beta, alpha, beta) at the complex points z (host only);
    returns an array [len(z), len(alpha)]."""
    a = np.ascontiguousarray(alpha, dtype=np.float64)
    b = np.ascontiguousarray(beta, dtype=np.float64) if len(beta) else np.zeros(1)
    zz = np.ascontiguousarray(np.asarray(z, dtype=np.complex128)).view(np.float64)
    out = np.zeros(2 * a.size * (zz.size // 2))
    _check(load().tdmrg_host_tridiag_exp(int(a.size), _dptr(a), _dptr(b), int(zz.size // 2),
                                         _dptr(zz), _dptr(out)))
    return (out[0::2] + 1j * out[1::2]).reshape(-1, a.size)


MPO_H, MPO_J, MPO_IDENTITY = 0, 1, 2


def host_mpo(N, omega, g, nmax, V, which=MPO_H, param=-1, peierls=None):
    """Every site of an MPO of the chain (or of its derivative with respect to parameter
    `param`: omega_m, g_m, V, then alpha, omega_p) through tdmrg_host_mpo_site, as complex
    arrays [Dl, Dr, d, d]; host only."""
    lib = load()
    om = np.ascontiguousarray(omega, dtype=np.float64)
    gg = np.ascontiguousarray(g, dtype=np.float64)
    nm = np.ascontiguousarray(nmax, dtype=np.int32)
    alpha, omega_p, nmax_p = peierls if peierls is not None else (0.0, 0.0, 0)
    L = int(N) * (1 + om.size + (1 if peierls is not None else 0))
    out = []
    dims = np.zeros(3, dtype=np.int32)
    for k in range(L):
        args = [int(N), int(om.size), _dptr(om), _dptr(gg), float(V), nm.ctypes.data_as(_ip),
                float(alpha), float(omega_p), int(nmax_p), int(which), int(param), k,
                dims.ctypes.data_as(_ip)]
        _check(lib.tdmrg_host_mpo_site(*args, None))
        Dl, Dr, d = (int(x) for x in dims)
        buf = np.zeros(2 * Dl * Dr * d * d)
        _check(lib.tdmrg_host_mpo_site(*args, _dptr(buf)))
        out.append((buf[0::2] + 1j * buf[1::2]).reshape(Dl, Dr, d, d))
    return out


# --- kernel-level entry points (device pointers from torch tensors) -------------------------

def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def kernel_heff(L, W, R, A, out, X, Y, d, precision=PREC_C128, ws32=None, stream=None):
    """out = H_eff A for one site; L, R, A, out, X, Y complex128 CUDA tensors, W numpy complex."""
    lib = load()
    Dl, Ml, _ = L.shape
    Dr, Mr, _ = R.shape
    Wc = np.ascontiguousarray(W, dtype=np.complex128).view(np.float64)
    _check(lib.tdmrg_kernel_heff(Ml, Mr, d, Dl, Dr, _dptr(Wc), _ptr(L), _ptr(R), _ptr(A),
                                 _ptr(out), _ptr(X), _ptr(Y), _ptr(ws32), int(precision),
                                 _stream_ptr(stream)))


def kernel_heff_timed(L, W, R, A, out, d, precision=PREC_C64_3XTF32, reps=20, stream=None):
    """Average milliseconds of the sweep's H_eff product (tdmrg_kernel_heff_timed)."""
    lib = load()
    Dl, Ml, _ = L.shape
    Dr, Mr, _ = R.shape
    Wc = np.ascontiguousarray(W, dtype=np.complex128).view(np.float64)
    ms = ctypes.c_double()
    _check(lib.tdmrg_kernel_heff_timed(Ml, Mr, d, Dl, Dr, _dptr(Wc), _ptr(L), _ptr(R), _ptr(A),
                                       _ptr(out), int(precision), int(reps), ctypes.byref(ms),
                                       _stream_ptr(stream)))
    return ms.value


def kernel_heff_vjp(L, W, R, A, ybar, Abar, Lbar, Rbar, X, Y, d, stream=None):
    """(Abar, Lbar, Rbar) of y = H_eff(L, W, R) A for the cotangent ybar (FP64, written into
    the given CUDA tensors); W numpy complex on the host."""
    lib = load()
    Dl, Ml, _ = L.shape
    Dr, Mr, _ = R.shape
    Wc = np.ascontiguousarray(W, dtype=np.complex128).view(np.float64)
    _check(lib.tdmrg_kernel_heff_vjp(Ml, Mr, d, Dl, Dr, _dptr(Wc), _ptr(L), _ptr(R), _ptr(A),
                                     _ptr(ybar), _ptr(Abar), _ptr(Lbar), _ptr(Rbar), _ptr(X),
                                     _ptr(Y), _stream_ptr(stream)))


def kernel_site_exp_vjp(L, W, R, A, ybar, tau, Abar, Lbar, Rbar, d, nodes=16, tol=1e-13,
                        stream=None):
    """(Abar, Lbar, Rbar) of y = exp(tau H_eff(L, W, R)) A for the cotangent ybar (FP64)."""
    lib = load()
    Dl, Ml, _ = L.shape
    Dr, Mr, _ = R.shape
    Wc = np.ascontiguousarray(W, dtype=np.complex128).view(np.float64)
    _check(lib.tdmrg_kernel_site_exp_vjp(Ml, Mr, d, Dl, Dr, _dptr(Wc), _ptr(L), _ptr(R), _ptr(A),
                                         _ptr(ybar), float(np.real(tau)), float(np.imag(tau)),
                                         int(nodes), float(tol), _ptr(Abar), _ptr(Lbar),
                                         _ptr(Rbar), _stream_ptr(stream)))


def kernel_qr_vjp(Q, R, Qbar, Rbar, Ybar, stream=None):
    """Ybar of the full-rank QR Y = Q R for the cotangents Qbar, Rbar (FP64 CUDA tensors)."""
    m, n = Q.shape
    _check(load().tdmrg_kernel_qr_vjp(int(m), int(n), _ptr(Q), _ptr(R), _ptr(Qbar), _ptr(Rbar),
                                      _ptr(Ybar), _stream_ptr(stream)))


def kernel_bond_exp_vjp(L, R, C, ybar, tau, Cbar, Lbar, Rbar, nodes=16, tol=1e-13,
                        stream=None):
    """(Cbar, Lbar, Rbar) of y = exp(tau K(L, R)) C for the cotangent ybar (FP64)."""
    Dw, M = L.shape[0], L.shape[1]
    _check(load().tdmrg_kernel_bond_exp_vjp(int(M), int(Dw), _ptr(L), _ptr(R), _ptr(C),
                                            _ptr(ybar), float(np.real(tau)), float(np.imag(tau)),
                                            int(nodes), float(tol), _ptr(Cbar), _ptr(Lbar),
                                            _ptr(Rbar), _stream_ptr(stream)))


def _dense_sites(dW, shape):
    """nparam dense MPO sites as one interleaved FP64 host array (None when there are none)."""
    if dW is None or len(dW) == 0:
        return 0, None
    arr = np.ascontiguousarray(np.stack([np.asarray(x).reshape(shape) for x in dW]),
                               dtype=np.complex128)
    return arr.shape[0], arr.view(np.float64)


def kernel_env_vjp(side, E, bra, W, ket, G, Ebar, brabar, ketbar, X, Y, d, dW=None,
                   stream=None):
    """(Ebar, brabar, ketbar) of an environment update (side 0: left, 1: right) for the
    cotangent G, written into the given CUDA tensors, and theta_bar[p] = Re<G, update with
    W -> dW[p]> (returned, numpy); W and dW numpy complex on the host."""
    lib = load()
    Ml, _, Mr = bra.shape
    Dl, Dr = W.shape[0], W.shape[1]
    Wc = np.ascontiguousarray(W, dtype=np.complex128).view(np.float64)
    npar, dWc = _dense_sites(dW, W.shape)
    tb = np.zeros(max(npar, 1))
    _check(lib.tdmrg_kernel_env_vjp(int(side), Ml, Mr, d, Dl, Dr, _dptr(Wc), npar,
                                    _dptr(dWc) if dWc is not None else None, _ptr(E), _ptr(bra),
                                    _ptr(ket), _ptr(G), _ptr(Ebar), _ptr(brabar), _ptr(ketbar),
                                    _dptr(tb), _ptr(X), _ptr(Y), _stream_ptr(stream)))
    return tb[:npar]


def kernel_expansion_vjp(side, E, W, A, Xbar, Ebar, Abar, X, Y, d, dW=None, stream=None):
    """(Ebar, Abar) of the gauge-completion candidates (side 0: left_expansion(L, W, A),
    side 1: right_expansion(W, A, R)) for the cotangent Xbar, and theta_bar (returned)."""
    lib = load()
    Ml, _, Mr = A.shape
    Dl, Dr = W.shape[0], W.shape[1]
    Wc = np.ascontiguousarray(W, dtype=np.complex128).view(np.float64)
    npar, dWc = _dense_sites(dW, W.shape)
    tb = np.zeros(max(npar, 1))
    _check(lib.tdmrg_kernel_expansion_vjp(int(side), Ml, Mr, d, Dl, Dr, _dptr(Wc), npar,
                                          _dptr(dWc) if dWc is not None else None, _ptr(E),
                                          _ptr(A), _ptr(Xbar), _ptr(Ebar), _ptr(Abar), _dptr(tb),
                                          _ptr(X), _ptr(Y), _stream_ptr(stream)))
    return tb[:npar]


def kernel_qr_vjp_completed(accepted, Q, R, Xsel, Qbar, Rbar, Ybar, Xselbar, stream=None):
    """(Ybar, Xselbar) of the gauge QR with completed columns (accepted: host flags)."""
    m, n = Q.shape
    acc = np.ascontiguousarray(accepted, dtype=np.int32)
    _check(load().tdmrg_kernel_qr_vjp_completed(int(m), int(n), acc.ctypes.data_as(_ip), _ptr(Q),
                                                _ptr(R), _ptr(Xsel), _ptr(Qbar), _ptr(Rbar),
                                                _ptr(Ybar), _ptr(Xselbar), _stream_ptr(stream)))


def heff_workspace_floats(Ml, Mr, d, Dl, Dr):
    return int(load().tdmrg_heff_workspace_floats(Ml, Mr, d, Dl, Dr))


def kernel_zgemm_tc(A, B, C, conjA=0, conjB=0, stream=None):
    """C = opA(A) opB(B)^T on the tensor cores (3xTF32); complex128 CUDA tensors."""
    lib = load()
    M, K = A.shape
    N = B.shape[0]
    _check(lib.tdmrg_kernel_zgemm_tc(M, N, K, _ptr(A), _ptr(B), int(conjA), int(conjB), _ptr(C),
                                     _stream_ptr(stream)))


def kernel_env_left(L, W, bra, ket, Lout, X, Y, d, stream=None):
    lib = load()
    Dl = L.shape[0]
    Dr = Lout.shape[0]
    Ml1, _, Mr1 = bra.shape
    Ml2, _, Mr2 = ket.shape
    Wc = np.ascontiguousarray(W, dtype=np.complex128).view(np.float64)
    _check(lib.tdmrg_kernel_env_left(Ml1, Mr1, Ml2, Mr2, d, Dl, Dr, _dptr(Wc), _ptr(L),
                                     _ptr(bra), _ptr(ket), _ptr(Lout), _ptr(X), _ptr(Y),
                                     _stream_ptr(stream)))


def kernel_gauge_qr(Y, Q, R, E=None, status=None, stream=None):
    lib = load()
    m, n = Y.shape
    p = 0 if E is None else E.shape[1]
    _check(lib.tdmrg_kernel_gauge_qr(m, n, _ptr(Y), p, _ptr(E), _ptr(Q), _ptr(R), _ptr(status),
                                     _stream_ptr(stream)))


def kernel_gauge_qr_blocked(Y, Q, R, E=None, status=None, stream=None):
    lib = load()
    m, n = Y.shape
    p = 0 if E is None else E.shape[1]
    _check(lib.tdmrg_kernel_gauge_qr_blocked(m, n, _ptr(Y), p, _ptr(E), _ptr(Q), _ptr(R),
                                             _ptr(status), _stream_ptr(stream)))


def kernel_gauge_qr_noalloc(Y, Q, R, E=None, status=None, stream=None):
    """tdmrg_kernel_gauge_qr with the scratch in the library's fixed device array: no device
    allocation happens in the call (for callers whose device memory is owned by another runtime
    or that may not allocate once set up); calls that overlap on the GPU race."""
    lib = load()
    m, n = Y.shape
    p = 0 if E is None else E.shape[1]
    _check(lib.tdmrg_kernel_gauge_qr_noalloc(m, n, _ptr(Y), p, _ptr(E), _ptr(Q), _ptr(R),
                                             _ptr(status), _stream_ptr(stream)))


def kernel_bond_exp(L, R, C, out, tau, tol=1e-7, kmax=32, stream=None):
    """out = exp(tau K) C, (K C)[a,b] = sum L[w,a,a'] C[a',b'] R[w,b,b'] (one launch)."""
    lib = load()
    k = ctypes.c_int()
    Dw, M = L.shape[0], L.shape[1]
    _check(lib.tdmrg_kernel_bond_exp(int(M), int(Dw), _ptr(L), _ptr(R), _ptr(C), _ptr(out),
                                     float(np.real(tau)), float(np.imag(tau)), float(tol),
                                     int(kmax), ctypes.byref(k), _stream_ptr(stream)))
    return k.value


def kernel_krylov_dense(H, v, out, tau, tol=1e-13, kmax=32, stream=None):
    lib = load()
    k = ctypes.c_int()
    _check(lib.tdmrg_kernel_krylov_dense(H.shape[0], _ptr(H), _ptr(v), _ptr(out),
                                         float(np.real(tau)), float(np.imag(tau)), float(tol),
                                         int(kmax), ctypes.byref(k), _stream_ptr(stream)))
    return k.value


# --- differentiable C(t) ----------------------------------------------------------------------

def _correlation_function():
    import torch

    class CorrelationFunction(torch.autograd.Function):
        """C(t_n), t_n = n dt (n = 0..nsteps), of the chain as a differentiable function of the
        parameters theta = (omega_0.., g_0.., V) (a float64 tensor): forward through
        tdmrg_thermal_prepare / tdmrg_correlation, backward through tdmrg_correlation_vjp
        (FP64).  spec: dict with N, nmax, beta, dtau, M, dt, nsteps and optionally every,
        rank_tol, nodes.  PyTorch's gradient of a real loss with respect to a complex output,
        dl/dRe C + i dl/dIm C, is the cotangent Cbar of dl = Re sum conj(Cbar_n) dC_n."""

        @staticmethod
        def forward(ctx, theta, spec):
            K = len(spec["nmax"])
            th = theta.detach().cpu().numpy().astype(np.float64)
            m = Model(spec["N"], th[:K], th[K:2 * K], spec["nmax"], float(th[2 * K]))
            try:
                if spec.get("rank_tol") is not None:
                    m.set_rank_tol(spec["rank_tol"])
                m.thermal_prepare(spec["beta"], spec["dtau"], spec["M"])
                t = np.arange(spec["nsteps"] + 1) * spec["dt"]
                C = m.correlation(t, spec["dt"])
            finally:
                m.close()
            ctx.spec = spec
            ctx.theta = th
            ctx.device = theta.device
            return torch.as_tensor(np.asarray(C), dtype=torch.complex128, device=theta.device)

        @staticmethod
        def backward(ctx, gC):
            spec, th = ctx.spec, ctx.theta
            K = len(spec["nmax"])
            m = Model(spec["N"], th[:K], th[K:2 * K], spec["nmax"], float(th[2 * K]))
            try:
                if spec.get("rank_tol") is not None:
                    m.set_rank_tol(spec["rank_tol"])
                cbar = gC.detach().cpu().numpy().astype(np.complex128)
                _, tb, _ = m.correlation_vjp(spec["beta"], spec["dtau"], spec["M"], spec["dt"],
                                             spec["nsteps"], cbar, every=spec.get("every", 2),
                                             nodes=spec.get("nodes", 16))
            finally:
                m.close()
            return torch.as_tensor(tb, dtype=torch.float64, device=ctx.device), None

    return CorrelationFunction


def correlation_autograd(theta, spec):
    """C(t) as a differentiable function of theta (see _correlation_function)."""
    return _correlation_function().apply(theta, spec)
