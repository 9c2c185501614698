"""Vector-Jacobian products of the TDVP building blocks (oracle for the adjoint step).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Convention: for y = f(x) with complex arrays and a real loss l, the cotangent ybar is defined
by dl = Re<ybar, dy> = Re sum conj(ybar) dy, and the VJP returns xbar with
dl = Re<xbar, dx> for every direction dx.  For a map that is linear in x (dy = J dx),
xbar = J^H ybar; for a map that depends on conj(x) (the bra of an environment update) the
conjugate pairing is taken accordingly.

* ``heff_vjp``        -- the H_eff product of the one-site step (Eq. S1),
                         y = sum L[w,x,y] W[w,v,s,u] A[y,u,t,c] R[v,b,c];
* ``bond_heff_vjp``   -- the zero-site (bond) product, y = sum L[w,x,y] C[y,c] R[w,b,c];
* ``update_left_vjp`` / ``update_right_vjp`` -- the environment updates;
* ``left_expansion_vjp`` / ``right_expansion_vjp`` -- the gauge completion candidates (what
  H_eff couples the site into), which move the completed directions of a gauge QR;
* ``expm_krylov_vjp`` -- y = exp(tau H) v for a Hermitian H given as a linear map:
  vbar = exp(conj(tau) H) ybar, and the cotangent of H as the integral
  Hbar = conj(tau) int_0^1 a(s) b(s)^H ds,  a(s) = exp((1-s) conj(tau) H) ybar,
  b(s) = exp(s tau H) v  (from d exp(X)[E] = int_0^1 e^{(1-s)X} E e^{sX} ds), evaluated by
  Gauss-Legendre quadrature and returned as weighted pairs (c_s, b_s) with
  Hbar = sum_s c_s b_s^H, which the caller maps to L, W, R through the VJPs above.  The
  energy offset of H cancels between a(s) and b(s), so the integrand varies on the scale of
  |tau| times the spread of the spectrum; 16 nodes integrate it to rounding for
  |tau| spread <= 5;
* ``qr_vjp`` / ``qr_vjp_completed`` / ``qr_vjp_selected`` -- the gauge QR at full column rank,
  with completed columns following their candidates, and with the completed columns fixed.

Reverse passes on tapes (``Tape``: values and the VJPs of the operations that made them):
``step_with_tape`` (one projector-splitting step, Eq. S1), ``correlation_vjp`` (C_n of two given
states, Eq. 6, stored every k steps), ``thermal_logz_gradient`` (the imaginary-time
preparation, Eq. 5), ``fit_with_tape`` (the variational j fit) and
``correlation_pipeline_gradient`` / ``mobility_pipeline_gradient`` (the whole C(t) and mu of
Eq. 2 as functions of omega_m, g_m, V through the MPO coefficients,
``step_parameter_gradient``).
"""
from typing import Callable, List, Tuple

import numpy as np

from .tdvp import (RANK_TOL, _split, bond_heff, gauge_qr, heff, krylov_expm, left_expansion,
                   right_expansion, update_left, update_right)


def heff_vjp(Lenv, W, Renv, A, d, ybar):
    """(Abar, Lbar, Wbar, Rbar) of y = heff(Lenv, W, Renv, A, d)."""
    A4 = _split(A, d)                                       # [y, u, t, c]
    Y4 = ybar.reshape(A.shape[0], d, d, A.shape[2])         # [x, s, t, b]
    Wc = np.conj(W)
    # Abar[y,u,t,c] = sum conj(L[w,x,y]) conj(W[w,v,s,u]) conj(R[v,b,c]) ybar[x,s,t,b]
    X = np.tensordot(np.conj(Lenv), Y4, axes=([1], [0]))    # [w, y, s, t, b]
    X = np.tensordot(Wc, X, axes=([0, 2], [0, 2]))          # [v, u, y, t, b]
    Ab = np.tensordot(X, np.conj(Renv), axes=([0, 4], [0, 1]))   # [u, y, t, c]
    Abar = Ab.transpose(1, 0, 2, 3).reshape(A.shape)
    # Lbar[w,x,y] = sum ybar[x,s,t,b] conj(W[w,v,s,u] A[y,u,t,c] R[v,b,c])
    AR = np.tensordot(np.conj(A4), np.conj(Renv), axes=([3], [2]))   # [y, u, t, v, b]
    WAR = np.tensordot(Wc, AR, axes=([1, 3], [3, 1]))       # [w, s, y, t, b]
    Lbar = np.tensordot(WAR, Y4, axes=([1, 3, 4], [1, 2, 3])).transpose(0, 2, 1)   # [w, x, y]
    # Rbar[v,b,c] = sum ybar[x,s,t,b] conj(L[w,x,y] W[w,v,s,u] A[y,u,t,c])
    LA = np.tensordot(np.conj(Lenv), np.conj(A4), axes=([2], [0]))   # [w, x, u, t, c]
    WLA = np.tensordot(Wc, LA, axes=([0, 3], [0, 2]))       # [v, s, x, t, c]
    Rbar = np.tensordot(WLA, Y4, axes=([1, 2, 3], [1, 0, 2])).transpose(0, 2, 1)   # [v, b, c]
    # Wbar[w,v,s,u] = sum ybar[x,s,t,b] conj(L[w,x,y] A[y,u,t,c] R[v,b,c])
    LAR = np.tensordot(LA, np.conj(Renv), axes=([4], [2]))  # [w, x, u, t, v, b]
    Wbar = np.tensordot(LAR, Y4, axes=([1, 3, 5], [0, 2, 3]))   # [w, u, v, s]
    Wbar = Wbar.transpose(0, 2, 3, 1)                       # [w, v, s, u]
    return Abar, Lbar, Wbar, Rbar


def bond_heff_vjp(Lenv, Renv, C, ybar):
    """(Cbar, Lbar, Rbar) of y = bond_heff(Lenv, Renv, C) = sum L[w,x,y] C[y,c] R[w,b,c]."""
    X = np.tensordot(np.conj(Lenv), ybar, axes=([1], [0]))          # [w, y, b]
    Cbar = np.tensordot(X, np.conj(Renv), axes=([0, 2], [0, 1]))    # [y, c]
    CR = np.tensordot(np.conj(C), np.conj(Renv), axes=([1], [2]))   # [y, w, b]
    Lbar = np.tensordot(ybar, CR, axes=([1], [2])).transpose(2, 0, 1)   # [x,y,w] -> [w,x,y]
    LC = np.tensordot(np.conj(Lenv), np.conj(C), axes=([2], [0]))   # [w, x, c]
    Rbar = np.tensordot(LC, ybar, axes=([1], [0])).transpose(0, 2, 1)   # [w, b, c]
    return Cbar, Lbar, Rbar


def update_left_vjp(Lenv, bra, W, ket, d, Lbar_out):
    """(Lbar, brabar, Wbar, ketbar) of L' = update_left(Lenv, bra, W, ket, d),
    L'[w', b, c] = sum conj(bra[a,s,t,b]) L[w,a,y] W[w,w',s,u] ket[y,u,t,c]."""
    K = _split(ket, d)
    B = _split(bra, d)
    G = Lbar_out                                                    # [w', b, c]
    # M[w',a,s,t,c] = sum L[w,a,y] W[w,w',s,u] ket[y,u,t,c]  (the part paired with conj(bra))
    X = np.tensordot(Lenv, K, axes=([2], [0]))                      # [w, a, u, t, c]
    M = np.tensordot(W, X, axes=([0, 3], [0, 2]))                   # [w', s, a, t, c]
    # brabar[a,s,t,b] = sum conj(G[w',b,c]) M[w',s,a,t,c]   (L' depends on conj(bra))
    brabar = np.tensordot(M, np.conj(G), axes=([0, 4], [0, 2]))     # [s, a, t, b]
    brabar = brabar.transpose(1, 0, 2, 3).reshape(bra.shape)
    # linear arguments: xbar = sum G conj(other factors), with conj(conj(bra)) = bra
    GB = np.tensordot(G, B, axes=([1], [3]))                        # [w', c, a, s, t]
    # ketbar[y,u,t,c] = sum G[w',b,c] bra[a,s,t,b] conj(L[w,a,y]) conj(W[w,w',s,u])
    T1 = np.tensordot(GB, np.conj(W), axes=([0, 3], [1, 2]))        # [c, a, t, w, u]
    ketbar = np.tensordot(T1, np.conj(Lenv), axes=([3, 1], [0, 1]))   # [c, t, u, y]
    ketbar = ketbar.transpose(3, 2, 1, 0).reshape(ket.shape)
    # Lbar[w,a,y] = sum G bra conj(W) conj(ket)
    T2 = np.tensordot(T1, np.conj(K), axes=([4, 2, 0], [1, 2, 3]))   # [a, w, y]
    Lbar = T2.transpose(1, 0, 2)
    # Wbar[w,w',s,u] = sum G[w',b,c] bra[a,s,t,b] conj(L[w,a,y]) conj(ket[y,u,t,c])
    LK = np.tensordot(np.conj(Lenv), np.conj(K), axes=([2], [0]))   # [w, a, u, t, c]
    Wbar = np.tensordot(GB, LK, axes=([1, 2, 4], [4, 1, 3]))        # [w', s, w, u]
    Wbar = Wbar.transpose(2, 0, 1, 3)
    return Lbar, brabar, Wbar, ketbar


def update_right_vjp(Renv, bra, W, ket, d, Rbar_out):
    """(Rbar, brabar, Wbar, ketbar) of R' = update_right(Renv, bra, W, ket, d),
    R'[w, a, y] = sum conj(bra[a,s,t,b]) R[w',b,c] W[w,w',s,u] ket[y,u,t,c]."""
    K = _split(ket, d)
    B = _split(bra, d)
    G = Rbar_out                                                    # [w, a, y]
    # M[w,s,y,t,b] = sum W[w,w',s,u] ket[y,u,t,c] R[w',b,c]
    X = np.tensordot(K, Renv, axes=([3], [2]))                      # [y, u, t, w', b]
    M = np.tensordot(W, X, axes=([1, 3], [3, 1]))                   # [w, s, y, t, b]
    brabar = np.tensordot(np.conj(G), M, axes=([0, 2], [0, 2]))     # [a, s, t, b]
    brabar = brabar.reshape(bra.shape)
    GB = np.tensordot(G, B, axes=([1], [0]))                        # [w, y, s, t, b]
    # ketbar[y,u,t,c] = sum G[w,a,y] bra[a,s,t,b] conj(W[w,w',s,u]) conj(R[w',b,c])
    T1 = np.tensordot(GB, np.conj(W), axes=([0, 2], [0, 2]))        # [y, t, b, w', u]
    ketbar = np.tensordot(T1, np.conj(Renv), axes=([3, 2], [0, 1]))   # [y, t, u, c]
    ketbar = ketbar.transpose(0, 2, 1, 3).reshape(ket.shape)
    # Rbar[w',b,c] = sum G bra conj(W) conj(ket)
    T2 = np.tensordot(T1, np.conj(K), axes=([0, 4, 1], [0, 1, 2]))   # [b, w', c]
    Rbar = T2.transpose(1, 0, 2)
    # Wbar[w,w',s,u] = sum G[w,a,y] bra[a,s,t,b] conj(ket[y,u,t,c]) conj(R[w',b,c])
    KR = np.tensordot(np.conj(K), np.conj(Renv), axes=([3], [2]))   # [y, u, t, w', b]
    Wbar = np.tensordot(GB, KR, axes=([1, 3, 4], [0, 2, 4]))        # [w, s, u, w']
    Wbar = Wbar.transpose(0, 3, 1, 2)
    return Rbar, brabar, Wbar, ketbar


def left_expansion_vjp(Lenv, W, A, d, Xbar):
    """VJP of ``tdvp.left_expansion``, X[(x,s,t), (v,c)] = sum L[w,x,y] W[w,v,s,u] A[y,u,t,c]:
    trilinear, so each cotangent is Xbar contracted with the conjugates of the other two
    factors.  Returns (Lbar, Wbar, Abar)."""
    As = _split(A, d)                                          # [y, u, t, c]
    Xb = Xbar.reshape(A.shape[0], d, d, W.shape[1], A.shape[2])  # [x, s, t, v, c]
    Lb = np.einsum("xstvc,wvsu,yutc->wxy", Xb, np.conj(W), np.conj(As))
    Wb = np.einsum("xstvc,wxy,yutc->wvsu", Xb, np.conj(Lenv), np.conj(As))
    Ab = np.einsum("xstvc,wxy,wvsu->yutc", Xb, np.conj(Lenv), np.conj(W))
    return Lb, Wb, Ab.reshape(A.shape)


def right_expansion_vjp(W, A, Renv, d, Xbar):
    """VJP of ``tdvp.right_expansion``, X = P^H with
    P[(w,y), (s,t,b)] = sum W[w,v,s,u] A[y,u,t,c] R[v,b,c]: Re<Xbar, P^H> = Re<Xbar^H, P>, so
    Pbar = Xbar^H and the trilinear rule applies.  Returns (Wbar, Abar, Rbar)."""
    As = _split(A, d)                                          # [y, u, t, c]
    Pb = Xbar.conj().T.reshape(W.shape[0], A.shape[0], d, d, Renv.shape[1])  # [w, y, s, t, b]
    Wb = np.einsum("wystb,yutc,vbc->wvsu", Pb, np.conj(As), np.conj(Renv))
    Ab = np.einsum("wystb,wvsu,vbc->yutc", Pb, np.conj(W), np.conj(Renv))
    Rb = np.einsum("wystb,wvsu,yutc->vbc", Pb, np.conj(W), np.conj(As))
    return Wb, Ab.reshape(A.shape), Rb


def expm_krylov_vjp(matvec: Callable[[np.ndarray], np.ndarray], v: np.ndarray, tau: complex,
                    ybar: np.ndarray, nodes: int = 16, tol: float = 1e-14
                    ) -> Tuple[np.ndarray, List[Tuple[np.ndarray, np.ndarray]]]:
    """VJP of y = exp(tau H) v for a Hermitian H given by `matvec`.

    Returns vbar = exp(conj(tau) H) ybar and pairs (c_s, b_s) with the cotangent of H
    Hbar = sum_s c_s b_s^H (Gauss-Legendre on [0, 1]; c_s already carries conj(tau) and the
    weight).  Every exponential is the oracle's Krylov exponential at tolerance `tol`."""
    vbar, _ = krylov_expm(matvec, ybar, np.conj(tau), tol=tol)
    x, w = np.polynomial.legendre.leggauss(nodes)
    s_nodes = 0.5 * (x + 1.0)
    weights = 0.5 * w
    pairs = []
    for s, ws in zip(s_nodes, weights):
        b, _ = krylov_expm(matvec, v, s * tau, tol=tol)
        a, _ = krylov_expm(matvec, ybar, (1.0 - s) * np.conj(tau), tol=tol)
        pairs.append((ws * np.conj(tau) * a, b))
    return vbar, pairs


def qr_vjp(Q, R, Qbar, Rbar):
    """VJP of the thin QR Y = Q R (m >= n, full column rank, diag(R) real positive: the gauge
    QR when no column is skipped).

    With M = R Rbar^H - Qbar^H Q, Ybar = (Qbar + Q copyltu(M)) R^{-H}, where copyltu(M) is the
    Hermitian matrix that keeps the strictly lower triangle of M, mirrors it (conjugated) into
    the upper triangle and keeps the real part of the diagonal (the imaginary part of a
    diagonal entry pairs with a phase of a column of Q, which the real-diagonal gauge fixes).
    From Q^H dQ anti-Hermitian, Q^H dY R^{-1} = Q^H dQ + dR R^{-1} with dR R^{-1} upper
    triangular with a real diagonal."""
    Rbar = np.triu(Rbar)               # entries below the diagonal of R are structural zeros
    M = R @ Rbar.conj().T - Qbar.conj().T @ Q
    low = np.tril(M, -1)
    sym = low + low.conj().T + np.diag(np.diag(M).real)
    rhs = Qbar + Q @ sym
    # Ybar = rhs R^{-H}: solve Ybar R^H = rhs, i.e. R Ybar^H = rhs^H (R upper triangular)
    return sl_solve_triangular(R, rhs.conj().T).conj().T


def sl_solve_triangular(R, B):
    """x with R x = B for upper-triangular R (back substitution, column by column of B)."""
    n = R.shape[0]
    X = np.zeros(B.shape, dtype=complex)
    for i in range(n - 1, -1, -1):
        X[i] = (B[i] - R[i, i + 1:] @ X[i + 1:]) / R[i, i]
    return X


# ---------------------------------------------------------------------------------
# discrete adjoint of one projector-splitting step
# ---------------------------------------------------------------------------------

class Tape:
    """Values and the operations that produced them, for reverse accumulation; rank_tol is
    the rank threshold of the gauge QRs recorded on it."""

    def __init__(self, rank_tol=RANK_TOL):
        self.rank_tol = rank_tol
        self.vals = {}
        self.ops = []            # (input ids, output ids, vjp(out_bars) -> in_bars)

    def var(self, x):
        i = len(self.vals)
        self.vals[i] = x
        return i

    def op(self, outs, ins, vjp):
        ids = [self.var(v) for v in outs]
        self.ops.append((ins, ids, vjp))
        return ids

    def backward(self, seeds):
        """Cotangents of every value from the cotangents `seeds` {id: bar} of some outputs."""
        bars = dict(seeds)
        for ins, outs, vjp in reversed(self.ops):
            obars = [bars.get(o) for o in outs]
            if all(b is None for b in obars):
                continue
            obars = [np.zeros_like(self.vals[o]) if b is None else b for o, b in zip(outs, obars)]
            for i, b in zip(ins, vjp(obars)):
                if b is not None:
                    bars[i] = b if i not in bars else bars[i] + b
        return bars


def _op_exp_heff(T, l, w, r, a, d, h, tol):
    Lk, Wk, Rk, A = T.vals[l], T.vals[w], T.vals[r], T.vals[a]
    mv = lambda x: heff(Lk, Wk, Rk, x, d)                      # noqa: E731
    y, _ = krylov_expm(mv, A, h, tol=tol)

    def vjp(bars):
        vbar, pairs = expm_krylov_vjp(mv, A, h, bars[0], tol=tol)
        Lb, Wb, Rb = np.zeros_like(Lk), np.zeros_like(Wk, dtype=complex), np.zeros_like(Rk)
        for c, b in pairs:
            _, l_, w_, r_ = heff_vjp(Lk, Wk, Rk, b, d, c)
            Lb, Wb, Rb = Lb + l_, Wb + w_, Rb + r_
        return [Lb, Wb, Rb, vbar]
    return T.op([y], [l, w, r, a], vjp)[0]


def _op_exp_bond(T, l, r, c, h, tol):
    Lk, Rk, C = T.vals[l], T.vals[r], T.vals[c]
    mv = lambda x: bond_heff(Lk, Rk, x)                        # noqa: E731
    y, _ = krylov_expm(mv, C, h, tol=tol)

    def vjp(bars):
        vbar, pairs = expm_krylov_vjp(mv, C, h, bars[0], tol=tol)
        Lb, Rb = np.zeros_like(Lk), np.zeros_like(Rk)
        for cs, b in pairs:
            _, l_, r_ = bond_heff_vjp(Lk, Rk, b, cs)
            Lb, Rb = Lb + l_, Rb + r_
        return [Lb, Rb, vbar]
    return T.op([y], [l, r, c], vjp)[0]


def _chosen_columns(X, chosen, m):
    """The vectors that completed a gauge QR: column i of X for a source i < p, e_{i-p}
    otherwise (the sources ``gauge_qr`` records)."""
    p = 0 if X is None else X.shape[1]
    out = np.zeros((m, len(chosen)), dtype=complex)
    for j, src in enumerate(chosen):
        if src < p:
            out[:, j] = X[:, src]
        else:
            out[src - p, j] = 1.0
    return out


def _scatter_chosen(Xsbar, chosen, shape):
    """Cotangent of the candidate matrix from that of its chosen columns (unit vectors are
    constants and take none)."""
    Xbar = np.zeros(shape, dtype=complex)
    for j, src in enumerate(chosen):
        if src < shape[1]:
            Xbar[:, src] += Xsbar[:, j]
    return Xbar


def _op_qr_right(T, a, cand=None):
    """A_k (Ml, Ds, Mr) = Q R with Q left-orthonormal; outputs (Q as a site tensor, R).
    Skipped columns are completed as the oracle sweep completes them: cand = (ids of L, W and
    the site tensor A_c, d) puts the candidates left_expansion(L, W, A_c) on the tape, so the
    reverse pass follows the completed directions as they move with L, W and A_c."""
    A = T.vals[a]
    Ml, Ds, Mr = A.shape
    m = Ml * Ds
    X = None if cand is None else left_expansion(T.vals[cand[0]], T.vals[cand[1]],
                                                 T.vals[cand[2]], cand[3])
    chosen = []
    Q, R = gauge_qr(A.reshape(m, Mr), X, rank_tol=T.rank_tol, chosen=chosen)
    Xs = _chosen_columns(X, chosen, m)

    def vjp(bars):
        Yb, Xsb = qr_vjp_completed(Q, R, bars[0].reshape(m, Mr), bars[1], Xs)
        out = [Yb.reshape(Ml, Ds, Mr)]
        if cand is not None:
            Xb = _scatter_chosen(Xsb, chosen, X.shape)
            out += list(left_expansion_vjp(T.vals[cand[0]], T.vals[cand[1]], T.vals[cand[2]],
                                           cand[3], Xb))
        return out
    ins = [a] if cand is None else [a, cand[0], cand[1], cand[2]]
    return T.op([Q.reshape(Ml, Ds, Mr), R], ins, vjp)


def _op_qr_left(T, a, cand=None):
    """A_k = C Q with Q right-orthonormal (QR of A^H); outputs (Q as a site tensor, C).
    cand = (ids of W, A_c and R, d) puts the candidates right_expansion(W, A_c, R) on the
    tape, as in _op_qr_right."""
    A = T.vals[a]
    Ml, Ds, Mr = A.shape
    m = Ds * Mr
    X = None if cand is None else right_expansion(T.vals[cand[0]], T.vals[cand[1]],
                                                  T.vals[cand[2]], cand[3])
    chosen = []
    Q2, R2 = gauge_qr(A.reshape(Ml, m).conj().T, X, rank_tol=T.rank_tol, chosen=chosen)
    Xs = _chosen_columns(X, chosen, m)

    def vjp(bars):
        Qb = bars[0].reshape(Ml, m).conj().T                    # output Q2^H
        Rb = bars[1].conj().T                                   # output C = R2^H
        Yb, Xsb = qr_vjp_completed(Q2, R2, Qb, Rb, Xs)
        out = [Yb.conj().T.reshape(Ml, Ds, Mr)]
        if cand is not None:
            Xb = _scatter_chosen(Xsb, chosen, X.shape)
            out += list(right_expansion_vjp(T.vals[cand[0]], T.vals[cand[1]],
                                            T.vals[cand[2]], cand[3], Xb))
        return out
    ins = [a] if cand is None else [a, cand[0], cand[1], cand[2]]
    return T.op([Q2.conj().T.reshape(Ml, Ds, Mr), R2.conj().T], ins, vjp)


def _op_env_left(T, l, q, w, d):
    Lk, Q, Wk = T.vals[l], T.vals[q], T.vals[w]

    def vjp(bars):
        Lb, bb, Wb, kb = update_left_vjp(Lk, Q, Wk, Q, d, bars[0])
        return [Lb, bb + kb, Wb]
    return T.op([update_left(Lk, Q, Wk, Q, d)], [l, q, w], vjp)[0]


def _op_env_right(T, r, q, w, d):
    Rk, Q, Wk = T.vals[r], T.vals[q], T.vals[w]

    def vjp(bars):
        Rb, bb, Wb, kb = update_right_vjp(Rk, Q, Wk, Q, d, bars[0])
        return [Rb, bb + kb, Wb]
    return T.op([update_right(Rk, Q, Wk, Q, d)], [r, q, w], vjp)[0]


def _op_absorb_left(T, c, a):
    """A' = C A (bond matrix into the left index of the next site)."""
    C, A = T.vals[c], T.vals[a]

    def vjp(bars):
        Ab = bars[0]
        return [np.einsum("asc,bsc->ab", Ab, np.conj(A)), np.einsum("ab,asc->bsc", np.conj(C), Ab)]
    return T.op([np.einsum("ab,bsc->asc", C, A)], [c, a], vjp)[0]


def _op_absorb_right(T, a, c):
    """A' = A C (bond matrix into the right index of the previous site)."""
    A, C = T.vals[a], T.vals[c]

    def vjp(bars):
        Ab = bars[0]
        return [np.einsum("asc,bc->asb", Ab, np.conj(C)), np.einsum("asb,asc->bc", np.conj(A), Ab)]
    return T.op([np.einsum("asb,bc->asc", A, C)], [a, c], vjp)[0]


def step_with_tape(Ws, d, A_in, tau, tol=1e-14, rank_tol=RANK_TOL):
    """The second-order projector-splitting step exp(tau H) of ``tdvp.PurifiedMPS.step`` written
    on a tape: right environments of the input (sites 1.. right-orthonormal, center at 0),
    left-to-right and right-to-left half-sweeps with dt/2 site exponentials, gauge shifts,
    environment updates, backward bond exponentials and absorption.  Skipped gauge columns
    are completed as the oracle step completes them (the H coupling of the site, then unit
    vectors), with the coupling candidates on the tape: below full bond dimension the span
    of the completed columns enters the projected evolution.  Returns (tape, ids of the
    output sites, ids of the input sites, ids of the MPO sites)."""
    T = Tape(rank_tol)
    L = len(A_in)
    a_in = [T.var(np.asarray(x, dtype=complex)) for x in A_in]
    w_ids = [T.var(np.asarray(W)) for W in Ws]
    a = list(a_in)
    one = np.ones((1, 1, 1), dtype=complex)
    Lenv, Renv = [None] * L, [None] * L
    Lenv[0] = T.var(one)
    Renv[L - 1] = T.var(one)
    for k in range(L - 1, 0, -1):
        Renv[k - 1] = _op_env_right(T, Renv[k], a[k], w_ids[k], d[k])
    h = 0.5 * tau
    for k in range(L):
        a[k] = _op_exp_heff(T, Lenv[k], w_ids[k], Renv[k], a[k], d[k], h, tol)
        if k < L - 1:
            a[k], r = _op_qr_right(T, a[k], (Lenv[k], w_ids[k], a[k], d[k]))
            Lenv[k + 1] = _op_env_left(T, Lenv[k], a[k], w_ids[k], d[k])
            c = _op_exp_bond(T, Lenv[k + 1], Renv[k], r, -h, tol)
            a[k + 1] = _op_absorb_left(T, c, a[k + 1])
    for k in range(L - 1, -1, -1):
        a[k] = _op_exp_heff(T, Lenv[k], w_ids[k], Renv[k], a[k], d[k], h, tol)
        if k > 0:
            a[k], c = _op_qr_left(T, a[k], (w_ids[k], a[k], Renv[k], d[k]))
            Renv[k - 1] = _op_env_right(T, Renv[k], a[k], w_ids[k], d[k])
            c = _op_exp_bond(T, Lenv[k], Renv[k - 1], c, -h, tol)
            a[k - 1] = _op_absorb_right(T, a[k - 1], c)
    return T, a, a_in, w_ids


def step_parameter_gradient(model, Wbars, mpo_builder) -> dict:
    """dl/dtheta for theta = omega_m, g_m, V from the MPO cotangents of a step: the MPO of
    Eq. 1 / Eq. 10 is affine in each parameter, so dW/dtheta = W(theta + 1) - W(theta)."""
    from .gradient import parameters, shifted
    W0 = mpo_builder(model)
    out = {}
    for p in parameters(model):
        W1 = mpo_builder(shifted(model, p, 1.0))
        out[p] = sum(float(np.vdot(b, w1 - w0).real) for b, w0, w1 in zip(Wbars, W0, W1))
    return out


# ---------------------------------------------------------------------------------
# real-time correlation: steps of both states and the overlaps, reversed with checkpoints
# ---------------------------------------------------------------------------------

def _overlap_with_tape(T, bra, w, ket, d):
    """<bra| W |ket> as a chain of left environment updates (Eq. 6 overlap, traced over P and
    Q by the fused sites); returns the id of the final 1 x 1 x 1 environment."""
    e = T.var(np.ones((1, 1, 1), dtype=complex))
    for k in range(len(bra)):
        Lk, B, Wk, K = T.vals[e], T.vals[bra[k]], T.vals[w[k]], T.vals[ket[k]]

        def vjp(bars, Lk=Lk, B=B, Wk=Wk, K=K, dk=d[k]):
            Lb, bb, Wb, kb = update_left_vjp(Lk, B, Wk, K, dk, bars[0])
            return [Lb, bb, Wb, kb]
        e = T.op([update_left(Lk, B, Wk, K, d[k])], [e, bra[k], w[k], ket[k]], vjp)[0]
    return e


def overlap_vjp(bra, Wj, ket, d, cbar):
    """(C, brabar, Wjbar, ketbar) of C = <bra| Wj |ket> for the cotangent cbar of C."""
    T = Tape()
    b = [T.var(x) for x in bra]
    w = [T.var(x) for x in Wj]
    k = [T.var(x) for x in ket]
    e = _overlap_with_tape(T, b, w, k, d)
    C = complex(T.vals[e][0, 0, 0])
    seed = np.zeros((1, 1, 1), dtype=complex)
    seed[0, 0, 0] = cbar
    bars = T.backward({e: seed})
    z = lambda i: bars.get(i, np.zeros_like(T.vals[i]))      # noqa: E731
    return C, [z(i) for i in b], [z(i) for i in w], [z(i) for i in k]


def correlation_vjp(Ws, Wj, d, psi1, psi2, dt, nsteps, cbar, every=2, tol=1e-14,
                    rank_tol=RANK_TOL):
    """C_n = <psi1(n dt)| j |psi2(n dt)>, n = 0 .. nsteps, both states evolved by the
    projector-splitting step exp(-i dt H); and the cotangents of psi1(0), psi2(0), of the
    H-MPO sites and of the j-MPO sites for the real loss Re sum_n conj(cbar_n) C_n.

    The states are stored every `every` steps on the forward pass; the backward pass
    recomputes each stretch of steps from its stored state, records it on a tape and
    reverses it (memory: nsteps / every stored states plus one stretch of tapes)."""
    tau = -1j * dt
    ckpt = {0: ([x.copy() for x in psi1], [x.copy() for x in psi2])}
    C = np.zeros(nsteps + 1, dtype=complex)
    s1, s2 = ckpt[0]
    for n in range(nsteps + 1):
        if n > 0:
            T1, o1, _, _ = step_with_tape(Ws, d, s1, tau, tol, rank_tol)
            T2, o2, _, _ = step_with_tape(Ws, d, s2, tau, tol, rank_tol)
            s1 = [T1.vals[i] for i in o1]
            s2 = [T2.vals[i] for i in o2]
            if n % every == 0:
                ckpt[n] = (s1, s2)
        C[n] = overlap_vjp(s1, Wj, s2, d, 0.0)[0]
    # reverse pass over the stretches between stored states, latest first
    Wbar = [np.zeros_like(np.asarray(W), dtype=complex) for W in Ws]
    Wjbar = [np.zeros_like(np.asarray(W), dtype=complex) for W in Wj]
    g1 = [np.zeros_like(x, dtype=complex) for x in psi1]
    g2 = [np.zeros_like(x, dtype=complex) for x in psi2]

    def add_overlap(n, a1, a2):
        nonlocal g1, g2, Wjbar
        _, b1, wjb, b2 = overlap_vjp(a1, Wj, a2, d, cbar[n])
        g1 = [x + y for x, y in zip(g1, b1)]
        g2 = [x + y for x, y in zip(g2, b2)]
        Wjbar = [x + y for x, y in zip(Wjbar, wjb)]

    cps = sorted(ckpt)
    segs = [(c, cps[i + 1] if i + 1 < len(cps) else nsteps) for i, c in enumerate(cps)]
    for s0, e0 in reversed([sg for sg in segs if sg[1] > sg[0]]):
        states = [ckpt[s0]]
        tapes = []
        for n in range(s0 + 1, e0 + 1):
            T1, o1, i1, w1 = step_with_tape(Ws, d, states[-1][0], tau, tol, rank_tol)
            T2, o2, i2, w2 = step_with_tape(Ws, d, states[-1][1], tau, tol, rank_tol)
            tapes.append((T1, o1, i1, w1, T2, o2, i2, w2))
            states.append(([T1.vals[i] for i in o1], [T2.vals[i] for i in o2]))
        for n in range(e0, s0, -1):
            add_overlap(n, *states[n - s0])
            T1, o1, i1, w1, T2, o2, i2, w2 = tapes[n - s0 - 1]
            bars1 = T1.backward(dict(zip(o1, g1)))
            bars2 = T2.backward(dict(zip(o2, g2)))
            g1 = [bars1.get(i, np.zeros_like(T1.vals[i])) for i in i1]
            g2 = [bars2.get(i, np.zeros_like(T2.vals[i])) for i in i2]
            Wbar = [x + bars1.get(a, 0) + bars2.get(b, 0) for x, a, b in zip(Wbar, w1, w2)]
    add_overlap(0, *ckpt[0])
    return C, g1, g2, Wbar, Wjbar


def qr_vjp_completed(Q, R, Qbar, Rbar, X):
    """VJP of the gauge QR with skipped columns (rows of R at completed positions are zero),
    with respect to Y and to the vectors X (m x |K|) that completed it.

    The completed columns are Gram-Schmidt residuals of the chosen candidates X against
    everything taken before them, so in processing order (accepted columns S first, then the
    completed ones K) the factorisation is the full-rank QR of Z = [Y_S | X] with
    R_Z = triu(Q_(S,K)^H Z), and R_S = Q_S^H Y.  The loss Re<Qbar, Q> + Re<Rbar_S, R_S> gives
        Zbar = qr_vjp(Q_(S,K), R_Z, [Qbar_S + Y Rbar_S^H | Qbar_K], 0),
        Ybar = Q_S Rbar_S + scatter_S(Zbar_S),   Xbar = Zbar_K.
    Returns (Ybar, Xbar)."""
    acc = np.abs(np.diag(R)) > 0
    S = np.flatnonzero(acc)
    K = np.flatnonzero(~acc)
    ns = len(S)
    Y = Q[:, S] @ R[S, :]
    Rb = np.triu(Rbar)
    order = np.concatenate([S, K])
    Qp = Q[:, order]
    Z = np.concatenate([Y[:, S], X], axis=1)
    Rp = np.triu(Qp.conj().T @ Z)
    Rp[:ns, :ns] = R[np.ix_(S, S)]
    Qbp = Qbar[:, order].astype(complex)
    Qbp[:, :ns] += Y @ Rb[S, :].conj().T
    Zbar = qr_vjp(Qp, Rp, Qbp, np.zeros_like(Rp))
    Ybar = Q[:, S] @ Rb[S, :]
    Ybar[:, S] += Zbar[:, :ns]
    return Ybar, Zbar[:, ns:]


def qr_vjp_selected(Q, R, Qbar, Rbar):
    """``qr_vjp_completed`` with the current completed columns Q_K themselves as the fixed
    candidates (every parameter value then gives a valid orthonormal gauge): R_Z has the
    identity in its K block.  Without skipped columns this equals ``qr_vjp``."""
    K = np.flatnonzero(~(np.abs(np.diag(R)) > 0))
    return qr_vjp_completed(Q, R, Qbar, Rbar, Q[:, K])[0]


def _canonicalize_with_tape(Ws, d, A_in, rank_tol=RANK_TOL):
    """``tdvp.PurifiedMPS.right_canonicalize`` on a tape: LQ shifts from the right end with
    the H coupling of each site as completion candidates, right environments on the way,
    the center ends at site 0.  Returns (tape, ids of the output sites, ids of the input
    sites, ids of the MPO sites)."""
    T = Tape(rank_tol)
    L = len(A_in)
    a_in = [T.var(np.asarray(x, dtype=complex)) for x in A_in]
    w_ids = [T.var(np.asarray(W)) for W in Ws]
    a = list(a_in)
    Renv = [None] * L
    Renv[L - 1] = T.var(np.ones((1, 1, 1), dtype=complex))
    for k in range(L - 1, 0, -1):
        a[k], c = _op_qr_left(T, a[k], (w_ids[k], a[k], Renv[k], d[k]))
        Renv[k - 1] = _op_env_right(T, Renv[k], a[k], w_ids[k], d[k])
        a[k - 1] = _op_absorb_right(T, a[k - 1], c)
    return T, a, a_in, w_ids


def _thermal_with_tapes(Ws, d, model, beta, dtau, M, tol, rank_tol=RANK_TOL):
    """``tdvp.thermal_state`` on tapes: the right-canonicalisation of |I> (theta enters its
    completed directions through W), then n = round(beta / (2 dtau)) steps exp(-dtau H), each
    followed by the normalisation of the center, log Z += log ||A_0||^2.  Returns (final
    normalised state, log Z, [(tape, output ids, input ids, MPO ids, ||A_0||)])."""
    from .tdvp import identity_state
    tapes = []
    T, out, inp, wids = _canonicalize_with_tape(Ws, d, identity_state(model, M), rank_tol)
    A = [T.vals[i] for i in out]
    nrm = np.linalg.norm(A[0])
    A[0] = A[0] / nrm
    logZ = 2.0 * np.log(nrm)
    tapes.append((T, out, inp, wids, nrm))
    for _ in range(int(round(beta / (2.0 * dtau)))):
        T, out, inp, wids = step_with_tape(Ws, d, A, -dtau, tol, rank_tol)
        A = [T.vals[i] for i in out]
        n = np.linalg.norm(A[0])
        logZ += 2.0 * np.log(n)
        A[0] = A[0] / n
        tapes.append((T, out, inp, wids, n))
    return A, logZ, tapes


def _thermal_reverse(tapes, Ws, state_bar, logz_bar):
    """Cotangents of the H-MPO sites for a loss with cotangent state_bar (or None) of the
    final normalised state and logz_bar of log Z.  Per tape, the normalisation
    A0n = A_0 / ||A_0|| has the VJP (abar - Re<A0n, abar> A0n) / ||A_0|| and log ||A_0||^2 the
    VJP 2 A_0 / ||A_0||^2; the input of the first tape (|I>) is a constant."""
    Wbar = [np.zeros_like(np.asarray(W), dtype=complex) for W in Ws]
    gbar = state_bar
    for T, out, inp, wids, n in reversed(tapes):
        A0 = T.vals[out[0]]
        A0n = A0 / n
        bar0 = logz_bar * 2.0 * A0 / n ** 2
        seeds = {}
        if gbar is not None:
            g0 = gbar[0]
            bar0 = bar0 + (g0 - np.vdot(A0n, g0).real * A0n) / n
            for i, g in zip(out[1:], gbar[1:]):
                seeds[i] = g
        seeds[out[0]] = bar0
        bars = T.backward(seeds)
        gbar = [bars.get(i, np.zeros_like(T.vals[i])) for i in inp]
        Wbar = [x + bars.get(wi, 0) for x, wi in zip(Wbar, wids)]
    return Wbar


def thermal_logz_gradient(model, beta, dtau, M, mpo_builder, tol=1e-14):
    """log Z of ``tdvp.thermal_state`` and dlogZ/dtheta (theta = omega_m, g_m, V) by reversing
    the canonicalisation and the imaginary-time steps on their tapes."""
    from .model import site_list
    Ws = mpo_builder(model)
    d = [s_[3] for s_ in site_list(model)]
    _, logZ, tapes = _thermal_with_tapes(Ws, d, model, beta, dtau, M, tol)
    Wbar = _thermal_reverse(tapes, Ws, None, 1.0)
    return logZ, step_parameter_gradient(model, Wbar, mpo_builder)


# ---------------------------------------------------------------------------------
# the whole C(t) pipeline: imaginary-time preparation, j fit, real-time steps, overlaps
# ---------------------------------------------------------------------------------

def _op_heff(T, l, w, r, a, d):
    """y = H_eff(L, W, R) A as a plain contraction (the fit's local projection)."""
    Lk, Wk, Rk, A = T.vals[l], T.vals[w], T.vals[r], T.vals[a]

    def vjp(bars):
        Ab, Lb, Wb, Rb = heff_vjp(Lk, Wk, Rk, A, d, bars[0])
        return [Lb, Wb, Rb, Ab]
    return T.op([heff(Lk, Wk, Rk, A, d)], [l, w, r, a], vjp)[0]


def _op_env_left2(T, l, bra, w, ket, d):
    Lk, B, Wk, K = T.vals[l], T.vals[bra], T.vals[w], T.vals[ket]

    def vjp(bars):
        Lb, bb, Wb, kb = update_left_vjp(Lk, B, Wk, K, d, bars[0])
        return [Lb, bb, Wb, kb]
    return T.op([update_left(Lk, B, Wk, K, d)], [l, bra, w, ket], vjp)[0]


def _op_env_right2(T, r, bra, w, ket, d):
    Rk, B, Wk, K = T.vals[r], T.vals[bra], T.vals[w], T.vals[ket]

    def vjp(bars):
        Rb, bb, Wb, kb = update_right_vjp(Rk, B, Wk, K, d, bars[0])
        return [Rb, bb, Wb, kb]
    return T.op([update_right(Rk, B, Wk, K, d)], [r, bra, w, ket], vjp)[0]


def fit_with_tape(Wop, d, psi, sweeps=2, rank_tol=RANK_TOL):
    """``tdvp.fit_apply`` (phi ~ Wop|psi> by one-site variational fitting) on a tape.
    Returns (tape, ids of phi, ids of psi, ids of the Wop sites)."""
    T = Tape(rank_tol)
    L = len(psi)
    p = [T.var(np.asarray(x, dtype=complex)) for x in psi]
    w = [T.var(np.asarray(x)) for x in Wop]
    phi = list(p)                                  # phi starts as psi
    one = np.ones((1, 1, 1), dtype=complex)
    Lf, Rf = [None] * L, [None] * L
    Lf[0] = T.var(one)
    Rf[L - 1] = T.var(one)
    for k in range(L - 1, 0, -1):
        Rf[k - 1] = _op_env_right2(T, Rf[k], phi[k], w[k], p[k], d[k])
    for _ in range(sweeps):
        for k in range(L):
            a = _op_heff(T, Lf[k], w[k], Rf[k], p[k], d[k])
            if k < L - 1:
                phi[k], _ = _op_qr_right(T, a, (Lf[k], w[k], p[k], d[k]))
                Lf[k + 1] = _op_env_left2(T, Lf[k], phi[k], w[k], p[k], d[k])
            else:
                phi[k] = a
        for k in range(L - 1, -1, -1):
            a = _op_heff(T, Lf[k], w[k], Rf[k], p[k], d[k])
            if k > 0:
                phi[k], _ = _op_qr_left(T, a, (w[k], p[k], Rf[k], d[k]))
                Rf[k - 1] = _op_env_right2(T, Rf[k], phi[k], w[k], p[k], d[k])
            else:
                phi[k] = a
    return T, phi, p, w


def correlation_pipeline_gradient(model, beta, dtau, M, dt, nsteps, cbar, mpo_h, mpo_j,
                                  every=2, tol=1e-14, rank_tol=RANK_TOL):
    """C_n (n = 0 .. nsteps) of the oracle pipeline (``tdvp.correlation`` with fit_sweeps=2)
    and dl/dtheta for l = Re sum_n conj(cbar_n) C_n: the real-time reverse pass, then the
    j fit, then the imaginary-time preparation, with the MPO cotangents of H and j mapped
    to omega_m, g_m, V.

    The gauge QRs use rank_tol.  Where a bond is wider than the rank of the state (the
    one-carrier sector at full bond dimension), columns whose exact residual is zero come out
    of Gram-Schmidt at rounding size; with the default 1e-12 some of them are accepted,
    their direction is set by rounding, and R^{-1} in the QR VJP amplifies it.  A threshold
    above rounding (1e-8) completes them from the candidates instead and keeps the reverse
    pass conditioned; the forward C then moves by the dropped residuals only."""
    from .model import site_list
    d = [s_[3] for s_ in site_list(model)]
    Ws, Wj = mpo_h(model), mpo_j(model)
    psi, _, ttapes = _thermal_with_tapes(Ws, d, model, beta, dtau, M, tol, rank_tol)
    Tf, phi_ids, psi_ids, wj_ids = fit_with_tape(Wj, d, psi, rank_tol=rank_tol)
    phi = [Tf.vals[i] for i in phi_ids]
    C, g1, g2, Wb, Wjb = correlation_vjp(Ws, Wj, d, psi, phi, dt, nsteps, cbar, every, tol,
                                         rank_tol)
    # the fit: phi = fit(Wj, psi)
    fb = Tf.backward(dict(zip(phi_ids, g2)))
    gpsi = [x + fb.get(i, np.zeros_like(x)) for x, i in zip(g1, psi_ids)]
    Wjb = [x + fb.get(i, 0) for x, i in zip(Wjb, wj_ids)]
    # the preparation
    Wb2 = _thermal_reverse(ttapes, Ws, gpsi, 0.0)
    Wb = [x + y for x, y in zip(Wb, Wb2)]
    gH = step_parameter_gradient(model, Wb, mpo_h)
    gJ = step_parameter_gradient(model, Wjb, mpo_j)
    return C, {p: gH[p] + gJ[p] for p in gH}


def mobility_pipeline_gradient(model, kT, dtau, M, dt, nsteps, mpo_h, mpo_j, every=2,
                               tol=1e-14, rank_tol=RANK_TOL):
    """mu of Eq. 2 from the oracle pipeline's C_n (t_n = n dt, n <= nsteps; trapezoid, cut off
    at nsteps dt) and dmu/dtheta.  mu = (1 / 2kT) 2 int_0^{t_max} Re C dt is linear in Re C_n,
    mu = sum_n w_n Re C_n with w_n = dt / kT (half at both ends), so dmu/dtheta is the
    pipeline gradient for the real cotangent cbar_n = w_n."""
    w = np.full(nsteps + 1, dt / kT)
    w[0] *= 0.5
    w[-1] *= 0.5
    C, g = correlation_pipeline_gradient(model, 1.0 / kT, dtau, M, dt, nsteps, w + 0j, mpo_h,
                                         mpo_j, every, tol, rank_tol)
    return float(np.sum(w * C.real)), g
