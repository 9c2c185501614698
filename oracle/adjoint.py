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
* ``expm_krylov_vjp`` -- y = exp(tau H) v for a Hermitian H given as a linear map:
  vbar = exp(conj(tau) H) ybar, and the cotangent of H as the integral
  Hbar = conj(tau) int_0^1 a(s) b(s)^H ds,  a(s) = exp((1-s) conj(tau) H) ybar,
  b(s) = exp(s tau H) v  (from d exp(X)[E] = int_0^1 e^{(1-s)X} E e^{sX} ds), evaluated by
  Gauss-Legendre quadrature and returned as weighted pairs (c_s, b_s) with
  Hbar = sum_s c_s b_s^H, which the caller maps to L, W, R through the VJPs above.  The
  energy offset of H cancels between a(s) and b(s), so the integrand varies on the scale of
  |tau| times the spread of the spectrum; 16 nodes integrate it to rounding for
  |tau| spread <= 5.
"""
from typing import Callable, List, Tuple

import numpy as np

from .tdvp import _split, krylov_expm


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
