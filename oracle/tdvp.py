"""Plain FP64 purified-MPS TD-DMRG with one-site TDVP projector splitting (oracle part ii).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

What it follows:
* Eq. S1: the MPS  |Psi> = sum A^{s1}_{a1} A^{s2}_{a1 a2} ... |s1 s2 ...>.
* Eq. 4-5 (purification): every degree of freedom carries a physical index (P) and an
  ancilla copy (Q); the thermal state is Psi_beta = exp(-beta H / 2)|I>, |I> = sum_i |i>_P|i>_Q,
  restricted to the one-carrier sector.  H acts on P only.  Here P and Q of one degree of
  freedom share one MPS site with fused index s = sigma * d + tau.
* Eq. 6: C(t) = <Psi_beta| e^{iHt} j e^{-iHt} j |Psi_beta> / Z, both states propagated in
  real time, the overlap traced over P and Q.
* Time evolution: the one-site TDVP projector-splitting integrator the paper uses (its ref.
  Haegeman et al. 2016), second-order symmetric form: a left-to-right half-sweep with half a
  step on every site and a backward bond step between sites, then the mirror sweep.

Readings where the paper is silent (each also listed in the design notes):
* bond dimensions M_k = min(M, prod of local dims left of bond k, prod right of it);
* the bond-2 start state |I> is zero padded to M_k; rank-deficient gauge shifts are
  completed deterministically by ``gauge_qr`` (Gram-Schmidt with skipped columns, then the
  unit vectors e_0, e_1, ... in index order);
* Krylov exponential: Lanczos with full re-orthogonalisation, stopped when
  beta_k |(exp(tau T_k) e_1)_k| < tol, or after a fixed number of vectors;
* the imaginary-time state is normalised after every step (log Z accumulated);
* j|Psi_beta> is compressed to the bond dimensions of Psi_beta by one-site variational
  fitting (two left-right + right-left sweeps) starting from Psi_beta itself.

Everything uses numpy tensordot / linalg; no blocking or fusion.
"""
import math
from dataclasses import dataclass
from typing import List, Optional

import numpy as np

from .model import HolsteinModel, mpo_current, mpo_hamiltonian, site_list

RANK_TOL = 1e-12      # column skipped if its residual norm <= RANK_TOL * ||Y||_F
COMPLETE_TOL = 1e-2   # unit vector e_i used for completion if its residual norm > this


# ---------------------------------------------------------------------------------
# gauge QR with deterministic completion
# ---------------------------------------------------------------------------------

def gauge_qr(Y: np.ndarray, extra: Optional[np.ndarray] = None,
             rank_tol: float = RANK_TOL, complete_tol: float = COMPLETE_TOL,
             chosen: Optional[list] = None):
    """Y (m x n, m >= n) = Q R with Q^H Q = I.

    Column j of Q is the Gram-Schmidt residual of Y[:, j] against the accepted earlier
    columns (computed twice), normalised, when its norm exceeds rank_tol * ||Y||_F; R_jj is
    then real and positive.  Skipped positions are filled, in increasing order, first by the
    columns of ``extra`` (m x p candidate directions, e.g. what the Hamiltonian couples the
    current state into) and then by the unit vectors e_0, e_1, ..., each projected against
    everything already in Q and taken when its residual norm exceeds complete_tol times its
    own norm.  R = Q^H Y, except that the rows of completed positions are set to zero
    (their entries are residuals below rank_tol * ||Y||_F, which the Gram-Schmidt
    coefficients of the skipped columns do not carry).

    If ``chosen`` is a list, the source of each completed position is appended to it, in
    increasing position order: i < p for column i of ``extra``, p + i for e_i.
    """
    m, n = Y.shape
    assert m >= n
    thr = rank_tol * np.linalg.norm(Y)
    Q = np.zeros((m, n), dtype=complex)
    B = np.zeros((m, n), dtype=complex)      # the columns of Q taken so far, in the order taken
    nb = 0
    have = set()

    def residual(v):
        for _ in range(2):
            if nb:
                Bv = B[:, :nb]
                v = v - Bv @ (Bv.conj().T @ v)
        return v

    for j in range(n):
        r = residual(Y[:, j].astype(complex))
        nr = np.linalg.norm(r)
        if nr > thr:
            Q[:, j] = r / nr
            B[:, nb] = Q[:, j]
            nb += 1
            have.add(j)

    p = 0 if extra is None else extra.shape[1]

    def candidates():
        for i in range(p):
            yield i, extra[:, i].astype(complex)
        for i in range(m):
            e = np.zeros(m, dtype=complex)
            e[i] = 1.0
            yield p + i, e

    gen = candidates()
    completed = []
    for j in range(n):
        if j in have:
            continue
        completed.append(j)
        while True:
            src, c = next(gen, (None, None))
            if c is None:
                raise RuntimeError("gauge_qr: ran out of completion vectors")
            n0 = np.linalg.norm(c)
            if n0 == 0.0:
                continue
            c = residual(c)
            nc = np.linalg.norm(c)
            if nc > complete_tol * n0:
                Q[:, j] = c / nc
                B[:, nb] = Q[:, j]
                nb += 1
                have.add(j)
                if chosen is not None:
                    chosen.append(src)
                break
    R = Q.conj().T @ Y
    R[completed, :] = 0.0
    return Q, R


# ---------------------------------------------------------------------------------
# MPS helpers
# ---------------------------------------------------------------------------------

def bond_dims(D: List[int], M: int) -> List[int]:
    """M_0 .. M_L with M_k = min(M, prod(D[:k]), prod(D[k:]))."""
    L = len(D)
    out = []
    for k in range(L + 1):
        left = math.prod(D[:k])
        right = math.prod(D[k:])
        out.append(min(M, left, right))
    return out


def identity_state(model: HolsteinModel, M: int) -> List[np.ndarray]:
    """|I> = sum_i |i>_P |i>_Q on the one-carrier sector (Eq. 5 start state), padded to M_k.

    Unpadded it has bond dimension 2: channel 0 'carrier not yet placed', 1 'placed'."""
    sites = site_list(model)
    d = [s[3] for s in sites]
    D = [x * x for x in d]
    Mk = bond_dims(D, M)
    L = len(sites)
    mps = []
    for k, (kind, n, m, dk) in enumerate(sites):
        T = np.zeros((2, dk * dk, 2), dtype=complex)
        if kind == "e":
            T[0, 0 * dk + 0, 0] = 1.0      # empty molecule, no carrier yet
            T[0, 1 * dk + 1, 1] = 1.0      # carrier here (P and Q)
            T[1, 0 * dk + 0, 1] = 1.0      # empty molecule, carrier already placed
        else:
            for c in range(2):
                for v in range(dk):
                    T[c, v * dk + v, c] = 1.0
        a_ch = [0] if k == 0 else [0, 1]
        b_ch = [1] if k == L - 1 else [0, 1]
        A = np.zeros((Mk[k], D[k], Mk[k + 1]), dtype=complex)
        for ia, ca in enumerate(a_ch):
            for ib, cb in enumerate(b_ch):
                A[ia, :, ib] = T[ca, :, cb]
        mps.append(A)
    return mps


def mps_to_dense(mps: List[np.ndarray]) -> np.ndarray:
    """Full coefficient vector in the fused (P,Q) site basis (tiny chains only)."""
    v = mps[0][0]                     # [s, b]
    for A in mps[1:]:
        v = np.einsum("xb,bsc->xsc", v, A).reshape(-1, A.shape[2])
    return v[:, 0]


# ---------------------------------------------------------------------------------
# environments and effective Hamiltonians
# ---------------------------------------------------------------------------------

def _split(A: np.ndarray, d: int) -> np.ndarray:
    """A[a, s, b] -> A[a, sigma, tau, b]."""
    return A.reshape(A.shape[0], d, d, A.shape[2])


def update_left(Lenv, bra, W, ket, d):
    """L'[w', b, c] = sum conj(bra[a,s,t,b]) L[w,a,y] W[w,w',s,u] ket[y,u,t,c].

    Contracted in the order written: ket with L, then W, then the conjugate bra."""
    K = _split(ket, d)
    X = np.tensordot(Lenv, K, axes=([2], [0]))            # [w, a, u, t, c]
    Y = np.tensordot(W, X, axes=([0, 3], [0, 2]))         # [w', s, a, t, c]
    B = _split(bra, d).conj()                              # [a, s, t, b]
    return np.tensordot(Y, B, axes=([2, 1, 3], [0, 1, 2])).transpose(0, 2, 1)  # [w', b, c]


def update_right(Renv, bra, W, ket, d):
    """R'[w, a, y] = sum conj(bra[a,s,t,b]) R[w',b,c] W[w,w',s,u] ket[y,u,t,c]."""
    K = _split(ket, d)
    X = np.tensordot(K, Renv, axes=([3], [2]))            # [y, u, t, w', b]
    Y = np.tensordot(W, X, axes=([1, 3], [3, 1]))         # [w, s, y, t, b]
    B = _split(bra, d).conj()                              # [a, s, t, b]
    return np.tensordot(Y, B, axes=([1, 3, 4], [1, 2, 3])).transpose(0, 2, 1)  # [w, a, y]


def heff(Lenv, W, Renv, A, d):
    """(H_eff A)[x,s,t,b] = sum L[w,x,y] W[w,v,s,u] A[y,u,t,c] R[v,b,c]; t (ancilla) is a spectator.

    Order: X = L A, Y = W X (mixes MPO channel and physical level), out = Y R."""
    X = np.tensordot(Lenv, _split(A, d), axes=([2], [0]))  # [w, x, u, t, c]
    Y = np.tensordot(W, X, axes=([0, 3], [0, 2]))          # [v, s, x, t, c]
    out = np.tensordot(Y, Renv, axes=([0, 4], [0, 2]))     # [s, x, t, b]
    return out.transpose(1, 0, 2, 3).reshape(A.shape)


def bond_heff(Lenv, Renv, C):
    """(K C)[x, b] = sum L[w,x,y] C[y,c] R[w,b,c] (zero-site effective Hamiltonian)."""
    X = np.tensordot(Lenv, C, axes=([2], [0]))             # [w, x, c]
    return np.tensordot(X, Renv, axes=([0, 2], [0, 2]))    # [x, b]


def left_expansion(Lenv, W, A, d):
    """Completion candidates for a left-to-right gauge shift: the columns of
    P[(x,s,t), (v,c)] = sum L[w,x,y] W[w,v,s,u] A[y,u,t,c] (H_eff without its right
    environment), column order v (MPO channel) outer, c inner."""
    X = np.tensordot(Lenv, _split(A, d), axes=([2], [0]))  # [w, x, u, t, c]
    Y = np.tensordot(W, X, axes=([0, 3], [0, 2]))          # [v, s, x, t, c]
    Y = Y.transpose(2, 1, 3, 0, 4)                          # [x, s, t, v, c]
    return Y.reshape(A.shape[0] * A.shape[1], -1)


def right_expansion(W, A, Renv, d):
    """Completion candidates for a right-to-left gauge shift (columns of Y = A^H): the
    conjugated rows of P[(w,y), (s,t,b)] = sum W[w,v,s,u] A[y,u,t,c] R[v,b,c],
    row order w outer, y inner."""
    X = np.tensordot(_split(A, d), Renv, axes=([3], [2]))  # [y, u, t, v, b]
    Y = np.tensordot(W, X, axes=([1, 3], [3, 1]))          # [w, s, y, t, b]
    Y = Y.transpose(0, 2, 1, 3, 4)                          # [w, y, s, t, b]
    P = Y.reshape(-1, A.shape[1] * A.shape[2])
    return P.conj().T


# ---------------------------------------------------------------------------------
# Krylov exponential
# ---------------------------------------------------------------------------------

def krylov_expm(matvec, v, tau: complex, tol: float = 1e-13, kmax: int = 32,
                fixed_k: Optional[int] = None):
    """exp(tau H) v by Lanczos with full re-orthogonalisation (H Hermitian).

    Returns (result, number of Krylov vectors used)."""
    v = np.asarray(v, dtype=complex)
    n = v.size
    b0 = np.linalg.norm(v)
    if b0 == 0.0:
        return v.copy(), 0
    cap = min(fixed_k if fixed_k is not None else kmax, n)
    Q = [v.reshape(-1) / b0]
    alpha, beta = [], []
    c = None
    for j in range(cap):
        w = matvec(Q[j].reshape(v.shape)).reshape(-1)
        Qm = np.array(Q)
        h = Qm.conj() @ w
        w = w - Qm.T @ h
        h2 = Qm.conj() @ w
        w = w - Qm.T @ h2
        alpha.append(float((h[j] + h2[j]).real))
        b = float(np.linalg.norm(w))
        k = j + 1
        T = np.diag(alpha) + np.diag(beta, 1) + np.diag(beta, -1)
        lam, U = np.linalg.eigh(T)                      # T real symmetric tridiagonal
        c = U @ (np.exp(tau * lam) * U[0, :])           # exp(tau T) e_1
        scale = max(abs(x) for x in alpha + beta + [1e-300])
        breakdown = b <= 1e-12 * scale
        if breakdown or k == cap:
            break
        if fixed_k is None and b * abs(c[-1]) < tol:
            break
        beta.append(b)
        Q.append(w / b)
    k = len(alpha)
    out = b0 * (np.array(Q[:k]).T @ c)
    return out.reshape(v.shape), k


# ---------------------------------------------------------------------------------
# TDVP state
# ---------------------------------------------------------------------------------

@dataclass
class KrylovOpts:
    tol: float = 1e-13
    kmax: int = 32
    fixed_k: Optional[int] = None


class PurifiedMPS:
    """Purified MPS with cached environments for one MPO (center kept at site 0 between steps)."""

    def __init__(self, model: HolsteinModel, tensors: List[np.ndarray], Ws: List[np.ndarray]):
        self.model = model
        self.d = [s[3] for s in site_list(model)]
        self.A = [t.copy() for t in tensors]
        self.W = Ws
        self.L = len(self.A)
        self.Lenv = [None] * self.L
        self.Renv = [None] * self.L

    def right_canonicalize(self):
        """LQ shifts from the right end (completion from the H coupling of each site), building
        the right environments on the way; the center ends at site 0."""
        self.Lenv[0] = np.ones((1, 1, 1), dtype=complex)
        self.Renv[self.L - 1] = np.ones((1, 1, 1), dtype=complex)
        for k in range(self.L - 1, 0, -1):
            C = self._shift_left(k)
            self.A[k - 1] = np.einsum("asb,bc->asc", self.A[k - 1], C)

    def _shift_left(self, k):
        """A_k = C Q (Q right-orthonormal); returns C and updates Renv[k-1]."""
        A = self.A[k]
        Ml, Ds, Mr = A.shape
        extra = right_expansion(self.W[k], A, self.Renv[k], self.d[k])
        Q, R = gauge_qr(A.reshape(Ml, Ds * Mr).conj().T, extra)
        self.A[k] = Q.conj().T.reshape(Ml, Ds, Mr)
        self.Renv[k - 1] = update_right(self.Renv[k], self.A[k], self.W[k], self.A[k], self.d[k])
        return R.conj().T

    def _shift_right(self, k):
        """A_k = Q C (Q left-orthonormal); returns C and updates Lenv[k+1]."""
        A = self.A[k]
        Ml, Ds, Mr = A.shape
        extra = left_expansion(self.Lenv[k], self.W[k], A, self.d[k])
        Q, R = gauge_qr(A.reshape(Ml * Ds, Mr), extra)
        self.A[k] = Q.reshape(Ml, Ds, Mr)
        self.Lenv[k + 1] = update_left(self.Lenv[k], self.A[k], self.W[k], self.A[k], self.d[k])
        return R

    def build_right_envs(self):
        """Right environments of an MPS whose sites 1..L-1 are already right-orthonormal."""
        self.Lenv[0] = np.ones((1, 1, 1), dtype=complex)
        self.Renv[self.L - 1] = np.ones((1, 1, 1), dtype=complex)
        for k in range(self.L - 1, 0, -1):
            self.Renv[k - 1] = update_right(self.Renv[k], self.A[k], self.W[k], self.A[k], self.d[k])

    def norm(self) -> float:
        return float(np.linalg.norm(self.A[0]))   # center at site 0

    def step(self, tau: complex, kopts: KrylovOpts, stats=None, on_site=None):
        """One second-order projector-splitting step exp(tau H) (tau = -i dt or -dtau).

        ``on_site`` (optional) is called after every site update (used to time a bounded
        sample of site updates)."""
        h = 0.5 * tau
        L = self.L
        # left to right
        for k in range(L):
            self._site(k, h, kopts, stats, on_site)
            if k < L - 1:
                C = self._shift_right(k)
                Lk, Rk = self.Lenv[k + 1], self.Renv[k]
                C, _ = krylov_expm(lambda x: bond_heff(Lk, Rk, x), C, -h, kopts.tol,
                                   kopts.kmax, kopts.fixed_k)
                self.A[k + 1] = np.einsum("ab,bsc->asc", C, self.A[k + 1])
        # right to left
        for k in range(L - 1, -1, -1):
            self._site(k, h, kopts, stats, on_site)
            if k > 0:
                C = self._shift_left(k)
                Lk, Rk = self.Lenv[k], self.Renv[k - 1]
                C, _ = krylov_expm(lambda x: bond_heff(Lk, Rk, x), C, -h, kopts.tol,
                                   kopts.kmax, kopts.fixed_k)
                self.A[k - 1] = np.einsum("asb,bc->asc", self.A[k - 1], C)

    def _site(self, k, h, kopts, stats, on_site=None):
        Lk, Rk, Wk, dk = self.Lenv[k], self.Renv[k], self.W[k], self.d[k]
        self.A[k], used = krylov_expm(lambda x: heff(Lk, Wk, Rk, x, dk), self.A[k], h,
                                      kopts.tol, kopts.kmax, kopts.fixed_k)
        if stats is not None:
            stats.append(used)
        if on_site is not None:
            on_site()


def overlap(bra: List[np.ndarray], Ws: List[np.ndarray], ket: List[np.ndarray], d: List[int]) -> complex:
    """<bra| W |ket> traced over P and Q by a left-to-right transfer contraction."""
    E = np.ones((1, 1, 1), dtype=complex)
    for k in range(len(bra)):
        E = update_left(E, bra[k], Ws[k], ket[k], d[k])
    return complex(E[0, 0, 0])


def reduced_density(model: HolsteinModel, mps: List[np.ndarray]) -> np.ndarray:
    """sigma_ij = <psi| c+_j c_i |psi> / <psi|psi> (Eq. 9 from a purified MPS), one overlap with
    an operator MPO per entry: c_i and c+_j on the P index of the electronic sites of molecules
    i and j (n_i when i = j), the identity elsewhere (hard-core carrier: no string)."""
    sites = site_list(model)
    d = [s[3] for s in sites]
    I = identity_mpo(model)
    norm = overlap(mps, I, mps, d)
    c = np.array([[0.0, 1.0], [0.0, 0.0]])          # |1> -> |0>
    N = model.N
    sig = np.zeros((N, N), dtype=complex)
    for i in range(N):
        for j in range(N):
            W = [w.copy() for w in I]
            for k, (kind, n, _, _) in enumerate(sites):
                if kind != "e":
                    continue
                op = np.eye(2)
                if n == i:
                    op = c @ op
                if n == j:
                    op = c.T @ op
                W[k] = op.astype(complex)[None, None]
            sig[i, j] = overlap(mps, W, mps, d) / norm
    return sig


def identity_mpo(model: HolsteinModel) -> List[np.ndarray]:
    return [np.eye(s[3], dtype=complex)[None, None] for s in site_list(model)]


def fit_apply(model, Wop, psi: List[np.ndarray], sweeps: int = 2) -> List[np.ndarray]:
    """phi ~ Wop|psi> with the bond dimensions of psi, by one-site variational fitting.

    psi must have its center at site 0 and right-canonical sites 1..L-1; phi starts as psi.
    Each site is set to the exact projection of Wop|psi> on phi's orthonormal environment."""
    d = [s[3] for s in site_list(model)]
    L = len(psi)
    phi = [t.copy() for t in psi]
    Lf = [None] * L
    Rf = [None] * L
    Lf[0] = np.ones((1, 1, 1), dtype=complex)
    Rf[L - 1] = np.ones((1, 1, 1), dtype=complex)
    for k in range(L - 1, 0, -1):
        Rf[k - 1] = update_right(Rf[k], phi[k], Wop[k], psi[k], d[k])
    for _ in range(sweeps):
        for k in range(L):
            A = heff(Lf[k], Wop[k], Rf[k], psi[k], d[k])
            if k < L - 1:
                Ml, Ds, Mr = A.shape
                extra = left_expansion(Lf[k], Wop[k], psi[k], d[k])
                Q, _ = gauge_qr(A.reshape(Ml * Ds, Mr), extra)
                phi[k] = Q.reshape(Ml, Ds, Mr)
                Lf[k + 1] = update_left(Lf[k], phi[k], Wop[k], psi[k], d[k])
            else:
                phi[k] = A
        for k in range(L - 1, -1, -1):
            A = heff(Lf[k], Wop[k], Rf[k], psi[k], d[k])
            if k > 0:
                Ml, Ds, Mr = A.shape
                extra = right_expansion(Wop[k], psi[k], Rf[k], d[k])
                Q, _ = gauge_qr(A.reshape(Ml, Ds * Mr).conj().T, extra)
                phi[k] = Q.conj().T.reshape(Ml, Ds, Mr)
                Rf[k - 1] = update_right(Rf[k], phi[k], Wop[k], psi[k], d[k])
            else:
                phi[k] = A
    return phi


# ---------------------------------------------------------------------------------
# the whole C(t) computation
# ---------------------------------------------------------------------------------

@dataclass
class CorrelationResult:
    t: np.ndarray
    C: np.ndarray
    logZ: float
    norm1: np.ndarray       # <Psi1|Psi1> along t (Z-normalised: 1)
    norm2: np.ndarray       # <Psi2|Psi2> along t (= C(0))
    energy: np.ndarray      # <Psi1|H|Psi1>
    krylov: List[int]


def thermal_state(model: HolsteinModel, beta: float, dtau: float, M: int,
                  kopts: Optional[KrylovOpts] = None):
    """Psi_beta = exp(-beta H/2)|I> (Eq. 5) by n = round(beta/(2 dtau)) imaginary steps.

    Returns the normalised state (center at site 0, environments for H built) and log Z."""
    kopts = kopts or KrylovOpts()
    WH = mpo_hamiltonian(model)
    psi = PurifiedMPS(model, identity_state(model, M), WH)
    psi.right_canonicalize()
    nrm = psi.norm()
    psi.A[0] = psi.A[0] / nrm
    logZ = 2.0 * math.log(nrm)
    nsteps = int(round(beta / (2.0 * dtau)))
    if abs(nsteps * 2.0 * dtau - beta) > 1e-9 * max(1.0, beta):
        raise ValueError("beta must be an even multiple of dtau")
    for _ in range(nsteps):
        psi.step(-dtau, kopts)
        nrm = psi.norm()
        psi.A[0] = psi.A[0] / nrm
        logZ += 2.0 * math.log(nrm)
    return psi, logZ


def correlation(model: HolsteinModel, beta: float, dtau: float, M: int, dt: float,
                nsteps: int, every: int = 1, kopts: Optional[KrylovOpts] = None,
                fit_sweeps: int = 2, observe: bool = False) -> CorrelationResult:
    """C(t) of Eq. 6 at t = 0, every*dt, ..., nsteps*dt."""
    kopts = kopts or KrylovOpts()
    psi, logZ = thermal_state(model, beta, dtau, M, kopts)
    WH = psi.W
    Wj = mpo_current(model)
    d = psi.d
    phi = fit_apply(model, Wj, psi.A, sweeps=fit_sweeps)
    s1 = psi
    s2 = PurifiedMPS(model, phi, WH)
    s2.build_right_envs()
    ts, Cs, n1, n2, en, kr = [], [], [], [], [], []
    I = identity_mpo(model)

    def record(i):
        ts.append(i * dt)
        Cs.append(overlap(s1.A, Wj, s2.A, d))
        if observe:
            n1.append(overlap(s1.A, I, s1.A, d).real)
            n2.append(overlap(s2.A, I, s2.A, d).real)
            en.append(overlap(s1.A, WH, s1.A, d).real)

    record(0)
    for i in range(1, nsteps + 1):
        s1.step(-1j * dt, kopts, kr)
        s2.step(-1j * dt, kopts, kr)
        if i % every == 0:
            record(i)
    return CorrelationResult(np.array(ts), np.array(Cs), logZ, np.array(n1), np.array(n2),
                             np.array(en), kr)
