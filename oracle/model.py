"""Model definition for the oracle: the periodic multi-mode Holstein(-Peierls) chain.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Paper passages restated here:
* Eq. 1: H = V sum_n (c+_{n+1} c_n + c+_n c_{n+1}) + sum_{n,m} w_m b+ b
             + sum_{n,m} g_m w_m (b+ + b) c+_n c_n        (periodic chain, one carrier)
* Eq. 3: j = (e0 V R / i) sum_n (c+_{n+1} c_n - c+_n c_{n+1})  (e0 = R = hbar = 1 here)
* Eq. 10 (Holstein-Peierls): one intermolecular mode per bond modulates the transfer
  integral.  Reading used here: V_n = V (1 + alpha (b_p + b_p^+)) on bond (n, n+1),
  and j = i[H, P] with P the carrier position, i.e. Eq. 3 with V -> V_n.

Site order along the MPS (Eq. S1): for each molecule n the electronic two-level site
e_n, then its K intramolecular modes v_{n,1..K}, then (Holstein-Peierls only) the
bond mode p_n of bond (n, n+1 mod N).

MPO convention: W[wl, wr, s, s'] with s the output (bra) and s' the input (ket) level of
the physical (P) index.  The first site only uses row 0, the last only the last column.
"""
from dataclasses import dataclass
from typing import List, Optional, Tuple

import numpy as np


@dataclass
class HolsteinModel:
    """Parameters of Eq. 1 (and Eq. 10 when ``alpha`` is not None)."""
    N: int
    omega: List[float]
    g: List[float]
    nmax: List[int]
    V: float
    alpha: Optional[float] = None      # Peierls modulation of V (Eq. 10 reading)
    omega_p: float = 0.2               # frequency of the bond mode
    nmax_p: int = 8                    # levels of the bond mode

    def __post_init__(self):
        if self.N < 3:
            raise ValueError("periodic chain needs N >= 3 (each bond counted once)")
        if not (len(self.omega) == len(self.g) == len(self.nmax)):
            raise ValueError("omega, g, nmax must have one entry per mode")

    @property
    def K(self) -> int:
        return len(self.omega)

    @property
    def peierls(self) -> bool:
        return self.alpha is not None


def site_list(model: HolsteinModel) -> List[Tuple[str, int, int, int]]:
    """Sites of the MPS in chain order: (kind, molecule n, mode m, levels d)."""
    sites = []
    for n in range(model.N):
        sites.append(("e", n, -1, 2))
        for m in range(model.K):
            sites.append(("v", n, m, int(model.nmax[m])))
        if model.peierls:
            sites.append(("p", n, -1, int(model.nmax_p)))
    return sites


# ---- local operators (truncated harmonic oscillator basis, two-level electron) ----

def op_b(d: int) -> np.ndarray:
    """Boson annihilator in the lowest d number states: b|v> = sqrt(v)|v-1>."""
    b = np.zeros((d, d))
    for v in range(1, d):
        b[v - 1, v] = np.sqrt(v)
    return b


def op_x(d: int) -> np.ndarray:
    b = op_b(d)
    return b + b.T


def op_num(d: int) -> np.ndarray:
    return np.diag(np.arange(d, dtype=float))


C_DAG = np.array([[0.0, 0.0], [1.0, 0.0]])   # |1><0| : puts the carrier on the molecule
C_ANN = np.array([[0.0, 1.0], [0.0, 0.0]])   # |0><1|
N_E = np.diag([0.0, 1.0])


# ---- MPO of H (Eq. 1 / Eq. 10) ----------------------------------------------------
# Channels of the finite-state automaton (bond dimension 7):
#   S  identities so far          F  a whole term has been placed
#   Cd c+_n placed, waiting for c_{n+1}       C  c_n placed, waiting for c+_{n+1}
#   Ne n_e(n) placed, waiting for one of molecule n's modes
#   Wd c+_1 placed, waiting for c_N (wrap-around bond)   Wc c_1 placed, waiting for c+_N
S, CD, CA, NE, WD, WC, F = range(7)


def mpo_hamiltonian(model: HolsteinModel) -> List[np.ndarray]:
    """MPO tensors of Eq. 1 (Eq. 10 with a bond mode) in the site order of ``site_list``."""
    N, V = model.N, model.V
    sites = site_list(model)
    Ws = []
    for (kind, n, m, d) in sites:
        I = np.eye(d)
        W = np.zeros((7, 7, d, d), dtype=complex)
        W[S, S] = I
        W[F, F] = I
        if kind == "e":
            hop = 1.0 if model.peierls else V       # with a bond mode, V sits on p_n
            if n < N - 1:
                W[S, CD] = hop * C_DAG
                W[S, CA] = hop * C_ANN
            if n > 0:
                W[CD, F] = C_ANN
                W[CA, F] = C_DAG
            if n == 0:
                W[S, WD] = hop * C_DAG
                W[S, WC] = hop * C_ANN
            elif n == N - 1:
                if model.peierls:   # wrap term still has to pass p_N
                    W[WD, WD] = C_ANN
                    W[WC, WC] = C_DAG
                else:
                    W[WD, F] = C_ANN
                    W[WC, F] = C_DAG
            else:
                W[WD, WD] = I
                W[WC, WC] = I
            W[S, NE] = N_E
        elif kind == "v":
            w, gm = model.omega[m], model.g[m]
            for ch in (CD, CA, WD, WC, NE):
                W[ch, ch] = I
            W[S, F] = w * op_num(d)
            W[NE, F] = gm * w * op_x(d)
        else:  # bond mode p_n (Eq. 10 reading)
            Vn = V * (I + model.alpha * op_x(d))
            W[S, F] = model.omega_p * op_num(d)
            W[NE, NE] = 0.0 * I
            if n < N - 1:
                # carried hopping of bond (n, n+1): c+_n / c_n placed at e_n
                W[CD, CD] = Vn
                W[CA, CA] = Vn
            else:
                # last bond mode closes the wrap-around term (c+_1 c_N and c+_N c_1)
                W[WD, F] = Vn
                W[WC, F] = Vn
            if n < N - 1:
                W[WD, WD] = I
                W[WC, WC] = I
        Ws.append(W)
    Ws[0] = Ws[0][S:S + 1]
    Ws[-1] = Ws[-1][:, F:F + 1]
    return Ws


# ---- MPO of the current operator (Eq. 3) ----------------------------------------
# Channels (bond dimension 6): S, Cd, Ca, Wd, Wc, F (same meaning as above)
JS, JCD, JCA, JWD, JWC, JF = range(6)


def mpo_current(model: HolsteinModel) -> List[np.ndarray]:
    """MPO of j = (V/i) sum_n (c+_{n+1} c_n - c+_n c_{n+1}), wrap bond included."""
    N, V = model.N, model.V
    sites = site_list(model)
    Ws = []
    for (kind, n, m, d) in sites:
        I = np.eye(d)
        W = np.zeros((6, 6, d, d), dtype=complex)
        W[JS, JS] = I
        W[JF, JF] = I
        hop = 1.0 if model.peierls else V
        if kind == "e":
            if n < N - 1:
                W[JS, JCD] = (1j * hop) * C_DAG     # + iV c+_n c_{n+1}
                W[JS, JCA] = (-1j * hop) * C_ANN    # - iV c+_{n+1} c_n
            if n > 0:
                W[JCD, JF] = C_ANN
                W[JCA, JF] = C_DAG
            if n == 0:
                W[JS, JWD] = (-1j * hop) * C_DAG    # - iV c+_1 c_N
                W[JS, JWC] = (1j * hop) * C_ANN     # + iV c+_N c_1
            elif n == N - 1:
                if model.peierls:
                    W[JWD, JWD] = C_ANN
                    W[JWC, JWC] = C_DAG
                else:
                    W[JWD, JF] = C_ANN
                    W[JWC, JF] = C_DAG
            else:
                W[JWD, JWD] = I
                W[JWC, JWC] = I
        elif kind == "v":
            for ch in (JCD, JCA, JWD, JWC):
                W[ch, ch] = I
        else:
            Vn = V * (I + model.alpha * op_x(d))
            if n < N - 1:
                W[JCD, JCD] = Vn
                W[JCA, JCA] = Vn
                W[JWD, JWD] = I
                W[JWC, JWC] = I
            else:
                W[JWD, JF] = Vn
                W[JWC, JF] = Vn
        Ws.append(W)
    Ws[0] = Ws[0][JS:JS + 1]
    Ws[-1] = Ws[-1][:, JF:JF + 1]
    return Ws


def mpo_to_dense(Ws: List[np.ndarray]) -> np.ndarray:
    """Contract an MPO into a dense matrix on the full product space (tiny chains only)."""
    T = Ws[0][0]                               # [wr, s, s']
    T = np.transpose(T, (1, 2, 0))             # [s, s', wr]
    dim = T.shape[0]
    for W in Ws[1:]:
        d = W.shape[2]
        T = np.einsum("ijw,wvab->iajbv", T, W).reshape(dim * d, dim * d, W.shape[1])
        dim *= d
    return T[:, :, 0]


def dense_from_definition(model: HolsteinModel):
    """H and j of Eq. 1/3/10 as dense matrices on the full product space, built term by
    term with Kronecker products (independent of the MPO automaton).  Tiny chains only."""
    sites = site_list(model)
    dims = [s[3] for s in sites]

    def embed(ops):
        out = np.array([[1.0 + 0j]])
        for i, d in enumerate(dims):
            out = np.kron(out, ops.get(i, np.eye(d)))
        return out

    e_index = {n: i for i, (k, n, m, d) in enumerate(sites) if k == "e"}
    v_index = {(n, m): i for i, (k, n, m, d) in enumerate(sites) if k == "v"}
    p_index = {n: i for i, (k, n, m, d) in enumerate(sites) if k == "p"}
    N = model.N
    D = int(np.prod(dims))
    H = np.zeros((D, D), dtype=complex)
    J = np.zeros((D, D), dtype=complex)
    for n in range(N):
        n1 = (n + 1) % N
        ops_f = {e_index[n1]: C_DAG, e_index[n]: C_ANN}   # c+_{n+1} c_n
        ops_b = {e_index[n]: C_DAG, e_index[n1]: C_ANN}   # c+_n c_{n+1}
        if model.peierls:
            pi = p_index[n]
            dp = dims[pi]
            Vop = model.V * (np.eye(dp) + model.alpha * op_x(dp))
            ops_f[pi] = Vop
            ops_b[pi] = Vop
            hf, hb = embed(ops_f), embed(ops_b)
        else:
            hf, hb = model.V * embed(ops_f), model.V * embed(ops_b)
        H += hf + hb
        J += -1j * hf + 1j * hb
        for m in range(model.K):
            vi = v_index[(n, m)]
            d = dims[vi]
            H += model.omega[m] * embed({vi: op_num(d)})
            H += model.g[m] * model.omega[m] * embed({vi: op_x(d), e_index[n]: N_E})
        if model.peierls:
            pi = p_index[n]
            H += model.omega_p * embed({pi: op_num(dims[pi])})
    return H, J


def carrier_number_dense(model: HolsteinModel) -> np.ndarray:
    sites = site_list(model)
    dims = [s[3] for s in sites]
    D = int(np.prod(dims))
    out = np.zeros((D, D))
    for i, (k, n, m, d) in enumerate(sites):
        if k == "e":
            M = np.array([[1.0]])
            for j, dj in enumerate(dims):
                M = np.kron(M, N_E if j == i else np.eye(dj))
            out += M
    return out
