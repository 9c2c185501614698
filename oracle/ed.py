"""Exact diagonalisation in the one-carrier sector (oracle part i).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

C(t) = Tr[rho j(t) j(0)],  rho = exp(-beta H) P_1 / Tr[exp(-beta H) P_1]    (Eq. 4-6)
     = sum_ab p_a exp(i (E_a - E_b) t) |j_ab|^2                            (eigenbasis)

P_1 projects on the one-carrier sector: the purified start state |I> is restricted to it
(the paper treats a single carrier; H conserves the carrier number).
The basis is |n> (carrier on molecule n) times the occupation numbers of every mode, and
H and j are assembled term by term from Eq. 1 / Eq. 3 / Eq. 10, without any MPO.
"""
import numpy as np

from .model import HolsteinModel, op_num, op_x


def _phonon_modes(model: HolsteinModel):
    """List of (kind, molecule, mode, d) for every phonon of the chain, in a fixed order."""
    modes = []
    for n in range(model.N):
        for m in range(model.K):
            modes.append(("v", n, m, int(model.nmax[m])))
        if model.peierls:
            modes.append(("p", n, -1, int(model.nmax_p)))
    return modes


def sector_operators(model: HolsteinModel):
    """H and j restricted to the one-carrier sector (dense, dimension N * prod(d))."""
    modes = _phonon_modes(model)
    dims = [m[3] for m in modes]
    Dph = int(np.prod(dims)) if dims else 1

    def ph_op(i, op):
        out = np.array([[1.0]])
        for k, d in enumerate(dims):
            out = np.kron(out, op if k == i else np.eye(d))
        return out

    N = model.N
    # phonon Hamiltonian (carrier independent part) and e-ph coupling per carrier site
    Hph = np.zeros((Dph, Dph))
    for i, (kind, n, m, d) in enumerate(modes):
        w = model.omega[m] if kind == "v" else model.omega_p
        Hph += w * ph_op(i, op_num(d))
    Hloc = []
    for n in range(N):
        h = Hph.copy()
        for i, (kind, nn, m, d) in enumerate(modes):
            if kind == "v" and nn == n:
                h += model.g[m] * model.omega[m] * ph_op(i, op_x(d))
        Hloc.append(h)
    # transfer integral of bond (n, n+1): V, or V (1 + alpha x_p) with a bond mode
    Vb = []
    for n in range(N):
        if model.peierls:
            i = [k for k, mm in enumerate(modes) if mm[0] == "p" and mm[1] == n][0]
            Vb.append(model.V * (np.eye(Dph) + model.alpha * ph_op(i, op_x(modes[i][3]))))
        else:
            Vb.append(model.V * np.eye(Dph))

    D = N * Dph
    H = np.zeros((D, D), dtype=complex)
    J = np.zeros((D, D), dtype=complex)

    def blk(a, b):
        return slice(a * Dph, (a + 1) * Dph), slice(b * Dph, (b + 1) * Dph)

    for n in range(N):
        H[blk(n, n)] += Hloc[n]
        n1 = (n + 1) % N
        # c+_{n+1} c_n moves the carrier n -> n+1 : block (n+1, n)
        H[blk(n1, n)] += Vb[n]
        H[blk(n, n1)] += Vb[n]
        J[blk(n1, n)] += -1j * Vb[n]
        J[blk(n, n1)] += 1j * Vb[n]
    return H, J


class ED:
    """Eigen-decomposition of the one-carrier sector at inverse temperature beta."""

    def __init__(self, model: HolsteinModel, beta: float):
        self.model = model
        self.beta = beta
        H, J = sector_operators(model)
        self.H, self.J = H, J
        E, U = np.linalg.eigh(H)
        self.E, self.U = E, U
        self.Jeig = U.conj().T @ J @ U
        w = np.exp(-beta * (E - E.min()))
        self.logZ = np.log(w.sum()) - beta * E.min()
        self.p = w / w.sum()

    def correlation(self, t) -> np.ndarray:
        """C(t) of Eq. 6 for an array of times."""
        t = np.atleast_1d(np.asarray(t, dtype=float))
        A = np.abs(self.Jeig) ** 2                    # |j_ab|^2
        out = np.empty(t.shape, dtype=complex)
        for i, ti in enumerate(t):
            ph_a = self.p * np.exp(1j * self.E * ti)  # p_a e^{i E_a t}
            ph_b = np.exp(-1j * self.E * ti)          # e^{-i E_b t}
            out[i] = ph_a @ A @ ph_b
        return out

    def thermal_energy(self) -> float:
        return float(self.p @ self.E)

    def rho(self) -> np.ndarray:
        return (self.U * self.p) @ self.U.conj().T

    def reduced_density(self) -> np.ndarray:
        """sigma = Tr_ph rho (Eq. 9): the thermal density matrix of the sector with every phonon
        traced out, sigma_nm = sum_ph rho[(n, ph), (m, ph)] = Tr[rho c+_m c_n]."""
        N = self.model.N
        Dph = self.H.shape[0] // N
        r = self.rho().reshape(N, Dph, N, Dph)
        return np.einsum("apbp->ab", r)

    def correlation_direct(self, t: float) -> complex:
        """Tr[rho e^{iHt} j e^{-iHt} j] with matrix exponentials (no eigen-sum)."""
        Ut = (self.U * np.exp(-1j * self.E * t)) @ self.U.conj().T
        return complex(np.trace(self.rho() @ Ut.conj().T @ self.J @ Ut @ self.J))
