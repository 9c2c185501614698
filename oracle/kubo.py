"""Kubo mobility (Eq. 2), the hopping-limit correlation function (Eq. 7), the mean free
path (Eq. 8) and the coherence length (Eq. 9).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).
"""
import numpy as np


def mobility(t: np.ndarray, C: np.ndarray, kT: float) -> float:
    """mu = 1/(2 kT) int_{-t_max}^{t_max} C(t) dt  (Eq. 2, e0 = 1, cut off at t_max).

    With C(-t) = C(t)^* the integral is 2 int_0^{t_max} Re C dt; the trapezoid rule is
    used on the given grid (which must start at t = 0)."""
    t = np.asarray(t, dtype=float)
    C = np.asarray(C)
    if t[0] != 0.0:
        raise ValueError("grid must start at t = 0")
    integral = 0.0
    for i in range(len(t) - 1):
        integral += 0.5 * (t[i + 1] - t[i]) * (C[i].real + C[i + 1].real)
    return float(2.0 * integral / (2.0 * kT))


def bose(omega: float, kT: float) -> float:
    return 1.0 / np.expm1(omega / kT)


def fgr_correlation(t, V, omega, g, kT, n_neighbours=2):
    """Hopping-limit C(t) for this model's C(t) convention (derived form of Eq. 7).

    Eq. 7 prints C/R^2 = V^2 exp{-sum g^2 [2n+1 - n e^{-iwt} - (n+1) e^{iwt}]}.  For the
    current of Eq. 3 on a periodic chain, to second order in V, a hop from molecule n
    relaxes the modes of both molecules, each carrier has two neighbours, and
    C(t) = Tr[rho e^{iHt} j e^{-iHt} j] carries the opposite time phase:
        C(t)/V^2 = 2 exp{-sum_m 2 g_m^2 [2n_m+1 - n_m e^{i w_m t} - (n_m+1) e^{-i w_m t}]}."""
    t = np.atleast_1d(np.asarray(t, dtype=float))
    expo = np.zeros(t.shape, dtype=complex)
    for w, gm in zip(omega, g):
        n = bose(w, kT)
        expo += 2.0 * gm * gm * (2 * n + 1 - n * np.exp(1j * w * t) - (n + 1) * np.exp(-1j * w * t))
    return n_neighbours * V * V * np.exp(-expo)


def free_band_correlation(N: int, V: float, beta: float) -> float:
    """g = 0: C(t) is constant, C = sum_k p_k (2 V sin k)^2, k = 2 pi m / N,
    p_k ~ exp(-beta 2 V cos k) (band of Eq. 1 without phonons)."""
    ks = 2.0 * np.pi * np.arange(N) / N
    eps = 2.0 * V * np.cos(ks)
    p = np.exp(-beta * (eps - eps.min()))
    p /= p.sum()
    return float(np.sum(p * (2.0 * V * np.sin(ks)) ** 2))


def mean_free_path(t: np.ndarray, C: np.ndarray):
    """Eq. 8: group velocity v = sqrt(<j(0) j(0)>) = sqrt(Re C(0)), relaxation time
    tau = 1/2 int_{-inf}^{inf} |Re C(t) / Re C(0)| dt, mean free path l = v tau.

    Re C is even in t (C(-t) = C(t)^*), so tau = int_0^{t_max} |Re C(t)| dt / Re C(0), cut off
    at the end of the grid and taken by the trapezoid rule on the grid values of |Re C|
    (the grid must start at t = 0).  Returns (v, tau, l)."""
    t = np.asarray(t, dtype=float)
    C = np.asarray(C)
    if t[0] != 0.0:
        raise ValueError("grid must start at t = 0")
    c0 = float(np.real(C[0]))
    if not c0 > 0.0:
        raise ValueError("Re C(0) = <j j> must be positive")
    area = 0.0
    for i in range(len(t) - 1):
        area += 0.5 * (t[i + 1] - t[i]) * (abs(C[i].real) + abs(C[i + 1].real))
    v = np.sqrt(c0)
    tau = area / c0
    return float(v), float(tau), float(v * tau)


def coherence_length(sigma: np.ndarray) -> float:
    """Eq. 9: L = (sum_ij |sigma_ij|)^2 / (N sum_ij |sigma_ij|^2) of the reduced electronic
    density matrix sigma = Tr_ph rho_beta (N x N)."""
    a = np.abs(np.asarray(sigma))
    N = a.shape[0]
    return float(a.sum() ** 2 / (N * (a * a).sum()))


def free_band_density(N: int, V: float, beta: float) -> np.ndarray:
    """g = 0: sigma = exp(-beta h) / Tr exp(-beta h) with h the N x N hopping matrix of Eq. 1
    (h_{n,n+1} = h_{n+1,n} = V on the ring)."""
    h = np.zeros((N, N))
    for n in range(N):
        h[n, (n + 1) % N] += V
        h[(n + 1) % N, n] += V
    e, u = np.linalg.eigh(h)
    w = np.exp(-beta * (e - e.min()))
    rho = (u * w) @ u.T
    return rho / np.trace(rho)
