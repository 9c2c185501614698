"""Exact parameter gradients of C(t) and of the mobility (oracle for the adjoint).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

C(t) = Tr[e^{-beta H} e^{iHt} j e^{-iHt} j] / Tr[e^{-beta H}] in the one-carrier sector
(Eq. 4-6).  Its derivative with respect to a parameter theta of Eq. 1 / Eq. 3 / Eq. 10 is
taken term by term:

    dC = ( Tr[dR A j] + Tr[R dA j] + Tr[R A dj] ) / Z  -  C dZ / Z,
    R = e^{-beta H},  Z = Tr R,  A = e^{iHt} j e^{-iHt},
    dA = dU j U^H + U dj U^H + U j dU^H,  U = e^{iHt},

where dR and dU are the Frechet derivatives of the matrix exponential in the direction of
dH (-beta dH and i t dH), read off the upper-right block of the exponential of the
block-triangular matrix [[X, E], [0, X]] (Van Loan, "Computing integrals involving the
matrix exponential", 1978); e^{-iHt} = (e^{iHt})^H, so its derivative is dU^H.

H is affine in each of omega_m, g_m and V, and j is linear in V (Eq. 1: omega_m b+b and
g_m omega_m (b+ + b) c+c; Eq. 3: j proportional to V; Eq. 10: V (1 + alpha x_p)), so dH and
dj are the exact differences of the operators at theta + 1 and theta.

The mobility of Eq. 2 is linear in C, so dmu = mobility(t, dC).  The isotope derivative
follows omega_m(m) = omega_m m^{-1/2}, lambda_m = g_m^2 omega_m fixed (g_m(m) = g_m m^{1/4}):
dmu/dm at m = 1 is sum_m (dmu/domega_m (-omega_m / 2) + dmu/dg_m (g_m / 4)).
"""
import dataclasses
from typing import Dict, List, Tuple

import numpy as np
import scipy.linalg

from . import kubo
from .ed import sector_operators
from .model import HolsteinModel

Param = Tuple[str, int]           # ("omega", m), ("g", m) or ("V", -1)


def parameters(model: HolsteinModel) -> List[Param]:
    return [("omega", m) for m in range(model.K)] + [("g", m) for m in range(model.K)] + \
        [("V", -1)]


def shifted(model: HolsteinModel, p: Param, delta: float) -> HolsteinModel:
    """The model with one parameter moved by delta."""
    name, m = p
    if name == "V":
        return dataclasses.replace(model, V=model.V + delta)
    vals = list(getattr(model, name))
    vals[m] = vals[m] + delta
    return dataclasses.replace(model, **{name: vals})


def operator_derivatives(model: HolsteinModel) -> Tuple[np.ndarray, np.ndarray,
                                                        Dict[Param, Tuple[np.ndarray, np.ndarray]]]:
    """H, j and (dH/dtheta, dj/dtheta) for every parameter (exact: affine dependence)."""
    H, J = sector_operators(model)
    out = {}
    for p in parameters(model):
        H1, J1 = sector_operators(shifted(model, p, 1.0))
        out[p] = (H1 - H, J1 - J)
    return H, J, out


def expm_and_frechet(X: np.ndarray, E: np.ndarray) -> Tuple[np.ndarray, np.ndarray]:
    """(e^X, d/ds e^{X + sE} at s = 0) from the block-triangular exponential."""
    n = X.shape[0]
    B = np.zeros((2 * n, 2 * n), dtype=complex)
    B[:n, :n] = X
    B[n:, n:] = X
    B[:n, n:] = E
    Y = scipy.linalg.expm(B)
    return Y[:n, :n], Y[:n, n:]


def correlation_gradient(model: HolsteinModel, beta: float, t_grid
                         ) -> Tuple[np.ndarray, Dict[Param, np.ndarray]]:
    """C(t) on t_grid and dC(t)/dtheta for every parameter."""
    t_grid = np.atleast_1d(np.asarray(t_grid, dtype=float))
    H, J, dops = operator_derivatives(model)
    C = np.zeros(t_grid.shape, dtype=complex)
    grads = {p: np.zeros(t_grid.shape, dtype=complex) for p in dops}
    first = True
    for p, (dH, dJ) in dops.items():
        R, dR = expm_and_frechet(-beta * H, -beta * dH)
        Z = np.trace(R).real
        dZ = np.trace(dR).real
        for i, t in enumerate(t_grid):
            U, dU = expm_and_frechet(1j * t * H, 1j * t * dH)
            Ud, dUd = U.conj().T, dU.conj().T
            A = U @ J @ Ud
            dA = dU @ J @ Ud + U @ dJ @ Ud + U @ J @ dUd
            c = np.trace(R @ A @ J) / Z
            if first:
                C[i] = c
            grads[p][i] = (np.trace(dR @ A @ J) + np.trace(R @ dA @ J) +
                           np.trace(R @ A @ dJ)) / Z - c * dZ / Z
        first = False
    return C, grads


def mobility_gradient(model: HolsteinModel, kT: float, t_grid) -> Tuple[float, Dict[Param, float]]:
    """mu of Eq. 2 on t_grid (trapezoid, cut off at t_grid[-1]) and dmu/dtheta."""
    C, dC = correlation_gradient(model, 1.0 / kT, t_grid)
    mu = kubo.mobility(t_grid, C, kT)
    return mu, {p: kubo.mobility(t_grid, g, kT) for p, g in dC.items()}


def isotope_derivative(model: HolsteinModel, dmu: Dict[Param, float]) -> float:
    """dmu/dm at m = 1 for omega_m ~ m^{-1/2} with g_m^2 omega_m fixed (g_m ~ m^{1/4})."""
    out = 0.0
    for m in range(model.K):
        out += dmu[("omega", m)] * (-0.5 * model.omega[m]) + dmu[("g", m)] * (0.25 * model.g[m])
    return out
