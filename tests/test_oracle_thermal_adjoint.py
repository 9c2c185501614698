"""Pins of the reverse pass of the imaginary-time preparation (oracle/adjoint.py).

* ``qr_vjp_selected`` (gauge QR with skipped columns): equal to ``qr_vjp`` without skipped
  columns; against central differences of an independent factorisation of [Y_S | Q_K]
  (numpy QR with a positive diagonal), the completed columns re-orthogonalised against the
  accepted ones, with perturbations that keep the rank (Y = B G).
* ``thermal_logz_gradient``: log Z equals ``tdvp.thermal_state`` and, at full bond dimension,
  dlogZ/dtheta equals -beta <dH/dtheta>_beta from exact diagonalisation (the identity
  d log Tr e^{-beta H} = -beta Tr[rho dH]); the first steps start from the rank-2 |I> and go
  through completed gauge columns, so this also pins their treatment.  Bound 1e-6: gauge
  columns accepted with residuals just above the rank threshold (1e-12 ||Y||_F) enter R^{-1}
  in the QR VJP and amplify rounding (measured 1e-9 for the first chain, 1.8e-7 for the
  second).
"""
import numpy as np
import pytest

from oracle import adjoint, ed, gradient, tdvp
from oracle.model import HolsteinModel, mpo_hamiltonian
from tests.inputs import random_complex


def ip(a, b):
    return float(np.vdot(a, b).real)


def test_selected_vjp_reduces_to_full_rank():
    rng = np.random.default_rng(80)
    Y = random_complex(rng, (12, 5))
    Q, R = tdvp.gauge_qr(Y)
    Qb, Rb = random_complex(rng, (12, 5)), random_complex(rng, (5, 5))
    assert np.abs(adjoint.qr_vjp_selected(Q, R, Qb, Rb) - adjoint.qr_vjp(Q, R, Qb, Rb)).max() < 1e-13


def test_selected_vjp_with_completed_columns():
    rng = np.random.default_rng(81)
    m, n, r = 12, 6, 4
    B = random_complex(rng, (m, r))
    G = random_complex(rng, (r, n))
    G[:, 3] = 0.7 * G[:, 0] - 0.2j * G[:, 1]            # columns 3 and 5 dependent
    G[:, 5] = G[:, 2] + G[:, 4]
    Q, R = tdvp.gauge_qr(B @ G)
    acc = np.abs(np.diag(R)) > 0
    S, K = np.flatnonzero(acc), np.flatnonzero(~acc)
    assert list(K) == [3, 5]
    QK0 = Q[:, K].copy()
    Qb, Rb = random_complex(rng, (m, n)), random_complex(rng, (n, n))
    Rb[K, :] = 0.0
    Yb = adjoint.qr_vjp_selected(Q, R, Qb, Rb)

    def factor(Yx):
        # accepted columns then the fixed candidates QK0, orthonormalised in that order
        Z = np.concatenate([Yx[:, S], QK0], axis=1)
        Qz, Rz = np.linalg.qr(Z)
        ph = np.diag(Rz) / np.abs(np.diag(Rz))
        Qz = Qz * ph
        Qx = np.zeros((m, n), dtype=complex)
        Qx[:, S] = Qz[:, :len(S)]
        Qx[:, K] = Qz[:, len(S):]
        Rx = Qx.conj().T @ Yx
        Rx[K, :] = 0.0
        return Qx, Rx

    Qf, Rf = factor(B @ G)
    assert np.abs(Qf - Q).max() < 1e-12 and np.abs(Rf - R).max() < 1e-12
    dB, dG = random_complex(rng, B.shape), random_complex(rng, G.shape)
    dG[:, 3] = 0.7 * dG[:, 0] - 0.2j * dG[:, 1]
    dG[:, 5] = dG[:, 2] + dG[:, 4]
    h = 1e-6
    Yp, Ym = (B + h * dB) @ (G + h * dG), (B - h * dB) @ (G - h * dG)
    (Qp, Rp), (Qm, Rm) = factor(Yp), factor(Ym)
    fd = (ip(Qb, Qp - Qm) + ip(Rb, Rp - Rm)) / (2 * h)
    assert abs(fd - ip(Yb, (Yp - Ym) / (2 * h))) <= 1e-8 * abs(fd)


@pytest.mark.parametrize("model", [
    HolsteinModel(N=3, omega=[1.0], g=[0.7], nmax=[2], V=0.8),
    HolsteinModel(N=3, omega=[0.6], g=[1.1], nmax=[2], V=0.4),
])
def test_thermal_logz_gradient_equals_exact(model):
    beta, dtau, M = 0.2, 0.05, 64          # M = 64 covers every cut of the 6-site chain
    lz, g = adjoint.thermal_logz_gradient(model, beta, dtau, M, mpo_hamiltonian)
    _, lz_ref = tdvp.thermal_state(model, beta, dtau, M, tdvp.KrylovOpts(tol=1e-14))
    assert lz == lz_ref
    E = ed.ED(model, beta)
    rho = E.rho()
    H0, _ = ed.sector_operators(model)
    for p in gradient.parameters(model):
        H1, _ = ed.sector_operators(gradient.shifted(model, p, 1.0))
        exact = -beta * np.trace(rho @ (H1 - H0)).real
        assert abs(g[p] - exact) <= 1e-6 * max(abs(exact), 1e-3), p
