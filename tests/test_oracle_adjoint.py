"""Pins of the VJP building blocks of the adjoint TDVP step (oracle/adjoint.py).

* The contractions (H_eff, bond operator, left/right environment updates) are linear in each
  argument (anti-linear in the bra), so the forward function applied to a direction is the
  exact derivative: dot-product tests Re<ybar, f(.., dX, ..)> = Re<Xbar, dX>.
* The Krylov-exponential VJP: vbar against the dense exponential, the operator cotangent
  against the Frechet derivative read off a block-triangular exponential (Van Loan), and the
  cotangent of the bond environments (pairs mapped through the bond VJP) against central
  differences of the Krylov exponential of the bond operator.
"""
import numpy as np
import pytest
import scipy.linalg as sl

from oracle import adjoint, tdvp
from tests.inputs import random_complex, random_mpo_site


def ip(a, b):
    return float(np.vdot(a, b).real)       # Re sum conj(a) b


def _close(x, y, rtol=1e-12):
    assert abs(x - y) <= rtol * max(abs(x), abs(y), 1e-300), (x, y)


@pytest.mark.parametrize("Ml,Mr,d,Dl,Dr", [(1, 4, 2, 1, 5), (5, 6, 3, 4, 3), (7, 3, 2, 7, 7)])
def test_heff_vjp_dot_product(Ml, Mr, d, Dl, Dr):
    rng = np.random.default_rng(40 + Ml * Mr)
    L = random_complex(rng, (Dl, Ml, Ml))
    R = random_complex(rng, (Dr, Mr, Mr))
    W = random_mpo_site(rng, Dl, Dr, d) + 0j
    A = random_complex(rng, (Ml, d * d, Mr))
    yb = random_complex(rng, (Ml, d * d, Mr))
    grads = dict(zip("ALWR", adjoint.heff_vjp(L, W, R, A, d, yb)))
    args = {"A": A, "L": L, "W": W, "R": R}
    for name, X in args.items():
        dX = random_complex(rng, X.shape)
        a = dict(args, **{name: dX})
        _close(ip(yb, tdvp.heff(a["L"], a["W"], a["R"], a["A"], d)), ip(grads[name], dX))


def test_bond_heff_vjp_dot_product():
    rng = np.random.default_rng(41)
    Ml, Mr, Dw = 5, 6, 4
    C = random_complex(rng, (Ml, Mr))
    L = random_complex(rng, (Dw, Ml, Ml))
    R = random_complex(rng, (Dw, Mr, Mr))
    yb = random_complex(rng, (Ml, Mr))
    grads = dict(zip("CLR", adjoint.bond_heff_vjp(L, R, C, yb)))
    args = {"C": C, "L": L, "R": R}
    for name, X in args.items():
        dX = random_complex(rng, X.shape)
        a = dict(args, **{name: dX})
        _close(ip(yb, tdvp.bond_heff(a["L"], a["R"], a["C"])), ip(grads[name], dX))


@pytest.mark.parametrize("side", ["left", "right"])
def test_environment_update_vjp_dot_product(side):
    rng = np.random.default_rng(42)
    Ml, Mr, d, Dl, Dr = 5, 6, 3, 4, 3
    W = random_mpo_site(rng, Dl, Dr, d) + 0j
    bra = random_complex(rng, (Ml, d * d, Mr))
    ket = random_complex(rng, (Ml, d * d, Mr))
    if side == "left":
        E = random_complex(rng, (Dl, Ml, Ml))
        G = random_complex(rng, (Dr, Mr, Mr))
        grads = adjoint.update_left_vjp(E, bra, W, ket, d, G)
        f = tdvp.update_left
    else:
        E = random_complex(rng, (Dr, Mr, Mr))
        G = random_complex(rng, (Dl, Ml, Ml))
        grads = adjoint.update_right_vjp(E, bra, W, ket, d, G)
        f = tdvp.update_right
    grads = dict(zip(["E", "bra", "W", "ket"], grads))
    args = {"E": E, "bra": bra, "W": W, "ket": ket}
    for name, X in args.items():
        dX = random_complex(rng, X.shape)
        a = dict(args, **{name: dX})
        # linear in E, W, ket; the bra enters conjugated, so f(.., d bra, ..) is the change of
        # the output along d bra and the pairing Re<G, .> equals Re<brabar, d bra>
        _close(ip(G, f(a["E"], a["bra"], a["W"], a["ket"], d)), ip(grads[name], dX))


@pytest.mark.parametrize("tau", [-0.3j, -0.2, 0.1 - 0.2j])
def test_krylov_vjp_against_frechet_derivative(tau):
    rng = np.random.default_rng(43)
    n = 24
    H = random_complex(rng, (n, n))
    H = (H + H.conj().T) / 4 + 40.0 * np.eye(n)     # an energy offset, as in the sweep
    v = random_complex(rng, (n,))
    yb = random_complex(rng, (n,))
    vbar, pairs = adjoint.expm_krylov_vjp(lambda x: H @ x, v, tau, yb)
    dv = random_complex(rng, (n,))
    _close(ip(yb, sl.expm(tau * H) @ dv), ip(vbar, dv), 1e-11)
    Hbar = sum(np.outer(c, b.conj()) for c, b in pairs)
    dH = random_complex(rng, (n, n))
    dH = (dH + dH.conj().T) / 2
    B = np.zeros((2 * n, 2 * n), dtype=complex)
    B[:n, :n] = tau * H
    B[n:, n:] = tau * H
    B[:n, n:] = tau * dH
    frechet = sl.expm(B)[:n, n:]
    _close(ip(yb, frechet @ v), ip(Hbar, dH), 1e-11)


def test_krylov_vjp_through_bond_environments():
    """d/dh Re<ybar, exp(tau K(L + h dL)) C> by central differences against the cotangent of
    L assembled from the pairs: Lbar = sum_s bond_heff_vjp(L, R, b_s, c_s)[1]."""
    rng = np.random.default_rng(44)
    M, Dw, tau = 6, 3, -0.4j

    def herm(shape):
        X = random_complex(rng, shape)
        return (X + np.conj(np.swapaxes(X, -1, -2))) / 2

    L = herm((Dw, M, M)) / np.sqrt(M)
    R = herm((Dw, M, M)) / np.sqrt(M)
    C = random_complex(rng, (M, M))
    yb = random_complex(rng, (M, M))
    _, pairs = adjoint.expm_krylov_vjp(lambda X: tdvp.bond_heff(L, R, X), C, tau, yb)
    Lbar = sum(adjoint.bond_heff_vjp(L, R, b, c)[1] for c, b in pairs)
    dL = herm((Dw, M, M))

    def loss(h):
        y, _ = tdvp.krylov_expm(lambda X: tdvp.bond_heff(L + h * dL, R, X), C, tau, tol=1e-15)
        return ip(yb, y)

    h = 1e-4
    fd = (loss(h) - loss(-h)) / (2 * h)
    _close(fd, ip(Lbar, dL), 1e-7)


def test_heff_vjp_is_forward_contractions_with_transformed_operands():
    """The cotangents of an H_eff product are forward contractions of the sweep:
    Abar = heff(L^dagger per channel, W^T conj, R^dagger per channel, ybar),
    Lbar = conj(update_right(R, ybar, W, A)),  Rbar = conj(update_left(L, ybar, W, A))
    (the cotangent takes the place of the bra), so an adjoint step can reuse the H_eff and
    environment kernels."""
    rng = np.random.default_rng(45)
    Ml, Mr, d, Dl, Dr = 5, 6, 3, 4, 3
    L = random_complex(rng, (Dl, Ml, Ml))
    R = random_complex(rng, (Dr, Mr, Mr))
    W = random_mpo_site(rng, Dl, Dr, d) + 0j
    A = random_complex(rng, (Ml, d * d, Mr))
    yb = random_complex(rng, (Ml, d * d, Mr))
    Abar, Lbar, Wbar, Rbar = adjoint.heff_vjp(L, W, R, A, d, yb)
    Lh = np.conj(np.swapaxes(L, 1, 2))
    Rh = np.conj(np.swapaxes(R, 1, 2))
    Wt = np.conj(np.swapaxes(W, 2, 3))
    assert np.abs(tdvp.heff(Lh, Wt, Rh, yb, d) - Abar).max() < 1e-12 * np.abs(Abar).max()
    assert np.abs(np.conj(tdvp.update_right(R, yb, W, A, d)) - Lbar).max() < 1e-12 * np.abs(Lbar).max()
    assert np.abs(np.conj(tdvp.update_left(L, yb, W, A, d)) - Rbar).max() < 1e-12 * np.abs(Rbar).max()


def test_environment_vjp_is_forward_contractions_with_transformed_operands():
    """The cotangents of an environment update are forward contractions too, with the
    cotangent G in place of an environment (per-channel daggers and transposes):
      left  L' = update_left(L, bra, W, ket):  ketbar = heff(L^dagger, W^T conj, G^T, bra),
            brabar = heff(L, W, conj G, ket),  Lbar = conj(update_right(conj G, bra, W, ket));
      right R' = update_right(R, bra, W, ket): ketbar = heff(G^T, W^T conj, R^dagger, bra),
            brabar = heff(conj G, W, R, ket),  Rbar = conj(update_left(conj G, bra, W, ket)),
    so a reverse sweep can run on the H_eff and environment kernels alone."""
    rng = np.random.default_rng(46)
    Ml, Mr, d, Dl, Dr = 5, 6, 3, 4, 3
    W = random_mpo_site(rng, Dl, Dr, d) + 0j
    bra = random_complex(rng, (Ml, d * d, Mr))
    ket = random_complex(rng, (Ml, d * d, Mr))
    Wt = np.conj(np.swapaxes(W, 2, 3))

    def dag(E):
        return np.conj(np.swapaxes(E, 1, 2))

    def tr(E):
        return np.swapaxes(E, 1, 2)

    def close(a, b):
        assert np.abs(a - b).max() < 1e-12 * np.abs(b).max()

    L = random_complex(rng, (Dl, Ml, Ml))
    G = random_complex(rng, (Dr, Mr, Mr))
    Lb, bb, _, kb = adjoint.update_left_vjp(L, bra, W, ket, d, G)
    close(tdvp.heff(dag(L), Wt, tr(G), bra, d), kb)
    close(tdvp.heff(L, W, np.conj(G), ket, d), bb)
    close(np.conj(tdvp.update_right(np.conj(G), bra, W, ket, d)), Lb)
    R = random_complex(rng, (Dr, Mr, Mr))
    G = random_complex(rng, (Dl, Ml, Ml))
    Rb, bb, _, kb = adjoint.update_right_vjp(R, bra, W, ket, d, G)
    close(tdvp.heff(tr(G), Wt, dag(R), bra, d), kb)
    close(tdvp.heff(np.conj(G), W, R, ket, d), bb)
    close(np.conj(tdvp.update_left(np.conj(G), bra, W, ket, d)), Rb)
