"""Pins of the reverse pass of the whole C(t) pipeline (oracle/adjoint.py,
``correlation_pipeline_gradient``): the imaginary-time preparation from |I>, the variational
fit of j|Psi_beta>, both real-time evolutions and the overlaps of Eq. 6, reversed on tapes.

* ``left_expansion_vjp`` / ``right_expansion_vjp``: dot-product tests (both maps are
  trilinear in L, W, A / W, A, R; right_expansion is P^H, real-linear in each factor).
* ``qr_vjp_completed``: against central differences of ``tdvp.gauge_qr`` itself, with the
  completion candidates moving with the parameter and perturbations that keep the rank.
* Truncated bond dimension (M = 4: every gauge QR of the sweep completes columns, and the
  span of the completions enters the projected evolution): dl/dtheta against central
  differences of ``tdvp.correlation`` (1e-6; measured 2e-9 at h = 1e-5).
* Full bond dimension with rank threshold 1e-8: one-site TDVP is then exact, so C_n and
  dl/dtheta must equal exact diagonalisation and its gradient (``gradient``, Frechet
  derivatives of dense exponentials) - an independent pin of the whole chain.  Bounds: C to
  1e-8 (measured 5e-10: residuals below 1e-8 dropped per gauge QR), the gradient to 1e-6
  relative (measured 5e-8).
* Mobility and isotope derivative: mu of Eq. 2 and dmu/dtheta from the pipeline (cotangent =
  the trapezoid weights), and dmu/dm for omega ~ m^{-1/2} at fixed g^2 omega, against exact
  diagonalisation at full bond dimension.
"""
import numpy as np

from oracle import adjoint, gradient, tdvp
from oracle.model import HolsteinModel, mpo_current, mpo_hamiltonian
from tests.inputs import random_complex, random_mpo_site


def ip(a, b):
    return float(np.vdot(a, b).real)


def _close(x, y, rtol):
    assert abs(x - y) <= rtol * max(abs(x), abs(y)), (x, y)


def test_expansion_vjps_dot_product():
    rng = np.random.default_rng(100)
    Ml, Mr, d, Dl, Dr = 4, 5, 3, 3, 4
    L = random_complex(rng, (Dl, Ml, Ml))
    R = random_complex(rng, (Dr, Mr, Mr))
    W = random_mpo_site(rng, Dl, Dr, d) + 0j
    A = random_complex(rng, (Ml, d * d, Mr))
    Xb = random_complex(rng, tdvp.left_expansion(L, W, A, d).shape)
    grads = dict(zip("LWA", adjoint.left_expansion_vjp(L, W, A, d, Xb)))
    args = {"L": L, "W": W, "A": A}
    for name, X in args.items():
        dX = random_complex(rng, X.shape)
        a = dict(args, **{name: dX})
        _close(ip(Xb, tdvp.left_expansion(a["L"], a["W"], a["A"], d)), ip(grads[name], dX), 1e-12)
    Xb = random_complex(rng, tdvp.right_expansion(W, A, R, d).shape)
    grads = dict(zip("WAR", adjoint.right_expansion_vjp(W, A, R, d, Xb)))
    args = {"W": W, "A": A, "R": R}
    for name, X in args.items():
        dX = random_complex(rng, X.shape)
        a = dict(args, **{name: dX})
        _close(ip(Xb, tdvp.right_expansion(a["W"], a["A"], a["R"], d)), ip(grads[name], dX), 1e-12)


def test_completed_qr_vjp_against_gauge_qr():
    rng = np.random.default_rng(101)
    m, n, r, p = 14, 6, 4, 3
    B, G = random_complex(rng, (m, r)), random_complex(rng, (r, n))
    G[:, 2] = 0.5 * G[:, 0] + 1j * G[:, 1]                 # columns 2 and 4 dependent
    G[:, 4] = G[:, 3] - G[:, 1]
    X0 = random_complex(rng, (m, p))
    chosen = []
    Q, R = tdvp.gauge_qr(B @ G, X0, chosen=chosen)
    assert chosen == [0, 1]
    Qb, Rb = random_complex(rng, (m, n)), random_complex(rng, (n, n))
    Yb, Xsb = adjoint.qr_vjp_completed(Q, R, Qb, Rb, X0[:, chosen])
    dB, dG, dX = random_complex(rng, B.shape), random_complex(rng, G.shape), random_complex(rng, X0.shape)
    dG[:, 2] = 0.5 * dG[:, 0] + 1j * dG[:, 1]
    dG[:, 4] = dG[:, 3] - dG[:, 1]
    h = 1e-6

    def loss(t):
        Qx, Rx = tdvp.gauge_qr((B + t * dB) @ (G + t * dG), X0 + t * dX)
        return ip(Qb, Qx) + ip(Rb, Rx)

    fd = (loss(h) - loss(-h)) / (2 * h)
    dY = (B + h * dB) @ (G + h * dG) - (B - h * dB) @ (G - h * dG)
    _close(fd, ip(Yb, dY / (2 * h)) + ip(Xsb, dX[:, chosen]), 1e-8)


def _loss_gradient(model, M, cbar, rank_tol=tdvp.RANK_TOL):
    return adjoint.correlation_pipeline_gradient(model, 0.2, 0.05, M, 0.1, len(cbar) - 1, cbar,
                                                 mpo_hamiltonian, mpo_current,
                                                 rank_tol=rank_tol)


def test_truncated_pipeline_gradient_matches_central_differences():
    model = HolsteinModel(N=3, omega=[1.0], g=[0.7], nmax=[2], V=0.8)
    rng = np.random.default_rng(90)
    cbar = random_complex(rng, (4,))
    M = 4
    C, g = _loss_gradient(model, M, cbar)

    def run(mdl):
        return tdvp.correlation(mdl, 0.2, 0.05, M, 0.1, 3, kopts=tdvp.KrylovOpts(tol=1e-14)).C

    assert np.array_equal(C, run(model))
    h = 1e-5
    for p in gradient.parameters(model):
        fd = (ip(cbar, run(gradient.shifted(model, p, h))) -
              ip(cbar, run(gradient.shifted(model, p, -h)))) / (2 * h)
        _close(fd, g[p], 1e-6)


def test_full_bond_pipeline_gradient_equals_exact():
    model = HolsteinModel(N=3, omega=[0.6], g=[1.1], nmax=[2], V=0.4)
    rng = np.random.default_rng(91)
    cbar = random_complex(rng, (4,))
    C, g = _loss_gradient(model, 64, cbar, rank_tol=1e-8)     # 64 covers every cut
    Cex, G = gradient.correlation_gradient(model, 0.2, np.arange(4) * 0.1)
    assert np.abs(C - Cex).max() <= 1e-8 * np.abs(Cex).max()
    for p in gradient.parameters(model):
        _close(g[p], float(np.sum(np.conj(cbar) * G[p]).real), 1e-6)


def test_mobility_and_isotope_derivative_equal_exact():
    """mu (Eq. 2, trapezoid cut off at t_max) and its derivatives from the TD-DMRG pipeline at
    full bond dimension (rank threshold 1e-8) equal exact diagonalisation, and so does the
    isotope derivative dmu/dm for omega ~ m^{-1/2} at fixed g^2 omega (the chain rule
    dmu/dm = -omega/2 dmu/domega + g/4 dmu/dg at m = 1)."""
    from oracle import kubo
    model = HolsteinModel(N=3, omega=[1.0], g=[0.7], nmax=[2], V=0.8)
    kT, dt, ns = 5.0, 0.1, 3
    mu, g = adjoint.mobility_pipeline_gradient(model, kT, 0.05, 64, dt, ns, mpo_hamiltonian,
                                               mpo_current, rank_tol=1e-8)
    t = np.arange(ns + 1) * dt
    mu_ex, g_ex = gradient.mobility_gradient(model, kT, t)
    Cex, _ = gradient.correlation_gradient(model, 1.0 / kT, t)
    assert abs(mu_ex - kubo.mobility(t, Cex, kT)) < 1e-15
    _close(mu, mu_ex, 1e-8)
    # the rank threshold drops residuals of absolute size, so the components are bounded
    # against the size of the whole gradient (measured: at most 1.9e-9 on a gradient of 0.23)
    scale = max(abs(x) for x in g_ex.values())
    for p in gradient.parameters(model):
        assert abs(g[p] - g_ex[p]) <= 1e-6 * scale, p
    iso, iso_ex = gradient.isotope_derivative(model, g), gradient.isotope_derivative(model, g_ex)
    assert abs(iso - iso_ex) <= 1e-6 * scale
