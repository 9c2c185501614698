"""Pins of the gradient oracle (oracle/gradient.py): dC(t)/dtheta and dmu/dtheta for
theta = omega_m, g_m, V.

* central finite differences of the exact-diagonalisation C(t) (eigen-sum, no matrix
  exponentials) on small chains;
* the free band (g = 0): C does not depend on omega, is even in g, and dC/dV follows from
  the closed form C = sum_k p_k (2 V sin k)^2 differentiated by hand;
* V = 0: j vanishes, so C and all its derivatives are zero;
* the isotope derivative against a finite difference along omega ~ m^{-1/2}, g ~ m^{1/4}.
"""
import numpy as np
import pytest

from oracle import ed, gradient, kubo
from oracle.model import HolsteinModel

T_GRID = np.linspace(0.0, 2.0, 6)


def _ed_corr(model, beta, t):
    return ed.ED(model, beta).correlation(t)


@pytest.mark.parametrize("model,beta", [
    (HolsteinModel(N=3, omega=[1.0], g=[0.8], nmax=[3], V=0.7), 1.0),
    (HolsteinModel(N=3, omega=[1.3, 0.4], g=[0.5, 0.9], nmax=[2, 2], V=1.1), 0.6),
    (HolsteinModel(N=4, omega=[0.9], g=[0.6], nmax=[2], V=0.5), 2.0),
])
def test_correlation_gradient_matches_central_differences(model, beta):
    C, G = gradient.correlation_gradient(model, beta, T_GRID)
    assert np.abs(C - _ed_corr(model, beta, T_GRID)).max() < 1e-12 * np.abs(C).max()
    h = 1e-5
    for p in gradient.parameters(model):
        fd = (_ed_corr(gradient.shifted(model, p, h), beta, T_GRID) -
              _ed_corr(gradient.shifted(model, p, -h), beta, T_GRID)) / (2 * h)
        # central differences: O(h^2) truncation and O(eps / h) rounding, both ~1e-10 here
        assert np.abs(G[p] - fd).max() <= 1e-8 * max(np.abs(fd).max(), np.abs(C).max()), p


def test_free_band_gradient_closed_form():
    """g = 0: C(t) = sum_k p_k (2 V sin k)^2 for all t, p_k ~ exp(-beta 2 V cos k).
    dC/dV = sum_k [ dp_k/dV (2 V sin k)^2 + p_k 8 V sin^2 k ],
    dp_k/dV = -beta p_k (2 cos k - <2 cos k>);  dC/domega = dC/dg = 0."""
    N, V, beta = 3, 1.0, 1.0
    model = HolsteinModel(N=N, omega=[1.0], g=[0.0], nmax=[3], V=V)
    C, G = gradient.correlation_gradient(model, beta, T_GRID)
    ks = 2 * np.pi * np.arange(N) / N
    p = np.exp(-beta * 2 * V * np.cos(ks))
    p /= p.sum()
    de = 2 * np.cos(ks)
    dp = -beta * p * (de - np.sum(p * de))
    dCdV = np.sum(dp * (2 * V * np.sin(ks)) ** 2 + p * 8 * V * np.sin(ks) ** 2)
    assert np.abs(C - kubo.free_band_correlation(N, V, beta)).max() < 1e-12
    assert np.abs(G[("V", -1)] - dCdV).max() < 1e-11
    assert np.abs(G[("omega", 0)]).max() < 1e-11
    assert np.abs(G[("g", 0)]).max() < 1e-11


def test_zero_transfer_integral_gradient_vanishes():
    model = HolsteinModel(N=3, omega=[1.0], g=[0.8], nmax=[3], V=0.0)
    C, G = gradient.correlation_gradient(model, 1.0, T_GRID)
    assert np.abs(C).max() == 0.0
    for p, g in G.items():
        assert np.abs(g).max() < 1e-14, p


def test_mobility_and_isotope_derivative():
    """dmu/dtheta against central differences of the ED mobility, and the isotope
    derivative against a difference along omega(m) = omega m^{-1/2}, g(m) = g m^{1/4}."""
    model = HolsteinModel(N=3, omega=[1.2, 0.6], g=[0.7, 0.5], nmax=[2, 2], V=0.9)
    kT = 1.0
    t = np.linspace(0.0, 3.0, 13)
    mu, dmu = gradient.mobility_gradient(model, kT, t)

    def mu_of(mdl):
        return kubo.mobility(t, _ed_corr(mdl, 1.0 / kT, t), kT)

    assert abs(mu - mu_of(model)) < 1e-12 * abs(mu)
    h = 1e-5
    for p in gradient.parameters(model):
        fd = (mu_of(gradient.shifted(model, p, h)) - mu_of(gradient.shifted(model, p, -h))) / (2 * h)
        assert abs(dmu[p] - fd) <= 1e-8 * max(abs(fd), abs(mu)), p

    def at_mass(m):
        return HolsteinModel(N=3, omega=[w * m ** -0.5 for w in model.omega],
                             g=[g * m ** 0.25 for g in model.g], nmax=model.nmax, V=model.V)

    fd = (mu_of(at_mass(1.0 + h)) - mu_of(at_mass(1.0 - h))) / (2 * h)
    assert abs(gradient.isotope_derivative(model, dmu) - fd) <= 1e-8 * max(abs(fd), abs(mu))
