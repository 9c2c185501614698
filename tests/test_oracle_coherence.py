"""Pins of the coherence length (Eq. 9) and of the reduced electronic density matrix
sigma = Tr_ph rho_beta it is defined from, in the oracle.

* definition limits of Eq. 9: sigma = I / N gives L = 1, |sigma_ij| = 1 / N gives L = N;
* the exact-diagonalisation sigma: trace one, Hermitian, positive; at g = 0 the phonons
  decouple and sigma is the free-band thermal matrix exp(-beta h) / Tr (closed form); at V = 0
  every molecule is equivalent and nothing hops, so sigma = I / N and L = 1; at g = 0 on an even
  ring at low temperature the ground state k = pi is uniform in modulus, so L -> N;
* the TD-DMRG oracle's sigma (one MPO overlap per entry) at full bond dimension equals ED's."""
import numpy as np
import pytest

from oracle import kubo
from oracle import model as om
from oracle import tdvp
from oracle.ed import ED


def test_coherence_length_definition_limits():
    for N in (3, 5, 16):
        assert abs(kubo.coherence_length(np.eye(N) / N) - 1.0) < 1e-14
        ph = np.exp(2j * np.pi * np.arange(N) / N)
        assert abs(kubo.coherence_length(np.outer(ph, ph.conj()) / N) - N) < 1e-12


@pytest.mark.parametrize("N,beta", [(3, 1.0), (4, 0.7)])
def test_ed_density_free_band_closed_form(N, beta):
    m = om.HolsteinModel(N=N, omega=[1.0], g=[0.0], nmax=[2], V=1.0)
    sig = ED(m, beta).reduced_density()
    assert np.abs(sig - kubo.free_band_density(N, 1.0, beta)).max() < 1e-13


def test_ed_density_properties_and_localised_limit():
    m = om.HolsteinModel(N=3, omega=[1.0], g=[1.0], nmax=[3], V=0.7)
    sig = ED(m, 1.0).reduced_density()
    assert abs(np.trace(sig) - 1.0) < 1e-13
    assert np.abs(sig - sig.conj().T).max() < 1e-14
    assert np.linalg.eigvalsh(sig).min() > -1e-14
    m0 = om.HolsteinModel(N=3, omega=[1.0], g=[1.0], nmax=[3], V=0.0)
    sig0 = ED(m0, 1.0).reduced_density()
    assert np.abs(sig0 - np.eye(3) / 3).max() < 1e-14
    assert abs(kubo.coherence_length(sig0) - 1.0) < 1e-13


def test_ed_delocalised_limit():
    """g = 0, N = 4, V = 1, beta = 40: the k = pi band bottom (-2V) is separated by 2V from the
    next level, so sigma = |pi><pi| up to e^{-80} and L = N."""
    m = om.HolsteinModel(N=4, omega=[1.0], g=[0.0], nmax=[2], V=1.0)
    assert abs(kubo.coherence_length(ED(m, 40.0).reduced_density()) - 4.0) < 1e-10


def test_tdvp_density_full_rank_equals_ed():
    m = om.HolsteinModel(N=3, omega=[1.0], g=[1.0], nmax=[2], V=1.0)
    psi, _ = tdvp.thermal_state(m, 1.0, 0.05, 64)
    sig = tdvp.reduced_density(m, psi.A)
    ref = ED(m, 1.0).reduced_density()
    assert np.abs(sig - ref).max() < 1e-10
    assert abs(kubo.coherence_length(sig) - kubo.coherence_length(ref)) < 1e-10
