"""Pins for the plain TD-DMRG oracle: full-rank exactness against ED, invariants, building blocks."""
import numpy as np
import pytest
import scipy.linalg

from oracle import kubo
from oracle import model as om
from oracle import tdvp
from oracle.ed import ED


def test_gauge_qr_properties():
    rng = np.random.default_rng(7)
    Y = rng.standard_normal((12, 5)) + 1j * rng.standard_normal((12, 5))
    Q, R = tdvp.gauge_qr(Y)
    assert np.abs(Q.conj().T @ Q - np.eye(5)).max() < 1e-14
    assert np.abs(Q @ R - Y).max() < 1e-13
    assert np.abs(np.tril(R, -1)).max() < 1e-13
    assert np.all(np.abs(np.diag(R).imag) < 1e-15) and np.all(np.diag(R).real > 0)
    # same Q as a library QR with the phases of diag(R) made positive
    Ql, Rl = np.linalg.qr(Y)
    ph = np.diag(Rl) / np.abs(np.diag(Rl))
    assert np.abs(Ql * ph - Q).max() < 1e-13


def test_gauge_qr_completion_is_canonical():
    """Skipped columns are filled by unit vectors in index order, orthogonalised."""
    Y = np.zeros((4, 3), dtype=complex)
    Y[0, 0] = 2.0          # column 0 -> e_0
    Y[0, 1] = 5.0          # column 1 parallel to column 0: skipped
    Y[2, 2] = -3.0         # column 2 -> -e_2
    Q, R = tdvp.gauge_qr(Y)
    # e_0 is already in the span, so the completion of position 1 is e_1
    assert np.allclose(Q[:, 0], [1, 0, 0, 0])
    assert np.allclose(Q[:, 1], [0, 1, 0, 0])
    assert np.allclose(Q[:, 2], [0, 0, -1, 0])
    assert np.allclose(Q @ R, Y)
    assert abs(R[1, 1]) == 0.0
    # a completion residual that is not a unit vector: span contains (e0+e1)/sqrt2
    Y = np.zeros((3, 2), dtype=complex)
    Y[0, 0] = Y[1, 0] = 1.0
    Q, R = tdvp.gauge_qr(Y)
    assert np.allclose(Q[:, 1], np.array([1, -1, 0]) / np.sqrt(2))


@pytest.mark.parametrize("tau", [-0.3j, -0.05, 0.05, -2.0j])
def test_krylov_expm_matches_expm(tau):
    rng = np.random.default_rng(3)
    n = 40
    A = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    H = (A + A.conj().T) / 4
    v = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    ref = scipy.linalg.expm(tau * H) @ v
    out, k = tdvp.krylov_expm(lambda x: H @ x, v, tau, tol=1e-14, kmax=40)
    assert np.abs(out - ref).max() / np.abs(ref).max() < 1e-12
    assert k <= 40
    # fixed k = dimension is exact
    out, k = tdvp.krylov_expm(lambda x: H @ x, v, tau, fixed_k=n)
    assert k == n and np.abs(out - ref).max() / np.abs(ref).max() < 1e-11


def test_identity_state_is_sector_trace():
    """|I> of Eq. 5 restricted to one carrier: sum over sector states of |i>_P |i>_Q."""
    m = om.HolsteinModel(N=3, omega=[1.0], g=[1.0], nmax=[2], V=1.0)
    mps = tdvp.identity_state(m, 64)
    v = tdvp.mps_to_dense(mps)
    sites = om.site_list(m)
    dims = [s[3] for s in sites]
    ref = np.zeros_like(v)
    import itertools
    for occ in itertools.product(*[range(d) for d in dims]):
        ne = sum(o for o, s in zip(occ, sites) if s[0] == "e")
        if ne != 1:
            continue
        idx = 0
        for o, d in zip(occ, dims):
            idx = idx * d * d + (o * d + o)
        ref[idx] = 1.0
    assert np.abs(v - ref).max() == 0.0
    assert abs(np.vdot(v, v).real - 3 * 2 ** 3) < 1e-12


def test_bond_dims_caps():
    assert tdvp.bond_dims([4, 16, 4, 16, 4, 16], 1000) == [1, 4, 64, 256, 64, 16, 1]
    assert tdvp.bond_dims([4, 16, 4, 16, 4, 16], 64) == [1, 4, 64, 64, 64, 16, 1]


def _full_rank_case():
    return om.HolsteinModel(N=3, omega=[1.0], g=[1.0], nmax=[2], V=1.0), 64


def test_full_rank_tdvp_equals_ed():
    """At bond dimensions equal to the full ranks the projector-splitting integrator is exact:
    log Z, <H>_beta and C(t) agree with ED to rounding and the Krylov tolerance."""
    m, M = _full_rank_case()
    beta, dtau, dt = 1.0, 0.05, 0.05
    r = tdvp.correlation(m, beta, dtau, M, dt, 12, every=4, observe=True)
    ed = ED(m, beta)
    assert abs(r.logZ - ed.logZ) < 1e-10
    C = ed.correlation(r.t)
    assert np.abs(r.C - C).max() / abs(C[0]) < 1e-10
    assert abs(r.energy[0] - ed.thermal_energy()) < 1e-10
    assert np.abs(r.norm1 - 1.0).max() < 1e-12
    assert np.abs(r.norm2 - C[0].real).max() < 1e-10


def test_full_rank_peierls_equals_ed():
    m = om.HolsteinModel(N=3, omega=[], g=[], nmax=[], V=1.0, alpha=0.4, omega_p=0.6, nmax_p=2)
    r = tdvp.correlation(m, 1.0, 0.1, 64, 0.1, 6, every=3)
    ed = ED(m, 1.0)
    C = ed.correlation(r.t)
    assert abs(r.logZ - ed.logZ) < 1e-10
    assert np.abs(r.C - C).max() / abs(C[0]) < 1e-10


def test_truncated_invariants():
    """Below full rank: norm and energy are conserved by one-site TDVP in real time,
    C(0) = <Psi2|Psi2> (Z = 1), and Im C(0) = 0."""
    m = om.HolsteinModel(N=3, omega=[1.0], g=[1.0], nmax=[3], V=1.0)
    r = tdvp.correlation(m, 1.0, 0.05, 12, 0.05, 10, every=2, observe=True)
    assert np.abs(r.norm1 - 1.0).max() < 1e-11
    assert np.abs(r.energy - r.energy[0]).max() < 1e-9
    assert np.abs(r.norm2 - r.norm2[0]).max() < 1e-9
    assert abs(r.C[0].imag) < 1e-12
    assert abs(r.C[0].real - r.norm2[0]) < 1e-3 * r.norm2[0]   # fit of j|Psi> is close


def test_free_band_tdvp():
    """g = 0: the purified state has Schmidt rank <= 4 on every cut; well below the full
    ranks (64) the truncated run reproduces the closed-form constant C."""
    m = om.HolsteinModel(N=3, omega=[1.0], g=[0.0], nmax=[2], V=1.0)
    r = tdvp.correlation(m, 1.0, 0.05, 16, 0.1, 6, every=2)
    ref = kubo.free_band_correlation(3, 1.0, 1.0)
    assert np.abs(r.C - ref).max() < 1e-9
    assert abs(r.logZ - ED(m, 1.0).logZ) < 1e-9


def test_zero_coupling_tdvp():
    m = om.HolsteinModel(N=3, omega=[1.0], g=[1.0], nmax=[2], V=0.0)
    r = tdvp.correlation(m, 1.0, 0.1, 16, 0.1, 2)
    assert np.abs(r.C).max() < 1e-14


def test_gauge_qr_uses_candidates_before_unit_vectors():
    Y = np.zeros((4, 2), dtype=complex)
    Y[0, 0] = 1.0                                    # column 1 is zero: skipped
    extra = np.zeros((4, 3), dtype=complex)
    extra[0, 0] = 3.0                                # in the span already: rejected
    extra[:, 1] = [1.0, 0.0, 1.0, 1.0]              # residual (0, 0, 1, 1)/sqrt2 taken
    Q, R = tdvp.gauge_qr(Y, extra)
    assert np.allclose(Q[:, 1], np.array([0, 0, 1, 1]) / np.sqrt(2))
    assert np.allclose(Q @ R, Y)
