"""Pins for the oracle's model layer: MPOs against an independent term-by-term construction."""
import numpy as np
import pytest

from oracle import model as om


def _models():
    return [
        om.HolsteinModel(N=3, omega=[1.0], g=[1.0], nmax=[2], V=1.0),
        om.HolsteinModel(N=4, omega=[0.7], g=[0.4], nmax=[2], V=0.3),
        om.HolsteinModel(N=3, omega=[0.2, 1.0], g=[1.5, 0.8], nmax=[2, 2], V=2.0),
        om.HolsteinModel(N=3, omega=[1.0], g=[0.5], nmax=[2], V=1.0, alpha=0.3, omega_p=0.5, nmax_p=2),
    ]


@pytest.mark.parametrize("m", _models())
def test_mpo_matches_definition(m):
    """Eq. 1/3/10 built term by term (Kronecker products) equals the contracted MPOs."""
    H, J = om.dense_from_definition(m)
    assert np.abs(om.mpo_to_dense(om.mpo_hamiltonian(m)) - H).max() < 1e-13
    assert np.abs(om.mpo_to_dense(om.mpo_current(m)) - J).max() < 1e-13


@pytest.mark.parametrize("m", _models())
def test_operators_hermitian_and_conserve_carrier(m):
    H, J = om.dense_from_definition(m)
    Ne = om.carrier_number_dense(m)
    assert np.abs(H - H.conj().T).max() < 1e-13
    assert np.abs(J - J.conj().T).max() < 1e-13
    assert np.abs(H @ Ne - Ne @ H).max() < 1e-12
    # j = i [H, P] with P the carrier position: checked on the one-carrier sector
    # through its matrix elements between neighbours (Eq. 3): <n+1|j|n> = -i V.
    if not m.peierls:
        sites = om.site_list(m)
        dims = [s[3] for s in sites]
        def basis(n):
            v = np.array([1.0])
            for (k, nn, mm, d) in sites:
                e = np.zeros(d)
                e[1 if (k == "e" and nn == n) else 0] = 1.0
                v = np.kron(v, e)
            return v
        for n in range(m.N):
            a, b = basis(n), basis((n + 1) % m.N)
            assert abs(b @ J @ a - (-1j * m.V)) < 1e-13
            assert abs(b @ H @ a - m.V) < 1e-13


def test_current_is_commutator_with_position():
    """j = i[H, X] restricted to the one-carrier sector, X = sum_n n c+_n c_n, on an open
    segment: away from the wrap bond the commutator fixes every matrix element of j."""
    m = om.HolsteinModel(N=5, omega=[1.0], g=[0.3], nmax=[2], V=0.7)
    H, J = om.dense_from_definition(m)
    sites = om.site_list(m)
    dims = [s[3] for s in sites]
    X = np.zeros_like(H)
    for i, (k, n, mm, d) in enumerate(sites):
        if k == "e":
            op = np.array([[1.0]])
            for jj, dj in enumerate(dims):
                op = np.kron(op, om.N_E if jj == i else np.eye(dj))
            X += n * op
    Jc = 1j * (H @ X - X @ H)
    # project both on states whose carrier is not on the wrap bond (molecules 0..N-2 <-> n+1)
    onec = np.isclose(np.diag(om.carrier_number_dense(m)), 1.0)
    pos = np.real(np.diag(X))
    inner = onec & (pos >= 0)
    Jw = J.copy()
    # remove the wrap-bond elements (carrier hops between molecule N-1 and 0)
    for a in np.where(inner)[0]:
        for b in np.where(inner)[0]:
            if abs(pos[a] - pos[b]) > 1.5:
                Jw[a, b] = 0.0
                Jc[a, b] = 0.0
    sel = np.ix_(inner, inner)
    assert np.abs(Jw[sel] - Jc[sel]).max() < 1e-12


def test_planted_mistakes_are_caught():
    """A dropped term, a wrong sign or a transposed operator in the MPO breaks the pin."""
    m = om.HolsteinModel(N=3, omega=[1.0], g=[1.0], nmax=[2], V=1.0)
    H, J = om.dense_from_definition(m)
    Ws = om.mpo_hamiltonian(m)
    bad = [w.copy() for w in Ws]
    bad[0][0, om.WD] = 0.0                       # drop the wrap-around hop
    assert np.abs(om.mpo_to_dense(bad) - H).max() > 0.5
    bad = [w.copy() for w in Ws]
    bad[1][om.NE, om.F] *= -1.0                  # wrong sign of the e-ph coupling
    assert np.abs(om.mpo_to_dense(bad) - H).max() > 0.5
    Wj = om.mpo_current(m)
    bad = [w.copy() for w in Wj]
    bad[0][0, om.JCD] = bad[0][0, om.JCD].T      # c+ <-> c
    assert np.abs(om.mpo_to_dense(bad) - J).max() > 0.5
