"""Pins of the gauge-completion reading of the oracle (one-site TDVP shifts of Eq. S1).

Below full bond dimension a gauge shift of a rank-deficient site must fill the skipped columns
of Q with some orthonormal directions, and those directions enter the projected dynamics.  The
oracle fills them from what the Hamiltonian couples the site into (``tdvp.left_expansion`` for a
left-to-right shift, ``tdvp.right_expansion`` for a right-to-left one), then unit vectors.
Two kinds of pin, each independent of the functions' own formulas:

* definition: the candidates are H_eff with one environment left out, so contracting them with
  that environment must give the full H_eff product (``tdvp.heff``, itself pinned by the
  full-rank TDVP == ED tests).  A transposed (channel, bond) column order or a dropped complex
  conjugation breaks this identity;
* physics: with these completions the truncated TD-DMRG of the c1 chain (N = 3, one mode,
  nmax = 4, full caps [4, 64, 256, 64, 16]) follows exact diagonalisation closely at M = 16
  and M = 32 (measured over ten real-time steps: 4.4e-4 and 1.8e-7 of C(0)), while unit-vector
  completion gives C(t) that is wrong at order one (C(0) ~ 0 at M = 16).
Planted mistakes are planted in the oracle, on the CPU, through monkeypatch."""
import numpy as np
import pytest

from oracle import model as om
from oracle import tdvp
from oracle.ed import ED
from tests.inputs import random_complex, random_mpo_site

SHAPES = [(3, 5, 2, 4, 3), (4, 3, 3, 2, 5)]     # Ml, Mr, d, Dl, Dr with Ml != Mr, Dl != Dr


def _env(rng, D, M):
    return random_complex(rng, (D, M, M))


@pytest.mark.parametrize("Ml,Mr,d,Dl,Dr", SHAPES)
def test_left_expansion_is_heff_without_right_environment(Ml, Mr, d, Dl, Dr):
    rng = np.random.default_rng(31 + Ml)
    L, R = _env(rng, Dl, Ml), _env(rng, Dr, Mr)
    W = random_mpo_site(rng, Dl, Dr, d, density=0.7)
    A = random_complex(rng, (Ml, d * d, Mr))
    P = tdvp.left_expansion(L, W, A, d)                      # rows (x,s,t), columns (v,c)
    assert P.shape == (Ml * d * d, Dr * Mr)
    got = np.einsum("rvc,vbc->rb", P.reshape(-1, Dr, Mr), R).reshape(Ml, d * d, Mr)
    ref = tdvp.heff(L, W, R, A, d)
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("Ml,Mr,d,Dl,Dr", SHAPES)
def test_right_expansion_is_heff_without_left_environment(Ml, Mr, d, Dl, Dr):
    rng = np.random.default_rng(47 + Ml)
    L, R = _env(rng, Dl, Ml), _env(rng, Dr, Mr)
    W = random_mpo_site(rng, Dl, Dr, d, density=0.7)
    A = random_complex(rng, (Ml, d * d, Mr))
    X = tdvp.right_expansion(W, A, R, d)                     # columns of Y = A^H: X = P^H
    assert X.shape == (d * d * Mr, Dl * Ml)
    P = X.conj().T.reshape(Dl, Ml, d * d * Mr)                # rows (w,y), columns (s,t,b)
    got = np.einsum("wxy,wyr->xr", L, P).reshape(Ml, d * d, Mr)
    ref = tdvp.heff(L, W, R, A, d)
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()


def _swapped_left(Lenv, W, A, d):
    X = np.tensordot(Lenv, tdvp._split(A, d), axes=([2], [0]))
    Y = np.tensordot(W, X, axes=([0, 3], [0, 2]))             # [v, s, x, t, c]
    return Y.transpose(2, 1, 3, 4, 0).reshape(A.shape[0] * A.shape[1], -1)   # c outer: wrong


def _unconjugated_right(W, A, Renv, d):
    X = np.tensordot(tdvp._split(A, d), Renv, axes=([3], [2]))
    Y = np.tensordot(W, X, axes=([1, 3], [3, 1])).transpose(0, 2, 1, 3, 4)
    return Y.reshape(-1, A.shape[1] * A.shape[2]).T          # conjugation dropped: wrong


@pytest.mark.parametrize("which", ["left", "right"])
def test_planted_candidate_mistakes_are_caught(which, monkeypatch):
    """The identity tests above fail on a transposed column order or a dropped conjugation."""
    if which == "left":
        monkeypatch.setattr(tdvp, "left_expansion", _swapped_left)
        with pytest.raises(AssertionError):
            test_left_expansion_is_heff_without_right_environment(*SHAPES[0])
    else:
        monkeypatch.setattr(tdvp, "right_expansion", _unconjugated_right)
        with pytest.raises(AssertionError):
            test_right_expansion_is_heff_without_left_environment(*SHAPES[0])


C1 = dict(N=3, omega=[1.0], g=[1.0], nmax=[4], V=1.0)


def _c1_error(M, nsteps=10):
    m = om.HolsteinModel(**C1)
    r = tdvp.correlation(m, 1.0, 0.05, M, 0.05, nsteps)
    ed = ED(m, 1.0)
    C = ed.correlation(r.t)
    return np.abs(r.C - C).max() / abs(C[0]), abs(r.logZ - ed.logZ)


@pytest.mark.parametrize("M,bound", [(16, 1e-3), (32, 1e-6)])
def test_truncated_c1_follows_ed(M, bound):
    """Below full rank (caps [4, 64, 256, 64, 16]) with Hamiltonian-coupled completion:
    ten real-time steps dt = 0.05 after the k_BT = 1 preparation stay within `bound` of C(0)
    (measured 4.4e-4 at M = 16 and 1.8e-7 at M = 32; log Z within 6e-5 and 6e-7)."""
    err, dlogz = _c1_error(M)
    assert err <= bound
    assert dlogz <= 1e3 * bound


def test_unit_vector_completion_is_wrong_physics(monkeypatch):
    """The survey's first proposal (completion by unit vectors only) gives order-one errors at
    M = 16; the Hamiltonian-coupled candidates are what make the truncated dynamics right."""
    monkeypatch.setattr(tdvp, "left_expansion", lambda *a: None)
    monkeypatch.setattr(tdvp, "right_expansion", lambda *a: None)
    err, _ = _c1_error(16, nsteps=2)
    assert err > 0.3
