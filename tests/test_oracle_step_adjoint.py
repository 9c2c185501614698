"""Pins of the discrete adjoint of one projector-splitting step (oracle/adjoint.py).

* ``step_with_tape`` reproduces ``tdvp.PurifiedMPS.step`` exactly (same operations);
* the reverse pass against central differences of ``PurifiedMPS.step``: along a random
  direction of the input state and for every model parameter (omega_m, g_m, V) through the
  MPO, in real and imaginary time.  Tolerance 1e-7 relative: the differences carry O(h^2)
  truncation (~1e-9 at h = 1e-4) and the Krylov stopping tolerance (1e-14 of |y|, divided
  by 2h: ~1e-9 here);
* the QR VJP against central differences of the gauge QR (full column rank).
"""
import numpy as np
import pytest

from oracle import adjoint, gradient, tdvp
from oracle.model import HolsteinModel, mpo_hamiltonian, site_list
from tests.inputs import random_complex


def ip(a, b):
    return float(np.vdot(a, b).real)


def _state(model, seed):
    rng = np.random.default_rng(seed)
    d = [s[3] for s in site_list(model)]
    D = [x * x for x in d]
    Mb = tdvp.bond_dims(D, 64)
    A = [random_complex(rng, (Mb[k], D[k], Mb[k + 1])) for k in range(len(D))]
    psi = tdvp.PurifiedMPS(model, A, mpo_hamiltonian(model))
    psi.right_canonicalize()
    return d, [x.copy() for x in psi.A], rng


def _oracle_step(model, A0, tau):
    p = tdvp.PurifiedMPS(model, A0, mpo_hamiltonian(model))
    p.build_right_envs()
    p.step(tau, tdvp.KrylovOpts(tol=1e-14))
    return p.A


@pytest.mark.parametrize("tau", [-0.2j, -0.1])
def test_step_adjoint_matches_central_differences(tau):
    model = HolsteinModel(N=3, omega=[1.0], g=[0.7], nmax=[2], V=0.8)
    d, A0, rng = _state(model, 61)
    Ws = mpo_hamiltonian(model)
    T, aout, ain, wids = adjoint.step_with_tape(Ws, d, A0, tau)
    ref = _oracle_step(model, A0, tau)
    assert max(np.abs(T.vals[i] - x).max() for i, x in zip(aout, ref)) == 0.0
    ybar = {i: random_complex(rng, T.vals[i].shape) for i in aout}
    bars = T.backward(ybar)

    def loss(mdl, As):
        return sum(ip(ybar[i], x) for i, x in zip(aout, _oracle_step(mdl, As, tau)))

    # input state
    # a direction of the size of each site tensor (entries of a right-orthonormal site are
    # ~1/sqrt(size)), so that h measures a relative change
    dA = []
    for x in A0:
        r = random_complex(rng, x.shape)
        dA.append(r * (np.linalg.norm(x) / np.linalg.norm(r)))
    h = 1e-6
    fd = (loss(model, [x + h * y for x, y in zip(A0, dA)]) -
          loss(model, [x - h * y for x, y in zip(A0, dA)])) / (2 * h)
    adj = sum(ip(bars[i], y) for i, y in zip(ain, dA))
    assert abs(fd - adj) <= 1e-7 * abs(adj)
    # model parameters through the MPO
    g = adjoint.step_parameter_gradient(model, [bars[i] for i in wids], mpo_hamiltonian)
    h = 1e-4
    for p in gradient.parameters(model):
        fd = (loss(gradient.shifted(model, p, h), A0) -
              loss(gradient.shifted(model, p, -h), A0)) / (2 * h)
        assert abs(fd - g[p]) <= 1e-7 * abs(g[p]), p


@pytest.mark.parametrize("m,n", [(12, 5), (30, 10), (8, 8)])
def test_qr_vjp_matches_central_differences(m, n):
    rng = np.random.default_rng(50 + m)
    Y = random_complex(rng, (m, n))
    Q, R = tdvp.gauge_qr(Y)
    Qb = random_complex(rng, (m, n))
    Rb = np.triu(random_complex(rng, (n, n)))
    Yb = adjoint.qr_vjp(Q, R, Qb, Rb)
    dY = random_complex(rng, (m, n))
    h = 1e-6
    Qp, Rp = tdvp.gauge_qr(Y + h * dY)
    Qm, Rm = tdvp.gauge_qr(Y - h * dY)
    fd = (ip(Qb, Qp - Qm) + ip(Rb, Rp - Rm)) / (2 * h)
    assert abs(fd - ip(Yb, dY)) <= 1e-8 * max(abs(fd), 1.0)
