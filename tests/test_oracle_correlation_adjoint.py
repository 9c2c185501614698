"""Pins of the reverse pass of the real-time correlation (oracle/adjoint.py,
``correlation_vjp``): C_n = <psi1(n dt)| j |psi2(n dt)> with both states stepped by the
projector-splitting integrator, reversed through stored states every two steps.

* A chain without modes at full bond dimension: one-site TDVP is then exact, so C_n and its
  derivative with respect to V must equal the dense e^{-iHt} evolution and its Frechet
  derivative (block-triangular exponential) to rounding.
* A chain with a mode: the gradients with respect to omega, g, V and to the initial states
  against central differences of the oracle's own steps and overlaps (1e-7: O(h^2) and the
  Krylov stopping tolerance).
"""
import numpy as np
import scipy.linalg as sl

from oracle import adjoint, gradient, tdvp
from oracle.model import HolsteinModel, mpo_current, mpo_hamiltonian, mpo_to_dense, site_list
from tests.inputs import random_complex


def ip(a, b):
    return float(np.vdot(a, b).real)


def _states(model, rng, n=2):
    d = [s[3] for s in site_list(model)]
    D = [x * x for x in d]
    Mb = tdvp.bond_dims(D, 64)
    Ws = mpo_hamiltonian(model)
    out = []
    for _ in range(n):
        A = [random_complex(rng, (Mb[k], D[k], Mb[k + 1])) for k in range(len(D))]
        p = tdvp.PurifiedMPS(model, A, Ws)
        p.right_canonicalize()
        A = [x.copy() for x in p.A]
        A[0] = A[0] / np.linalg.norm(A[0])
        out.append(A)
    return d, out


def _embed(op, d):
    """An operator on the physical indices as an operator on the fused (sigma, tau) sites."""
    L, n = len(d), int(np.prod(d))
    T = op.reshape(d + d)
    I = np.eye(n).reshape(d + d)
    out = np.einsum(T, list(range(2 * L)), I, list(range(2 * L, 4 * L)),
                    [x for k in range(L) for x in (k, 2 * L + k)] +
                    [x for k in range(L) for x in (L + k, 3 * L + k)])
    return out.reshape(n * n, n * n)


def test_full_rank_gradient_equals_exact_evolution():
    model = HolsteinModel(N=3, omega=[], g=[], nmax=[], V=0.8)
    rng = np.random.default_rng(71)
    d, (p1, p2) = _states(model, rng)
    Ws, Wj = mpo_hamiltonian(model), mpo_current(model)
    dt, ns = 0.3, 3
    cbar = random_complex(rng, (ns + 1,))
    C, g1, g2, Wb, Wjb = adjoint.correlation_vjp(Ws, Wj, d, p1, p2, dt, ns, cbar, every=2)
    V = ("V", -1)
    gV = (adjoint.step_parameter_gradient(model, Wb, mpo_hamiltonian)[V] +
          adjoint.step_parameter_gradient(model, Wjb, mpo_current)[V])
    H, J = _embed(mpo_to_dense(Ws), d), _embed(mpo_to_dense(Wj), d)
    up = gradient.shifted(model, V, 1.0)
    dH = _embed(mpo_to_dense(mpo_hamiltonian(up)), d) - H
    dJ = _embed(mpo_to_dense(mpo_current(up)), d) - J
    v1, v2 = tdvp.mps_to_dense(p1), tdvp.mps_to_dense(p2)
    n = H.shape[0]
    Cex, dC = [], []
    for k in range(ns + 1):
        B = np.zeros((2 * n, 2 * n), dtype=complex)
        B[:n, :n] = B[n:, n:] = -1j * k * dt * H
        B[:n, n:] = -1j * k * dt * dH
        E = sl.expm(B)
        a, b = E[:n, :n] @ v1, E[:n, :n] @ v2
        da, db = E[:n, n:] @ v1, E[:n, n:] @ v2
        Cex.append(np.vdot(a, J @ b))
        dC.append(np.vdot(da, J @ b) + np.vdot(a, dJ @ b) + np.vdot(a, J @ db))
    assert np.abs(C - np.array(Cex)).max() <= 1e-12 * np.abs(Cex).max()
    ref = float(np.sum(np.conj(cbar) * np.array(dC)).real)
    assert abs(gV - ref) <= 1e-11 * abs(ref)


def test_gradient_with_modes_matches_central_differences():
    model = HolsteinModel(N=3, omega=[1.0], g=[0.7], nmax=[2], V=0.8)
    rng = np.random.default_rng(70)
    d, (p1, p2) = _states(model, rng)
    dt, ns = 0.1, 3
    cbar = random_complex(rng, (ns + 1,))
    C, g1, g2, Wb, Wjb = adjoint.correlation_vjp(mpo_hamiltonian(model), mpo_current(model), d,
                                                 p1, p2, dt, ns, cbar, every=2)

    def loss(mdl, q1, q2):
        W, Jm = mpo_hamiltonian(mdl), mpo_current(mdl)
        a = tdvp.PurifiedMPS(mdl, q1, W)
        b = tdvp.PurifiedMPS(mdl, q2, W)
        a.build_right_envs()
        b.build_right_envs()
        out = 0.0
        for n in range(ns + 1):
            if n > 0:
                a.step(-1j * dt, tdvp.KrylovOpts(tol=1e-14))
                b.step(-1j * dt, tdvp.KrylovOpts(tol=1e-14))
            out += ip(cbar[n], tdvp.overlap(a.A, Jm, b.A, d))
        return out

    gH = adjoint.step_parameter_gradient(model, Wb, mpo_hamiltonian)
    gJ = adjoint.step_parameter_gradient(model, Wjb, mpo_current)
    h = 1e-4
    for p in gradient.parameters(model):
        fd = (loss(gradient.shifted(model, p, h), p1, p2) -
              loss(gradient.shifted(model, p, -h), p1, p2)) / (2 * h)
        assert abs(fd - (gH[p] + gJ[p])) <= 1e-7 * abs(fd), p
    h = 1e-6
    for which, g in ((0, g1), (1, g2)):
        base = [p1, p2]
        dA = []
        for x in base[which]:
            r = random_complex(rng, x.shape)
            dA.append(r * (np.linalg.norm(x) / np.linalg.norm(r)))
        plus = [list(base[0]), list(base[1])]
        minus = [list(base[0]), list(base[1])]
        plus[which] = [x + h * y for x, y in zip(base[which], dA)]
        minus[which] = [x - h * y for x, y in zip(base[which], dA)]
        fd = (loss(model, *plus) - loss(model, *minus)) / (2 * h)
        adj = sum(ip(a, b) for a, b in zip(g, dA))
        assert abs(fd - adj) <= 1e-7 * abs(adj), which
