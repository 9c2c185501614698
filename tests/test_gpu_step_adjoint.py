"""Parity of the reverse of one projector-splitting step (tdmrg_step_vjp, FP64) with the
oracle's tape (``oracle/adjoint.step_with_tape``): the output sites, the cotangents of the input
sites and the parameter cotangents (omega, g, V).

* A random state (full-rank bonds, no completed columns), real and imaginary tau: every part is
  a smooth function of its inputs; bound 1e-8 of the largest entry (the Krylov tolerances).
* The right-canonicalised |I> at M = 4, real tau: rank-2 bonds, so 12 gauge-QR columns per
  step are completed from their coupling candidates, accepted with residuals down to 1e-2 of
  their norm; two CPU rounding orders of the same algorithm differ by 2.6e-9 of the parameter
  cotangents, so the bound there is 1e-7; 1e-14 relative noise on the input sites moves the
  oracle's own output sites by 3.7e-9 of their largest entry, so they are held to 4e-8 there
  (10x that spread; measured on GB300: 4e-10).  (Wider bonds around |I>, or imaginary tau from it,
  put columns at the rank threshold and are not a parity case: two rounding orders differ by
  1e-6 and more.)
"""
import numpy as np
import pytest

from tests.inputs import random_complex

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2003_13245_gb300.build import build_library
    build_library()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


@pytest.mark.parametrize("basis", [False, True])
@pytest.mark.parametrize("M,tau,start,bound,out_bound", [(4, -0.1j, "random", 1e-8, 1e-10),
                                                         (4, -0.05, "random", 1e-8, 1e-10),
                                                         (64, -0.1j, "random", 1e-8, 1e-10),
                                                         (4, -0.1j, "identity", 1e-7, 4e-8)])
def test_step_vjp_matches_oracle_tape(M, tau, start, bound, out_bound, basis):
    from oracle import adjoint, tdvp
    from oracle.model import HolsteinModel, mpo_hamiltonian, site_list
    from paper_2003_13245_gb300 import binding
    model = HolsteinModel(N=3, omega=[1.0], g=[0.7], nmax=[2], V=0.8)
    rng = np.random.default_rng(9000 + M)
    d = [s[3] for s in site_list(model)]
    Ws = mpo_hamiltonian(model)
    if start == "random":
        Mb = tdvp.bond_dims([x * x for x in d], M)
        A0 = [random_complex(rng, (Mb[k], d[k] ** 2, Mb[k + 1])) for k in range(len(d))]
    else:
        A0 = tdvp.identity_state(model, M)
    p = tdvp.PurifiedMPS(model, A0, Ws)
    p.right_canonicalize()
    A = [x.copy() for x in p.A]
    A[0] = A[0] / np.linalg.norm(A[0])
    Abar = [random_complex(rng, x.shape) for x in A]
    T, out, inp, wids = adjoint.step_with_tape(Ws, d, A, tau, tol=1e-14)
    bars = T.backward(dict(zip(out, Abar)))
    ref_out = [T.vals[i] for i in out]
    ref_in = [bars.get(i, np.zeros_like(T.vals[i])) for i in inp]
    ref_th = adjoint.step_parameter_gradient(model, [bars.get(w, 0) for w in wids],
                                             mpo_hamiltonian)
    m = binding.Model(model.N, model.omega, model.g, model.nmax, model.V)
    try:
        m.set_adjoint_krylov_basis(basis)
        A_out, Abar_in, th = m.step_vjp(M, [dev(x) for x in A], tau, [dev(x) for x in Abar])
    finally:
        m.close()
    for got, ref in zip(A_out, ref_out):
        assert np.abs(got.cpu().numpy() - ref).max() <= out_bound * max(np.abs(ref).max(), 1e-300)
    scale = max(np.abs(x).max() for x in ref_in)
    for got, ref in zip(Abar_in, ref_in):
        assert np.abs(got.cpu().numpy() - ref).max() <= bound * scale
    ref_vec = [ref_th[("omega", 0)], ref_th[("g", 0)], ref_th[("V", -1)]]
    tscale = max(abs(x) for x in ref_vec)
    for got, ref in zip(th, ref_vec):
        assert abs(got - ref) <= bound * tscale


def test_correlation_states_vjp_matches_oracle():
    """C_n and the reverse pass of the real-time correlation of two given states
    (tdmrg_correlation_states_vjp) against ``oracle/adjoint.correlation_vjp``: random states at
    M = 4, three steps stored every two (one recomputed stretch of two, one of one)."""
    from oracle import adjoint, tdvp
    from oracle.model import HolsteinModel, mpo_current, mpo_hamiltonian, site_list
    from paper_2003_13245_gb300 import binding
    model = HolsteinModel(N=3, omega=[1.0], g=[0.7], nmax=[2], V=0.8)
    rng = np.random.default_rng(9100)
    d = [s[3] for s in site_list(model)]
    Ws, Wj = mpo_hamiltonian(model), mpo_current(model)
    Mb = tdvp.bond_dims([x * x for x in d], 4)
    states = []
    for _ in range(2):
        A0 = [random_complex(rng, (Mb[k], d[k] ** 2, Mb[k + 1])) for k in range(len(d))]
        p = tdvp.PurifiedMPS(model, A0, Ws)
        p.right_canonicalize()
        A = [x.copy() for x in p.A]
        A[0] = A[0] / np.linalg.norm(A[0])
        states.append(A)
    dt, ns = 0.1, 3
    cbar = random_complex(rng, (ns + 1,))
    C, g1, g2, Wb, Wjb = adjoint.correlation_vjp(Ws, Wj, d, states[0], states[1], dt, ns, cbar,
                                                 every=2)
    gH = adjoint.step_parameter_gradient(model, Wb, mpo_hamiltonian)
    gJ = adjoint.step_parameter_gradient(model, Wjb, mpo_current)
    ref_th = [gH[p] + gJ[p] for p in (("omega", 0), ("g", 0), ("V", -1))]
    m = binding.Model(model.N, model.omega, model.g, model.nmax, model.V)
    try:
        Cg, h1, h2, th = m.correlation_states_vjp(4, [dev(x) for x in states[0]],
                                                  [dev(x) for x in states[1]], dt, ns, cbar)
    finally:
        m.close()
    assert np.abs(Cg - C).max() <= 1e-10 * np.abs(C).max()
    for got, ref in zip(h1 + h2, g1 + g2):
        assert np.abs(got.cpu().numpy() - ref).max() <= 1e-8 * max(np.abs(x).max() for x in g1 + g2)
    tscale = max(abs(x) for x in ref_th)
    for got, ref in zip(th, ref_th):
        assert abs(got - ref) <= 1e-8 * tscale


@pytest.mark.parametrize("basis", [False, True])
@pytest.mark.parametrize("M,rank_tol", [(4, None), (64, 1e-8)])
def test_correlation_vjp_matches_oracle_pipeline(M, rank_tol, basis):
    """The gradient of the whole C(t) computation (tdmrg_correlation_vjp) against the oracle's
    reverse pass of its pipeline: below full bond dimension (M = 4, completed gauge columns
    everywhere; the oracle matches central differences to 2e-9 there) and at full bond
    dimension with rank threshold 1e-8 (the oracle matches the ED gradient to 5e-8)."""
    from oracle import adjoint, gradient
    from oracle.model import HolsteinModel, mpo_current, mpo_hamiltonian
    from paper_2003_13245_gb300 import binding
    model = HolsteinModel(N=3, omega=[1.0], g=[0.7], nmax=[2], V=0.8)
    rng = np.random.default_rng(9200 + M)
    beta, dtau, dt, ns = 0.2, 0.05, 0.1, 3
    cbar = random_complex(rng, (ns + 1,))
    kw = {} if rank_tol is None else dict(rank_tol=rank_tol)
    C, g = adjoint.correlation_pipeline_gradient(model, beta, dtau, M, dt, ns, cbar,
                                                 mpo_hamiltonian, mpo_current, **kw)
    ref = [g[p] for p in gradient.parameters(model)]
    m = binding.Model(model.N, model.omega, model.g, model.nmax, model.V)
    try:
        if rank_tol is not None:
            m.set_rank_tol(rank_tol)
        m.set_adjoint_krylov_basis(basis)
        Cg, th, _ = m.correlation_vjp(beta, dtau, M, dt, ns, cbar)
    finally:
        m.close()
    assert np.abs(Cg - C).max() <= 1e-9 * np.abs(C).max()
    scale = max(abs(x) for x in ref)
    for got, r in zip(th, ref):
        assert abs(got - r) <= 1e-6 * scale


def test_autograd_gradient_matches_central_differences():
    """The torch.autograd.Function over the library (forward tdmrg_correlation, backward
    tdmrg_correlation_vjp): d/dtheta of Re sum conj(w_n) C(t_n) against central differences of
    the library's own forward C(t) in omega, g and V, to 1e-6 relative (h = 1e-4: O(h^2)
    1e-8, Krylov stopping 1e-13 / h)."""
    from paper_2003_13245_gb300 import binding
    spec = dict(N=3, nmax=[2], beta=0.2, dtau=0.05, M=4, dt=0.1, nsteps=3)
    rng = np.random.default_rng(9300)
    w = torch.as_tensor(random_complex(rng, (spec["nsteps"] + 1,)))
    theta = torch.tensor([1.0, 0.7, 0.8], dtype=torch.float64, requires_grad=True)
    loss = (torch.conj(w) * binding.correlation_autograd(theta, spec)).real.sum()
    loss.backward()
    grad = theta.grad.numpy()

    def value(t):
        with torch.no_grad():
            C = binding.correlation_autograd(torch.tensor(t, dtype=torch.float64), spec)
            return float((torch.conj(w) * C).real.sum())

    h = 1e-4
    base = theta.detach().numpy()
    fd = np.array([(value(base + h * e) - value(base - h * e)) / (2 * h) for e in np.eye(3)])
    assert np.abs(grad - fd).max() <= 1e-6 * np.abs(fd).max()
