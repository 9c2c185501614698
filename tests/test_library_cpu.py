"""Host-side checks of the C ABI library (no GPU needed): it loads, exports every declared
symbol, its pure-host mobility matches the oracle's quadrature, and it reports errors."""
import os

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2003_13245_gb300.build import build_library
    build_library()
    from paper_2003_13245_gb300 import binding
    return binding.load()


def test_exports_every_declared_symbol(lib):
    from paper_2003_13245_gb300 import binding
    names = binding.declared_symbols(os.path.join(ROOT, "include", "tdmrg.h"))
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n


def test_mobility_matches_oracle(lib):
    from oracle import kubo
    from paper_2003_13245_gb300 import binding
    t = np.linspace(0, 8, 161)
    C = np.exp(-0.3 * t) * (np.cos(t) + 0.2j * np.sin(t))
    assert abs(binding.mobility(t, C, 0.7) - kubo.mobility(t, C, 0.7)) < 1e-14


def test_mean_free_path_matches_oracle(lib):
    """Eq. 8 through the C ABI equals the oracle's quadrature on a sign-changing Re C."""
    from oracle import kubo
    from paper_2003_13245_gb300 import binding
    t = np.linspace(0, 8, 161)
    C = np.exp(-0.3 * t) * (1.7 * np.cos(2.1 * t) + 0.2j * np.sin(t))
    got = binding.mean_free_path(t, C)
    ref = kubo.mean_free_path(t, C)
    assert max(abs(a - b) for a, b in zip(got, ref)) < 1e-14
    with pytest.raises(binding.TdmrgError):
        binding.mean_free_path(t, -C)          # <j j> must be positive


def test_argument_errors_are_reported(lib):
    from paper_2003_13245_gb300 import binding
    with pytest.raises(binding.TdmrgError) as e:
        binding.mobility([0.0], [1.0], 1.0)
    assert e.value.code == -1
    with pytest.raises(binding.TdmrgError) as e:
        binding.mobility([0.5, 1.0], [1.0, 1.0], 1.0)
    assert "t_grid[0]" in str(e.value)
    with pytest.raises(binding.TdmrgError) as e:
        binding.Model(2, [1.0], [1.0], [4], 1.0)     # N < 3 is rejected before any CUDA call
    assert e.value.code == -1
    # non-finite parameters (a corrupted configuration) are rejected before any CUDA call
    for bad in (dict(omega=[float("nan")]), dict(g=[float("inf")]), dict(V=float("nan"))):
        a = {**dict(N=3, omega=[1.0], g=[1.0], nmax=[4], V=1.0), **bad}
        with pytest.raises(binding.TdmrgError) as e:
            binding.Model(a["N"], a["omega"], a["g"], a["nmax"], a["V"])
        assert e.value.code == -1 and "non-finite" in str(e.value)
        with pytest.raises(binding.TdmrgError) as e:
            binding.host_mpo(a["N"], a["omega"], a["g"], a["nmax"], a["V"])
        assert e.value.code == -1
    # kernel-level entry points check their arguments before touching the device
    rc = lib.tdmrg_kernel_bond_exp(0, 7, None, None, None, None, 0.0, -0.05, 1e-7, 32, None, None)
    assert rc == -1
    rc = lib.tdmrg_kernel_bond_exp(16, 7, 1, 1, 1, 1, 0.0, -0.05, 1e-7, 33, None, None)
    assert rc == -1
    rc = lib.tdmrg_kernel_bond_exp(257, 7, 1, 1, 1, 1, 0.0, -0.05, 1e-7, 32, None, None)
    assert rc == -1
    # tile widths other than 0, 64 and 128 are rejected before any allocation
    import ctypes
    ms = ctypes.c_double()
    for tile_n in (32, 96, -64):
        rc = lib.tdmrg_kernel_tc_gemm_timed(128, 64, 256, 1, 1, 1, tile_n, 2, ctypes.byref(ms),
                                            None)
        assert rc == -1
    # the quadrature node rule checks its bound, cap and tolerance
    for args in ((-1.0, 16, 1e-15), (float("nan"), 16, 1e-15), (1.0, 0, 1e-15), (1.0, 65, 1e-15),
                 (1.0, 16, 0.0)):
        with pytest.raises(binding.TdmrgError) as e:
            binding.host_quadrature_nodes(*args)
        assert e.value.code == -1


def _mpo_params(peierls):
    from oracle.model import HolsteinModel
    extra = {} if peierls is None else dict(zip(("alpha", "omega_p", "nmax_p"), peierls))
    return HolsteinModel(N=3, omega=[0.7], g=[1.3], nmax=[2], V=0.6, **extra)


def _host_mpo(model, which, param=-1):
    from paper_2003_13245_gb300 import binding
    peierls = (model.alpha, model.omega_p, model.nmax_p) if model.peierls else None
    return binding.host_mpo(model.N, model.omega, model.g, model.nmax, model.V, which, param,
                            peierls)


@pytest.mark.parametrize("peierls", [None, (0.3, 0.5, 2)])
def test_host_mpo_equals_definition(lib, peierls):
    """The library's MPOs of H and j (built on the host, no GPU) contract to the operators of
    Eq. 1 / Eq. 10 and Eq. 3 written term by term with Kronecker products."""
    from oracle.model import dense_from_definition, mpo_to_dense
    from paper_2003_13245_gb300 import binding
    model = _mpo_params(peierls)
    H, J = dense_from_definition(model)
    assert np.abs(mpo_to_dense(_host_mpo(model, binding.MPO_H)) - H).max() < 1e-13
    assert np.abs(mpo_to_dense(_host_mpo(model, binding.MPO_J)) - J).max() < 1e-13
    Id = mpo_to_dense(_host_mpo(model, binding.MPO_IDENTITY))
    assert np.array_equal(Id, np.eye(H.shape[0]))


@pytest.mark.parametrize("peierls", [None, (0.3, 0.5, 2)])
def test_host_mpo_parameter_derivatives(lib, peierls):
    """sum_k (MPO with site k replaced by its derivative site) == dH/dtheta and dj/dtheta of
    the term-by-term operators, for omega, g, V (and alpha, omega_p with a bond mode); both
    operators are affine in each parameter, so the derivative is the difference at +1."""
    import dataclasses
    from oracle.model import dense_from_definition, mpo_to_dense
    from paper_2003_13245_gb300 import binding
    model = _mpo_params(peierls)
    shifts = [dict(omega=[model.omega[0] + 1.0]), dict(g=[model.g[0] + 1.0]),
              dict(V=model.V + 1.0)]
    if peierls is not None:
        shifts += [dict(alpha=model.alpha + 1.0), dict(omega_p=model.omega_p + 1.0)]
    H0, J0 = dense_from_definition(model)
    W0 = {w: _host_mpo(model, w) for w in (binding.MPO_H, binding.MPO_J)}
    for p, sh in enumerate(shifts):
        H1, J1 = dense_from_definition(dataclasses.replace(model, **sh))
        for w, ref in ((binding.MPO_H, H1 - H0), (binding.MPO_J, J1 - J0)):
            dW = _host_mpo(model, w, p)
            D = sum(mpo_to_dense(W0[w][:k] + [dW[k]] + W0[w][k + 1:]) for k in range(len(dW)))
            assert np.abs(D - ref).max() < 1e-12, (p, w)
    with pytest.raises(binding.TdmrgError):
        _host_mpo(model, binding.MPO_H, len(shifts))      # one past the last parameter


@pytest.mark.parametrize("k,spread", [(1, 1.0), (5, 1.0), (17, 30.0), (32, 40.0)])
def test_host_tridiagonal_exponential_matches_dense_expm(lib, k, spread):
    """exp(z T) e_1 of a real symmetric tridiagonal T from the library's host Jacobi
    eigendecomposition against scipy's dense matrix exponential, at real, imaginary and complex
    z over [0, 1] of a step (the points a reverse pass needs from one Krylov basis); T carries
    an energy offset like the Lanczos matrices of the sweep.  |tau| times the spectral spread
    reaches 14 here (the sweep's steps stay below 5); at 68 two FP64 methods already differ by
    2e-10 through cancellation, which is no test of either."""
    import scipy.linalg as sl
    from paper_2003_13245_gb300 import binding
    rng = np.random.default_rng(600 + k)
    alpha = spread * rng.standard_normal(k) + 40.0
    beta = np.abs(spread * rng.standard_normal(k - 1))
    T = np.diag(alpha) + np.diag(beta, 1) + np.diag(beta, -1)
    zs = [s * tau for tau in (-0.05, -0.1j, 0.02 - 0.05j) for s in np.linspace(0.0, 1.0, 5)]
    got = binding.host_tridiag_exp(alpha, beta, zs)
    for z, g in zip(zs, got):
        ref = sl.expm(z * T)[:, 0]
        assert np.abs(g - ref).max() <= 1e-12 * np.abs(ref).max(), z


def test_host_tridiagonal_exponential_rejects_bad_input(lib):
    from paper_2003_13245_gb300 import binding
    with pytest.raises(binding.TdmrgError):
        binding.host_tridiag_exp(np.zeros(65), np.zeros(64), [0.1])
    with pytest.raises(binding.TdmrgError):
        binding.host_tridiag_exp([1.0, float("nan")], [0.5], [0.1])


@pytest.mark.parametrize("n", [1, 2, 7, 16, 64])
def test_host_gauss_legendre_rule(lib, n):
    """The quadrature of the exponential VJPs: nodes and weights on [0, 1] equal numpy's
    Gauss-Legendre rule mapped from [-1, 1], and the rule integrates polynomials of degree
    2n - 1 exactly."""
    from paper_2003_13245_gb300 import binding
    s, w = binding.host_gauss_legendre(n)
    x, v = np.polynomial.legendre.leggauss(n)
    assert np.abs(s - 0.5 * (x + 1)).max() < 1e-14 and np.abs(w - 0.5 * v).max() < 1e-14
    for deg in (0, n, 2 * n - 1):
        assert abs(np.sum(w * s ** deg) - 1.0 / (deg + 1)) < 1e-13


@pytest.mark.parametrize("r", [0.0, 0.05, 0.5, 1.5, 4.0, 12.0])
def test_host_quadrature_node_count_meets_its_bound(lib, r):
    """The node count of the Krylov-basis quadrature, pinned by closed forms: with the count
    chosen for the bound r, Gauss-Legendre integrates the scalar Frechet integrands
    e^{s x} e^{(1-s) y} on [0, 1] with |x| + |y| = r to within 1e-15 e^{r/2} of
    (e^x - e^y)/(x - y), for real (imaginary time) and imaginary (real time) exponents, and one
    node fewer violates the bound (the count is the smallest)."""
    from math import log, lgamma
    from paper_2003_13245_gb300 import binding
    eps = 1e-15
    n = binding.host_quadrature_nodes(r, 64, eps)
    assert 2 <= n <= 64
    s, w = binding.host_gauss_legendre(n)
    for x, y in ((0.5 * r, -0.5 * r), (0.5j * r, -0.5j * r), (0.3 * r, -0.7 * r)):
        f = np.exp(s * x) * np.exp((1 - s) * y)
        exact = (np.exp(x) - np.exp(y)) / (x - y) if r > 0 else 1.0
        assert abs(np.sum(w * f) - exact) <= eps * np.exp(0.5 * r) + 4e-16 * n
    if n > 2:
        m = n - 1
        lc = 4 * lgamma(m + 1) - log(2 * m + 1) - 3 * lgamma(2 * m + 1)
        assert lc + 2 * m * log(r) + r > log(eps)
    assert binding.host_quadrature_nodes(r, 3, eps) == min(n, 3)


def test_tile_table_parsing(lib, tmp_path, monkeypatch):
    """The tile table read beside the library (or from TDMRG_SPLITK_TABLE): lines
    "M N K nred nbatch ksplit [tile_n]" with the width 64 when absent, comments skipped, lines
    with a width other than 64 / 128 or a split below 1 ignored, unlisted shapes (0, 0); and
    the committed table lists the shapes of the c2 bulk-site H_eff contractions."""
    from paper_2003_13245_gb300 import binding
    table = tmp_path / "table.txt"
    table.write_text("# comment\n128 64 4096 1 1 3\n165 197 4096 1 1 2 128   # ms\n"
                     "10 10 10 1 1 2 96\n11 11 11 1 1 0 64\n")
    monkeypatch.setenv("TDMRG_SPLITK_TABLE", str(table))
    binding.tune_reload_table()
    try:
        assert binding.tune_table_lookup(128, 64, 4096, 1, 1) == (3, 64)
        assert binding.tune_table_lookup(165, 197, 4096, 1, 1) == (2, 128)
        assert binding.tune_table_lookup(10, 10, 10, 1, 1) == (0, 0)
        assert binding.tune_table_lookup(11, 11, 11, 1, 1) == (0, 0)
        assert binding.tune_table_lookup(1, 2, 3, 4, 5) == (0, 0)
    finally:
        monkeypatch.delenv("TDMRG_SPLITK_TABLE")
        binding.tune_reload_table()
    ks, bn = binding.tune_table_lookup(8192, 128, 128, 7, 1)     # second contraction, c2 bulk
    assert ks >= 1 and bn in (64, 128)
    ks, bn = binding.tune_table_lookup(896, 8192, 128, 1, 1)     # first contraction, c2 bulk
    assert ks >= 1 and bn in (64, 128)
