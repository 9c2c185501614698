"""Parameter sweeps on the GPU: the hopping-limit (Fermi golden rule) mobility of Eq. 7 for a
batch of parameter sets, and the frequency-scaling isotope scan (omega_m ~ m^-1/2 with the
reorganisation energy g_m^2 omega_m held fixed, so g_m ~ m^1/4) on the batched TD-DMRG path and
through the adjoint, each against the oracle."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2003_13245_gb300.build import build_library
    build_library()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def isotope(omega, g, m):
    """Approach 2 of the isotope study: all frequencies scaled by m^-1/2, g^2 omega fixed."""
    return [w / np.sqrt(m) for w in omega], [x * m ** 0.25 for x in g]


@pytest.mark.parametrize("K", [1, 4])
def test_fgr_batch_matches_oracle(K):
    """tdmrg_fgr_mobility_batch against the oracle's derived hopping-limit C(t) integrated by
    the oracle's Eq. 2 quadrature, on 37 random parameter sets (a partial last warp of blocks)
    and on the isotope scan of one of them; 1e-12 relative."""
    from oracle import kubo
    from paper_2003_13245_gb300 import binding
    rng = np.random.default_rng(700 + K)
    P, dt, nt = 37, 0.02, 1501
    om = rng.uniform(0.1, 1.5, (P, K))
    g = rng.uniform(0.1, 1.2, (P, K))
    V = rng.uniform(0.01, 0.3, P)
    kT = rng.uniform(0.3, 2.0, P)
    ms = np.array([1.0, 13.0 / 12.0, 20.0 / 12.0])
    om_i = np.array([isotope(om[0], g[0], m)[0] for m in ms])
    g_i = np.array([isotope(om[0], g[0], m)[1] for m in ms])
    om = np.vstack([om, om_i])
    g = np.vstack([g, g_i])
    V = np.concatenate([V, np.full(3, V[0])])
    kT = np.concatenate([kT, np.full(3, kT[0])])
    mu = binding.fgr_mobility_batch(om, g, V, kT, dt, nt)
    t = np.arange(nt) * dt
    for p in range(om.shape[0]):
        ref = kubo.mobility(t, kubo.fgr_correlation(t, V[p], om[p], g[p], kT[p]), kT[p])
        assert abs(mu[p] - ref) <= 1e-12 * abs(ref) + 1e-300


MASSES = [1.0, 1.1, 1.2]
CHAIN = dict(N=3, omega=[1.0], g=[0.9], nmax=[2], V=0.7, kT=1.0)


def test_isotope_scan_batch_matches_ed():
    """The isotope scan as one batch of TD-DMRG instances (tdmrg_batch_correlation, full bond
    dimension M = 64): mu(m) of every instance through tdmrg_mobility equals ED's mu(m) to
    1e-10 of C(0) t_max / kT."""
    from oracle import kubo
    from oracle.ed import ED
    from oracle.model import HolsteinModel
    from paper_2003_13245_gb300 import Batch, Model, binding
    c = CHAIN
    models = []
    for m in MASSES:
        w, g = isotope(c["omega"], c["g"], m)
        mod = Model(c["N"], w, g, c["nmax"], c["V"], krylov=(1e-13, 32, 12))
        mod.thermal_prepare(1.0 / c["kT"], 0.05, 64)
        mod.realtime_init()
        models.append(mod)
    b = Batch(models)
    t = np.arange(0, 41) * 0.05
    C = b.correlation(t, 0.05)
    b.close()
    for mod in models:
        mod.close()
    for m, cm in zip(MASSES, C):
        w, g = isotope(c["omega"], c["g"], m)
        ref = ED(HolsteinModel(N=c["N"], omega=w, g=g, nmax=c["nmax"], V=c["V"]),
                 1.0 / c["kT"]).correlation(t)
        scale = abs(ref[0]) * t[-1] / c["kT"]
        assert abs(binding.mobility(t, cm, c["kT"]) - kubo.mobility(t, ref, c["kT"])) < 1e-10 * scale


@pytest.mark.parametrize("m", [1.0, 1.1])
def test_isotope_derivative_by_adjoint_matches_ed(m):
    """dmu/dm at m = 1 and 1.1 from the adjoint (tdmrg_correlation_vjp with the trapezoid
    weights of Eq. 2 as the cotangent, then d omega/dm = -omega / 2m, dg/dm = g / 4m) against
    the exact Frechet gradient of ED (oracle.gradient), full bond dimension with the gauge-QR
    rank threshold 1e-8 (the pipeline adjoint equals the ED gradient there to 5e-8); 1e-6 of
    the largest dmu/dtheta."""
    from oracle import gradient
    from oracle.model import HolsteinModel
    from paper_2003_13245_gb300 import Model
    c = CHAIN
    kT = 5.0                           # beta = 0.2: two imaginary steps (GPU test time)
    w, g = isotope(c["omega"], c["g"], m)
    dt, ns = 0.1, 4
    t = np.arange(ns + 1) * dt
    wts = np.full(ns + 1, dt / kT)
    wts[0] *= 0.5
    wts[-1] *= 0.5
    mod = Model(c["N"], w, g, c["nmax"], c["V"])
    try:
        mod.set_rank_tol(1e-8)
        mod.set_adjoint_krylov_basis(True)
        _, th, _ = mod.correlation_vjp(1.0 / kT, 0.05, 64, dt, ns, wts)
    finally:
        mod.close()
    model = HolsteinModel(N=c["N"], omega=w, g=g, nmax=c["nmax"], V=c["V"])
    _, dmu = gradient.mobility_gradient(model, kT, t)
    ref = [dmu[p] for p in gradient.parameters(model)]
    scale = max(abs(x) for x in ref)
    for got, r in zip(th, ref):
        assert abs(got - r) <= 1e-6 * scale
    K = len(w)
    dmdm = sum(-0.5 * w[i] / m * th[i] + 0.25 * g[i] / m * th[K + i] for i in range(K))
    assert abs(dmdm - gradient.isotope_derivative(model, dmu) / m) <= 1e-6 * scale


def test_holstein_peierls_paradigms_batch_match_ed():
    """The three coupling paradigms of the Holstein-Peierls study (Eq. 10) as one batch at full
    bond dimension (N = 3, one local mode and one bond mode of two levels each: caps 4^k, so
    M = 256 is exact): Holstein only (alpha = 0), Peierls only (g = 0) and both.  Each
    instance's mu equals ED's to 1e-10 of C(0) t_max / kT; Matthiessen's mu_M is the harmonic
    combination of the first two."""
    from oracle import kubo
    from oracle.ed import ED
    from oracle.model import HolsteinModel
    from paper_2003_13245_gb300 import Batch, Model, binding
    specs = [("H", 0.0, [0.9]), ("P", 0.4, [0.0]), ("HP", 0.4, [0.9])]
    wp, nmp, V, kT = 0.6, 2, 0.7, 2.0
    models = []
    for _, alpha, g in specs:
        m = Model(3, [1.0], g, [2], V, peierls=(alpha, wp, nmp), krylov=(1e-13, 32, 12))
        m.thermal_prepare(1.0 / kT, 0.05, 256)
        m.realtime_init()
        models.append(m)
    b = Batch(models)
    t = np.arange(0, 9) * 0.05
    C = b.correlation(t, 0.05)
    b.close()
    for m in models:
        m.close()
    mus = {}
    for (name, alpha, g), c in zip(specs, C):
        ref = ED(HolsteinModel(N=3, omega=[1.0], g=g, nmax=[2], V=V, alpha=alpha, omega_p=wp,
                               nmax_p=nmp), 1.0 / kT).correlation(t)
        mu = binding.mobility(t, c, kT)
        assert abs(mu - kubo.mobility(t, ref, kT)) < 1e-10 * abs(ref[0]) * t[-1] / kT
        mus[name] = mu
    mu_M = 1.0 / (1.0 / mus["H"] + 1.0 / mus["P"])
    assert min(mus["H"], mus["P"]) > mu_M > 0.0
