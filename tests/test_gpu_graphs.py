"""Graph mode (captured half-sweeps with a fixed Krylov dimension) and batched stepping of
independent instances against the plain stream path."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    torch = pytest.importorskip("torch")
    from paper_2003_13245_gb300.build import build_library
    build_library()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _run(graphs, precision=0, V=1.0, nsteps=6):
    from paper_2003_13245_gb300 import Model
    m = Model(3, [1.0], [1.0], [2], V, precision=precision, krylov=(1e-13, 32, 12))
    if graphs:
        m.set_graphs(True)
    m.thermal_prepare(1.0, 0.05, 64)
    m.realtime_init()
    out = [m.realtime_observe()]
    for _ in range(nsteps):
        m.realtime_step(1, 0.05)
        out.append(m.realtime_observe())
    lz = m.logz()
    m.close()
    return lz, np.array(out)


@pytest.mark.parametrize("precision", [0, 1])
def test_graph_replay_equals_stream_execution(precision):
    lz0, c0 = _run(False, precision)
    lz1, c1 = _run(True, precision)
    assert abs(lz1 - lz0) < 1e-13
    assert np.abs(c1 - c0).max() < 1e-12 * abs(c0[0])


def test_fixed_krylov_full_rank_matches_ed():
    from oracle.ed import ED
    from oracle.model import HolsteinModel
    lz, C = _run(True, 0)
    ed = ED(HolsteinModel(N=3, omega=[1.0], g=[1.0], nmax=[2], V=1.0), 1.0)
    ref = ed.correlation(np.arange(7) * 0.05)
    assert abs(lz - ed.logZ) < 1e-10
    assert np.abs(C - ref).max() / abs(ref[0]) < 1e-10


def test_batch_equals_individual_runs():
    from paper_2003_13245_gb300 import Batch, Model
    Vs = [0.5, 1.0, 2.0]
    singles = [_run(False, 0, V=V, nsteps=4)[1] for V in Vs]
    models = []
    for V in Vs:
        m = Model(3, [1.0], [1.0], [2], V, krylov=(1e-13, 32, 12))
        m.thermal_prepare(1.0, 0.05, 64)
        m.realtime_init()
        models.append(m)
    b = Batch(models)
    got = [[m.realtime_observe()] for m in models]
    for _ in range(4):
        b.realtime_step(1, 0.05)
        for i, m in enumerate(models):
            got[i].append(m.realtime_observe())
    b.close()
    for m in models:
        m.close()
    for g, s in zip(got, singles):
        g = np.array(g)
        assert np.abs(g - s).max() < 1e-10 * abs(s[0])


# (N, V, kT, M): three chains of two lengths and uneven bond dimensions, each at its full rank
BATCH_ED = [(3, 0.5, 1.0, 64), (3, 2.0, 0.5, 64), (4, 1.0, 2.0, 256)]


def test_batch_correlation_matches_ed():
    """tdmrg_batch_correlation (Eq. 6 for every instance, all advanced together by half-steps)
    against exact diagonalisation of each instance: full bond dimension, so 1e-10 of C(0)."""
    from oracle.ed import ED
    from oracle.model import HolsteinModel
    from paper_2003_13245_gb300 import Batch, Model
    models = []
    for N, V, kT, M in BATCH_ED:
        m = Model(N, [1.0], [1.0], [2], V, krylov=(1e-13, 32, 12))
        m.thermal_prepare(1.0 / kT, 0.05, M)
        m.realtime_init()
        models.append(m)
    b = Batch(models)
    t = np.arange(0, 9, 2) * 0.05
    C = b.correlation(t, 0.05)
    b.close()
    for m in models:
        m.close()
    for (N, V, kT, M), c in zip(BATCH_ED, C):
        ref = ED(HolsteinModel(N=N, omega=[1.0], g=[1.0], nmax=[2], V=V), 1.0 / kT).correlation(t)
        assert np.abs(c - ref).max() / abs(ref[0]) < 1e-10


def test_batch_half_steps_equal_whole_steps():
    """Two tdmrg_batch_step_half calls are one second-order step: same C as tdmrg_batch_
    realtime_step of a twin batch (bit for bit up to 1e-13), and a whole step is refused while
    a second half is pending."""
    from paper_2003_13245_gb300 import Batch, Model, TdmrgError
    twins = []
    for _ in range(2):
        ms = []
        for N, V, kT, M in BATCH_ED[:2]:
            m = Model(N, [1.0], [1.0], [2], V, krylov=(1e-13, 32, 12))
            m.thermal_prepare(1.0 / kT, 0.05, M)
            m.realtime_init()
            ms.append(m)
        twins.append(ms)
    b_half, b_whole = Batch(twins[0]), Batch(twins[1])
    for _ in range(3):
        b_half.step_half(0.05)
        with pytest.raises(TdmrgError):
            b_half.realtime_step(1, 0.05)
        b_half.step_half(0.05)
        b_whole.realtime_step(1, 0.05)
    got = [m.realtime_observe() for m in twins[0]]
    ref = [m.realtime_observe() for m in twins[1]]
    b_half.close()
    b_whole.close()
    for ms in twins:
        for m in ms:
            m.close()
    for g, r in zip(got, ref):
        assert abs(g - r) < 1e-13 * abs(r) + 1e-15
