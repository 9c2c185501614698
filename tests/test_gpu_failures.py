"""Failure paths of the library on the GPU, exercised without faulting, trapping or hanging it.

* Timeout: every grid barrier of the cooperative kernels is a bounded wait.  Lowering the
  handle's limit to one clock cycle makes the barriers of multi-block launches give up; the
  blocks leave, the status word is read on the host and the call returns TDMRG_ERR_TIMEOUT.
  Restoring the limit and preparing again reproduces exact diagonalisation: the handle and the
  context stay usable.
* Non-convergence: a site Krylov exponential limited to two vectors at tolerance 1e-15 stops
  unconverged; the call returns TDMRG_ERR_NOCONV, and the next preparation with the default
  Krylov settings is exact again."""
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


def _ed_check(m):
    from oracle.ed import ED
    from oracle.model import HolsteinModel
    ed = ED(HolsteinModel(N=3, omega=[1.0], g=[1.0], nmax=[2], V=1.0), 1.0)
    t = np.arange(0, 5) * 0.05
    C = m.correlation(t, 0.05)
    assert abs(m.logz() - ed.logZ) < 1e-10
    assert np.abs(C - ed.correlation(t)).max() / abs(ed.correlation(t)[0]) < 1e-10


@pytest.mark.parametrize("precision", [0, 1])
def test_barrier_timeout_is_reported_and_recoverable(precision):
    from paper_2003_13245_gb300 import Model, TdmrgError
    m = Model(3, [1.0], [1.0], [2], 1.0, precision=precision)
    try:
        m.set_wait_cycles(1)
        with pytest.raises(TdmrgError) as e:
            m.thermal_prepare(1.0, 0.05, 64)
        assert e.value.code == -6
        assert "timed out" in str(e.value)
        m.set_wait_cycles(0)
        if precision == 0:
            m.thermal_prepare(1.0, 0.05, 64)
            _ed_check(m)
        else:
            m.thermal_prepare(1.0, 0.05, 64)
            assert np.isfinite(m.logz())
    finally:
        m.close()


def test_krylov_nonconvergence_is_reported_and_recoverable():
    from paper_2003_13245_gb300 import Model, TdmrgError
    m = Model(3, [1.0], [1.0], [2], 1.0, krylov=(1e-15, 2, 0))
    try:
        with pytest.raises(TdmrgError) as e:
            m.thermal_prepare(1.0, 0.05, 64)
        assert e.value.code == -5
        m.set_krylov(1e-13, 32, 0)
        m.thermal_prepare(1.0, 0.05, 64)
        _ed_check(m)
    finally:
        m.close()
