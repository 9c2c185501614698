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
    # kernel-level entry points check their arguments before touching the device
    rc = lib.tdmrg_kernel_bond_exp(0, 7, None, None, None, None, 0.0, -0.05, 1e-7, 32, None, None)
    assert rc == -1
    rc = lib.tdmrg_kernel_bond_exp(16, 7, 1, 1, 1, 1, 0.0, -0.05, 1e-7, 33, None, None)
    assert rc == -1
    rc = lib.tdmrg_kernel_bond_exp(257, 7, 1, 1, 1, 1, 0.0, -0.05, 1e-7, 32, None, None)
    assert rc == -1
