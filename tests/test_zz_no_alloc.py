"""The allocation-free gauge QR (tdmrg_kernel_gauge_qr_noalloc) against the allocating one.

It serves callers that cannot allocate device memory (all device memory owned by another
runtime or pool, or no allocation allowed once set up);
two calls in a row must give the same Q and R as tdmrg_kernel_gauge_qr, which also shows that
the shared scratch left by one call does not leak into the next."""
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


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


@pytest.mark.parametrize("m,n,rank,p", [(4096, 128, 128, 0), (1000, 130, 97, 40)])
def test_noalloc_matches_allocating_entry_point(m, n, rank, p):
    from paper_2003_13245_gb300 import binding
    rng = np.random.default_rng(11 * m + n)
    Y = random_complex(rng, (m, rank)) @ random_complex(rng, (rank, n))
    E = _dev(random_complex(rng, (m, p))) if p else None
    Yd = _dev(Y)
    Qa = torch.zeros((m, n), dtype=torch.complex128, device="cuda")
    Ra = torch.zeros((n, n), dtype=torch.complex128, device="cuda")
    binding.kernel_gauge_qr(Yd, Qa, Ra, E)
    for _ in range(2):
        Qn = torch.full((m, n), float("nan"), dtype=torch.complex128, device="cuda")
        Rn = torch.full((n, n), float("nan"), dtype=torch.complex128, device="cuda")
        binding.kernel_gauge_qr_noalloc(Yd, Qn, Rn, E)
        assert torch.abs(Qn - Qa).max().item() < 1e-12
        assert torch.abs(Rn - Ra).max().item() < 1e-12 * torch.abs(Ra).max().item()


def test_noalloc_rejects_sizes_beyond_its_scratch():
    from paper_2003_13245_gb300 import binding
    Y = torch.zeros((300, 257), dtype=torch.complex128, device="cuda")
    Q = torch.zeros_like(Y)
    R = torch.zeros((257, 257), dtype=torch.complex128, device="cuda")
    with pytest.raises(binding.TdmrgError) as e:
        binding.kernel_gauge_qr_noalloc(Y, Q, R)
    assert "n <= 256" in str(e.value)


def test_noalloc_rejects_rows_beyond_shared_memory():
    """m so large that one block's row slice exceeds the kernel's 200 KB of shared memory is
    refused on the host with a message, before any launch (no buffer is touched)."""
    import ctypes
    from paper_2003_13245_gb300 import binding
    lib = binding.load()
    Y = torch.zeros((1, 1), dtype=torch.complex128, device="cuda")
    p = ctypes.c_void_p(Y.data_ptr())
    rc = lib.tdmrg_kernel_gauge_qr_noalloc(4_200_000, 1, p, 0, None, p, p, None, None)
    assert rc == -1
    assert "shared memory" in lib.tdmrg_last_global_error().decode()
