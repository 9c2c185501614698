"""Tensor-core (tcgen05, 3xTF32) contractions against FP64 references on the same seeded
inputs.  Tolerance: 3xTF32 keeps about 21 significant bits per product with FP32
accumulation, so the error of a length-K complex dot product of O(1) entries is bounded by
~ 1e-6 * sqrt(K) relative to the largest output; the tests use 2e-5 of max|C|."""
import numpy as np
import pytest

from tests.inputs import random_complex, random_mpo_site

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

TOL = 2e-5


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2003_13245_gb300.build import build_library
    build_library()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


@pytest.mark.parametrize("M,N,K,cA,cB", [(128, 64, 32, 0, 0), (1, 1, 1, 0, 0), (130, 70, 33, 1, 0),
                                         (300, 200, 700, 0, 1), (64, 129, 96, 1, 1),
                                         (1000, 130, 128, 0, 0), (128, 128, 4096, 1, 0),
                                         (40, 70, 900, 0, 1)])
def test_zgemm_tc(M, N, K, cA, cB):
    from paper_2003_13245_gb300 import binding
    rng = np.random.default_rng(M + 3 * N + 7 * K)
    A = random_complex(rng, (M, K))
    B = random_complex(rng, (N, K))
    ref = (A.conj() if cA else A) @ (B.conj() if cB else B).T
    C = torch.zeros((M, N), dtype=torch.complex128, device="cuda")
    binding.kernel_zgemm_tc(dev(A), dev(B), C, cA, cB)
    err = np.abs(C.cpu().numpy() - ref).max() / np.abs(ref).max()
    assert err < TOL, err


HEFF_CASES = [(1, 4, 2, 1, 7), (4, 16, 4, 7, 7), (37, 53, 3, 7, 7), (64, 64, 2, 7, 7),
              (96, 70, 4, 6, 6), (130, 129, 2, 7, 1), (128, 128, 8, 7, 7)]


@pytest.mark.parametrize("Ml,Mr,d,Dl,Dr", HEFF_CASES)
def test_heff_tc_matches_oracle(Ml, Mr, d, Dl, Dr):
    from oracle import tdvp
    from paper_2003_13245_gb300 import binding
    rng = np.random.default_rng(2000 + Ml + Mr)
    L = random_complex(rng, (Dl, Ml, Ml))
    R = random_complex(rng, (Dr, Mr, Mr))
    W = random_mpo_site(rng, Dl, Dr, d)
    A = random_complex(rng, (Ml, d * d, Mr))
    ref = tdvp.heff(L, W, R, A, d)
    n = Ml * d * d * Mr
    ws = torch.zeros(binding.heff_workspace_floats(Ml, Mr, d, Dl, Dr), dtype=torch.float32,
                     device="cuda")
    out = torch.zeros(n, dtype=torch.complex128, device="cuda")
    binding.kernel_heff(dev(L), W, dev(R), dev(A), out, None, None, d,
                        precision=binding.PREC_C64_3XTF32, ws32=ws)
    got = out.cpu().numpy().reshape(ref.shape)
    err = np.abs(got - ref).max() / np.abs(ref).max()
    assert err < TOL, err


@pytest.mark.parametrize("ksplit,tile_n,M,N", [(1, 64, 128, 64), (3, 64, 128, 64),
                                               (8, 64, 128, 64), (1, 128, 165, 197),
                                               (3, 128, 165, 197), (2, None, 165, 197)])
def test_splitk_table_is_applied_and_exact(ksplit, tile_n, M, N, tmp_path, monkeypatch):
    """A tile-table entry for a contraction shape (split-K factor and tile width, 64 or 128
    columns; a line without a width means 64) changes only the summation order: with the entry
    forced through a table file, C = A B^T still matches FP64 to the 3xTF32 bound for its
    length: an FP32 sum of K products carries up to K 2^-24 of the sum of their moduli, which
    for random entries is about K 2^-24 of max|C| (2.4e-4 at K = 4096; an unsplit loop sums all
    4096 products in one FP32 accumulator, measured 7e-5), ragged row and column tiles
    included, and the timed entry point runs that shape at every candidate."""
    from paper_2003_13245_gb300 import binding
    K = 4096
    table = tmp_path / "table.txt"
    table.write_text("# test\n%d %d %d 1 1 %d%s\n" % (M, N, K, ksplit,
                                                      "" if tile_n is None else " %d" % tile_n))
    monkeypatch.setenv("TDMRG_SPLITK_TABLE", str(table))
    binding.tune_reload_table()
    try:
        rng = np.random.default_rng(77 + ksplit)
        A = random_complex(rng, (M, K))
        B = random_complex(rng, (N, K))
        C = torch.zeros((M, N), dtype=torch.complex128, device="cuda")
        binding.kernel_zgemm_tc(dev(A), dev(B), C, 0, 0)
        ref = A @ B.T
        assert np.abs(C.cpu().numpy() - ref).max() / np.abs(ref).max() < K * 2.0 ** -24
        assert binding.kernel_tc_gemm_timed(M, N, K, 1, 1, ksplit, reps=2,
                                            tile_n=tile_n or 64) > 0.0
    finally:
        monkeypatch.delenv("TDMRG_SPLITK_TABLE")
        binding.tune_reload_table()


@pytest.mark.parametrize("Ml,Mr,d,Dl,Dr", HEFF_CASES + [(128, 128, 6, 7, 7), (50, 130, 10, 8, 3),
                                           (37, 64, 8, 7, 7), (20, 32, 4, 5, 3),
                                           (50, 32, 2, 6, 6)])
def test_sweep_heff_path_matches_oracle(Ml, Mr, d, Dl, Dr):
    """The H_eff product as the sweep runs it (tdmrg_kernel_heff_timed: split, L.A contraction,
    MPO mixing into split planes, contraction with R, with the tile table) against the oracle,
    3xTF32 bound; ragged row and column tiles, local dimensions d = 2 .. 10."""
    from oracle import tdvp
    from paper_2003_13245_gb300 import binding
    rng = np.random.default_rng(3000 + Ml + Mr + d)
    L = random_complex(rng, (Dl, Ml, Ml))
    R = random_complex(rng, (Dr, Mr, Mr))
    W = random_mpo_site(rng, Dl, Dr, d)
    A = random_complex(rng, (Ml, d * d, Mr))
    ref = tdvp.heff(L, W, R, A, d)
    out = torch.zeros((Ml, d * d, Mr), dtype=torch.complex128, device="cuda")
    ms = binding.kernel_heff_timed(dev(L), W, dev(R), dev(A), out, d, binding.PREC_C64_3XTF32,
                                   reps=1)
    assert ms > 0.0
    err = np.abs(out.cpu().numpy() - ref).max() / np.abs(ref).max()
    assert err < TOL, err
