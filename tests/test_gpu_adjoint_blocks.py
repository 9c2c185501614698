"""Parity of the remaining building blocks of a reverse sweep through the C ABI against the
oracle's VJPs (FP64): environment updates (both sides, with parameter cotangents through
derivative MPO sites), gauge-completion candidates (both sides) and the gauge QR with completed
columns.  Sizes span several 64-wide tiles with ragged tails."""
import numpy as np
import pytest

from tests.inputs import random_complex, random_mpo_site

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


def zeros(shape):
    return torch.zeros(shape, dtype=torch.complex128, device="cuda")


CASES = [(5, 6, 3, 4, 3), (37, 70, 2, 7, 7), (96, 65, 3, 6, 1)]


@pytest.mark.parametrize("side", [0, 1])
@pytest.mark.parametrize("Ml,Mr,d,Dl,Dr", CASES)
def test_env_vjp_matches_oracle(side, Ml, Mr, d, Dl, Dr):
    from oracle import adjoint
    from paper_2003_13245_gb300 import binding
    rng = np.random.default_rng(6000 + 2 * Ml + side)
    W = random_mpo_site(rng, Dl, Dr, d) + 0.3j * random_mpo_site(rng, Dl, Dr, d)
    dW = [random_mpo_site(rng, Dl, Dr, d) + 0j for _ in range(2)] + [np.zeros_like(W)]
    bra = random_complex(rng, (Ml, d * d, Mr))
    ket = random_complex(rng, (Ml, d * d, Mr))
    if side == 0:
        E, G = random_complex(rng, (Dl, Ml, Ml)), random_complex(rng, (Dr, Mr, Mr))
        Er, br, Wr, kr = adjoint.update_left_vjp(E, bra, W, ket, d, G)
    else:
        E, G = random_complex(rng, (Dr, Mr, Mr)), random_complex(rng, (Dl, Ml, Ml))
        Er, br, Wr, kr = adjoint.update_right_vjp(E, bra, W, ket, d, G)
    n = Ml * d * d * Mr
    X, Y = zeros(max(Dl, Dr) * n), zeros(max(Dl, Dr) * n)
    Eb, bb, kb = zeros(E.shape), zeros(bra.shape), zeros(ket.shape)
    tb = binding.kernel_env_vjp(side, dev(E), dev(bra), W, dev(ket), dev(G), Eb, bb, kb, X, Y, d,
                                dW=dW)
    for got, ref in ((Eb, Er), (bb, br), (kb, kr)):
        assert np.abs(got.cpu().numpy() - ref).max() <= 1e-12 * np.abs(ref).max()
    for t, x in zip(tb, dW):
        ref = float(np.vdot(Wr, x).real)
        assert abs(t - ref) <= 1e-12 * max(abs(ref), np.abs(Wr).max())


@pytest.mark.parametrize("side", [0, 1])
@pytest.mark.parametrize("Ml,Mr,d,Dl,Dr", CASES)
def test_expansion_vjp_matches_oracle(side, Ml, Mr, d, Dl, Dr):
    from oracle import adjoint, tdvp
    from paper_2003_13245_gb300 import binding
    rng = np.random.default_rng(7000 + 2 * Ml + side)
    W = random_mpo_site(rng, Dl, Dr, d) + 0.3j * random_mpo_site(rng, Dl, Dr, d)
    dW = [random_mpo_site(rng, Dl, Dr, d) + 0j for _ in range(2)]
    A = random_complex(rng, (Ml, d * d, Mr))
    if side == 0:
        E = random_complex(rng, (Dl, Ml, Ml))
        Xb = random_complex(rng, tdvp.left_expansion(E, W, A, d).shape)
        Er, Wr, Ar = adjoint.left_expansion_vjp(E, W, A, d, Xb)
    else:
        E = random_complex(rng, (Dr, Mr, Mr))
        Xb = random_complex(rng, tdvp.right_expansion(W, A, E, d).shape)
        Wr, Ar, Er = adjoint.right_expansion_vjp(W, A, E, d, Xb)
    n = Ml * d * d * Mr
    X, Y = zeros(max(Dl, Dr) * n), zeros(max(Dl, Dr) * n)
    Eb, Ab = zeros(E.shape), zeros(A.shape)
    tb = binding.kernel_expansion_vjp(side, dev(E), W, dev(A), dev(Xb), Eb, Ab, X, Y, d, dW=dW)
    for got, ref in ((Eb, Er), (Ab, Ar)):
        assert np.abs(got.cpu().numpy() - ref).max() <= 1e-12 * np.abs(ref).max()
    for t, x in zip(tb, dW):
        ref = float(np.vdot(Wr, x).real)
        assert abs(t - ref) <= 1e-12 * max(abs(ref), np.abs(Wr).max())


@pytest.mark.parametrize("m,n,rank,p", [(14, 6, 4, 3), (300, 96, 70, 40), (256, 256, 200, 64)])
def test_qr_vjp_completed_matches_oracle(m, n, rank, p):
    """Rank-deficient Y = B G (dependent columns skipped) completed from candidates X; the
    chosen candidates and the factors come from the oracle's gauge QR."""
    from oracle import adjoint, tdvp
    from paper_2003_13245_gb300 import binding
    rng = np.random.default_rng(8000 + m + n)
    Y = random_complex(rng, (m, rank)) @ random_complex(rng, (rank, n))
    X0 = random_complex(rng, (m, p))
    chosen = []
    Q, R = tdvp.gauge_qr(Y, X0, chosen=chosen)
    acc = (np.abs(np.diag(R)) > 0).astype(np.int32)
    assert acc.sum() == rank
    Xs = np.ascontiguousarray(np.concatenate(
        [X0[:, [c]] if c < p else np.eye(m)[:, [c - p]] for c in chosen], axis=1))
    Qb, Rb = random_complex(rng, (m, n)), random_complex(rng, (n, n))
    Yr, Xr = adjoint.qr_vjp_completed(Q, R, Qb, Rb, Xs)
    Yb, Xb = zeros((m, n)), zeros(Xs.shape)
    binding.kernel_qr_vjp_completed(acc, dev(Q), dev(R), dev(Xs), dev(Qb), dev(Rb), Yb, Xb)
    assert np.abs(Yb.cpu().numpy() - Yr).max() <= 1e-9 * np.abs(Yr).max()
    assert np.abs(Xb.cpu().numpy() - Xr).max() <= 1e-9 * np.abs(Xr).max()
