"""Kernel-level parity: each hot-path contraction through the C ABI against the oracle's
plain FP64 implementation on the same seeded inputs (sizes span several 64-wide tiles and
ragged tails)."""
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


HEFF_CASES = [
    # Ml, Mr, d, Dl, Dr
    (1, 4, 2, 1, 7),
    (4, 16, 4, 7, 7),
    (37, 53, 3, 7, 7),
    (64, 64, 2, 7, 7),
    (96, 70, 4, 6, 6),
    (130, 129, 2, 7, 1),
]


@pytest.mark.parametrize("Ml,Mr,d,Dl,Dr", HEFF_CASES)
def test_heff_matches_oracle(Ml, Mr, d, Dl, Dr):
    from oracle import tdvp
    from paper_2003_13245_gb300 import binding
    rng = np.random.default_rng(1000 + Ml + Mr)
    L = random_complex(rng, (Dl, Ml, Ml))
    R = random_complex(rng, (Dr, Mr, Mr))
    W = random_mpo_site(rng, Dl, Dr, d)
    A = random_complex(rng, (Ml, d * d, Mr))
    ref = tdvp.heff(L, W, R, A, d)
    n = Ml * d * d * Mr
    X = torch.zeros(max(Dl, Dr) * n, dtype=torch.complex128, device="cuda")
    Y = torch.zeros_like(X)
    out = torch.zeros(n, dtype=torch.complex128, device="cuda")
    binding.kernel_heff(dev(L), W, dev(R), dev(A), out, X, Y, d)
    got = out.cpu().numpy().reshape(ref.shape)
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("Ml1,Mr1,Ml2,Mr2,d,Dl,Dr", [
    (1, 4, 1, 4, 2, 1, 7), (16, 64, 16, 64, 2, 7, 7), (33, 47, 29, 51, 3, 7, 6), (70, 70, 70, 70, 4, 6, 1)])
def test_env_left_matches_oracle(Ml1, Mr1, Ml2, Mr2, d, Dl, Dr):
    from oracle import tdvp
    from paper_2003_13245_gb300 import binding
    rng = np.random.default_rng(77 + Ml1 + Mr2)
    L = random_complex(rng, (Dl, Ml1, Ml2))
    W = random_mpo_site(rng, Dl, Dr, d)
    bra = random_complex(rng, (Ml1, d * d, Mr1))
    ket = random_complex(rng, (Ml2, d * d, Mr2))
    ref = tdvp.update_left(L, bra, W, ket, d)
    X = torch.zeros(max(Dl, Dr) * Ml1 * d * d * Mr2, dtype=torch.complex128, device="cuda")
    Y = torch.zeros_like(X)
    out = torch.zeros((Dr, Mr1, Mr2), dtype=torch.complex128, device="cuda")
    binding.kernel_env_left(dev(L), W, dev(bra), dev(ket), out, X, Y, d)
    assert np.abs(out.cpu().numpy() - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("blocked", [False, True])
@pytest.mark.parametrize("m,n,rank,p", [(12, 5, 5, 0), (300, 64, 64, 0), (1000, 130, 97, 40),
                                        (64, 64, 30, 0), (4096, 128, 128, 0), (256, 70, 3, 300),
                                        (8192, 128, 128, 0), (2048, 128, 60, 200)])
def test_gauge_qr_matches_oracle(m, n, rank, p, blocked):
    """Full-rank and rank-deficient (with and without completion candidates) gauge QR."""
    from oracle import tdvp
    from paper_2003_13245_gb300 import binding
    rng = np.random.default_rng(m * 7 + n)
    Y = random_complex(rng, (m, rank)) @ random_complex(rng, (rank, n))
    if rank < n:
        Y[:, rng.choice(n, size=min(n - rank, 5), replace=False)] = 0.0
    E = random_complex(rng, (m, p)) if p else None
    Qr, Rr = tdvp.gauge_qr(Y, E)
    # the C ABI zeroes R rows of completed positions (the oracle returns Q^H Y there)
    Q = torch.zeros((m, n), dtype=torch.complex128, device="cuda")
    R = torch.zeros((n, n), dtype=torch.complex128, device="cuda")
    qr = binding.kernel_gauge_qr_blocked if blocked else binding.kernel_gauge_qr
    qr(dev(Y), Q, R, dev(E) if E is not None else None)
    Qg, Rg = Q.cpu().numpy(), R.cpu().numpy()
    assert np.abs(Qg.conj().T @ Qg - np.eye(n)).max() < 1e-12
    assert np.abs(Qg @ Rg - Y).max() <= 1e-10 * np.abs(Y).max()
    # the same columns are taken and the same completion vectors are chosen
    if rank == n:
        assert np.abs(Qg - Qr).max() < 1e-9
    else:
        acc = np.abs(np.diag(Rr)) > 0
        assert np.array_equal(np.abs(np.diag(Rg)) > 0, acc)
        # accepted columns are well defined up to rounding amplified by small residuals
        assert np.abs(np.abs(np.einsum("ij,ij->j", Qg.conj(), Qr)) - 1).max() < 1e-6


def test_gauge_qr_blocked_too_wide_for_shared_memory():
    """A factor whose row slices and block coefficients exceed a block's shared memory
    (24576 x 640 on 152 blocks) is factorised by the column-wise kernel instead: for a full-rank
    Y the result is the QR with a real positive diagonal, which Q^H Q = 1, Q R = Y and R upper
    triangular with diag(R) > 0 fix uniquely."""
    from paper_2003_13245_gb300 import binding
    rng = np.random.default_rng(24576)
    m, n = 24576, 640
    Y = random_complex(rng, (m, n))
    Q = torch.zeros((m, n), dtype=torch.complex128, device="cuda")
    R = torch.zeros((n, n), dtype=torch.complex128, device="cuda")
    binding.kernel_gauge_qr_blocked(dev(Y), Q, R, None)
    Qg, Rg = Q.cpu().numpy(), R.cpu().numpy()
    assert np.abs(Qg.conj().T @ Qg - np.eye(n)).max() < 1e-12
    assert np.abs(Qg @ Rg - Y).max() <= 1e-10 * np.abs(Y).max()
    assert np.abs(np.tril(Rg, -1)).max() == 0.0
    dg = np.diag(Rg)
    assert np.all(dg.real > 0) and np.abs(dg.imag).max() == 0.0


@pytest.mark.parametrize("tau", [-0.3j, -0.05, 0.05, -2.0j, 0.4 - 1.5j])
def test_krylov_dense_matches_expm(tau):
    import scipy.linalg
    from paper_2003_13245_gb300 import binding
    rng = np.random.default_rng(3)
    n = 100
    A = random_complex(rng, (n, n))
    H = (A + A.conj().T) / 8
    v = random_complex(rng, (n,))
    ref = scipy.linalg.expm(tau * H) @ v
    out = torch.zeros(n, dtype=torch.complex128, device="cuda")
    k = binding.kernel_krylov_dense(dev(H), dev(v), out, tau, tol=1e-14, kmax=32)
    got = out.cpu().numpy()
    assert 1 <= k <= 32
    assert np.abs(got - ref).max() / np.abs(ref).max() < 1e-11


def _hermitian(rng, shape):
    A = random_complex(rng, shape)
    return (A + np.conj(np.swapaxes(A, -1, -2))) / 2


@pytest.mark.parametrize("M,Dw,tau", [(1, 3, -0.05), (5, 7, 0.025), (33, 7, -0.025j),
                                      (64, 7, -0.05j), (100, 6, 0.025), (128, 7, -0.025j),
                                      (150, 5, -0.05)])
def test_bond_exp_matches_oracle(M, Dw, tau):
    """Fused bond exponential (one cooperative launch, complex FP32 contractions, FP64
    Lanczos) against the oracle's Krylov exponential of the zero-site operator.  The bound
    2e-5 of max|ref| allows the FP32 contraction error (2^-24 per product, summed over
    Dw*M terms in FP32, amplified by |tau| ||K|| <= ~2) with a margin of ~10."""
    from oracle import tdvp
    from paper_2003_13245_gb300 import binding
    rng = np.random.default_rng(500 + M + Dw)
    L = _hermitian(rng, (Dw, M, M)) / np.sqrt(M)
    R = _hermitian(rng, (Dw, M, M)) / np.sqrt(M)
    C = random_complex(rng, (M, M))
    ref, _ = tdvp.krylov_expm(lambda X: tdvp.bond_heff(L, R, X), C, tau, tol=1e-13)
    out = torch.zeros((M, M), dtype=torch.complex128, device="cuda")
    k = binding.kernel_bond_exp(dev(L), dev(R), dev(C), out, tau, tol=1e-7)
    assert 1 <= k <= 32
    got = out.cpu().numpy()
    assert np.abs(got - ref).max() <= 2e-5 * np.abs(ref).max()
    # fixed reduction order: a second launch gives the same bits
    out2 = torch.zeros_like(out)
    binding.kernel_bond_exp(dev(L), dev(R), dev(C), out2, tau, tol=1e-7)
    assert torch.equal(out, out2)


@pytest.mark.parametrize("Ml,Mr,d,Dl,Dr", HEFF_CASES)
def test_heff_vjp_matches_oracle(Ml, Mr, d, Dl, Dr):
    """VJP of the H_eff product (the adjoint step's building block, made of the forward
    H_eff and environment kernels with daggered operands) against the oracle's contraction
    VJP, FP64."""
    from oracle import adjoint
    from paper_2003_13245_gb300 import binding
    rng = np.random.default_rng(2000 + Ml + Mr)
    L = random_complex(rng, (Dl, Ml, Ml))
    R = random_complex(rng, (Dr, Mr, Mr))
    W = random_mpo_site(rng, Dl, Dr, d) + 0.3j * random_mpo_site(rng, Dl, Dr, d)
    A = random_complex(rng, (Ml, d * d, Mr))
    yb = random_complex(rng, (Ml, d * d, Mr))
    Ar, Lr, _, Rr = adjoint.heff_vjp(L, W, R, A, d, yb)
    n = Ml * d * d * Mr
    X = torch.zeros(max(Dl, Dr) * n, dtype=torch.complex128, device="cuda")
    Y = torch.zeros_like(X)
    Ab = torch.zeros(A.shape, dtype=torch.complex128, device="cuda")
    Lb = torch.zeros(L.shape, dtype=torch.complex128, device="cuda")
    Rb = torch.zeros(R.shape, dtype=torch.complex128, device="cuda")
    binding.kernel_heff_vjp(dev(L), W, dev(R), dev(A), dev(yb), Ab, Lb, Rb, X, Y, d)
    for got, ref in ((Ab, Ar), (Lb, Lr), (Rb, Rr)):
        g = got.cpu().numpy()
        assert np.abs(g - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("tau", [-0.1j, -0.05])
def test_site_exp_vjp_matches_oracle(tau):
    """VJP of a site exponential exp(tau H_eff) A (environments of a Hermitian MPO, so H_eff
    is Hermitian) against the oracle: Krylov-exponential VJP with the same 16 Gauss-Legendre
    nodes, mapped onto L and R through the contraction VJP.  Both sides take 33 Lanczos
    exponentials (GPU tol 1e-13, oracle 1e-14): bound 1e-9 of the largest entry."""
    from oracle import adjoint, tdvp
    from oracle.model import HolsteinModel, mpo_hamiltonian, site_list
    from paper_2003_13245_gb300 import binding
    model = HolsteinModel(N=3, omega=[1.0], g=[0.7], nmax=[3], V=0.8)
    rng = np.random.default_rng(3000)
    d_all = [s[3] for s in site_list(model)]
    D = [x * x for x in d_all]
    Mb = tdvp.bond_dims(D, 64)
    Ws = mpo_hamiltonian(model)
    psi = tdvp.PurifiedMPS(model, [random_complex(rng, (Mb[k], D[k], Mb[k + 1]))
                                   for k in range(len(D))], Ws)
    psi.right_canonicalize()
    psi.step(-0.05j, tdvp.KrylovOpts(tol=1e-13))      # builds left and right environments
    k = 2
    L, R, W, d = psi.Lenv[k], psi.Renv[k], Ws[k], d_all[k]
    A = random_complex(rng, (Mb[k], D[k], Mb[k + 1]))
    yb = random_complex(rng, A.shape)
    mv = lambda x: tdvp.heff(L, W, R, x, d)            # noqa: E731
    Ar, pairs = adjoint.expm_krylov_vjp(mv, A, tau, yb, nodes=16, tol=1e-14)
    Lr = sum(adjoint.heff_vjp(L, W, R, b, d, c)[1] for c, b in pairs)
    Rr = sum(adjoint.heff_vjp(L, W, R, b, d, c)[3] for c, b in pairs)
    Ab = torch.zeros(A.shape, dtype=torch.complex128, device="cuda")
    Lb = torch.zeros(L.shape, dtype=torch.complex128, device="cuda")
    Rb = torch.zeros(R.shape, dtype=torch.complex128, device="cuda")
    binding.kernel_site_exp_vjp(dev(L), W, dev(R), dev(A), dev(yb), tau, Ab, Lb, Rb, d,
                                nodes=16, tol=1e-13)
    for got, ref in ((Ab, Ar), (Lb, Lr), (Rb, Rr)):
        assert np.abs(got.cpu().numpy() - ref).max() <= 1e-9 * np.abs(ref).max()


@pytest.mark.parametrize("m,n", [(12, 5), (300, 64), (1000, 128), (64, 64)])
def test_qr_vjp_matches_oracle(m, n):
    """VJP of the full-rank gauge QR against the oracle's formula on the oracle's factors."""
    from oracle import adjoint, tdvp
    from paper_2003_13245_gb300 import binding
    rng = np.random.default_rng(4000 + m + n)
    Y = random_complex(rng, (m, n))
    Q, R = tdvp.gauge_qr(Y)
    Qb = random_complex(rng, (m, n))
    Rb = random_complex(rng, (n, n))
    ref = adjoint.qr_vjp(Q, R, Qb, Rb)
    out = torch.zeros((m, n), dtype=torch.complex128, device="cuda")
    binding.kernel_qr_vjp(dev(Q), dev(R), dev(Qb), dev(Rb), out)
    assert np.abs(out.cpu().numpy() - ref).max() <= 1e-10 * np.abs(ref).max()


@pytest.mark.parametrize("M,Dw,tau", [(5, 3, -0.2j), (40, 7, -0.05), (64, 7, -0.1j)])
def test_bond_exp_vjp_matches_oracle(M, Dw, tau):
    """VJP of the bond exponential exp(tau K) C (Hermitian K) against the oracle's Krylov VJP
    (same 16 nodes) mapped through the bond-product VJP; bound 1e-9 of the largest entry."""
    from oracle import adjoint, tdvp
    from paper_2003_13245_gb300 import binding
    rng = np.random.default_rng(5000 + M)
    L = _hermitian(rng, (Dw, M, M)) / np.sqrt(M)
    R = _hermitian(rng, (Dw, M, M)) / np.sqrt(M)
    C = random_complex(rng, (M, M))
    yb = random_complex(rng, (M, M))
    mv = lambda X: tdvp.bond_heff(L, R, X)             # noqa: E731
    Cr, pairs = adjoint.expm_krylov_vjp(mv, C, tau, yb, nodes=16, tol=1e-14)
    Lr = sum(adjoint.bond_heff_vjp(L, R, b, c)[1] for c, b in pairs)
    Rr = sum(adjoint.bond_heff_vjp(L, R, b, c)[2] for c, b in pairs)
    Cb = torch.zeros((M, M), dtype=torch.complex128, device="cuda")
    Lb = torch.zeros((Dw, M, M), dtype=torch.complex128, device="cuda")
    Rb = torch.zeros((Dw, M, M), dtype=torch.complex128, device="cuda")
    binding.kernel_bond_exp_vjp(dev(L), dev(R), dev(C), dev(yb), tau, Cb, Lb, Rb)
    for got, ref in ((Cb, Cr), (Lb, Lr), (Rb, Rr)):
        assert np.abs(got.cpu().numpy() - ref).max() <= 1e-9 * np.abs(ref).max()
