"""Pins for the exact-diagonalisation oracle: closed forms, limits and invariants of Eq. 2-7."""
import numpy as np
import scipy.linalg

from oracle import kubo
from oracle import model as om
from oracle.ed import ED, sector_operators


def test_sector_matches_full_space():
    """The one-carrier-sector ED equals the full product space restricted by the projector."""
    m = om.HolsteinModel(N=3, omega=[1.0], g=[0.7], nmax=[2], V=0.8)
    beta = 1.3
    H, J = om.dense_from_definition(m)
    P = np.diag(np.isclose(np.diag(om.carrier_number_dense(m)), 1.0).astype(float))
    rho = P @ scipy.linalg.expm(-beta * H) @ P
    Z = np.trace(rho).real
    rho /= Z
    ed = ED(m, beta)
    assert abs(ed.logZ - np.log(Z)) < 1e-12
    for t in (0.0, 0.4, 1.7):
        U = scipy.linalg.expm(-1j * H * t)
        c_full = np.trace(rho @ U.conj().T @ J @ U @ J)
        assert abs(ed.correlation(t)[0] - c_full) < 1e-12


def test_free_band_closed_form():
    """g = 0: C(t) is constant and equals sum_k p_k (2 V sin k)^2."""
    for N, V, beta in [(3, 1.0, 1.0), (5, 0.6, 2.0), (4, 1.3, 0.5)]:
        m = om.HolsteinModel(N=N, omega=[1.0], g=[0.0], nmax=[3], V=V)
        ed = ED(m, beta)
        ref = kubo.free_band_correlation(N, V, beta)
        C = ed.correlation(np.linspace(0, 7, 11))
        assert np.abs(C - ref).max() < 1e-12
    # the N=3, V=1, beta=1 value in closed form: 6e / (e^-2 + 2e)
    assert abs(kubo.free_band_correlation(3, 1.0, 1.0) - 6 * np.e / (np.exp(-2) + 2 * np.e)) < 1e-14


def test_zero_transfer_integral_gives_zero():
    m = om.HolsteinModel(N=3, omega=[1.0], g=[1.0], nmax=[3], V=0.0)
    ed = ED(m, 1.0)
    assert np.abs(ed.correlation(np.linspace(0, 5, 6))).max() == 0.0


def test_correlation_symmetries():
    """C(-t) = C(t)*, Im C(0) = 0, C(0) = Tr[rho j^2] > 0, Tr rho = 1."""
    m = om.HolsteinModel(N=3, omega=[1.0], g=[1.0], nmax=[4], V=1.0)
    ed = ED(m, 1.0)
    t = np.linspace(0.1, 6, 9)
    assert np.abs(ed.correlation(-t) - ed.correlation(t).conj()).max() < 1e-12
    c0 = ed.correlation(0.0)[0]
    rho = ed.rho()
    assert abs(np.trace(rho) - 1.0) < 1e-13
    assert abs(c0 - np.trace(rho @ ed.J @ ed.J)) < 1e-12
    assert abs(c0.imag) < 1e-14 and c0.real > 0
    # direct matrix exponentials, not the eigen-sum
    H, J = sector_operators(m)
    w, U = np.linalg.eigh(H)
    for ti in (0.3, 2.2):
        Ut = scipy.linalg.expm(-1j * H * ti)
        direct = np.trace(rho @ Ut.conj().T @ J @ Ut @ J)
        assert abs(ed.correlation(ti)[0] - direct) < 1e-11


def test_hopping_limit_matches_derived_fgr():
    """Small V: C(t)/V^2 -> 2 exp{-sum 2 g^2 [2n+1 - n e^{iwt} - (n+1) e^{-iwt}]} (Eq. 7 in this
    model's conventions).  Agreement is O(V^2) plus phonon truncation; 1e-2 relative to C(0)."""
    V, w, g, kT = 1e-3, 1.0, 0.5, 1.0
    m = om.HolsteinModel(N=3, omega=[w], g=[g], nmax=[8], V=V)
    ed = ED(m, 1.0 / kT)
    t = np.array([0.0, 0.5, 1.0, 2.0, 3.0, 4.5])
    C = ed.correlation(t)
    ref = kubo.fgr_correlation(t, V, [w], [g], kT)
    assert np.abs(C - ref).max() / abs(ref[0]) < 1e-2
    # the printed form of Eq. 7 (no factors 2, opposite phase) does not match this model
    printed = V * V * np.exp(-(g * g) * (2 * kubo.bose(w, kT) + 1
                                         - kubo.bose(w, kT) * np.exp(-1j * w * t)
                                         - (kubo.bose(w, kT) + 1) * np.exp(1j * w * t)))
    assert np.abs(C - printed).max() / abs(ref[0]) > 0.1


def test_kubo_trapezoid():
    """Eq. 2 on a Gaussian C(t) = e^{-t^2/2}: mu = sqrt(pi/2) / kT; exact for linear pieces."""
    t = np.linspace(0, 12, 4801)
    C = np.exp(-t * t / 2) + 0j
    assert abs(kubo.mobility(t, C, 2.0) - np.sqrt(np.pi / 2) / 2.0) < 1e-6
    t = np.array([0.0, 1.0, 3.0])
    C = np.array([2.0, 1.0, 0.0]) + 1j
    assert abs(kubo.mobility(t, C, 1.0) - (1.5 + 1.0)) < 1e-15


# ---- mean free path (Eq. 8) -------------------------------------------------------------------

def test_mean_free_path_gaussian_closed_form():
    """C(t) = C0 exp(-t^2 / (2 s^2)): v = sqrt(C0), tau = s sqrt(pi / 2) (t_max = 12 s)."""
    from oracle import kubo
    C0, s = 2.5, 0.7
    t = np.linspace(0.0, 12 * s, 4001)
    C = C0 * np.exp(-t ** 2 / (2 * s * s)) * (1 + 0.3j * t)     # Im C does not enter
    v, tau, l = kubo.mean_free_path(t, C)
    assert abs(v - np.sqrt(C0)) < 1e-15
    assert abs(tau - s * np.sqrt(np.pi / 2)) < 1e-9
    assert abs(l - v * tau) < 1e-15


def test_mean_free_path_free_band_grows_with_cutoff():
    """g = 0: C is constant (free band), so tau equals the cut-off t_max."""
    from oracle import kubo
    c = kubo.free_band_correlation(3, 1.0, 1.0)
    t = np.arange(0, 201) * 0.05
    v, tau, l = kubo.mean_free_path(t, np.full(t.size, c + 0j))
    assert abs(tau - t[-1]) < 1e-12 and abs(v - np.sqrt(c)) < 1e-15


def test_mean_free_path_takes_absolute_values():
    """Re C = cos(w t) exp(-g t) changes sign: tau = int_0^T |cos w t| e^{-g t} dt (adaptive
    quadrature split at the zeros of the cosine) -- dropping the absolute value fails this."""
    import scipy.integrate
    from oracle import kubo
    w, gam, T = 3.0, 0.4, 12.0
    t = np.linspace(0.0, T, 24001)
    C = np.cos(w * t) * np.exp(-gam * t) + 0j
    zeros = [(k + 0.5) * np.pi / w for k in range(int(T * w / np.pi) + 1) if (k + 0.5) * np.pi / w < T]
    ref = scipy.integrate.quad(lambda x: abs(np.cos(w * x)) * np.exp(-gam * x), 0.0, T,
                               points=zeros, limit=200, epsabs=1e-13)[0]
    _, tau, _ = kubo.mean_free_path(t, C)
    assert abs(tau - ref) < 1e-6
    signed = np.trapezoid(C.real, t)
    assert abs(signed - ref) > 0.1
