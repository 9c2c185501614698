"""Writes the stored expected values of the GPU parity tests.  Calls only ``oracle/``.

    python tests/golden/make_golden.py
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import tdvp  # noqa: E402
from oracle.model import HolsteinModel  # noqa: E402


def perturbed_spread(run, rel=1e-14, seeds=(1, 2, 3)):
    """Spread of the oracle's own result when every gauge-QR input is perturbed by a relative
    Gaussian noise of size `rel` (a few ulp of accumulated FP64 rounding).  Below full rank the
    one-site TDVP dynamics depends on basis directions of tiny singular values, so this spread
    -- not machine precision -- bounds the attainable agreement of two correct FP64 codes."""
    ref_logz, ref_C = run()
    orig = tdvp.gauge_qr
    dz, dc = 0.0, 0.0
    for sd in seeds:
        rng = np.random.default_rng(sd)

        def noisy(Y, extra=None, **kw):
            return orig(Y * (1.0 + rel * rng.standard_normal(Y.shape)), extra, **kw)

        tdvp.gauge_qr = noisy
        try:
            lz, C = run()
        finally:
            tdvp.gauge_qr = orig
        dz = max(dz, abs(lz - ref_logz))
        dc = max(dc, float(np.abs(C - ref_C).max() / abs(ref_C[0])))
    return dz, dc


def c1_prefix():
    """N=3 Holstein chain, one mode (w = g = V = kT = 1, nmax = 4), M = 64 (below the full
    ranks), dtau = dt = 0.05: the oracle TD-DMRG C(t) on the first 20 real-time steps, with the
    tolerances set to 10x the oracle's spread under 1e-14 relative perturbations."""
    p = dict(N=3, omega=[1.0], g=[1.0], nmax=[4], V=1.0, beta=1.0, dtau=0.05, M=64, dt=0.05)
    m = HolsteinModel(N=p["N"], omega=p["omega"], g=p["g"], nmax=p["nmax"], V=p["V"])

    def run():
        r = tdvp.correlation(m, p["beta"], p["dtau"], p["M"], p["dt"], 20, every=5)
        run.last = r
        return r.logZ, r.C

    dz, dc = perturbed_spread(run)
    logz, C = run()
    r = run.last
    p.update(t=r.t.tolist(), C_re=C.real.tolist(), C_im=C.imag.tolist(), logZ=logz,
             spread_logZ=dz, spread_C=dc, tol=max(1e-10, 10 * dc), logz_tol=max(1e-10, 10 * dz),
             source="oracle.tdvp.correlation; spread: 3 runs with 1e-14 relative noise on every "
                    "gauge-QR input")
    with open(os.path.join(HERE, "c1_M64_prefix.json"), "w") as f:
        json.dump(p, f, indent=1)


def c2_modes_prefix():
    """The c2 chain's two modes per molecule, (w, g, nmax) = (0.2, 1.5, 8) and (1.0, 0.8, 4),
    on N = 3 molecules at V = 0.5, kT = 2 (5 imaginary steps of dtau = 0.05), M = 128: the bulk
    sites are 128 x 64 x 128 as in the N = 16 benchmark chain, so every kernel path of the
    benchmark runs (split-K tensor-core H_eff, fused bond exponential at M = 128, blocked QR of
    8192 x 128).  The oracle's C(t) on the first 10 real-time steps (dt = 0.05), with the
    tolerances set to 10x the oracle's spread under 1e-14 relative perturbations."""
    p = dict(N=3, omega=[0.2, 1.0], g=[1.5, 0.8], nmax=[8, 4], V=0.5, beta=0.5, dtau=0.05, M=128,
             dt=0.05)
    m = HolsteinModel(N=p["N"], omega=p["omega"], g=p["g"], nmax=p["nmax"], V=p["V"])

    def run():
        r = tdvp.correlation(m, p["beta"], p["dtau"], p["M"], p["dt"], 10, every=2)
        run.last = r
        return r.logZ, r.C

    dz, dc = perturbed_spread(run, seeds=(1, 2))
    logz, C = run()
    r = run.last
    p.update(t=r.t.tolist(), C_re=C.real.tolist(), C_im=C.imag.tolist(), logZ=logz,
             spread_logZ=dz, spread_C=dc, tol=max(1e-10, 10 * dc), logz_tol=max(1e-10, 10 * dz),
             source="oracle.tdvp.correlation; spread: 2 runs with 1e-14 relative noise on every "
                    "gauge-QR input")
    with open(os.path.join(HERE, "c2modes_N3_M128_prefix.json"), "w") as f:
        json.dump(p, f, indent=1)


if __name__ == "__main__":
    which = sys.argv[1:] or ["c1"]
    if "c1" in which:
        c1_prefix()
    if "c2modes" in which:
        c2_modes_prefix()
