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


def c1_prefix():
    """N=3 Holstein chain, one mode (w = g = V = kT = 1, nmax = 4), M = 64 (below the full
    ranks), dtau = dt = 0.05: the oracle TD-DMRG C(t) on the first 20 real-time steps."""
    p = dict(N=3, omega=[1.0], g=[1.0], nmax=[4], V=1.0, beta=1.0, dtau=0.05, M=64, dt=0.05)
    m = HolsteinModel(N=p["N"], omega=p["omega"], g=p["g"], nmax=p["nmax"], V=p["V"])
    r = tdvp.correlation(m, p["beta"], p["dtau"], p["M"], p["dt"], 20, every=5)
    p.update(t=r.t.tolist(), C_re=r.C.real.tolist(), C_im=r.C.imag.tolist(), logZ=r.logZ,
             tol=1e-8, source="oracle.tdvp.correlation")
    with open(os.path.join(HERE, "c1_M64_prefix.json"), "w") as f:
        json.dump(p, f, indent=1)


if __name__ == "__main__":
    c1_prefix()
