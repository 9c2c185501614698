"""Seeded synthetic inputs shared by the oracle tests and the GPU parity tests.

Only random numbers and shapes live here: no arithmetic of the method."""
import numpy as np


def random_complex(rng, shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def random_mpo_site(rng, Dl, Dr, d, density=0.4):
    """A sparse complex MPO site W[wl, wr, s, u] with about `density` of its blocks nonzero."""
    W = np.zeros((Dl, Dr, d, d), dtype=complex)
    for wl in range(Dl):
        for wr in range(Dr):
            if rng.random() < density or (wl == 0 and wr == 0):
                W[wl, wr] = random_complex(rng, (d, d))
    return W
