"""Synthetic CLS workloads: the case parameters the tests and the benchmark use.

Inputs only -- no step of the method is computed here.  A case is the 9-tuple
(sigma0, sigma1, lambda0, lambda1, c0, c1, L, d, nbins) of include/cls.h.
"""
from __future__ import annotations

import numpy as np

# Rod, L = 10, Sigma = (0.5, 5), Lambda = (2, 0.5), c = (0.5, 0.9), 100 bins; 1e5 histories.
ROD_L10 = (0.5, 5.0, 2.0, 0.5, 0.5, 0.9, 10.0, 1, 100)
ROD_L10_HISTORIES = 100_000

# Box of side 10, Sigma = (0.1, 10), Lambda = (1, 0.1), c = 0.99 (long histories), 200 bins; 1e8 histories.
BOX_L10 = (0.1, 10.0, 1.0, 0.1, 0.99, 0.99, 10.0, 3, 200)
# The same box walked by its x-marginal (geometry 13): same law of the tallies.
BOX_L10_X = (0.1, 10.0, 1.0, 0.1, 0.99, 0.99, 10.0, 13, 200)
BOX_L10_HISTORIES = 100_000_000

# Diffusive box: L = 100, Sigma = (1, 10), Lambda = (0.5, 0.2), c = 0.999, 500 bins; 1e8 histories.
BOX_DIFFUSIVE = (1.0, 10.0, 0.5, 0.2, 0.999, 0.999, 100.0, 3, 500)
BOX_DIFFUSIVE_HISTORIES = 100_000_000

# Benchmark suite I materials (paper Tables 1-2): case -> (Sigma, Lambda), sub-case -> c.
SUITE_MATERIALS = {
    "1": ((10 / 99, 100 / 11), (99 / 100, 11 / 100)),
    "2": ((10 / 99, 100 / 11), (99 / 10, 11 / 10)),
    "3": ((2 / 101, 200 / 101), (101 / 20, 101 / 20)),
}
SUITE_SCATTERING = {"a": (0.0, 1.0), "b": (1.0, 0.0), "c": (0.9, 0.9)}


GEOM_ROD, GEOM_EXTRUDED, GEOM_BOX, GEOM_SLAB, GEOM_BOX_X = 1, 2, 3, 11, 13


def suite_case(name: str, d: int = 3, L: float = 10.0, nbins: int = 100):
    """Benchmark configuration like '1a' (paper Tables 1-2) as a case tuple;
    d = 3 for the box, 2 for the extruded 2D box, 11 for the paper's d = 1 slab."""
    (s0, s1), (l0, l1) = SUITE_MATERIALS[name[0]]
    c0, c1 = SUITE_SCATTERING[name[1]]
    return (s0, s1, l0, l1, c0, c1, L, d, nbins)


def batch_sweep(ncases: int = 256, seed: int = 7, nbins: int = 100) -> np.ndarray:
    """The batched sweep: per case, d in {1, 3} (probability 1/2 each),
    L in {0.1, 1, 10} (1/3 each), Sigma_0, Sigma_1 log-uniform in [0.02, 10],
    Lambda_0, Lambda_1 log-uniform in [0.05, 10], c_0, c_1 uniform in [0, 1],
    drawn in this order from numpy's PCG64 seeded with `seed`."""
    rng = np.random.default_rng(seed)
    out = np.zeros((ncases, 9))

    def logu(a, b):
        return float(np.exp(np.log(a) + rng.random() * np.log(b / a)))

    for k in range(ncases):
        d = 1 if rng.random() < 0.5 else 3
        L = (0.1, 1.0, 10.0)[min(2, int(rng.random() * 3))]
        s0, s1 = logu(0.02, 10.0), logu(0.02, 10.0)
        l0, l1 = logu(0.05, 10.0), logu(0.05, 10.0)
        c0, c1 = float(rng.random()), float(rng.random())
        out[k] = (s0, s1, l0, l1, c0, c1, L, d, nbins)
    return out
