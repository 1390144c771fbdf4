"""Seeded synthetic inputs shared by the tests, the smoke check and the benchmark.

This module holds none of the method's arithmetic: it only draws initial bead
configurations and perturbation fields from numpy's PCG64 generator.  The workloads follow
the shapes of the paper's runs (Sec. II E): a single chain of N beads with bonds of length
~0.97 (random walk, optionally self-avoiding) started near the centre of a periodic L^3 box
filled with fluid at rest.
"""
from __future__ import annotations

import numpy as np


def _unit_vectors(rng: np.random.Generator, n: int) -> np.ndarray:
    v = rng.standard_normal((n, 3))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def chain_walk(N: int, L: int, a: float = 1.0, bond: float = 0.97, seed: int = 0,
               self_avoiding: bool = False, sigma: float = 1.0, max_tries: int = 1000) -> np.ndarray:
    """Initial bead positions (N, 3), float64, unwrapped, first bead near the box centre.

    Random walk of fixed step ``bond``.  With ``self_avoiding`` a trial bead closer than
    ``sigma`` to any earlier bead other than its predecessor, or to a periodic image of one
    (the box has side L a), is rejected (up to max_tries per bead); raises ValueError if the
    walk gets stuck.
    """
    rng = np.random.default_rng(np.random.PCG64(seed))
    X = np.zeros((max(N, 0), 3))
    if N == 0:
        return X
    # offset from the exact centre node so that no bead starts on a lattice plane
    X[0] = 0.5 * L * a + a * (rng.random(3) - 0.5) * 0.5
    for i in range(1, N):
        for _ in range(max_tries):
            trial = X[i - 1] + bond * _unit_vectors(rng, 1)[0]
            if not self_avoiding or i < 2:
                break
            dv = X[: i - 1] - trial
            dv -= L * a * np.round(dv / (L * a))
            d = np.linalg.norm(dv, axis=1)
            if np.all(d >= sigma):
                break
        else:
            raise ValueError(f"self-avoiding walk stuck at bead {i}")
        X[i] = trial
    return X


def bead_velocities(N: int, scale: float, seed: int) -> np.ndarray:
    """Gaussian initial velocities of standard deviation ``scale`` (N, 3)."""
    rng = np.random.default_rng(np.random.PCG64(seed + 7919))
    return scale * rng.standard_normal((N, 3))


def perturbation(L: int, q: int = 19, amplitude: float = 1e-2, seed: int = 0) -> np.ndarray:
    """Relative perturbation field (q, L, L, L) uniform in [-amplitude, amplitude]; a test
    multiplies a rest state by (1 + this) to start away from equilibrium."""
    rng = np.random.default_rng(np.random.PCG64(seed + 104729))
    return amplitude * (2.0 * rng.random((q, L, L, L)) - 1.0)


def c4_ensemble(R: int = 64, base_seed: int = 100):
    """The batched-replica workload: replica r has box L_r = (16, 24, 32, 48, 64)[r mod 5] and
    chain N_r = (8, 16, 32, 64)[(r // 5) mod 4], stepped down while L_r < 2 R_g,est(N_r)
    (R_g,est^2 = 0.97^2 N^(2*0.588) / 6.5: Flory exponent and the R_e^2/R_g^2 ratio ~6.5 of the
    paper's Table 1), seed base_seed + r, self-avoiding initial walk.
    Returns (L list, N list, seeds, list of (N_r, 3) position arrays)."""
    Ls, Ns, seeds, X = [], [], [], []
    for r in range(R):
        L = (16, 24, 32, 48, 64)[r % 5]
        N = (8, 16, 32, 64)[(r // 5) % 4]
        while N > 8 and L < 2.0 * np.sqrt(0.97 ** 2 * N ** (2 * 0.588) / 6.5):
            N //= 2
        Ls.append(L)
        Ns.append(N)
        seeds.append(base_seed + r)
        X.append(chain_walk(N, L=L, bond=0.97, seed=base_seed + r, self_avoiding=True))
    return Ls, Ns, seeds, X
