"""Pins of the Brownian-dynamics oracle (Sec. II C/D): the regularised RPY tensor (continuity
at contact, symmetry, positive definiteness, the two-bead relative mobility in closed form),
Fixman's Chebyshev square root against the exact matrix square root, the single-bead limit,
the free-draining diffusion constant, and the unit mapping of Sec. II D."""
import math

import numpy as np
import pytest

from oracle import bd
from paper_0903_5067_gb300 import inputs


def test_parameter_mapping_of_sec_2d():
    eta = 0.864 * 2.8
    ze = bd.zeta_eff(20.8, eta)
    assert 1.0 / ze == pytest.approx(1.0 / 20.8 + 1.0 / (25.0 * eta), rel=1e-15)
    assert ze == pytest.approx(15.48, abs=0.01)
    p = bd.BDParams(N=32)
    tau_k = p.zeta / (4.0 * p.k_fene)  # BD time unit in MD/LB units
    assert p.dt == pytest.approx(0.005 * tau_k, rel=1e-12)
    hstar = p.zeta / (6.0 * math.pi ** 1.5 * p.eta_s) * math.sqrt(p.k_fene / p.kT)
    d = p.zeta / (6.0 * math.pi * p.eta_s)
    assert hstar * math.sqrt(math.pi) * math.sqrt(p.kT / p.k_fene) == pytest.approx(d, rel=1e-14)


def test_rpy_continuity_symmetry_and_self_mobility():
    radius, eta = 0.34, 2.4
    u = np.array([0.3, -0.5, 0.8])
    u /= np.linalg.norm(u)
    below = bd.rpy_block(u * (2 * radius * (1 - 1e-12)), radius, eta)
    above = bd.rpy_block(u * (2 * radius * (1 + 1e-12)), radius, eta)
    assert np.allclose(below, above, rtol=1e-9, atol=0)
    # at r -> 0 the overlap form tends to the self-mobility 1/(6 pi eta a) = 1/zeta
    tiny = bd.rpy_block(u * 1e-9, radius, eta)
    assert np.allclose(tiny, np.eye(3) / (6 * math.pi * eta * radius), rtol=1e-8)
    p = bd.BDParams(N=12)
    rng = np.random.default_rng(1)
    for trial in range(5):  # coils with some overlapping beads: D stays symmetric positive definite
        X = rng.normal(scale=0.8 + trial * 0.5, size=(12, 3))
        M = bd.mobility(X, p)
        assert np.allclose(M, M.T, rtol=0, atol=1e-15)
        assert np.linalg.eigvalsh(M).min() > 0


def test_two_bead_relative_mobility_closed_form():
    """Two beads along x pulled together by +-f: the separation changes at the rate
    -2 (1/zeta - Omega_par(r)) f, Omega_par = (2 - 4 a^2 / 3 r^2) / (8 pi eta r) (r >= 2a) and
    (1 - 3r / 16a) / (6 pi eta a) (r < 2a)."""
    p = bd.BDParams(N=2)
    a = p.zeta / (6 * math.pi * p.eta_s)
    f = 0.7
    for r in (0.5 * a, 1.5 * a, 3.0 * a, 7.0):
        X = np.array([[0.0, 0, 0], [r, 0, 0]])
        F = np.array([[f, 0, 0], [-f, 0, 0]]).reshape(-1)
        v = (bd.mobility(X, p) @ F).reshape(2, 3)
        par = (2 - 4 * a * a / (3 * r * r)) / (8 * math.pi * p.eta_s * r) if r >= 2 * a else \
            (1 - 3 * r / (16 * a)) / (6 * math.pi * p.eta_s * a)
        assert v[1, 0] - v[0, 0] == pytest.approx(-2 * (1 / p.zeta - par) * f, rel=1e-12)
        assert np.allclose(v[:, 1:], 0, atol=1e-15)


def test_chebyshev_square_root_against_exact():
    p = bd.BDParams(N=16)
    X = inputs.chain_walk(16, L=1000, bond=0.97, seed=3, self_avoiding=True)
    D = p.kT * bd.mobility(X, p)
    w, V = np.linalg.eigh(D)
    S = V @ np.diag(np.sqrt(w)) @ V.T  # symmetric square root
    rng = np.random.default_rng(4)
    W = rng.standard_normal(48)
    lo, hi = bd.eigen_bounds(D, 20)
    assert lo <= w.min() * 1.0001 and hi >= w.max() * 0.9999  # the bounds bracket the spectrum
    y = bd.chebyshev_sqrt_apply(D, W, 20, 20)
    assert np.linalg.norm(y - S @ W) <= 1e-4 * np.linalg.norm(S @ W)
    y40 = bd.chebyshev_sqrt_apply(D, W, 40, 20)  # converges with the degree
    assert np.linalg.norm(y40 - S @ W) < np.linalg.norm(y - S @ W)
    # B.W has covariance D: for a batch of vectors, <y y^T> = D
    Ws = rng.standard_normal((48, 4000))
    Y = np.stack([bd.chebyshev_sqrt_apply(D, Ws[:, k], 20, 20) for k in range(4000)], axis=1)
    assert np.allclose(Y @ Y.T / 4000, D, atol=0.1 * np.abs(D).max())


def test_single_bead_limits():
    p = bd.BDParams(N=1, seed=5)
    q = bd.BDParams(N=1, seed=5, hi=False)
    X = np.zeros((1, 3))
    a = bd.run(X, p, 20)
    b = bd.run(X, q, 20)
    assert np.allclose(a, b, rtol=0, atol=1e-12)  # Chebyshev of a multiple of the identity
    # free diffusion: <|dr|^2> = 6 kT / zeta t
    n = 20000
    disp = np.array([bd.step(X, q, r, 0)[0] for r in range(n)])
    assert np.mean(np.sum(disp ** 2, axis=1)) == pytest.approx(6 * q.kT / q.zeta * q.dt, rel=0.03)
