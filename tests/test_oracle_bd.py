"""Pins of the Brownian-dynamics oracle (Sec. II C/D): the regularised RPY tensor (continuity
at contact, symmetry, positive definiteness, the two-bead relative mobility in closed form),
Fixman's Chebyshev square root against the exact matrix square root, the single-bead limit,
the free-draining diffusion constant, and the unit mapping of Sec. II D."""
import math

import numpy as np
import pytest

from oracle import bd
from oracle import lbchain as o
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


# ---------------------------------------------------------------------------------------
# The BD chain's conservative forces (Sec. II A, Eqs. 1-2, in an infinite medium)
# ---------------------------------------------------------------------------------------
def _folded_chain():
    """Six beads, bonds between 0.9 and 1.9 (the production model's R0 = 2), and two
    non-bonded pairs, (0, 5) and (2, 4), inside the WCA range 2^(1/6) sigma."""
    return np.array([[0.0, 0.0, 0.0], [0.95, 0.1, 0.0], [1.6, 0.9, 0.3], [1.3, 1.8, 0.9],
                     [0.55, 1.0, 0.55], [-0.4, 0.6, 0.5]])


def _wca_energy(r, eps, sigma):
    """Eq. 2 restated: 4 eps ((sigma/r)^12 - (sigma/r)^6 + 1/4) below 2^(1/6) sigma, else 0."""
    return 4.0 * eps * ((sigma / r) ** 12 - (sigma / r) ** 6 + 0.25) if r < 2.0 ** (1.0 / 6.0) * sigma else 0.0


def _chain_energy(X, p):
    """FENE (Eq. 1) on the bonds plus WCA on all pairs, infinite medium: a second, independent
    statement of the potential whose negative gradient the BD forces are."""
    N = X.shape[0]
    e = 0.0
    for i in range(N - 1):
        r2 = float(((X[i] - X[i + 1]) ** 2).sum())
        e += -0.5 * p.k_fene * p.R0 ** 2 * math.log(1.0 - r2 / p.R0 ** 2)
    for i in range(N):
        for j in range(i + 1, N):
            e += _wca_energy(math.sqrt(float(((X[i] - X[j]) ** 2).sum())), p.eps, p.sigma)
    return e


def _force_pin_failures(forces):
    """Names of the properties a BD force routine misses (empty when all hold):
    - F = -grad V by central differences of the restated energy above (folded chain);
    - two beads: |F| = k r / (1 - r^2/R0^2) attractive for a bond beyond the WCA range, and
      the FENE pull minus the WCA push 24 eps (2 (sigma/r)^12 - (sigma/r)^6) / r inside it;
    - Newton's third law (zero net force) and zero net torque (central pair forces);
    - equal to the LB oracle's chain forces in a box far larger than the chain."""
    fails = []
    p = bd.BDParams(N=6)
    X = _folded_chain()
    F = forces(X, p)
    h = 1e-6
    for b in range(6):
        for al in range(3):
            Xp, Xm = X.copy(), X.copy()
            Xp[b, al] += h
            Xm[b, al] -= h
            fd = -(_chain_energy(Xp, p) - _chain_energy(Xm, p)) / (2 * h)
            if abs(F[b, al] - fd) > 1e-6 * max(1.0, abs(fd)):
                fails.append(f"-grad V bead {b} axis {al}")
    if np.abs(F.sum(axis=0)).max() > 1e-10:
        fails.append("net force")
    if np.abs(np.cross(X, F).sum(axis=0)).max() > 1e-10:
        fails.append("net torque")
    q = bd.BDParams(N=2)
    for r in (0.95, 1.5):
        X2 = np.array([[0.0, 0.0, 0.0], [r, 0.0, 0.0]])
        F2 = forces(X2, q)
        fene = q.k_fene * r / (1.0 - r * r / q.R0 ** 2)
        wca = 24.0 * q.eps * (2.0 * (q.sigma / r) ** 12 - (q.sigma / r) ** 6) / r if r < 2 ** (1 / 6) else 0.0
        want = -fene + wca  # x component on bead 1 (positive: pushed away from bead 0)
        if abs(F2[1, 0] - want) > 1e-12 * abs(want) or abs(F2[0, 0] + want) > 1e-12 * abs(want):
            fails.append(f"two beads r={r}")
    cp = o.ChainParams(N=6, k_fene=p.k_fene, R0=p.R0, eps=p.eps, sigma=p.sigma)
    if not np.allclose(forces(X + 50.0, p), o.chain_forces(X + 50.0, cp, 1.0e6), rtol=1e-13, atol=1e-13):
        fails.append("LB oracle chain forces")
    return fails


def test_bd_forces_are_minus_the_gradient_of_fene_plus_wca():
    assert _force_pin_failures(bd.forces) == []


def _forces_wca_sign(X, p):  # planted: the WCA pair force with the wrong sign
    F = bd.forces(X, bd.BDParams(N=p.N, k_fene=0.0, R0=p.R0, eps=p.eps, sigma=p.sigma))
    G = bd.forces(X, bd.BDParams(N=p.N, k_fene=p.k_fene, R0=p.R0, eps=0.0, sigma=p.sigma))
    return G - F


def _forces_fene_linear(X, p):  # planted: a harmonic bond k r in place of FENE
    F = bd.forces(X, bd.BDParams(N=p.N, k_fene=0.0, R0=p.R0, eps=p.eps, sigma=p.sigma))
    for i in range(X.shape[0] - 1):
        d = X[i] - X[i + 1]
        F[i] -= p.k_fene * d
        F[i + 1] += p.k_fene * d
    return F


def _forces_bonded_wca_only(X, p):  # planted: WCA between chain neighbours only
    F = bd.forces(X, bd.BDParams(N=p.N, k_fene=p.k_fene, R0=p.R0, eps=0.0, sigma=p.sigma))
    rc2 = 2.0 ** (1.0 / 3.0) * p.sigma ** 2
    for i in range(X.shape[0] - 1):
        d = X[i] - X[i + 1]
        r2 = d @ d
        if r2 < rc2:
            sr6 = (p.sigma ** 2 / r2) ** 3
            f = 24.0 * p.eps / r2 * (2.0 * sr6 * sr6 - sr6) * d
            F[i] += f
            F[i + 1] -= f
    return F


def _forces_one_sided(X, p):  # planted: the reaction on the second bead of each pair dropped
    F = np.zeros_like(X)
    full = bd.forces(X, p)
    F[: X.shape[0] // 2] = full[: X.shape[0] // 2]
    F[X.shape[0] // 2:] = 0.5 * full[X.shape[0] // 2:]
    return F


@pytest.mark.parametrize("fn", [_forces_wca_sign, _forces_fene_linear, _forces_bonded_wca_only, _forces_one_sided],
                         ids=["wca_sign", "fene_linear", "wca_bonded_only", "reaction_halved"])
def test_planted_bd_force_mistakes_are_caught(fn):
    assert _force_pin_failures(fn)
