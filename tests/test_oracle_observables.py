"""Pins of the observable definitions (Sec. III A/B): the isotropic structure factor
against a direct average of exp(i k.r) over wave-vector directions, displacement functions
against rigid motions, the Rouse transform against a single-mode shape and its inverse, and
the Rouse correlation against the exact relaxation of a Gaussian Rouse chain (the paper's
own check of its Rouse-mode analysis)."""
import math

import numpy as np
import pytest

from oracle import observables as ob


def _directions(n):
    """Fibonacci-sphere unit vectors (near-uniform)."""
    i = np.arange(n) + 0.5
    phi = np.arccos(1 - 2 * i / n)
    th = math.pi * (1 + 5 ** 0.5) * i
    return np.stack([np.cos(th) * np.sin(phi), np.sin(th) * np.sin(phi), np.cos(phi)], axis=1)


def _sk_direct(frame, k, dirs):
    """(1/N) |sum_j exp(i k.r_j)|^2 averaged over the directions of k."""
    ph = k * frame @ dirs.T  # (N, ndir)
    re = np.cos(ph).sum(axis=0)
    im = np.sin(ph).sum(axis=0)
    return float(np.mean(re * re + im * im)) / frame.shape[0]


def test_static_sk_is_the_direction_average_of_the_fourier_definition():
    rng = np.random.default_rng(1)
    traj = rng.normal(scale=1.5, size=(2, 6, 3))
    dirs = _directions(40000)
    ks = [0.3, 1.0, 2.5]
    S = ob.static_structure_factor(traj, ks)
    for a, k in enumerate(ks):
        direct = np.mean([_sk_direct(traj[t], k, dirs) for t in range(2)])
        assert S[a] == pytest.approx(direct, rel=2e-4, abs=2e-4)


def test_static_sk_special_cases():
    d = 1.7
    two = np.array([[[0.0, 0, 0], [d, 0, 0]]])
    for k in (0.5, 2.0):
        assert ob.static_structure_factor(two, [k])[0] == pytest.approx(1.0 + math.sin(k * d) / (k * d), rel=1e-14)
    rng = np.random.default_rng(2)
    traj = rng.normal(size=(3, 7, 3))
    assert ob.static_structure_factor(traj, [1e-9])[0] == pytest.approx(7.0, rel=1e-12)  # k -> 0: N


def test_dynamic_sk_matches_the_fourier_definition_and_reduces_to_static_at_lag_zero():
    rng = np.random.default_rng(3)
    traj = np.cumsum(rng.normal(scale=0.4, size=(5, 4, 3)), axis=0)
    ks = [0.7, 1.9]
    Skt = ob.dynamic_structure_factor(traj, ks, max_lag=3)
    Sk = ob.static_structure_factor(traj, ks)
    assert np.allclose(Skt[:, 0], Sk, rtol=1e-14)
    dirs = _directions(40000)
    for a, k in enumerate(ks):
        lag = 2
        vals = []
        for t0 in range(5 - lag):
            p1 = k * traj[t0 + lag] @ dirs.T
            p0 = k * traj[t0] @ dirs.T
            s1 = np.cos(p1).sum(0) + 1j * np.sin(p1).sum(0)
            s0 = np.cos(p0).sum(0) + 1j * np.sin(p0).sum(0)
            vals.append(float(np.mean((s1 * np.conj(s0)).real)) / 4)
        assert Skt[a, lag] == pytest.approx(np.mean(vals), rel=3e-4, abs=3e-4)
    # origin stride: the average over the chosen origins only
    Skt2 = ob.dynamic_structure_factor(traj, ks, max_lag=1, origin_stride=2)
    ref = np.mean([ob.dynamic_structure_factor(traj[[t0, t0 + 1]], ks, max_lag=1)[:, 1] for t0 in (0, 2)], axis=0)
    assert np.allclose(Skt2[:, 1], ref, rtol=1e-14)


def test_msd_rigid_translation_and_rotation():
    N, T = 6, 8
    rng = np.random.default_rng(4)
    base = rng.normal(size=(N, 3))
    v = np.array([0.3, -0.1, 0.2])
    traj = np.stack([base + t * v for t in range(T)])
    g1, g2, g3 = ob.msd(traj, 5)
    lags = np.arange(6)
    assert np.allclose(g1, (lags ** 2) * (v @ v), rtol=1e-12, atol=1e-14)
    assert np.allclose(g3, (lags ** 2) * (v @ v), rtol=1e-12, atol=1e-14)
    assert np.allclose(g2, 0.0, atol=1e-12)
    # rotation about the centre of mass (z axis, angle w per frame): a monomer at distance
    # rho from the axis moves 2 rho^2 (1 - cos(w lag)); the centre of mass stays
    w = 0.3
    base = base - base.mean(axis=0)
    rot = lambda a: np.array([[math.cos(a), -math.sin(a), 0], [math.sin(a), math.cos(a), 0], [0, 0, 1]])
    traj = np.stack([base @ rot(w * t).T for t in range(T)])
    g1, g2, g3 = ob.msd(traj, 4)
    i0, i1 = ob.inner_pair(N)
    rho2 = np.mean([base[i, 0] ** 2 + base[i, 1] ** 2 for i in (i0, i1)])
    expect = 2 * rho2 * (1 - np.cos(w * np.arange(5)))
    assert np.allclose(g2, expect, rtol=1e-12, atol=1e-14)
    assert np.allclose(g1, expect, rtol=1e-12, atol=1e-14)
    assert np.allclose(g3, 0.0, atol=1e-20)
    assert ob.inner_pair(8) == (3, 4) and ob.inner_pair(7) == (3, 3)


def test_rouse_transform_single_mode_and_inverse():
    N = 9
    n = np.arange(1, N + 1)
    for q in (1, 4, 8):
        shape = np.cos(q * math.pi * (n - 0.5) / N)
        frame = np.stack([2.5 * shape, -1.0 * shape, 0.5 * shape], axis=1)[None]
        X = ob.rouse_modes(frame)[0]
        for p in range(1, N):
            expect = np.array([2.5, -1.0, 0.5]) / 2 if p == q else np.zeros(3)
            assert np.allclose(X[p - 1], expect, atol=1e-14)
    rng = np.random.default_rng(5)
    frame = rng.normal(size=(1, N, 3))
    X = ob.rouse_modes(frame)[0]
    cm = frame[0].mean(axis=0)
    rebuilt = cm + 2 * np.array([sum(X[p - 1] * math.cos(p * math.pi * (m - 0.5) / N) for p in range(1, N))
                                 for m in n])
    assert np.allclose(rebuilt, frame[0], atol=1e-13)


def test_rouse_correlation_of_a_gaussian_rouse_chain_decays_with_the_rouse_times():
    N, T, dt = 8, 40000, 0.05
    traj, tau, var = ob.rouse_chain_trajectory(N, T, dt, b=1.0, zeta=1.0, kT=1.0, seed=6)
    X = ob.rouse_modes(traj)
    c, x2 = ob.rouse_correlation(X, max_lag=40)
    assert np.allclose(x2, c[:, 0])
    for p in (1, 2, 3):
        assert x2[p - 1] == pytest.approx(3 * var[p - 1], rel=0.05)  # 3 components
        for lag in (5, 10, 20, 40):
            expect = math.exp(-lag * dt / tau[p - 1])
            if expect < 0.1:
                continue
            assert c[p - 1, lag] / x2[p - 1] == pytest.approx(expect, abs=0.03)
    # centre of mass diffuses with D = kT / (N zeta): g3 = 6 D t
    g1, g2, g3 = ob.msd(traj[:4000], 20)
    assert g3[20] == pytest.approx(6 * (1.0 / N) * 20 * dt, rel=0.1)


def test_inverse_hydrodynamic_radius_closed_forms():
    d = 1.7
    two = np.array([[[0.0, 0, 0], [d, 0, 0]]])
    assert ob.inverse_hydrodynamic_radius(two) == pytest.approx(2 / (4 * d), rel=1e-15)  # 2 ordered pairs / N^2
    s = 1.3
    tri = np.array([[[0.0, 0, 0], [s, 0, 0], [s / 2, s * math.sqrt(3) / 2, 0]]])
    assert ob.inverse_hydrodynamic_radius(tri) == pytest.approx(6 / (9 * s), rel=1e-14)
    # average over frames: a rod whose spacing doubles in the second frame
    rod = np.array([[[0.0, 0, 0], [1.0, 0, 0], [2.0, 0, 0]], [[0.0, 0, 0], [2.0, 0, 0], [4.0, 0, 0]]])
    one = 2 * (1 + 1 + 0.5) / 9
    assert ob.inverse_hydrodynamic_radius(rod) == pytest.approx((one + one / 2) / 2, rel=1e-14)


def test_table1_tau_tr_row_is_rg2_over_six_d_cm():
    """The golden Table 1 rows are read consistently: the printed tau_tr estimate equals
    <R_g^2> / (6 D_CM) with D_CM = (printed value) x 1e-3 (reading of the row label
    'D_CM x 10^-3') within 0.5 %, for the three LB boxes and the BD column."""
    import os

    g = os.path.join(os.path.dirname(__file__), "golden")
    tau = {int(r[0]): r[1] for r in np.loadtxt(os.path.join(g, "table1_tau_tr.txt"), ndmin=2)}
    stat = {int(r[0]): r for r in np.loadtxt(os.path.join(g, "table1_lb_statics.txt"), ndmin=2)}
    dyn = {int(r[0]): r for r in np.loadtxt(os.path.join(g, "table1_lb_dynamics.txt"), ndmin=2)}
    bd = np.loadtxt(os.path.join(g, "table1_bd.txt"))
    for L in (10, 15, 25):
        assert stat[L][3] / (6.0 * dyn[L][3]) == pytest.approx(tau[L], rel=5e-3)
    assert bd[2] / (6.0 * bd[6]) == pytest.approx(tau[0], rel=5e-3)
