"""GPU chain observables (Sec. III A/B) against the oracle's definitions: trajectory
recording (bit-exact against the bead read-back), g1/g2/g3, Rouse modes and their
correlation, S(k) and S(k,t) at 1e-12 relative on the same frames, and the Rouse-mode
analysis validated on a Gaussian Rouse chain as in the paper."""
import math

import numpy as np
import pytest

from gpu_helpers import Case, gpu_sim
from oracle import observables as ob

pytestmark = pytest.mark.gpu


def _close(a, b, rtol=1e-12):
    a, b = np.asarray(a), np.asarray(b)
    scale = max(float(np.max(np.abs(b))), 1e-300)
    assert np.max(np.abs(a - b)) <= rtol * scale, (np.max(np.abs(a - b)), scale)


def test_recorded_frames_equal_the_bead_read_back_and_wrap(lblib):
    case = Case(L=12, N=8, steps=0, seed=3)
    for prec in (lblib.LB_FP64, lblib.LB_FP32):
        sim = gpu_sim(lblib, case, prec)
        sim.record_trajectory(stride=3, capacity=5)
        ref = [sim.beads()[0]]
        for _ in range(6):  # 6 calls of 3 steps: frames 1..6, the ring keeps 2..6
            sim.step(3)
            ref.append(sim.beads()[0])
        assert lblib.lb_trajectory_frames(sim.ctx) == 7
        traj = sim.trajectory().cpu().numpy()
        assert traj.shape == (5, 8, 3)
        assert np.array_equal(traj, np.array(ref[2:]))
        # frames recorded inside one multi-step call
        sim.record_trajectory(stride=2, capacity=8)
        x0 = sim.beads()[0]
        sim.step(6)
        traj = sim.trajectory().cpu().numpy()
        assert traj.shape == (4, 8, 3)
        assert np.array_equal(traj[0], x0) and np.array_equal(traj[3], sim.beads()[0])
        sim.close()


def _lb_trajectory(lblib):
    case = Case(L=10, N=8, steps=0, seed=4)
    sim = gpu_sim(lblib, case, lblib.LB_FP64)
    sim.record_trajectory(stride=5, capacity=64)
    sim.step(5 * 40)
    traj = sim.trajectory()
    sim.close()
    return traj


def test_analysis_matches_oracle_on_an_lb_trajectory(lblib):
    import torch
    from paper_0903_5067_gb300 import analysis as an

    traj = _lb_trajectory(lblib)
    t = traj.cpu().numpy()
    assert t.shape == (41, 8, 3)
    g = an.msd(traj, 45)  # lags beyond the trajectory: no origins, zeros
    r = ob.msd(t, 45)
    for a, b in zip(g, r):
        _close(a, b)
    assert np.all(g[0][41:] == 0.0)
    g = an.msd(traj, 10, pair=(0, 7))
    for a, b in zip(g, ob.msd(t, 10, pair=(0, 7))):
        _close(a, b)
    X = an.rouse_modes(traj)
    Xo = ob.rouse_modes(t)
    _close(X.cpu().numpy(), Xo)
    c, x2 = an.rouse_correlation(X, 20)
    co, x2o = ob.rouse_correlation(Xo, 20)
    _close(c, co)
    _close(x2, x2o)
    ks = [0.2, 0.8, 1.7, 3.1]
    _close(an.static_sk(traj, ks), ob.static_structure_factor(t, ks))
    _close(an.dynamic_sk(traj, ks[:2], 6, origin_stride=3), ob.dynamic_structure_factor(t, ks[:2], 6, origin_stride=3))
    assert an.inverse_radius(traj) == pytest.approx(ob.inverse_hydrodynamic_radius(t), rel=1e-12)
    assert torch.cuda.is_available()


def test_rouse_analysis_recovers_rouse_times_of_a_gaussian_chain(lblib):
    """The paper's validation of its Rouse-mode analysis: a Gaussian Rouse chain of N = 8
    without hydrodynamic or excluded-volume interactions; the normalised correlation of X_p
    decays as exp(-t / tau_p) with the analytic tau_p."""
    import torch
    from paper_0903_5067_gb300 import analysis as an

    N, T, dt = 8, 40000, 0.05
    t, tau, var = ob.rouse_chain_trajectory(N, T, dt, b=1.0, zeta=1.0, kT=1.0, seed=8)
    traj = torch.tensor(t, device="cuda")
    X = an.rouse_modes(traj)
    c, x2 = an.rouse_correlation(X, 60)
    for p in range(1, 6):
        assert x2[p - 1] == pytest.approx(3 * var[p - 1], rel=0.05)
        for lag in (5, 10, 20, 40, 60):
            expect = math.exp(-lag * dt / tau[p - 1])
            if expect < 0.1:
                continue
            assert c[p - 1, lag] / x2[p - 1] == pytest.approx(expect, abs=0.03)
    # the same numbers as the oracle's analysis of the same frames
    co, _ = ob.rouse_correlation(ob.rouse_modes(t[:3000]), 10)
    cg, _ = an.rouse_correlation(an.rouse_modes(traj[:3000]), 10)
    _close(cg, co)


def test_structure_factor_edge_cases(lblib):
    import torch
    from paper_0903_5067_gb300 import analysis as an

    one = torch.zeros((3, 1, 3), dtype=torch.float64, device="cuda")
    assert an.static_sk(one, [1.0])[0] == 1.0  # a single bead
    two = torch.tensor([[[0.0, 0, 0], [1.3, 0, 0]]], dtype=torch.float64, device="cuda")
    assert an.static_sk(two, [0.9])[0] == pytest.approx(1 + math.sin(0.9 * 1.3) / (0.9 * 1.3), rel=1e-14)
    rng = np.random.default_rng(9)
    t = rng.normal(size=(7, 5, 3))
    traj = torch.tensor(t, device="cuda")
    Skt = an.dynamic_sk(traj, [0.5, 2.0], 9)  # lags 7..9 have no origins
    _close(Skt, ob.dynamic_structure_factor(t, [0.5, 2.0], 9))
    _close(Skt[:, 0], an.static_sk(traj, [0.5, 2.0]))
