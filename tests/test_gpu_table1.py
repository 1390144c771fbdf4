"""Chain properties against the paper's Table 1 (LB columns, N = 32, L = 10, 15, 25), with the
production parameters of Sec. II E (two MD steps per LB step).

64 independent replicas per box run together as one batch.  Statics: <R_g^2> and <R_e^2> are
averaged over time within each replica and their standard error taken over the replicas.
From the same runs, bead positions every 2 time units give each replica's trajectory, which
the library's analysis kernels turn into <1/R_H> (Kirkwood), g1 and g3; D_CM is the slope of
g3 / 6 over lags 40..400 time units, fitted per replica.  Equilibrium statics depend only on
the chain potential, the thermostat's temperature and the periodic images (the L = 10 chain
is compressed); D_CM carries the hydrodynamic finite-size effect of the box."""
import os

import numpy as np
import pytest

from paper_0903_5067_gb300 import inputs

pytestmark = pytest.mark.gpu

HERE = os.path.join(os.path.dirname(__file__), "golden")
PAPER = dict(rho=0.864, eta=0.864 * 2.8, eta_b=0.864 * 2.8, kT=1.2, h=0.02, a=1.0, m=1.0, zeta=20.8, k_fene=7.0,
             R0=2.0, eps=1.0, sigma=1.0)
FRAME = 100  # LB steps between recorded frames: 2 time units


def _rows(name):
    rows = {}
    with open(os.path.join(HERE, name)) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                v = line.split()
                rows[int(v[0])] = [float(x) for x in v[1:]]
    return rows


def _fit_slope(t, y):
    A = np.stack([t, np.ones_like(t)], axis=1)
    return float(np.linalg.lstsq(A, y, rcond=None)[0][0])


def _production(lblib, L, stress_only=False):
    """64 replicas of the paper's production run in an L box: per-replica time averages of
    R_g^2 and R_e^2, and from the recorded trajectories <1/R_H>, D_CM and the g1, g3
    exponents."""
    import torch
    from paper_0903_5067_gb300 import analysis as an

    R, N = 64, 32
    seeds = [1000 * L + r for r in range(R)]
    X = [inputs.chain_walk(N, L=L, bond=0.97, seed=s, self_avoiding=True) for s in seeds]
    b = lblib.Batch([L] * R, [N] * R, seeds, X, precision=lblib.LB_FP32, md_substeps=2, stress_only=stress_only,
                    **PAPER)
    b.step(40000)  # equilibration: 800 time units
    frames = []
    for k in range(1600):  # sampling: 3200 time units per replica
        b.step(FRAME)
        if k % 4 == 3:
            b.accumulate()
        frames.append(np.stack([b.beads(r)[0] for r in range(R)]))
    b.sync()
    obs = np.array([b.observables(r) for r in range(R)])
    b.close()
    traj = np.stack(frames, axis=1)  # (R, T, N, 3), unwrapped
    rh, dcm, e1, e3 = [], [], [], []
    dt = FRAME * PAPER["h"]
    lags = np.arange(0, 201)
    t = lags * dt
    fit = (t >= 40) & (t <= 400)
    sub = (t >= 20) & (t <= 80)
    for r in range(R):
        tr = torch.tensor(traj[r], device="cuda")
        rh.append(an.inverse_radius(tr))
        g1, g2, g3 = an.msd(tr, int(lags[-1]))
        dcm.append(_fit_slope(t[fit], g3[fit]) / 6.0)
        e1.append(_fit_slope(np.log(t[sub]), np.log(g1[sub])))
        e3.append(_fit_slope(np.log(t[sub]), np.log(g3[sub])))
    return dict(R=R, rg2=obs[:, 18], re2=obs[:, 19], rh=np.array(rh), dcm=np.array(dcm), e1=np.array(e1),
                e3=np.array(e3))


def _se(a):
    return a.std(ddof=1) / np.sqrt(a.size)


@pytest.mark.parametrize("L", [10, 15, 25])
def test_chain_properties_match_table1(lblib, L):
    res = _production(lblib, L)
    rg2, re2, rh, dcm, e1, e3 = (res[k] for k in ("rg2", "re2", "rh", "dcm", "e1", "e3"))
    re2_p, dre2_p, rg2_p, drg2_p = _rows("table1_lb_statics.txt")[L]
    se_rg, se_re = _se(rg2), _se(re2)
    rh_p, drh_p, d_p, dd_p, e1_p, de1_p, e3_p, de3_p = _rows("table1_lb_dynamics.txt")[L]
    se = _se
    print(f"L={L}: Rg2 {rg2.mean():.2f} +- {se_rg:.2f} (paper {rg2_p} +- {drg2_p}); "
          f"Re2 {re2.mean():.2f} +- {se_re:.2f} (paper {re2_p} +- {dre2_p}); "
          f"1/RH {rh.mean():.4f} +- {se(rh):.4f} (paper {rh_p}); "
          f"D_CM {dcm.mean():.3e} +- {se(dcm):.1e} (paper {d_p:.3e}); "
          f"g1 exp {e1.mean():.3f} +- {se(e1):.3f} (paper {e1_p}); g3 exp {e3.mean():.3f} +- {se(e3):.3f} "
          f"(paper {e3_p})")
    assert abs(rg2.mean() - rg2_p) <= 3 * np.hypot(se_rg, drg2_p)
    assert abs(re2.mean() - re2_p) <= 3 * np.hypot(se_re, dre2_p)
    assert abs(rh.mean() - rh_p) <= 3 * np.hypot(se(rh), drh_p)
    assert abs(dcm.mean() - d_p) <= 3 * np.hypot(se(dcm), dd_p)
    assert abs(e1.mean() - e1_p) <= 3 * np.hypot(se(e1), de1_p)
    assert abs(e3.mean() - e3_p) <= 3 * np.hypot(se(e3), de3_p)
    # tau_tr = <R_g^2> / (6 D_CM), the paper's estimate (Table 1, last row), with the error of
    # the two measured means propagated
    tau = rg2.mean() / (6.0 * dcm.mean())
    se_tau = tau * np.hypot(se_rg / rg2.mean(), se(dcm) / dcm.mean())
    tau_p, dtau_p = _rows("table1_tau_tr.txt")[L]
    print(f"L={L}: tau_tr {tau:.1f} +- {se_tau:.1f} (paper {tau_p} +- {dtau_p})")
    assert abs(tau - tau_p) <= 3 * np.hypot(se_tau, dtau_p)


@pytest.mark.parametrize("L", [10, 15, 25])
def test_stress_only_thermalization_matches_table1_note_b(lblib, L):
    """The original thermalization, noise on the stress modes only (Table 1, note b; Sec. II B):
    the same production runs give the note-b g1 exponents.  D_CM and <1/R_H> are printed for
    the record (the paper compares the stress-only D_CM only through its L -> infinity
    extrapolation, Sec. III B)."""
    res = _production(lblib, L, stress_only=True)
    rh, dcm, e1, e3 = (res[k] for k in ("rh", "dcm", "e1", "e3"))
    e1_p, de1_p = _rows("table1_lb_stress_only.txt")[L]
    print(f"L={L} stress-only: 1/RH {rh.mean():.4f} +- {_se(rh):.4f}; D_CM {dcm.mean():.3e} +- {_se(dcm):.1e}; "
          f"g1 exp {e1.mean():.3f} +- {_se(e1):.3f} (paper {e1_p}); g3 exp {e3.mean():.3f} +- {_se(e3):.3f}")
    assert abs(e1.mean() - e1_p) <= 3 * np.hypot(_se(e1), de1_p)
