"""Brownian dynamics with hydrodynamic interaction (Sec. II C) on the GPU against the FP64
oracle on identical inputs and noise: positions after a few steps (RPY mobility, power
iterations, Chebyshev square root, Ito-Euler update), free draining, several replicas with
their own noise streams, and the FENE-break status."""
import numpy as np
import pytest

from oracle import bd
from paper_0903_5067_gb300 import inputs

pytestmark = pytest.mark.gpu


def _chains(R, N, seed):
    return np.stack([inputs.chain_walk(N, L=1000, bond=0.97, seed=seed + r, self_avoiding=True) for r in range(R)])


def _run_gpu(lblib, X0, p, steps, prec):
    b = lblib.BD(X0, kT=p.kT, zeta=p.zeta, eta_s=p.eta_s, dt=p.dt, k_fene=p.k_fene, R0=p.R0, eps=p.eps,
                 sigma=p.sigma, hi=p.hi, degree=p.degree, power_iters=p.power_iters, seed=p.seed, precision=prec)
    b.step(steps)
    x = b.beads()
    b.close()
    return x


@pytest.mark.parametrize("hi", [True, False])
def test_bd_fp64_matches_oracle(lblib, hi):
    R, N, steps = 3, 8, 12
    p = bd.BDParams(N=N, hi=hi, seed=4)
    X0 = _chains(R, N, 10)
    x = _run_gpu(lblib, X0, p, steps, lblib.LB_FP64)
    for r in range(R):
        ref = bd.run(X0[r], p, steps, replica=r)
        disp = np.abs(ref - X0[r]).max()
        assert np.abs(x[r] - ref).max() <= 1e-10 * max(disp, 1.0), r


def test_bd_fp32_matches_oracle(lblib):
    R, N, steps = 2, 16, 10
    p = bd.BDParams(N=N, seed=6)
    X0 = _chains(R, N, 20)
    x = _run_gpu(lblib, X0, p, steps, lblib.LB_FP32)
    for r in range(R):
        ref = bd.run(X0[r], p, steps, replica=r)
        disp = np.abs(ref - X0[r]).max()
        assert np.abs(x[r] - ref).max() <= 2e-4 * disp, r


def test_bd_reports_a_broken_bond(lblib):
    X0 = np.array([[[0.0, 0, 0], [2.05, 0, 0]]])  # a bond beyond the FENE limit R0 = 2
    b = lblib.BD(X0, kT=5.0, precision=lblib.LB_FP32, seed=1)
    b.step(2)
    with pytest.raises(lblib.LBError) as ei:
        b.sync()
    assert ei.value.code == lblib.LB_ERR_FENE
    b.close()


def test_bd_chain_properties_match_table1_bd_column(lblib):
    """The paper's BD model (Sec. II C/D: N = 32, kT = 1.2, FENE k = 7, R0 = 2, WCA, RPY with
    eta_s = 0.864 x 2.8 and zeta = zeta_eff(20.8), dt = 0.005 tau_k, in MD/LB units), 64
    chains for 800 + 3200 time units: statics, <1/R_H>, D_CM from g3 and the g1/g3 exponents
    against Table 1's BD column, within three combined standard errors."""
    import os

    import torch
    from paper_0903_5067_gb300 import analysis as an

    row = np.loadtxt(os.path.join(os.path.dirname(__file__), "golden", "table1_bd.txt"))
    re2_p, dre2_p, rg2_p, drg2_p, rh_p, drh_p, d_p, dd_p, e1_p, de1_p, e3_p, de3_p = row
    R, N = 64, 32
    X0 = _chains(R, N, 500)
    b = lblib.BD(X0, precision=lblib.LB_FP32, seed=11)
    dt = 0.005 * lblib.zeta_eff(20.8, 0.864 * 2.8) / 28.0
    per_frame = int(round(2.0 / dt))  # a frame every 2 time units
    b.step(int(800 / dt))
    frames = []
    for _ in range(1600):
        b.step(per_frame)
        frames.append(b.beads())
    b.close()
    traj = np.stack(frames, axis=1)  # (R, T, N, 3)
    t = np.arange(0, 201) * per_frame * dt
    fit, sub = (t >= 40) & (t <= 400), (t >= 20) & (t <= 80)
    rg2, re2, rh, dcm, e1, e3 = [], [], [], [], [], []
    for r in range(R):
        c = traj[r] - traj[r].mean(axis=1, keepdims=True)
        rg2.append(np.mean(np.sum(c ** 2, axis=2)))
        re2.append(np.mean(np.sum((traj[r][:, -1] - traj[r][:, 0]) ** 2, axis=1)))
        tr = torch.tensor(traj[r], device="cuda")
        rh.append(an.inverse_radius(tr))
        g1, _, g3 = an.msd(tr, 200)
        A = np.stack([t[fit], np.ones(fit.sum())], axis=1)
        dcm.append(np.linalg.lstsq(A, g3[fit], rcond=None)[0][0] / 6.0)
        B = np.stack([np.log(t[sub]), np.ones(sub.sum())], axis=1)
        e1.append(np.linalg.lstsq(B, np.log(g1[sub]), rcond=None)[0][0])
        e3.append(np.linalg.lstsq(B, np.log(g3[sub]), rcond=None)[0][0])
    vals = {k: np.array(v) for k, v in dict(rg2=rg2, re2=re2, rh=rh, dcm=dcm, e1=e1, e3=e3).items()}
    se = {k: v.std(ddof=1) / np.sqrt(R) for k, v in vals.items()}
    m = {k: v.mean() for k, v in vals.items()}
    print(f"BD: Rg2 {m['rg2']:.2f} +- {se['rg2']:.2f} (paper {rg2_p}); Re2 {m['re2']:.1f} +- {se['re2']:.1f} "
          f"(paper {re2_p}); 1/RH {m['rh']:.4f} +- {se['rh']:.4f} (paper {rh_p}); D_CM {m['dcm']:.3e} +- "
          f"{se['dcm']:.1e} (paper {d_p:.3e}); g1 exp {m['e1']:.3f} +- {se['e1']:.3f} (paper {e1_p}); "
          f"g3 exp {m['e3']:.3f} +- {se['e3']:.3f} (paper {e3_p})")
    for k, (ref, err) in dict(rg2=(rg2_p, drg2_p), re2=(re2_p, dre2_p), rh=(rh_p, drh_p), dcm=(d_p, dd_p),
                              e1=(e1_p, de1_p), e3=(e3_p, de3_p)).items():
        assert abs(m[k] - ref) <= 3 * np.hypot(se[k], err), k
    # tau_tr = <R_g^2> / (6 D_CM) against Table 1's last row (BD column)
    tau_rows = np.loadtxt(os.path.join(os.path.dirname(__file__), "golden", "table1_tau_tr.txt"))
    tau_p, dtau_p = tau_rows[tau_rows[:, 0] == 0][0, 1:]
    tau = m["rg2"] / (6.0 * m["dcm"])
    se_tau = tau * np.hypot(se["rg2"] / m["rg2"], se["dcm"] / m["dcm"])
    print(f"BD: tau_tr {tau:.1f} +- {se_tau:.1f} (paper {tau_p} +- {dtau_p})")
    assert abs(tau - tau_p) <= 3 * np.hypot(se_tau, dtau_p)
