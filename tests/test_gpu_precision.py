"""Reduced-precision population storage (deviations n_i - w_i rho0 stored in BF16 or FP16,
arithmetic in FP32) against the FP64 oracle on the same seeded inputs and noise.

Quantising every population every step is a random error of relative size 2^-9 (BF16) or
2^-12 (FP16) of the deviation, so these are stated error bounds per observable, not the FP32
parity bar: the populations, the bead trajectory after 100 steps, the exact invariants
(mass, total momentum) that storage rounding breaks only at the level of that noise, and
the thermal averages (fluid velocity variance, bead temperature) that must stay unbiased."""
import numpy as np
import pytest

from gpu_helpers import Case, bead_errs, gpu_run, gpu_sim, oracle_run, pop_rel_err

pytestmark = pytest.mark.gpu

C1_100 = Case(L=16, N=8, steps=100, seed=1)
BOUNDS = {  # precision: (population, bead x / box, bead v / thermal velocity)
    "bf16": (5e-3, 5e-4, 2e-2),
    "fp16": (1e-3, 1e-4, 3e-3),
}


@pytest.mark.parametrize("name", ["bf16", "fp16"])
def test_16bit_storage_error_against_oracle(lblib, name):
    prec = lblib.LB_BF16 if name == "bf16" else lblib.LB_FP16
    st = oracle_run(C1_100)
    n, x, v, _ = gpu_run(lblib, C1_100, prec)
    bp, bx, bv = BOUNDS[name]
    assert pop_rel_err(n, st.n) <= bp
    ex, ev = bead_errs(x, v, st, C1_100)
    assert ex <= bx and ev <= bv


@pytest.mark.parametrize("name", ["bf16", "fp16"])
def test_16bit_storage_invariants_and_thermal_averages(lblib, name):
    """Mass and momentum drift over 400 steps stay at the storage-noise level; the fluid
    velocity variance (kT / rho a^3) and bead temperature (kT / m) stay unbiased."""
    prec = lblib.LB_BF16 if name == "bf16" else lblib.LB_FP16
    case = Case(L=32, N=16, steps=0, seed=7)
    sim = gpu_sim(lblib, case, prec)
    o0 = sim.observables()
    temps, varu = [], []
    for _ in range(8):
        sim.step(50)
        ob = sim.observables()
        temps.append(ob[15])
        n = sim.populations()
        rho = n.sum(axis=0)
        ux = (n[1] - n[2] + n[7] - n[8] + n[9] - n[10] + n[11] - n[12] + n[13] - n[14]) / rho / case.h
        varu.append(ux.var())
    o1 = sim.observables()
    sim.close()
    q = 2.0 ** -8 if name == "bf16" else 2.0 ** -11  # half an ulp at 1
    nodes = case.L ** 3
    # rounding noise: ~q * |deviation| (~0.02) per population and step, random in sign
    drift_bound = 10 * q * 0.02 * np.sqrt(19 * nodes * 400)
    assert abs(o1[1] - o0[1]) <= drift_bound
    assert np.all(np.abs(o1[2:5] - o0[2:5]) <= drift_bound / case.h)
    assert np.mean(varu) == pytest.approx(case.kT / case.rho, rel=0.05)
    assert np.mean(temps) == pytest.approx(case.kT / case.m, rel=0.25)


def _c3_run(lblib, prec, steps=10000, snaps=5, frames=100):
    """The L = 128, N = 128 workload (seed 3) over `steps` coupled steps in one precision:
    mass and total momentum at the start and the end, the fluid velocity variance of
    `snaps` population snapshots, the bead temperature sampled every steps/frames steps, and
    the chain trajectory every steps/frames steps (FP64 unwrapped positions)."""
    import torch
    from paper_0903_5067_gb300 import analysis as an

    case = Case(L=128, N=128, steps=0, seed=3)
    sim = gpu_sim(lblib, case, prec)
    stride = steps // frames
    sim.record_trajectory(stride=stride, capacity=frames + 1)
    o0 = sim.observables()
    varu, v2 = [], []
    E = np.array([[0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0],
                  [0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1],
                  [0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1]], dtype=np.float64)
    for s in range(frames):
        sim.step(stride)
        _, v = sim.beads()
        v2.append((v ** 2).mean())
        if (s + 1) % (frames // snaps) == 0:
            n = sim.populations().reshape(19, -1)
            u = (E @ n) / n.sum(axis=0)[None] * case.a / case.h
            varu.append(u.var(axis=1).mean())
            del n, u
    o1 = sim.observables()
    traj = sim.trajectory()
    sim.close()
    X = traj.cpu().numpy()
    cm = X.mean(axis=1, keepdims=True)
    rg2 = ((X - cm) ** 2).sum(axis=2).mean(axis=1)
    g1, _, g3 = an.msd(traj, frames // 2)
    scale = case.L ** 3 * case.rho * case.a ** 4 / case.h
    return dict(mass_drift=abs(o1[1] / o0[1] - 1.0), mom_drift=float(np.abs(o1[2:5] - o0[2:5]).max() / scale),
                varu=np.array(varu), v2=np.array(v2), rg2=rg2, g1=np.asarray(g1), g3=np.asarray(g3), X=X,
                steps=int(o1[0]))


def test_c3_precision_study_fp32_bf16_fp16_against_fp64(lblib):
    """Precision study at the roofline workload (L = 128, N = 128, 10^4 steps, seed 3): FP32
    deviations, BF16 and FP16 storage with FP32 arithmetic, each against the FP64 path (itself
    held to the oracle at 1e-12).  Per observable: mass and momentum drift (FP64 and FP32:
    rounding only, about 1e-9, stated bound 1e-7; 16-bit storage: the random storage rounding
    of ~q |n - w rho0| per population and step, bound 10 q 0.02 sqrt(19 L^3 steps) / L^3 with
    q half an ulp at 1); the fluid velocity variance and the bead temperature against
    kT/(rho a^3) and kT/m (three standard errors, plus 3 mu for the fluid and the coupled step's
    O(h) excess, 4 h, for the beads: test_gpu_bead_temperature); R_g^2, the bead MSD
    g1 and the centre-of-mass MSD g3 at lags of 100, 1000 and 5000 steps against the FP64 run:
    FP32 within 1e-4 (R_g^2) and 1e-3 (g1, g3), since it follows the FP64 trajectory; BF16 and
    FP16 within 2 % and 5 %, their trajectories decorrelating from the FP64 one (statistical
    differences of one chain over 100 time units)."""
    steps = 10000
    runs = {"fp64": _c3_run(lblib, lblib.LB_FP64, steps), "fp32": _c3_run(lblib, lblib.LB_FP32, steps),
            "bf16": _c3_run(lblib, lblib.LB_BF16, steps), "fp16": _c3_run(lblib, lblib.LB_FP16, steps)}
    ref = runs["fp64"]
    L, kT, rho, mu = 128, 1.0, 1.0, 3.0 * 1.0 * 0.01 ** 2
    q = {"fp64": 0.0, "fp32": 0.0, "bf16": 2.0 ** -8, "fp16": 2.0 ** -11}
    lags = [1, 10, 50]  # frames of 100 steps
    failures = []
    for name, r in runs.items():
        assert r["steps"] == steps
        se_u = r["varu"].std(ddof=1) / np.sqrt(r["varu"].size)
        se_v = r["v2"].std(ddof=1) / np.sqrt(r["v2"].size)
        d_rg = float(np.abs(r["rg2"] - ref["rg2"]).max() / ref["rg2"].mean())
        d_x = float(np.abs(r["X"][-1] - ref["X"][-1]).max())
        g1r = [r["g1"][k] / ref["g1"][k] - 1.0 for k in lags]
        g3r = [r["g3"][k] / ref["g3"][k] - 1.0 for k in lags]
        print(f"{name}: mass drift {r['mass_drift']:.2e}, momentum drift {r['mom_drift']:.2e}; "
              f"var u/(kT/rho) - 1 = {r['varu'].mean() / kT - 1:+.2e} (se {se_u:.1e}); "
              f"bead <v^2>/3 = {r['v2'].mean():.4f} +- {se_v:.4f}; <R_g^2> = {r['rg2'].mean():.4f} "
              f"(fp64 {ref['rg2'].mean():.4f}), max |dR_g^2|/R_g^2 over the run {d_rg:.2e}, "
              f"max |dx| at the end {d_x:.2e}; g1 rel. diff at 1e2/1e3/5e3 steps "
              f"{', '.join(f'{v:+.1e}' for v in g1r)}; g3 {', '.join(f'{v:+.1e}' for v in g3r)}")
        drift = 1e-7 if q[name] == 0.0 else 10 * q[name] * 0.02 * np.sqrt(19 * L ** 3 * steps) / L ** 3
        if not (r["mass_drift"] <= drift and r["mom_drift"] <= drift):
            failures.append(f"{name}: drift")
        if not abs(r["varu"].mean() - kT / rho) <= 3 * se_u + 3 * mu:
            failures.append(f"{name}: var u")
        if not abs(r["v2"].mean() - kT) <= 3 * se_v + 4 * 0.01:  # O(h) coupling excess, h = 0.01
            failures.append(f"{name}: bead temperature")
        # chain observables against the FP64 run: FP32 follows the FP64 trajectory (rounding
        # grows over the 10^4 steps but stays far below the chain's own motion); 16-bit
        # storage decorrelates the trajectory, so its averages differ by statistics only
        if name != "fp64":
            rg_tol, g_tol = (1e-4, 1e-3) if name == "fp32" else (2e-2, 5e-2)
            if abs(r["rg2"].mean() / ref["rg2"].mean() - 1.0) > rg_tol:
                failures.append(f"{name}: <R_g^2>")
            if max(abs(v) for v in g1r + g3r) > g_tol:
                failures.append(f"{name}: g1/g3")
    assert not failures, failures
