"""Equipartition and conservation of the FP32 fast path at the L = 64, N = 64 workload
(self-avoiding chain, seed 2) over 10^4 coupled steps: the fluctuation-dissipation balance of
the fluctuating LB (Sec. II B) fixes the stationary moment statistics of the stored
populations, which at equilibrium are independent per population with variance mu rho0 w_i
(mu = 3 kT h^2 / a^5), so that every node moment m_k = sum_i e_k(c_i) n_i has

    var(m_k) = mu rho0 b_k              k = 4..18 (every non-conserved mode)
    var(rho) = mu rho0 (1 - 1/L^3)      var(u_alpha) = kT / (rho0 a^3) (1 - 1/L^3)

(the conserved totals remove one degree of freedom per conserved mode); the coupled beads
reach <v^2>/3 = kT/m up to the O(h) excess of the discrete coupling; the collision and the coupling conserve mass and total momentum, so in
FP32 they drift only by rounding.  The moments are formed here from lb_get_populations
snapshots with the oracle's (pinned) mode matrix.  Statistical bands: three standard errors
of the mean over the snapshots (taken 500 steps apart), plus O(mu) = 3e-4 for the
non-linear equilibrium terms, which the linear statement above leaves out."""
import numpy as np
import pytest

from gpu_helpers import Case, gpu_sim
from oracle import lbchain as o

pytestmark = pytest.mark.gpu


def test_c2_equipartition_and_conservation_fp32(lblib):
    case = Case(L=64, N=64, steps=0, seed=2)
    fp = case.fluid()
    L, rho0, kT, a, h = case.L, case.rho, case.kT, case.a, case.h
    mu = o.mu_thermal(fp)
    sim = gpu_sim(lblib, case, lblib.LB_FP32)
    obs0 = sim.observables()
    sim.step(1000)  # the fluid starts at rest: let every mode reach its stationary variance
    var_m, var_u, v2 = [], [], []
    for snap in range(18):
        for _ in range(10):
            sim.step(50)
            _, v = sim.beads()
            v2.append((v ** 2).mean())
        n = sim.populations().reshape(19, -1)
        m = o.M @ n
        var_m.append(m.var(axis=1))
        rho = m[0]
        u = m[1:4] / rho[None] * a / h
        var_u.append(u.var(axis=1))
    obs1 = sim.observables()
    steps = int(obs1[0])
    sim.close()
    assert steps == 10000

    var_m, var_u = np.array(var_m), np.array(var_u)
    n_s = var_m.shape[0]
    mean_m = var_m.mean(axis=0)
    se_m = var_m.std(axis=0, ddof=1) / np.sqrt(n_s)
    want = mu * rho0 * o.B
    want[0] *= 1.0 - 1.0 / L ** 3
    rel = mean_m / want - 1.0
    band = 3.0 * se_m / want + 3.0 * mu
    for k in range(19):
        print(f"mode {k:2d}: var/expected - 1 = {rel[k]:+.2e} (band {band[k]:.1e})")
    for k in [0] + list(range(4, 19)):
        assert abs(rel[k]) <= band[k], k
    # velocity: kT/(rho0 a^3) (1 - 1/L^3) per component
    want_u = kT / (rho0 * a ** 3) * (1.0 - 1.0 / L ** 3)
    mu_u = var_u.mean(axis=0)
    se_u = var_u.std(axis=0, ddof=1) / np.sqrt(n_s)
    print("var(u)/expected - 1:", mu_u / want_u - 1.0)
    assert np.all(np.abs(mu_u / want_u - 1.0) <= 3.0 * se_u / want_u + 3.0 * mu)
    # beads: 180 samples of 64 beads (velocity correlation time m / zeta_eff ~ 7 steps << 50);
    # allowance 4 h for the coupled step's O(h) excess (test_gpu_bead_temperature measures the
    # slope, 2 to 3.5 per unit step, and the extrapolation to kT/m at h = 0)
    v2 = np.array(v2)
    se_v = v2.std(ddof=1) / np.sqrt(v2.size)
    print(f"bead <v^2>/3 = {v2.mean():.4f} +- {se_v:.4f} (kT/m = {kT / case.m})")
    assert abs(v2.mean() - kT / case.m) <= 3.0 * se_v + 4.0 * h
    # conservation in FP32: rounding only (about 1e-9 of the mass and of the box momentum at
    # one lattice unit of velocity over 10^4 steps); bounds 1e-7
    scale = L ** 3 * rho0 * a ** 4 / h
    dm = abs(obs1[1] / obs0[1] - 1.0)
    dp = float(np.abs(obs1[2:5] - obs0[2:5]).max() / scale)
    print(f"mass drift {dm:.1e}, total momentum drift {dp:.1e} of the box momentum at unit lattice velocity")
    assert dm <= 1e-7 and dp <= 1e-7
