"""Bead kinetic temperature of the coupled step as the time step shrinks.

The dissipative coupling (Sec. II B: friction -zeta (v - u) plus a Langevin force balancing it)
satisfies the fluctuation-dissipation theorem of the continuous-time equations, so the beads
reach <v^2>/3 = kT/m as h -> 0.  At finite h the velocity-Verlet discretisation of the coupled
step (reading: friction at the half-step velocity, plain J/rho of the post-stream fluid) is
exact only in a frozen fluid (var v = kT/m, pinned on the oracle); with the fluid responding to
the bead's own reaction it runs slightly warm, by an amount linear in h.  This test measures
free beads (no FENE, no WCA) in the fluctuating fluid at h = 0.01, 0.005, 0.0025 (same
physical parameters and duration, FP32) and requires the straight line T(h) - kT/m = a + c h
fitted to the three temperatures to extrapolate to kT/m at h = 0 (|a| within three standard
errors) with every point on the line within three standard errors; the slope c is printed
(about 2 to 3.5 per unit time step: +2 to +3.5 % at the paper's MD step 0.01)."""
import numpy as np
import pytest

from paper_0903_5067_gb300 import inputs

pytestmark = pytest.mark.gpu


def _free_bead_temperature(lb, h, L=32, N=64, seed=11):
    sim = lb.Simulation(L=L, rho=1.0, eta=3.0, eta_b=3.0, kT=1.0, h=h, a=1.0, seed=seed, precision=lb.LB_FP32)
    X0 = inputs.chain_walk(N, L=L, bond=0.97, seed=seed, self_avoiding=True)
    sim.add_chain(N, m=1.0, zeta=20.8, k_fene=0.0, R0=1e6, eps=0.0, sigma=1.0, x0=X0)
    every = int(round(0.2 / h))  # samples 0.2 time units apart (velocity memory m / zeta_eff ~ 0.07)
    sim.step(int(round(20.0 / h)))
    v2 = []
    for _ in range(1500):
        sim.step(every)
        _, v = sim.beads()
        v2.append((v ** 2).mean())
    sim.close()
    v2 = np.array(v2)
    return v2.mean(), v2.std(ddof=1) / np.sqrt(v2.size)


def test_bead_temperature_converges_to_kT_over_m_as_the_step_shrinks(lblib):
    hs = np.array([0.01, 0.005, 0.0025])
    T, se = np.array([_free_bead_temperature(lblib, h) for h in hs]).T
    w = 1.0 / se ** 2
    A = np.stack([np.ones_like(hs), hs], axis=1)
    cov = np.linalg.inv(A.T @ (w[:, None] * A))
    a, c = cov @ (A.T @ (w * (T - 1.0)))
    sa = np.sqrt(cov[0, 0])
    print("bead temperature:", ", ".join(f"h={h}: {t:.4f} +- {s:.4f}" for h, t, s in zip(hs, T, se)),
          f"; fit T - 1 = {a:+.4f} (+- {sa:.4f}) + {c:.2f} h")
    assert abs(a) <= 3 * sa
    assert np.all(np.abs(T - 1.0 - (a + c * hs)) <= 3 * se)
