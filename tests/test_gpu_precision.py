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
