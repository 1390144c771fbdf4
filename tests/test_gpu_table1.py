"""Static chain properties against the paper's Table 1 (LB columns, N = 32, L = 10, 15, 25),
with the production parameters of Sec. II E (two MD steps per LB step).

Equilibrium statics depend only on the chain potential (FENE + WCA between all monomers)
and the temperature the coupled thermostat delivers, and on the box through the periodic
images (the paper's L = 10 chain is compressed).  64 independent replicas per box run
together as one batch; <R_g^2> and <R_e^2> are averaged over time within each replica and
their standard error taken over the replicas."""
import os

import numpy as np
import pytest

from paper_0903_5067_gb300 import inputs

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "table1_lb_statics.txt")
PAPER = dict(rho=0.864, eta=0.864 * 2.8, eta_b=0.864 * 2.8, kT=1.2, h=0.02, a=1.0, m=1.0, zeta=20.8, k_fene=7.0,
             R0=2.0, eps=1.0, sigma=1.0)


def _table1():
    rows = {}
    with open(GOLDEN) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                L, re2, dre2, rg2, drg2 = line.split()
                rows[int(L)] = (float(re2), float(dre2), float(rg2), float(drg2))
    return rows


@pytest.mark.parametrize("L", [10, 15, 25])
def test_static_chain_size_matches_table1(lblib, L):
    R, N = 64, 32
    seeds = [1000 * L + r for r in range(R)]
    X = [inputs.chain_walk(N, L=L, bond=0.97, seed=s, self_avoiding=True) for s in seeds]
    b = lblib.Batch([L] * R, [N] * R, seeds, X, precision=lblib.LB_FP32, md_substeps=2, **PAPER)
    b.step(40000)  # equilibration: 800 time units
    for _ in range(400):  # sampling: 400 x 400 LB steps = 3200 time units per replica
        b.step(400)
        b.accumulate()
    b.sync()
    obs = np.array([b.observables(r) for r in range(R)])
    b.close()
    rg2, re2 = obs[:, 18], obs[:, 19]
    re2_p, dre2_p, rg2_p, drg2_p = _table1()[L]
    se_rg, se_re = rg2.std(ddof=1) / np.sqrt(R), re2.std(ddof=1) / np.sqrt(R)
    print(f"L={L}: Rg2 {rg2.mean():.2f} +- {se_rg:.2f} (paper {rg2_p} +- {drg2_p}); "
          f"Re2 {re2.mean():.2f} +- {se_re:.2f} (paper {re2_p} +- {dre2_p})")
    assert abs(rg2.mean() - rg2_p) <= 3 * np.hypot(se_rg, drg2_p)
    assert abs(re2.mean() - re2_p) <= 3 * np.hypot(se_re, dre2_p)
