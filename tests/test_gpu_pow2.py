"""Power-of-two boxes beyond the benchmark sizes against the FP64 oracle (Sec. II B, Eq. 3):
the whole box at L = 32 with a chain, body forces and deferred corrections, in FP32 and in
16-bit storage, and sampled nodes after one step at L = 256 (twice the largest workload),
including every node whose pull sources wrap around in x, y or z."""
import numpy as np
import pytest

from gpu_helpers import Case, bead_errs, gpu_run, gpu_sim, oracle_run, pop_rel_err
from oracle import lbchain as o
from paper_0903_5067_gb300 import inputs

pytestmark = pytest.mark.gpu

L32 = Case(L=32, N=16, steps=20, seed=21, perturb=0.05, ext=(0.3, -0.2, 0.1), counter=True)


def test_box_32_with_chain_and_forces_fp32(lblib):
    st = oracle_run(L32)
    n, x, v, _ = gpu_run(lblib, L32, lblib.LB_FP32)
    err = pop_rel_err(n, st.n)
    ex, ev = bead_errs(x, v, st, L32)
    print(f"L=32 N=16 20 steps FP32: populations {err:.2e}, bead x {ex:.2e}, bead v {ev:.2e}")
    assert err <= 1e-5
    assert ex <= 1e-5 and ev <= 1e-5


@pytest.mark.parametrize("prec,p", [("bf16", 8), ("fp16", 11)])
def test_box_32_in_16bit_storage(lblib, prec, p):
    """Deviations n_i - w_i rho0 stored in 16 bits (significands of p bits, unit roundoff
    2^-p) and computed in FP32.  Each step's stores round the deviations by at most 2^-p of
    their size and the collision carries these errors, of random sign, on with a gain well
    below 8, so after k steps the population error stays below 8 k 2^-p max|deviation|; a
    wrong pull source would give errors of the order of the deviations themselves."""
    case = Case(L=32, N=16, steps=3, seed=22, perturb=0.05, ext=(0.3, -0.2, 0.1), counter=True)
    st = oracle_run(case)
    n, x, v, _ = gpu_run(lblib, case, getattr(lblib, "LB_" + prec.upper()))
    rest = o.fluid_at_rest(case.fluid())
    dev = float(np.max(np.abs(st.n - rest)))
    err = float(np.max(np.abs(n - st.n)))
    print(f"L=32 {prec}: population error {err:.2e} of max deviation {dev:.2e}")
    assert err <= 8 * case.steps * 2.0 ** -p * dev
    ex, _ = bead_errs(x, v, st, case)
    assert ex <= 1e-3


def _sample_nodes(L, rng, extra=300):
    edge = [0, 1, L // 2 - 1, L // 2, L - 2, L - 1]
    nodes = {(x, y, z) for x in edge for y in edge for z in (0, 1, L - 1)}
    nodes |= {tuple(int(c) for c in rng.integers(0, L, 3)) for _ in range(extra)}
    return sorted(nodes)


def test_sampled_nodes_after_one_step_at_256(lblib):
    """One step of a perturbed fluid (noise on, no chain) at L = 256 against the oracle's
    single-node update at sampled nodes: every combination of x, y in {0, 1, L/2 - 1, L/2,
    L - 2, L - 1} and z in {0, 1, L - 1} (the periodic wrap of the pull in each direction, the
    middle of each row and column) and 300 random nodes."""
    case = Case(L=256, N=0, steps=1, seed=23)
    fp = case.fluid()
    n0 = o.fluid_at_rest(fp)
    n0 *= 1.0 + inputs.perturbation(case.L, amplitude=0.05, seed=23)
    sim = gpu_sim(lblib, case, lblib.LB_FP32)
    sim.set_populations(n0)
    sim.step(1)
    sim.sync()
    n1 = sim.populations()
    sim.close()
    rng = np.random.default_rng(5)
    worst = 0.0
    for (x, y, z) in _sample_nodes(case.L, rng):
        want = o.node_update(n0, fp, 0, (x, y, z))
        got = n1[:, z, y, x]
        worst = max(worst, float(np.max(np.abs(got - want) / np.abs(want))))
    print(f"L=256 sampled nodes: max relative error {worst:.2e}")
    assert worst <= 1e-5
