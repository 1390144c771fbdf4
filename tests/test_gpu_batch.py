"""Batched replicas (one launch per kernel stage for many boxes of different L and N) against
the oracle with each replica's own noise stream, and the batch's own invariances: results do
not depend on the tile shape, on CUDA-graph replay or on autotuning."""
import numpy as np
import pytest

from gpu_helpers import Case, pop_rel_err
from oracle import lbchain as o
from paper_0903_5067_gb300 import inputs

pytestmark = pytest.mark.gpu

PARAMS = dict(rho=1.0, eta=3.0, eta_b=3.0, kT=1.0, h=0.01, a=1.0, m=1.0, zeta=20.8, k_fene=30.0, R0=1.5,
              eps=1.0, sigma=1.0)


def _ensemble():
    L = [8, 12, 5, 16, 24, 7]
    N = [4, 8, 0, 3, 16, 1]
    seeds = [11, 12, 13, 14, 15, 16]
    X = [inputs.chain_walk(n, L=l, bond=0.97, seed=s, self_avoiding=True) for n, l, s in zip(N, L, seeds)]
    return L, N, seeds, X


def _oracle_replica(r, L, N, seed, X0, steps, stress_only=False):
    fp = o.FluidParams(L=L, rho=1.0, eta=3.0, eta_b=3.0, kT=1.0, h=0.01, a=1.0, seed=seed, stress_only=stress_only)
    cp = o.ChainParams(N=N) if N > 0 else None
    st = o.init_state(fp, cp, X0 if N > 0 else None)
    return o.run(st, fp, cp, steps, replica=r)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_batch_replicas_match_oracle(lblib, prec):
    """40 steps = two replays of the 16-step graph + 8 direct steps."""
    L, N, seeds, X = _ensemble()
    p = lblib.LB_FP64 if prec == "fp64" else lblib.LB_FP32
    tol = 1e-12 if prec == "fp64" else 1e-5
    b = lblib.Batch(L, N, seeds, X, precision=p, **PARAMS)
    b.step(40)
    b.sync()
    for r in range(len(L)):
        st = _oracle_replica(r, L[r], N[r], seeds[r], X[r], 40)
        assert pop_rel_err(b.populations(r), st.n) <= tol, r
        if N[r] > 0:
            x, v = b.beads(r)
            assert np.max(np.abs(x - st.X)) / L[r] <= tol, r
    b.close()


def test_batch_stress_only_replicas_match_oracle(lblib):
    """lb_batch_set_options(stress_only): noise on the six stress modes of every replica
    (Table 1, note b), FP64 against the oracle."""
    L, N, seeds, X = _ensemble()
    b = lblib.Batch(L, N, seeds, X, precision=lblib.LB_FP64, stress_only=True, **PARAMS)
    b.step(20)
    b.sync()
    for r in range(len(L)):
        st = _oracle_replica(r, L[r], N[r], seeds[r], X[r], 20, stress_only=True)
        assert pop_rel_err(b.populations(r), st.n) <= 1e-12, r
        if N[r] > 0:
            x, v = b.beads(r)
            assert np.max(np.abs(x - st.X)) / L[r] <= 1e-12, r
    b.close()


def test_batch_results_do_not_depend_on_shape_graphs_or_autotuning(lblib):
    L, N, seeds, X = _ensemble()
    runs = []
    for shape, chunks in (((128, 0), [32]), ((512, 4), [1] * 32), ((256, 2), [20, 12]), ("auto", [32])):
        b = lblib.Batch(L, N, seeds, X, precision=lblib.LB_FP32, **PARAMS)
        if shape == "auto":
            t, k = lblib.lb_batch_autotune(b.b)
            assert t in (128, 256, 512) and 0 <= k <= 8
        else:
            lblib.lb_batch_set_shape(b.b, *shape)
        for c in chunks:
            b.step(c)
        b.sync()
        runs.append([b.populations(r) for r in range(len(L))] + [b.beads(r)[0] for r in range(len(L)) if N[r]])
        b.close()
    for other in runs[1:]:
        for a_, b_ in zip(runs[0], other):
            assert np.array_equal(a_, b_)


def test_c4_ensemble_64_replicas(lblib):
    """The 64-replica workload (5,242,368 nodes per step) for 2000 graph-replayed steps: every
    replica keeps its mass and total momentum; five small replicas match the oracle after 100
    steps (parity spot check)."""
    L, N, seeds, X = inputs.c4_ensemble()
    assert sum(l ** 3 for l in L) == 5242368
    b = lblib.Batch(L, N, seeds, X, precision=lblib.LB_FP32, **PARAMS)
    obs0 = [b.observables(r) for r in range(64)]
    b.step(100)
    b.sync()
    for r in (0, 1, 2, 5, 6):  # L = 16, 24, 32 replicas
        st = _oracle_replica(r, L[r], N[r], seeds[r], X[r], 100)
        assert pop_rel_err(b.populations(r), st.n) <= 1e-5, r
    b.step(1900)
    b.sync()
    temps = []
    for r in range(64):
        ob = b.observables(r)
        assert ob[1] == pytest.approx(obs0[r][1], rel=2e-6)
        scale = L[r] ** 3 / 0.01
        assert np.allclose(ob[2:5], obs0[r][2:5], rtol=0, atol=2e-6 * scale)
        temps.append(ob[15])
    # bead temperature averaged over the ensemble stays at kT/m = 1 (about 4 sigma)
    assert np.mean(temps) == pytest.approx(1.0, abs=0.15)
    b.close()
