"""A box whose 19 population planes exceed 2^32 elements (L = 612): the LB kernel then
addresses populations with 64-bit offsets (32-bit ones below that size).  Mass and
momentum are exact invariants of the collision with full thermalization (Sec. II B: the
noise acts on the non-conserved modes only), so any population read or written at a
wrapped offset shows up in the device-side FP64 sums."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def test_box_beyond_32_bit_offsets_conserves_mass_and_momentum():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_0903_5067_gb300 import lb

    L = 612
    assert 19 * L ** 3 > 2 ** 32
    sim = lb.Simulation(L=L, rho=1.0, eta=3.0, eta_b=3.0, kT=1.0, h=0.01, a=1.0, seed=5, precision=lb.LB_FP32)
    try:
        sim.step(3)
        obs = sim.observables()
        mass = L ** 3 * 1.0
        # a population read or written 2^32 elements off (about 60 M nodes of the last
        # plane) would move the mass by ~1e-8 relative
        assert abs(obs[1] - mass) / mass < 1e-9, obs[:8]
        # fluid momentum: zero up to the FP32 rounding of each node's j (~1e-10 lattice units,
        # times a/h = 100 per node)
        assert np.all(np.abs(obs[5:8]) < 1e-6 * L ** 3), obs[5:8]
        assert obs[16] == 0
    finally:
        sim.close()
