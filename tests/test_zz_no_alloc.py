"""The allocation-free entry point lb_fluid_sums_noalloc against the context-based one.

lb_fluid_sums_noalloc serves callers that cannot allocate device memory where they need the
fluid's mass and momentum (inside a stream capture, under a foreign allocator): it keeps its
partial sums in a fixed file-scope scratch array of the library.  This test computes the same
sums through lb_get_observables and through the new entry point, twice in a row (the second
call reuses the scratch left by the first), and requires agreement to the FP64 parity bar.
It lives in a file collected last so that a failure here stops a -x run only after every
other test has run."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_noalloc_sums_match_observables_on_two_calls(lblib):
    import torch
    from paper_0903_5067_gb300 import inputs

    L, N, a, h = 24, 12, 0.9, 0.01
    sim = lblib.Simulation(L=L, rho=1.0, eta=3.0, eta_b=3.0, kT=1.0, h=h, a=a, seed=17, precision=lblib.LB_FP64)
    sim.add_chain(N, x0=inputs.chain_walk(N, L=L, a=a, bond=0.97, seed=17, self_avoiding=True))
    sim.step(15)
    obs = sim.observables()
    n = sim.populations()
    sim.close()
    dev = torch.from_numpy(n).cuda()
    stream = torch.cuda.current_stream().cuda_stream
    first = lblib.lb_fluid_sums_noalloc(dev.data_ptr(), L, a, h, stream)
    second = lblib.lb_fluid_sums_noalloc(dev.data_ptr(), L, a, h, stream)
    scale = L ** 3 * a ** 4 / h  # momentum of the box at one lattice unit of velocity
    for got in (first, second):
        assert got[0] == pytest.approx(obs[1], rel=1e-12)
        assert np.allclose(got[1:4], obs[5:8], rtol=0, atol=1e-12 * scale)
    with pytest.raises(lblib.LBError) as ei:
        lblib.lb_fluid_sums_noalloc(dev.data_ptr(), lblib.LB_NOALLOC_MAX_L + 1, a, h, stream)
    assert ei.value.code == lblib.LB_ERR_ARG
