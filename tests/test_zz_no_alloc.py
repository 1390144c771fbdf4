"""The allocation-free entry point lb_fluid_sums_noalloc against the context-based one.

lb_fluid_sums_noalloc serves callers that cannot allocate device memory where they need the
fluid's mass and momentum: an application whose device memory is all held by another
allocator, or a time-critical loop that must not pay for cudaMalloc/cudaFree.  It keeps its
partial sums in a fixed file-scope scratch array of the library.  These tests compute the same
sums through lb_get_observables and through the new entry point, twice in a row (the second
call reuses the scratch left by the first), and require agreement to the FP64 parity bar; they
also check that the calls leave the device's free memory unchanged, the size limit, and a box
whose last block of 256 nodes is partial.  The file is collected last so that a failure here
stops a -x run only after every other test has run."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _context_sums(lblib, L, N, a, h, seed, steps):
    from paper_0903_5067_gb300 import inputs

    sim = lblib.Simulation(L=L, rho=1.0, eta=3.0, eta_b=3.0, kT=1.0, h=h, a=a, seed=seed, precision=lblib.LB_FP64)
    sim.add_chain(N, x0=inputs.chain_walk(N, L=L, a=a, bond=0.97, seed=seed, self_avoiding=True))
    sim.step(steps)
    obs = sim.observables()
    n = sim.populations()
    sim.close()
    return obs, n


@pytest.mark.parametrize("L,N,a", [(24, 12, 0.9), (7, 3, 1.0)], ids=["L24", "L7_partial_block"])
def test_noalloc_sums_match_observables_on_two_calls(lblib, L, N, a):
    import torch

    h = 0.01
    obs, n = _context_sums(lblib, L, N, a, h, seed=17 + L, steps=15)
    dev = torch.from_numpy(n).cuda()
    stream = torch.cuda.current_stream().cuda_stream
    first = lblib.lb_fluid_sums_noalloc(dev.data_ptr(), L, a, h, stream)
    second = lblib.lb_fluid_sums_noalloc(dev.data_ptr(), L, a, h, stream)
    scale = L ** 3 * a ** 4 / h  # momentum of the box at one lattice unit of velocity
    for got in (first, second):
        assert got[0] == pytest.approx(obs[1], rel=1e-12)
        assert np.allclose(got[1:4], obs[5:8], rtol=0, atol=1e-12 * scale)


def test_noalloc_calls_leave_device_memory_unchanged_and_reject_oversized_boxes(lblib):
    """Two calls at the capacity edge (L = LB_NOALLOC_MAX_L: every scratch slot in use) change
    neither the device's free memory nor torch's allocation, and agree with a plain PyTorch
    FP64 sum of the same field; one more node per edge is refused with LB_ERR_ARG and a reason."""
    import torch

    L, a, h = lblib.LB_NOALLOC_MAX_L, 1.0, 0.01
    g = torch.Generator(device="cuda").manual_seed(5)
    pop = torch.rand((19, L ** 3), dtype=torch.float64, device="cuda", generator=g)
    c = torch.tensor([[0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0],
                      [0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1],
                      [0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1]], dtype=torch.float64,
                     device="cuda")
    per_dir = pop.sum(dim=1)
    want = np.concatenate([[float(per_dir.sum()) * a ** 3], (c @ per_dir).cpu().numpy() * a ** 4 / h])
    stream = torch.cuda.current_stream().cuda_stream
    lblib.lb_fluid_sums_noalloc(pop.data_ptr(), L, a, h, stream)  # the first call on the device sets up
    torch.cuda.synchronize()
    free0, alloc0 = torch.cuda.mem_get_info()[0], torch.cuda.memory_allocated()
    got = [lblib.lb_fluid_sums_noalloc(pop.data_ptr(), L, a, h, stream) for _ in range(2)]
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert torch.cuda.memory_allocated() == alloc0
    total = float(pop.sum()) * a ** 4 / h
    for r in got:
        assert r[0] == pytest.approx(want[0], rel=1e-12)
        assert np.allclose(r[1:], want[1:], rtol=0, atol=1e-12 * total)
    with pytest.raises(lblib.LBError) as ei:
        lblib.lb_fluid_sums_noalloc(pop.data_ptr(), L + 1, a, h, stream)
    assert ei.value.code == lblib.LB_ERR_ARG
    assert "LB_NOALLOC_MAX_L" in ei.value.detail
