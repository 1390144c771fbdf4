"""Parity of the CUDA path (through the C ABI) with the FP64 oracle on identical seeded inputs
and identical Philox noise streams.

Bars: FP64 context <= 1e-12 relative per population; FP32 context <= 1e-5 relative per
population after 100 steps (populations are O(w_i rho0), so this is also an absolute bar
of ~1e-5 w_i rho0); bead positions relative to the box and velocities relative to the
thermal velocity sqrt(kT/m) at the same bars."""
import numpy as np
import pytest

from gpu_helpers import Case, bead_errs, gpu_run, gpu_sim, oracle_run, pop_rel_err
from oracle import lbchain as o

pytestmark = pytest.mark.gpu

C1 = Case(L=16, N=8, steps=200, seed=1)  # plain FP64 config: L=16, N=8, 200 steps, seed 1
C1_FP32 = Case(L=16, N=8, steps=100, seed=1)


def test_c1_fp64_matches_oracle(lblib):
    st = oracle_run(C1)
    n, x, v, obs = gpu_run(lblib, C1, lblib.LB_FP64)
    assert pop_rel_err(n, st.n) <= 1e-12
    ex, ev = bead_errs(x, v, st, C1)
    assert ex <= 1e-12 and ev <= 1e-11


def test_c1_fp32_matches_oracle_after_100_steps(lblib):
    st = oracle_run(C1_FP32)
    n, x, v, obs = gpu_run(lblib, C1_FP32, lblib.LB_FP32)
    assert pop_rel_err(n, st.n) <= 1e-5
    ex, ev = bead_errs(x, v, st, C1_FP32)
    assert ex <= 1e-5 and ev <= 1e-5


@pytest.mark.parametrize("L", [4, 5, 7, 40])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_ragged_boxes_with_forces_and_perturbed_fluid(lblib, L, prec):
    """Box sizes that leave partial thread blocks (odd L, L not a multiple of the 32-wide
    rows), a fluid started away from equilibrium, a constant force on the beads balanced by
    the uniform counter-force on the fluid."""
    N = 3 if L >= 5 else 1
    case = Case(L=L, N=N, steps=12, seed=4 + L, perturb=0.05, ext=(0.3, -0.2, 0.1), counter=True)
    st = oracle_run(case)
    p = lblib.LB_FP64 if prec == "fp64" else lblib.LB_FP32
    n, x, v, _ = gpu_run(lblib, case, p)
    tol = 1e-12 if prec == "fp64" else 1e-5
    vtol = 10 * tol if prec == "fp64" else tol
    assert pop_rel_err(n, st.n) <= tol
    ex, ev = bead_errs(x, v, st, case)
    assert ex <= tol and ev <= vtol


@pytest.mark.parametrize("variant", ["stress_only", "noise_off", "beads_noise_off", "kT0"])
def test_noise_variants(lblib, variant):
    kw = dict(L=8, N=4, steps=30, seed=9, perturb=0.02)
    if variant == "stress_only":
        kw["stress_only"] = True
    elif variant == "noise_off":
        kw["noise_fluid"] = False
        kw["noise_beads"] = False
    elif variant == "beads_noise_off":
        kw["noise_beads"] = False
    else:
        kw["kT"] = 0.0
    case = Case(**kw)
    st = oracle_run(case)
    for prec, tol in ((lblib.LB_FP64, 1e-12), (lblib.LB_FP32, 1e-5)):
        n, x, v, _ = gpu_run(lblib, case, prec)
        assert pop_rel_err(n, st.n) <= tol, (variant, prec)


def test_fluid_without_chain(lblib):
    case = Case(L=12, N=0, steps=40, seed=3, perturb=0.03)
    st = oracle_run(case)
    for prec, tol in ((lblib.LB_FP64, 1e-12), (lblib.LB_FP32, 1e-5)):
        n, _, _, _ = gpu_run(lblib, case, prec)
        assert pop_rel_err(n, st.n) <= tol


def test_single_bead_and_general_spacing(lblib):
    """N = 1 and a lattice spacing a != 1 (positions, forces and velocities rescale)."""
    case = Case(L=6, N=1, steps=25, seed=12, a=0.8, h=0.02, eta=1.7, eta_b=2.2, kT=0.7)
    st = oracle_run(case)
    for prec, tol in ((lblib.LB_FP64, 1e-12), (lblib.LB_FP32, 1e-5)):
        n, x, v, _ = gpu_run(lblib, case, prec)
        assert pop_rel_err(n, st.n) <= tol
        ex, ev = bead_errs(x, v, st, case)
        assert ex <= tol and ev <= (10 * tol if prec == lblib.LB_FP64 else tol)


def test_c2_full_size_fp32_after_100_steps(lblib):
    """The L = 64, N = 64 workload at full size, every population and every bead compared
    after 100 coupled steps at the FP32 bar."""
    case = Case(L=64, N=64, steps=100, seed=2)
    st = oracle_run(case)
    n, x, v, _ = gpu_run(lblib, case, lblib.LB_FP32)
    err = pop_rel_err(n, st.n)
    ex, ev = bead_errs(x, v, st, case)
    print(f"C2 L=64 N=64 100 steps: populations {err:.2e}, bead x {ex:.2e}, bead v {ev:.2e}")
    assert err <= 1e-5
    assert ex <= 1e-5 and ev <= 1e-5


def test_c3_full_size_fp32_after_100_steps(lblib):
    """The benchmark's L = 128, N = 128 workload, in the same kernels and launch shapes the
    benchmark times (one lb_step call of 100 deferred steps), every one of the 39.8 M
    populations and every bead compared after 100 coupled steps at the FP32 bar."""
    case = Case(L=128, N=128, steps=100, seed=3)
    st = oracle_run(case)
    n, x, v, _ = gpu_run(lblib, case, lblib.LB_FP32)
    err = pop_rel_err(n, st.n)
    ex, ev = bead_errs(x, v, st, case)
    print(f"C3 L=128 N=128 100 steps: populations {err:.2e}, bead x {ex:.2e}, bead v {ev:.2e}")
    assert err <= 1e-5
    assert ex <= 1e-5 and ev <= 1e-5


def test_observables_match_oracle(lblib):
    case = Case(L=16, N=8, steps=50, seed=5)
    st = oracle_run(case)
    fp, cp = case.fluid(), case.chain()
    _, _, _, obs = gpu_run(lblib, case, lblib.LB_FP64)
    assert obs[0] == case.steps
    assert obs[1] == pytest.approx(o.total_mass(st, fp), rel=1e-13)
    scale = fp.L ** 3 * fp.rho * fp.a ** 4 / fp.h
    assert np.allclose(obs[2:5], o.total_momentum(st, fp, cp), rtol=0, atol=1e-12 * scale)
    assert np.allclose(obs[5:8], o.fluid_momentum(st, fp), rtol=0, atol=1e-12 * scale)
    assert obs[8] == pytest.approx(o.radius_of_gyration2(st.X), rel=1e-12)
    assert obs[9] == pytest.approx(o.end_to_end2(st.X), rel=1e-12)
    assert np.allclose(obs[10:13], st.X.mean(axis=0), rtol=1e-13)
    X0 = case.x0()
    g1 = 0.5 * sum(((st.X[i] - X0[i]) ** 2).sum() for i in (3, 4))
    assert obs[13] == pytest.approx(g1, rel=1e-9)
    g3 = ((st.X.mean(axis=0) - X0.mean(axis=0)) ** 2).sum()
    assert obs[14] == pytest.approx(g3, rel=1e-8, abs=1e-14)
    assert obs[15] == pytest.approx(cp.m * (st.V ** 2).sum() / (3 * cp.N), rel=1e-12)


def test_observables_match_oracle_in_fp32(lblib):
    """The FP32 context's observables (per-node sums formed in FP32 from the stored
    deviations, accumulated in FP64) against the oracle.  Bounds from the arithmetic: the
    mass is rho0 L^3 plus FP32 deviation sums, whose rounding (~6e-8 of |n - w rho0| ~ 1e-2
    per population) adds up to ~1e-10 of the mass over 50 steps: 1e-8 relative is stated;
    momentum: the same rounding on J, stated as 1e-7 of the box momentum at one lattice unit
    of velocity; chain observables follow the beads' FP32 bar (1e-5 of the box per coordinate):
    R_g^2, R_e^2 and the centre of mass within 1e-4 relative, the bead temperature 1e-4."""
    case = Case(L=16, N=8, steps=50, seed=5)
    st = oracle_run(case)
    fp, cp = case.fluid(), case.chain()
    _, _, _, obs = gpu_run(lblib, case, lblib.LB_FP32)
    scale = fp.L ** 3 * fp.rho * fp.a ** 4 / fp.h
    errs = {
        "mass": abs(obs[1] / o.total_mass(st, fp) - 1),
        "P_total": float(np.abs(obs[2:5] - o.total_momentum(st, fp, cp)).max() / scale),
        "P_fluid": float(np.abs(obs[5:8] - o.fluid_momentum(st, fp)).max() / scale),
        "Rg2": abs(obs[8] / o.radius_of_gyration2(st.X) - 1),
        "Re2": abs(obs[9] / o.end_to_end2(st.X) - 1),
        "cm": float(np.abs(obs[10:13] / st.X.mean(axis=0) - 1).max()),
        "T_bead": abs(obs[15] / (cp.m * (st.V ** 2).sum() / (3 * cp.N)) - 1),
    }
    print("FP32 observables vs oracle:", {k: f"{v:.1e}" for k, v in errs.items()})
    assert obs[0] == case.steps
    assert errs["mass"] <= 1e-8
    assert errs["P_total"] <= 1e-7 and errs["P_fluid"] <= 1e-7
    assert errs["Rg2"] <= 1e-4 and errs["Re2"] <= 1e-4 and errs["cm"] <= 1e-4
    assert errs["T_bead"] <= 1e-4


def test_mass_and_momentum_invariants_on_gpu(lblib):
    """Exact invariants of the coupled step (collision and coupling conserve mass and total
    momentum) at the full L = 64 size, FP64 and FP32."""
    for prec, tol in ((lblib.LB_FP64, 1e-12), (lblib.LB_FP32, 1e-5)):
        case = Case(L=64, N=64, steps=0, seed=2)
        sim = gpu_sim(lblib, case, prec)
        o0 = sim.observables()
        sim.step(50)
        o1 = sim.observables()
        sim.close()
        assert o1[1] == pytest.approx(o0[1], rel=tol)
        scale = 64 ** 3 * 1.0 / 0.01  # momentum of the box at one lattice velocity unit
        assert np.allclose(o1[2:5], o0[2:5], rtol=0, atol=tol * scale)


def test_checkpoint_resume_is_bit_exact(lblib, tmp_path):
    case = Case(L=12, N=6, steps=0, seed=8)
    for prec in (lblib.LB_FP64, lblib.LB_FP32):
        a = gpu_sim(lblib, case, prec)
        a.step(10)
        path = str(tmp_path / f"ck{prec}.bin")
        a.save(path)
        a.step(10)
        na = a.populations()
        xa, va = a.beads()
        b = gpu_sim(lblib, case, prec)
        b.load(path)
        assert lblib.lb_get_step(b.ctx) == 10
        b.step(10)
        nb = b.populations()
        xb, vb = b.beads()
        assert np.array_equal(na, nb) and np.array_equal(xa, xb) and np.array_equal(va, vb)
        a.close()
        b.close()


def test_runs_are_deterministic_and_workspace_owner_independent(lblib):
    case = Case(L=16, N=16, steps=20, seed=6)
    r1 = gpu_run(lblib, case, lblib.LB_FP32)
    sim = gpu_sim(lblib, case, lblib.LB_FP32)
    sim._torch_workspace = False  # library-owned cudaMalloc workspace
    sim.step(case.steps)
    n2 = sim.populations()
    x2, _ = sim.beads()
    sim.close()
    assert np.array_equal(r1[0], n2) and np.array_equal(r1[1], x2)


def test_fene_break_is_reported_not_faulted(lblib):
    """A bond pulled past R0 latches LB_ERR_FENE in the device status word; the host reads
    it at the next synchronising call and the context stays usable."""
    ctx = lblib.lb_create(8, 1.0, 3.0, 3.0, 0.0, 0.01, 1.0, 1, lblib.LB_FP32)
    lblib.lb_add_chain(ctx, 2, 1.0, 20.8, 30.0, 1.5, 1.0, 1.0, x0=[[3.0, 4, 4], [4.4, 4, 4]],
                       v0=[[-60.0, 0, 0], [60.0, 0, 0]])
    lblib.lb_step(ctx, 5)
    with pytest.raises(lblib.LBError) as ei:
        lblib.lb_sync(ctx)
    assert ei.value.code == lblib.LB_ERR_FENE
    lblib.lb_destroy(ctx)


def test_philox_gpu_is_bit_identical_to_oracle(lblib):
    import torch

    rng = np.random.default_rng(1)
    ctr = rng.integers(0, 2 ** 32, size=(4096, 4), dtype=np.uint64).astype(np.uint32)
    ctr[0] = 0
    ctr[1] = 0xFFFFFFFF
    dev = torch.from_numpy(ctr.view(np.int32)).cuda()
    out = torch.empty_like(dev)
    for k0, k1 in ((0, 0), (1, 0), (0xDEADBEEF, 0x102), (0xFFFFFFFF, 0xFFFFFFFF)):
        lblib.lb_philox4x32_10(dev.data_ptr(), 4096, k0, k1, out.data_ptr(), torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        got = out.cpu().numpy().view(np.uint32)
        want = np.stack(o.philox4x32_10(ctr[:, 0], ctr[:, 1], ctr[:, 2], ctr[:, 3], k0, k1), axis=1)
        assert np.array_equal(got, want)


def test_cell_index_is_bit_exact(lblib):
    import torch

    L = 16
    xs = [0.0, -0.0, 1.0, 15.0, 16.0, -1.0, -16.0, 1e4 * L, -1e4 * L - 0.5, 31.999]
    for k in (1, 5, 15, 16, 17, -1, -16, 160000):
        xk = np.float32(k)
        xs += [np.nextafter(xk, np.float32(np.inf)), np.nextafter(xk, np.float32(-np.inf))]
    rng = np.random.default_rng(2)
    xs += list(rng.uniform(-100, 100, 2000))
    x = np.array(xs, dtype=np.float32)
    for a in (1.0, 0.7, 1.3):
        xd = torch.from_numpy(x).cuda()
        out = torch.empty(x.size, dtype=torch.int32, device="cuda")
        lblib.lb_cell_index_f32(xd.data_ptr(), x.size, a, L, out.data_ptr(), torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        want = o.cell_index(x, np.float32(a), L)
        assert np.array_equal(out.cpu().numpy(), want), a


def test_md_substeps_with_paper_parameters(lblib):
    """The paper's production setting (Sec. II E): kT = 1.2, rho = 0.864, nu = 2.8, k = 7,
    R0 = 2, zeta = 20.8, MD step 0.01 with an LB step of 0.02 (two MD substeps)."""
    case = Case(L=10, N=8, steps=25, seed=31, rho=0.864, eta=0.864 * 2.8, eta_b=0.864 * 2.8, kT=1.2, h=0.02,
                k_fene=7.0, R0=2.0, substeps=2)
    st = oracle_run(case)
    for prec, tol in ((lblib.LB_FP64, 1e-12), (lblib.LB_FP32, 1e-5)):
        n, x, v, _ = gpu_run(lblib, case, prec)
        assert pop_rel_err(n, st.n) <= tol
        ex, ev = bead_errs(x, v, st, case)
        assert ex <= tol and ev <= (10 * tol if prec == lblib.LB_FP64 else tol)


@pytest.mark.parametrize("case", [
    Case(L=12, N=24, steps=30, seed=3),
    Case(L=40, N=32, steps=12, seed=4, ext=(0.5, -0.2, 0.1), counter=True),
    Case(L=9, N=10, steps=15, seed=5, substeps=3),
    Case(L=12, N=48, steps=6, seed=6, substeps=3),
], ids=["L12", "L40_body_force", "L9_substeps", "L12_sorted_spreading"])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_deferred_corrections_are_bit_exact(lblib, case, prec):
    """Consecutive steps keep each step's bead force correction pending and add it where the
    next step reads the populations (LB kernel at the marked nodes, bead gather from the dense
    correction field).  In FP64 and FP32 that is the same arithmetic as
    applying it at the end of every step: K deferred steps and K steps each completed by a
    read of the fluid agree bit for bit."""
    p = getattr(lblib, "LB_" + prec.upper())
    a = gpu_sim(lblib, case, p)
    a.step(case.steps)
    na = a.populations()
    xa, va = a.beads()
    b = gpu_sim(lblib, case, p)
    for _ in range(case.steps):
        b.step(1)
        b.observables()  # reads the fluid: applies the pending correction (a complete step)
    nb = b.populations()
    xb, vb = b.beads()
    a.close()
    b.close()
    assert np.array_equal(na, nb)
    assert np.array_equal(xa, xb) and np.array_equal(va, vb)


@pytest.mark.parametrize("N", [0, 24], ids=["fluid", "chain"])
def test_chained_and_ordinary_launches_agree_bit_for_bit(lblib, N):
    """Without timing, consecutive kernels are chained by programmatic dependent launch (each
    grid released at the start of the one before it, waiting for it before it reads; the LB
    kernel beside the bead kernel of its step waits for it before completing).  With
    lb_set_timing every launch is an ordinary one.  The two give the same state bit for bit."""
    case = Case(L=24, N=N, steps=25, seed=12)
    a = gpu_sim(lblib, case, lblib.LB_FP32)
    a.step(case.steps)
    na = a.populations()
    b = gpu_sim(lblib, case, lblib.LB_FP32)
    lblib.lb_set_timing(b.ctx, True)
    b.step(case.steps)
    lblib.lb_set_timing(b.ctx, False)
    nb = b.populations()
    assert np.array_equal(na, nb)
    if N:
        xa, va = a.beads()
        xb, vb = b.beads()
        assert np.array_equal(xa, xb) and np.array_equal(va, vb)
    a.close()
    b.close()


def test_deferred_corrections_with_observable_stride(lblib):
    """Observables taken inside a multi-step call flush the pending correction first."""
    case = Case(L=10, N=12, steps=20, seed=9)
    a = gpu_sim(lblib, case, lblib.LB_FP64)
    lblib.lb_set_obs_stride(a.ctx, 3)
    a.step(case.steps)
    na = a.populations()
    st = oracle_run(case)
    assert pop_rel_err(na, st.n) <= 1e-12
    a.close()


def test_spreading_of_many_entries_matches_oracle(lblib):
    """More than 1024 corner entries per step (N = 48 beads, 3 MD substeps: 1152) take the
    sorted grouping instead of the shared-memory table; FP64 parity with the oracle."""
    case = Case(L=12, N=48, steps=6, seed=6, substeps=3)
    st = oracle_run(case)
    n, x, v, obs = gpu_run(lblib, case, lblib.LB_FP64)
    assert pop_rel_err(n, st.n) <= 1e-12
    ex, ev = bead_errs(x, v, st, case)
    assert ex <= 1e-12 and ev <= 1e-11


@pytest.mark.parametrize("N", [12, 48], ids=["one_block", "cluster"])
def test_asynchronous_bead_read_back(lblib, N, tmp_path):
    """lb_get_beads_async + lb_wait return what lb_get_beads returns, step after step, with
    reads queued behind later steps (copied from the bead kernel's per-step snapshot, off the
    context's stream); after a checkpoint load (the snapshot no longer holds the state) the
    read-back of the loaded state; a ticket not yet issued is an argument error."""
    import torch

    case = Case(L=10, N=N, steps=0, seed=12)
    a = gpu_sim(lblib, case, lblib.LB_FP32)
    b = gpu_sim(lblib, case, lblib.LB_FP32)
    a._bind()
    bufs = [(torch.empty((N, 3), dtype=torch.float64, pin_memory=True).numpy(),
             torch.empty((N, 3), dtype=torch.float64, pin_memory=True).numpy()) for _ in range(3)]
    tickets, ref = [], {}
    for k in range(9):
        a.step(1)
        tickets.append(lblib.lb_get_beads_async(a.ctx, bufs[k % 3][0], bufs[k % 3][1], 3 * N))
        b.step(1)
        xr, vr = b.beads()
        ref[k] = (xr.copy(), vr.copy())
        if k >= 2:  # the read-back of step k-2 while steps k-1 and k are queued behind it
            lblib.lb_wait(a.ctx, tickets[k - 2])
            xo, vo = bufs[(k - 2) % 3]
            assert np.array_equal(xo, ref[k - 2][0]) and np.array_equal(vo, ref[k - 2][1])
    for t in tickets[-2:]:
        lblib.lb_wait(a.ctx, t)
    path = str(tmp_path / "state.lb")
    lblib.lb_save(a.ctx, path)
    xs, vs = a.beads()
    a.step(3)
    lblib.lb_load(a.ctx, path)
    t = lblib.lb_get_beads_async(a.ctx, bufs[0][0], bufs[0][1], 3 * N)
    lblib.lb_wait(a.ctx, t)
    assert np.array_equal(bufs[0][0], xs) and np.array_equal(bufs[0][1], vs)
    with pytest.raises(lblib.LBError) as ei:
        lblib.lb_wait(a.ctx, t + 1)
    assert ei.value.code == lblib.LB_ERR_ARG
    a.close()
    b.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32", "bf16"])
def test_populations_through_pinned_and_pageable_host_memory(lblib, prec):
    """lb_get_populations / lb_set_populations address page-locked host memory directly (one
    conversion kernel over the 19 planes) and copy other host memory through the second
    population buffer in chunks of planes: both routes give the same populations bit for bit,
    a round trip through either reproduces the state, and stepping on goes the same way."""
    import torch

    p = {"fp64": lblib.LB_FP64, "fp32": lblib.LB_FP32, "bf16": lblib.LB_BF16}[prec]
    case = Case(L=24, N=8, steps=0, seed=13, perturb=0.02)
    a = gpu_sim(lblib, case, p)
    a.step(6)
    pageable = a.populations()
    pinned = torch.empty((19, 24, 24, 24), dtype=torch.float64).pin_memory().numpy()
    lblib.lb_get_populations(a.ctx, pinned)
    assert np.array_equal(pageable, pinned)
    lblib.lb_set_populations(a.ctx, pinned)  # round trip through page-locked memory
    assert np.array_equal(a.populations(), pageable)
    a.set_populations(pageable)  # and through pageable memory
    assert np.array_equal(a.populations(), pageable)
    a.step(4)
    ref = a.populations()
    a.close()
    b = gpu_sim(lblib, case, p)
    b.step(6)
    lblib.lb_set_populations(b.ctx, pinned)
    b.step(4)
    assert np.array_equal(b.populations(), ref)
    b.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_bead_kernel_cells_match_the_oracle_step_by_step(lblib, prec):
    """The 8 cells around each bead that the running bead kernel coupled to (Sec. II B, last
    paragraph), read back after every step of the L = 16, N = 8 workload (100 steps):
    (1) bit-exact against the oracle's cell function applied to the kernel's own stored
    coordinate (floor(x/a) mod L in the stored precision), and (2) equal to the cells of the
    oracle's own FP64 trajectory except for coordinates closer to a cell face than the path's
    parity bar on positions (1e-9 of the box in FP64, 1e-5 in FP32), which are counted."""
    p = lblib.LB_FP64 if prec == "fp64" else lblib.LB_FP32
    dtype = np.float64 if prec == "fp64" else np.float32
    band = (1e-9 if prec == "fp64" else 1e-5) * 16
    case = Case(L=16, N=8, steps=0, seed=1)
    fp, cp = case.fluid(), case.chain()
    L, a = case.L, case.a
    st = o.init_state(fp, cp, case.x0())
    sim = gpu_sim(lblib, case, p)
    offs = np.array([[c & 1, (c >> 1) & 1, (c >> 2) & 1] for c in range(8)])

    def corners(cells):  # (N, 3) cells -> (N, 8) node indices in the kernel's corner order
        q = (cells[:, None, :] + offs[None]) % L
        return q[..., 0] + L * (q[..., 1] + L * q[..., 2])

    near = compared = 0
    for _ in range(100):
        sim.step(1)
        st = o.step(st, fp, cp)
        nodes, xs = lblib.lb_debug_coupling_cells(sim.ctx, case.N)
        nodes = nodes[0]
        assert np.array_equal(nodes, corners(o.cell_index(xs.astype(dtype), dtype(a), L)))
        s = st.X / a
        frac = s - np.floor(s)
        ok = np.all(np.minimum(frac, 1.0 - frac) * a > band, axis=1)
        near += int((~ok).sum())
        compared += int(ok.sum())
        assert np.array_equal(nodes[ok], corners(o.cell_index(st.X, a, L))[ok])
    sim.close()
    print(f"{prec}: {compared} bead-steps compared against the oracle trajectory, {near} within the band")
    assert compared >= 0.95 * 100 * case.N
