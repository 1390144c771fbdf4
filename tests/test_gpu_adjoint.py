"""The adjoint of the coupled step (noise held fixed, checkpoints every K steps) against finite
differences: of the library's own FP64 forward path, and of the FP64 oracle on the
L = 32, N = 16 workload (100 steps, checkpoint every 10, seed 7); and against the oracle's
tangent-linear (forward-mode) derivative on that workload.

Objective O = sum_b |x_b(T) - x_b(0)|^2; derivatives with respect to the initial positions
(checked along random directions) and zeta.  The trilinear weights have kinks on the cell
faces, where a one-sided adjoint and a central difference differ; the oracle-based test uses
a perturbation of 1e-5 (smaller steps are dominated by round-off of the 100-step objective)
and verifies that no bead changes cell between the two perturbed trajectories."""
import numpy as np
import pytest

from oracle import lbchain as o
from paper_0903_5067_gb300 import inputs

pytestmark = pytest.mark.gpu

CHAIN = dict(m=1.0, k_fene=30.0, R0=1.5, eps=1.0, sigma=1.0)


def _gpu_objective(lb, L, X0, zeta, T, seed, prec, kT=1.0):
    sim = lb.Simulation(L=L, rho=1.0, eta=3.0, eta_b=3.0, kT=kT, h=0.01, a=1.0, seed=seed, precision=prec)
    sim.add_chain(X0.shape[0], zeta=zeta, x0=X0, **CHAIN)
    sim.step(T)
    x, _ = sim.beads()
    sim.close()
    return float(((x - X0) ** 2).sum())


def _gpu_adjoint(lb, L, X0, zeta, T, K, seed, prec, kT=1.0):
    sim = lb.Simulation(L=L, rho=1.0, eta=3.0, eta_b=3.0, kT=kT, h=0.01, a=1.0, seed=seed, precision=prec)
    sim.add_chain(X0.shape[0], zeta=zeta, x0=X0, **CHAIN)
    sim._bind()
    O, gx, gz = lb.lb_adjoint_displacement(sim.ctx, T, K, X0.shape[0])
    assert lb.lb_get_step(sim.ctx) == T
    sim.close()
    return O, gx, gz


def _oracle_objective(L, X0, zeta, T, seed):
    """O and the per-step cells of every bead (to detect face crossings)."""
    fp = o.FluidParams(L=L, rho=1.0, eta=3.0, eta_b=3.0, kT=1.0, h=0.01, a=1.0, seed=seed)
    cp = o.ChainParams(N=X0.shape[0], zeta=zeta, **CHAIN)
    st = o.init_state(fp, cp, X0)
    cells = []
    for _ in range(T):
        st = o.step(st, fp, cp)
        cells.append(np.floor(st.X).astype(np.int64))
    return float(((st.X - X0) ** 2).sum()), np.array(cells)


def test_adjoint_fp64_matches_finite_differences_of_the_gpu_path(lblib):
    L, N, T, K, seed = 8, 4, 12, 5, 21  # segments of 5, 5, 2 steps
    X0 = inputs.chain_walk(N, L=L, bond=0.97, seed=seed, self_avoiding=True)
    zeta = 20.8
    O, gx, gz = _gpu_adjoint(lblib, L, X0, zeta, T, K, seed, lblib.LB_FP64)
    assert O == pytest.approx(_gpu_objective(lblib, L, X0, zeta, T, seed, lblib.LB_FP64), rel=1e-13)
    rng = np.random.default_rng(3)
    eps = 1e-6
    for _ in range(3):
        d = rng.standard_normal((N, 3))
        fd = (_gpu_objective(lblib, L, X0 + eps * d, zeta, T, seed, lblib.LB_FP64)
              - _gpu_objective(lblib, L, X0 - eps * d, zeta, T, seed, lblib.LB_FP64)) / (2 * eps)
        assert (gx * d).sum() == pytest.approx(fd, rel=1e-5, abs=1e-8)
    fdz = (_gpu_objective(lblib, L, X0, zeta + eps, T, seed, lblib.LB_FP64)
           - _gpu_objective(lblib, L, X0, zeta - eps, T, seed, lblib.LB_FP64)) / (2 * eps)
    assert gz == pytest.approx(fdz, rel=1e-5, abs=1e-8)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_adjoint_is_independent_of_the_checkpoint_interval(lblib, prec):
    """The gradient does not depend on how the T steps are cut into checkpoint segments: a
    single segment longer than T (launched directly), full segments replayed as graphs with a
    partial last segment, and full segments only, all against one segment of T steps (the same
    states are recomputed bit for bit, so the results agree to round-off of nothing)."""
    p = lblib.LB_FP64 if prec == "fp64" else lblib.LB_FP32
    L, N, seed = 8, 4, 21
    X0 = inputs.chain_walk(N, L=L, bond=0.97, seed=seed, self_avoiding=True)
    for T, Ks in ((7, (10, 3)), (23, (5, 4)), (24, (6, 5))):
        O, gx, gz = _gpu_adjoint(lblib, L, X0, 20.8, T, T, seed, p)
        for K in Ks:
            O2, gx2, gz2 = _gpu_adjoint(lblib, L, X0, 20.8, T, K, seed, p)
            assert O2 == O and np.array_equal(gx2, gx) and gz2 == gz, (T, K)


def test_adjoint_c5_workload_matches_oracle_finite_differences(lblib):
    """L=32, N=16, 100 steps, checkpoints every 10, noise fixed by seed 7: FP32 adjoint
    within 1e-3 and FP64 adjoint within 1e-6 of central differences of the FP64 oracle with
    the step 1e-5.  The configured step 1e-4 is checked beside it: its truncation error
    (O(eps^2) times the third derivative of the 100-step objective) is larger, so the FP64
    bar there is 1e-4; both differences are printed."""
    L, N, T, K, seed, zeta = 32, 16, 100, 10, 7, 20.8
    X0 = inputs.chain_walk(N, L=L, bond=0.97, seed=seed, self_avoiding=True)
    O64, gx64, gz64 = _gpu_adjoint(lblib, L, X0, zeta, T, K, seed, lblib.LB_FP64)
    O32, gx32, gz32 = _gpu_adjoint(lblib, L, X0, zeta, T, K, seed, lblib.LB_FP32)
    O_or, _ = _oracle_objective(L, X0, zeta, T, seed)
    assert O64 == pytest.approx(O_or, rel=1e-10)
    assert O32 == pytest.approx(O_or, rel=1e-5)
    bars = {1e-5: (1e-6, 1e-3), 1e-4: (1e-4, 1e-3)}  # step: (FP64, FP32) relative bars

    def fd(eps, d=None, dz=0.0):
        """central difference along (d, dz), or None when a bead changes cell between the two
        perturbed trajectories (a kink of the trilinear weights)"""
        dX = np.zeros((N, 3)) if d is None else d
        op, cp_ = _oracle_objective(L, X0 + eps * dX, zeta + eps * dz, T, seed)
        om, cm_ = _oracle_objective(L, X0 - eps * dX, zeta - eps * dz, T, seed)
        return None if not np.array_equal(cp_, cm_) else (op - om) / (2 * eps)

    rng = np.random.default_rng(11)
    checked = {1e-5: 0, 1e-4: 0}
    for _ in range(4):
        d = rng.standard_normal((N, 3))
        for eps, (b64, b32) in bars.items():
            q = fd(eps, d)
            if q is None:
                continue
            print(f"direction {checked[eps]}: step {eps:.0e}: FD {q:.10e}, FP64 adjoint rel. diff "
                  f"{(gx64 * d).sum() / q - 1:+.2e}, FP32 {(gx32 * d).sum() / q - 1:+.2e}")
            assert (gx64 * d).sum() == pytest.approx(q, rel=b64, abs=1e-8)
            assert (gx32 * d).sum() == pytest.approx(q, rel=b32, abs=1e-6)
            checked[eps] += 1
        if min(checked.values()) >= 2:
            break
    assert min(checked.values()) >= 1
    for eps, (b64, b32) in bars.items():
        q = fd(eps, dz=1.0)
        if q is not None:
            print(f"zeta: step {eps:.0e}: FD {q:.10e}, FP64 adjoint rel. diff {gz64 / q - 1:+.2e}, "
                  f"FP32 {gz32 / q - 1:+.2e}")
            assert gz64 == pytest.approx(q, rel=b64, abs=1e-8)
            assert gz32 == pytest.approx(q, rel=b32, abs=1e-6)


def test_adjoint_c5_workload_matches_the_oracle_tangent(lblib):
    """The reverse-mode gradient against the oracle's forward-mode (tangent-linear)
    derivative along the same directions, L=32, N=16, 100 steps, checkpoints every 10,
    seed 7.  Both are exact derivatives of the same trajectory (same cells, same WCA
    branches), so no finite-difference step enters: FP64 within 1e-7, FP32 within 1e-3."""
    from oracle import tangent as tg

    L, N, T, K, seed, zeta = 32, 16, 100, 10, 7, 20.8
    X0 = inputs.chain_walk(N, L=L, bond=0.97, seed=seed, self_avoiding=True)
    O64, gx64, gz64 = _gpu_adjoint(lblib, L, X0, zeta, T, K, seed, lblib.LB_FP64)
    O32, gx32, gz32 = _gpu_adjoint(lblib, L, X0, zeta, T, K, seed, lblib.LB_FP32)
    fp = o.FluidParams(L=L, rho=1.0, eta=3.0, eta_b=3.0, kT=1.0, h=0.01, a=1.0, seed=seed)
    cp = o.ChainParams(N=N, zeta=zeta, **CHAIN)
    rng = np.random.default_rng(23)
    for dz in (0.0, 1.0):
        d = rng.standard_normal((N, 3))
        O, dO = tg.displacement_jvp(fp, cp, X0, T, d, dzeta=dz)
        assert O64 == pytest.approx(O, rel=1e-10)
        assert (gx64 * d).sum() + gz64 * dz == pytest.approx(dO, rel=1e-7, abs=1e-10)
        assert (gx32 * d).sum() + gz32 * dz == pytest.approx(dO, rel=1e-3, abs=1e-6)


def test_autograd_function_returns_the_adjoint(lblib):
    import torch
    from paper_0903_5067_gb300.autograd import chain_displacement

    L, N, T, K, seed = 8, 4, 10, 4, 5
    X0 = inputs.chain_walk(N, L=L, bond=0.97, seed=seed, self_avoiding=True)
    x = torch.tensor(X0, dtype=torch.float64, requires_grad=True)
    z = torch.tensor(20.8, dtype=torch.float64, requires_grad=True)
    params = dict(L=L, seed=seed, precision=lblib.LB_FP64)
    O = chain_displacement(x, z, params, T=T, K=K)
    (3.0 * O).backward()
    O_ref, gx, gz = _gpu_adjoint(lblib, L, X0, 20.8, T, K, seed, lblib.LB_FP64)
    assert O.item() == pytest.approx(O_ref, rel=1e-14)
    assert np.allclose(x.grad.numpy(), 3.0 * gx, rtol=1e-12)
    assert float(z.grad) == pytest.approx(3.0 * gz, rel=1e-12)


def test_autograd_function_keeps_the_device_and_skips_the_adjoint_without_grad(lblib):
    """x0 and zeta on the GPU: O and the gradients come back on that device in the inputs'
    dtypes; without requires_grad the forward gives the same O from the steps alone."""
    import torch
    from paper_0903_5067_gb300.autograd import chain_displacement

    L, N, T, K, seed = 8, 4, 10, 4, 5
    X0 = inputs.chain_walk(N, L=L, bond=0.97, seed=seed, self_avoiding=True)
    x = torch.tensor(X0, dtype=torch.float64, device="cuda", requires_grad=True)
    z = torch.tensor(20.8, dtype=torch.float32, device="cuda", requires_grad=True)
    params = dict(L=L, seed=seed, precision=lblib.LB_FP64)
    O = chain_displacement(x, z, params, T=T, K=K)
    assert O.device == x.device and O.dtype == torch.float64
    O.backward()
    assert x.grad.device == x.device and x.grad.dtype == torch.float64
    assert z.grad.device == z.device and z.grad.dtype == torch.float32
    O_ref, gx, gz = _gpu_adjoint(lblib, L, X0, float(z.item()), T, K, seed, lblib.LB_FP64)  # zeta as FP32 holds it
    assert O.item() == pytest.approx(O_ref, rel=1e-14)
    assert np.allclose(x.grad.cpu().numpy(), gx, rtol=1e-12)
    assert float(z.grad) == pytest.approx(gz, rel=1e-6)
    with torch.no_grad():
        O2 = chain_displacement(x, z, params, T=T, K=K)
    assert O2.item() == pytest.approx(O.item(), rel=1e-13) and not O2.requires_grad


def test_adjoint_rejects_a_stepped_context(lblib):
    sim = lblib.Simulation(L=8, seed=1, precision=lblib.LB_FP64)
    sim.add_chain(3, x0=inputs.chain_walk(3, L=8, seed=1, self_avoiding=True))
    sim.step(1)
    with pytest.raises(lblib.LBError) as ei:
        lblib.lb_adjoint_displacement(sim.ctx, 5, 2, 3)
    assert ei.value.code == lblib.LB_ERR_STATE
    sim.close()
