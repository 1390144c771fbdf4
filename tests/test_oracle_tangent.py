"""Pins of the oracle's tangent-linear derivative (forward mode) against central finite
differences of the oracle itself: the chain force field (Sec. II A, Eqs. 1-2), the
trilinear interpolation and spreading (Sec. II B, last paragraph), the collision with noise
and forcing (Sec. II B, Eqs. 3-4), and whole coupled trajectories.  A dropped or mis-signed
term in any of the derivative rules moves the tangent away from the difference quotient by
far more than the tolerances below."""
import numpy as np
import pytest

from oracle import lbchain as o
from oracle import tangent as t
from paper_0903_5067_gb300 import inputs


def _chain_params(**kw):
    base = dict(N=6, m=1.0, zeta=20.8, k_fene=30.0, R0=1.5, eps=1.0, sigma=1.0)
    base.update(kw)
    return o.ChainParams(**base)


def _folded_chain():
    # bonds between 0.9 and 1.3, two non-bonded pairs inside the WCA range, one pair across
    # the periodic boundary of a box of 10
    return np.array([[9.6, 5.0, 5.0], [0.5, 5.1, 5.0], [1.3, 5.8, 5.2], [1.0, 6.6, 5.9],
                     [0.3, 5.9, 5.4], [9.4, 5.9, 5.3]])


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def test_force_jvp_matches_finite_differences_of_the_force_field():
    cp = _chain_params()
    X = _folded_chain()
    rng = np.random.default_rng(1)
    for _ in range(4):
        dX = rng.standard_normal(X.shape)
        eps = 1e-6
        fd = (o.chain_forces(X + eps * dX, cp, 10.0) - o.chain_forces(X - eps * dX, cp, 10.0)) / (2 * eps)
        assert _rel(t.force_jvp(X, dX, cp, 10.0), fd) < 1e-7
    # a single stretched FENE bond and a single WCA pair, each alone
    X2 = np.array([[0.0, 0.0, 0.0], [1.4, 0.1, 0.0]])
    dX2 = np.array([[0.0, 0.0, 0.0], [1.0, 0.0, 0.0]])
    cp2 = _chain_params(N=2)
    fd = (o.chain_forces(X2 + 1e-7 * dX2, cp2, 50.0) - o.chain_forces(X2 - 1e-7 * dX2, cp2, 50.0)) / 2e-7
    assert _rel(t.force_jvp(X2, dX2, cp2, 50.0), fd) < 1e-6


def test_interpolation_and_spreading_jvp_match_finite_differences():
    fp = o.FluidParams(L=5, a=1.3)
    rng = np.random.default_rng(2)
    field = rng.standard_normal((3, 5, 5, 5))
    dfield = rng.standard_normal((3, 5, 5, 5))
    # positions inside cells (away from faces), including one across the periodic wrap
    X = np.array([[0.4, 1.7, 2.9], [6.1, 0.2, 3.3], [-0.65, 5.0, 4.1]])
    dX = rng.standard_normal(X.shape)
    Fc = rng.standard_normal(X.shape)
    dFc = rng.standard_normal(X.shape)
    eps = 1e-6
    val, dval = t.interp_field_jvp(field, dfield, X, dX, fp)
    assert np.array_equal(val, o.interp_field(field, X, fp))
    fd = (o.interp_field(field + eps * dfield, X + eps * dX, fp)
          - o.interp_field(field - eps * dfield, X - eps * dX, fp)) / (2 * eps)
    assert _rel(dval, fd) < 1e-8
    f, df = t.spread_jvp(Fc, dFc, X, dX, fp)
    assert np.array_equal(f, o.spread(Fc, X, fp))
    fd = (o.spread(Fc + eps * dFc, X + eps * dX, fp) - o.spread(Fc - eps * dFc, X - eps * dX, fp)) / (2 * eps)
    assert _rel(df, fd) < 1e-8


@pytest.mark.parametrize("stress_only", [False, True])
def test_collide_jvp_matches_finite_differences_of_the_collision(stress_only):
    # a large kT makes the density dependence of the noise amplitude visible next to the
    # relaxation; forcing at three nodes, and a force derivative at a fourth node where the
    # force itself is zero
    L = 4
    fp = o.FluidParams(L=L, kT=200.0, seed=5, stress_only=stress_only)
    rng = np.random.default_rng(3)
    n = o.fluid_at_rest(fp) * (1.0 + 0.05 * rng.standard_normal((o.Q, L, L, L)))
    dn = 0.01 * rng.standard_normal(n.shape)
    f = np.zeros((3, L, L, L))
    df = np.zeros_like(f)
    for (z, y, x) in [(0, 0, 0), (1, 2, 3), (3, 3, 1)]:
        f[:, z, y, x] = rng.standard_normal(3) * 40.0
        df[:, z, y, x] = rng.standard_normal(3) * 40.0
    df[:, 2, 1, 0] = rng.standard_normal(3) * 40.0
    eps = 1e-6
    fd = (o.collide(n + eps * dn, fp, 7, force_density=f + eps * df)
          - o.collide(n - eps * dn, fp, 7, force_density=f - eps * df)) / (2 * eps)
    jv = t.collide_jvp(n, dn, fp, 7, force_density=f, dforce_density=df)
    assert _rel(jv, fd) < 1e-7
    # without the noise-amplitude term the tangent misses the difference quotient
    fp0 = o.FluidParams(L=L, kT=200.0, seed=5, stress_only=stress_only, noise_fluid=False)
    jv0 = t.collide_jvp(n, dn, fp0, 7, force_density=f, dforce_density=df)
    assert _rel(jv0, fd) > 1e-4


def test_step_jvp_carries_the_oracle_state_unchanged():
    fp = o.FluidParams(L=6, seed=4)
    cp = _chain_params(N=4)
    X0 = inputs.chain_walk(4, L=6, bond=0.97, seed=4, self_avoiding=True)
    st = o.init_state(fp, cp, X0)
    ref = o.run(st, fp, cp, 3)
    tg = t.init_tangent(st, fp, cp, np.ones((4, 3)))
    for _ in range(3):
        st, tg = t.step_jvp(st, tg, fp, cp, dzeta=1.0)
    for name in ("n", "X", "V", "F", "Fc"):
        assert np.array_equal(getattr(st, name), getattr(ref, name)), name
    assert st.step == ref.step


def _objective_and_cells(fp, cp, X0, T):
    st = o.init_state(fp, cp, X0)
    cells = []
    for _ in range(T):
        st = o.step(st, fp, cp)
        cells.append(np.floor(st.X / fp.a).astype(np.int64))
    return float(((st.X - X0) ** 2).sum()), np.array(cells)


@pytest.mark.parametrize("case", ["noise", "no_noise", "substeps2", "stress_only"])
def test_trajectory_derivative_matches_central_differences(case):
    L, N, T, seed = 8, 4, 12, 21
    fp = o.FluidParams(L=L, seed=seed, noise_fluid=(case != "no_noise"),
                       stress_only=(case == "stress_only"))
    cp = _chain_params(N=N, substeps=2 if case == "substeps2" else 1,
                       noise_beads=(case != "no_noise"))
    if case == "no_noise":
        cp.ext_force = (3.0, -1.0, 0.5)  # something to move the chain without noise
    X0 = inputs.chain_walk(N, L=L, bond=0.97, seed=seed, self_avoiding=True)
    rng = np.random.default_rng(7)
    eps = 1e-6
    checked = 0
    for trial in range(4):
        dX = rng.standard_normal((N, 3))
        dz = 0.0 if trial == 0 else 1.0
        O, dO = t.displacement_jvp(fp, cp, X0, T, dX, dzeta=dz)
        cpp = _chain_params(N=N, zeta=cp.zeta + eps * dz, substeps=cp.substeps,
                            noise_beads=cp.noise_beads, ext_force=cp.ext_force)
        cpm = _chain_params(N=N, zeta=cp.zeta - eps * dz, substeps=cp.substeps,
                            noise_beads=cp.noise_beads, ext_force=cp.ext_force)
        op, cellp = _objective_and_cells(fp, cpp, X0 + eps * dX, T)
        om, cellm = _objective_and_cells(fp, cpm, X0 - eps * dX, T)
        assert O == pytest.approx(_objective_and_cells(fp, cp, X0, T)[0], rel=1e-15)
        if not np.array_equal(cellp, cellm):
            continue  # a bead changed cell between the two runs: a kink of the weights
        assert dO == pytest.approx((op - om) / (2 * eps), rel=1e-6, abs=1e-9)
        checked += 1
    assert checked >= 2


def test_zeta_derivative_includes_the_noise_amplitude():
    """With the bead noise on, dO/dzeta has a term from d sqrt(2 kT zeta / h) / d zeta; with
    that term left out (noise amplitude held fixed) the derivative differs."""
    L, N, T, seed = 8, 4, 10, 3
    fp = o.FluidParams(L=L, seed=seed)
    cp = _chain_params(N=N)
    X0 = inputs.chain_walk(N, L=L, bond=0.97, seed=seed, self_avoiding=True)
    zero = np.zeros((N, 3))
    _, dz = t.displacement_jvp(fp, cp, X0, T, zero, dzeta=1.0)
    eps = 1e-6
    op, _ = _objective_and_cells(fp, _chain_params(N=N, zeta=cp.zeta + eps), X0, T)
    om, _ = _objective_and_cells(fp, _chain_params(N=N, zeta=cp.zeta - eps), X0, T)
    fd = (op - om) / (2 * eps)
    assert dz == pytest.approx(fd, rel=1e-6)
    # the same run with the Langevin amplitude frozen at zeta: a visibly different slope
    amp = np.sqrt(2.0 * fp.kT * cp.zeta / fp.h)

    op2 = _frozen_amplitude_objective(fp, cp, X0, T, cp.zeta + eps, amp)
    om2 = _frozen_amplitude_objective(fp, cp, X0, T, cp.zeta - eps, amp)
    assert abs((op2 - om2) / (2 * eps) - fd) > 1e-3 * abs(fd)


def _frozen_amplitude_objective(fp, cp, X0, T, zeta, amp):
    """The oracle trajectory with the friction at zeta but the bead noise amplitude fixed."""
    cpz = _chain_params(N=cp.N, zeta=zeta, noise_beads=False)
    st = o.init_state(fp, cpz, X0)
    box = fp.L * fp.a
    for _ in range(T):
        k = st.step
        n_ps = o.stream(st.n)
        X, Vh = o.bead_kick_drift(st.X, st.V, st.F, cpz, fp.h)
        Fcons = o.chain_forces(X, cpz, box)
        ub = o.interpolate_u(n_ps, fp, X)
        Fc = -zeta * (Vh - ub) + amp * o.bead_gaussians(fp.seed, 0, k, cp.N)
        f = o.spread(Fc, X, fp)
        F = Fcons + Fc
        V = o.bead_kick(Vh, F, cpz, fp.h)
        st = o.State(o.collide(n_ps, fp, k, force_density=f), X, V, F, Fc, k + 1)
    return float(((st.X - X0) ** 2).sum())
