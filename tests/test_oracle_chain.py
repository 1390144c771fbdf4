"""Pins of the oracle's bead-spring chain and its dissipative coupling to the fluid
(Sec. II A Eqs. 1-2; Sec. II B last paragraph; Sec. II D Eq. 7)."""
import math

import numpy as np
import pytest

from oracle import lbchain as o
from paper_0903_5067_gb300 import inputs


def _chain_params(**kw):
    base = dict(N=6, m=1.0, zeta=20.8, k_fene=30.0, R0=1.5, eps=1.0, sigma=1.0)
    base.update(kw)
    return o.ChainParams(**base)


def test_forces_are_minus_gradient_of_fene_plus_wca():
    cp = _chain_params()
    box = 10.0
    # a folded chain: bonds between 0.9 and 1.3, non-bonded pairs (1,4) and (0,5) inside the
    # WCA range, plus one pair across the periodic boundary
    X = np.array([[9.6, 5.0, 5.0], [0.5, 5.1, 5.0], [1.3, 5.8, 5.2], [1.0, 6.6, 5.9],
                  [0.3, 5.9, 5.4], [9.4, 5.9, 5.3]])
    d = np.linalg.norm(o.min_image(X[:, None] - X[None], box), axis=-1)
    assert d[1, 4] < 2 ** (1 / 6) and d[0, 5] < 2 ** (1 / 6)
    assert all(d[i, i + 1] < cp.R0 for i in range(5))
    F = o.chain_forces(X, cp, box)
    h = 1e-5
    for b in range(6):
        for al in range(3):
            Xp, Xm = X.copy(), X.copy()
            Xp[b, al] += h
            Xm[b, al] -= h
            fd = -(o.chain_energy(Xp, cp, box) - o.chain_energy(Xm, cp, box)) / (2 * h)
            assert F[b, al] == pytest.approx(fd, rel=1e-6, abs=1e-6)
    assert np.allclose(F.sum(axis=0), 0.0, atol=1e-10)  # pairwise: Newton's third law


def test_wca_is_cut_and_shifted_at_two_to_the_sixth():
    rc = 2 ** (1 / 6)
    assert float(o.v_wca(np.array(rc), 1.0, 1.0)) == pytest.approx(0.0, abs=1e-15)
    assert float(o.v_wca(np.array(rc * 1.0001), 1.0, 1.0)) == 0.0
    assert float(o.v_wca(np.array(1.0), 1.0, 1.0)) == pytest.approx(1.0)  # 4(1 - 1 + 1/4)
    cp = _chain_params(N=3)
    X = np.array([[0.0, 0, 0], [0.97, 0, 0], [rc + 0.2, 0.9, 0]])
    F1 = o.chain_forces(X, cp, 50.0)
    X2 = X.copy()
    X2[2] = [0.97 + rc + 1e-9, 0, 0]  # bead 2 just outside the WCA range of bead 1 along x
    cpn = _chain_params(N=2)
    assert np.allclose(o.chain_forces(X2[:2], cpn, 50.0), o.chain_forces(X[:2], cpn, 50.0))
    assert np.all(np.isfinite(F1))


def test_fene_beyond_max_extension_is_an_error():
    cp = _chain_params(N=2)
    with pytest.raises(o.FeneBroken):
        o.chain_forces(np.array([[0.0, 0, 0], [1.5, 0, 0]]), cp, 20.0)


def test_minimum_image_for_pairs_across_the_box():
    cp = _chain_params(N=2)
    L = 8.0
    a = np.array([[0.2, 4.0, 4.0], [L - 0.6, 4.0, 4.0]])  # 0.8 apart through the boundary
    b = np.array([[4.2, 4.0, 4.0], [3.4, 4.0, 4.0]])
    assert np.allclose(o.chain_forces(a, cp, L), o.chain_forces(b, cp, L))


def test_trilinear_interpolation_reproduces_linear_fields():
    fp = o.FluidParams(L=12, a=0.5)
    L = fp.L
    zz, yy, xx = np.meshgrid(np.arange(L), np.arange(L), np.arange(L), indexing="ij")
    G = np.array([[0.3, -1.1, 0.7], [2.0, 0.1, -0.4], [-0.5, 0.9, 1.3]])
    c = np.array([0.1, -0.2, 0.3])
    pos = np.stack([xx, yy, zz]) * fp.a  # node positions (3, z, y, x)
    field = c[:, None, None, None] + np.einsum("ab,bzyx->azyx", G, pos)
    rng = np.random.default_rng(0)
    X = fp.a * (2 + (L - 5) * rng.random((20, 3)))
    got = o.interp_field(field, X, fp)
    assert np.allclose(got, c[None] + X @ G.T, rtol=1e-12, atol=1e-12)
    # a bead exactly on a node sees exactly that node's value
    node = np.array([[3 * fp.a, 7 * fp.a, 5 * fp.a]])
    assert np.array_equal(o.interp_field(field, node, fp)[0], field[:, 5, 7, 3])


def test_spreading_is_minus_the_transpose_of_interpolation():
    """Momentum given to the fluid equals minus the momentum taken from the beads, with the
    same weights: sum_r f(r).u(r) a^3 = -sum_b F_b.u(x_b) for any field u."""
    fp = o.FluidParams(L=7, a=1.3)
    rng = np.random.default_rng(1)
    u = rng.standard_normal((3, 7, 7, 7))
    X = rng.random((9, 3)) * 30 - 10  # unwrapped, outside the primary box too
    Fc = rng.standard_normal((9, 3))
    f = o.spread(Fc, X, fp)
    lhs = (f * u).sum() * fp.a ** 3
    rhs = -(Fc * o.interp_field(u, X, fp)).sum()
    assert lhs == pytest.approx(rhs, rel=1e-12)
    assert np.allclose(f.reshape(3, -1).sum(axis=1) * fp.a ** 3, -Fc.sum(axis=0), atol=1e-12)


def test_bead_velocity_variance_in_frozen_fluid_is_exactly_kT_over_m():
    """Velocity-Verlet Langevin with friction at the half-step velocity: for u = 0 the
    stationary variance of v is kT/m exactly and that of v_half kT/(m (1 - alpha)),
    alpha = h zeta / 2m (fluctuation-dissipation, Sec. II B)."""
    nb = 2000
    fp = o.FluidParams(L=4, kT=1.3, h=0.01, seed=5)
    cp = _chain_params(N=nb, m=1.7, zeta=20.8)
    X = np.zeros((nb, 3))
    V = np.zeros((nb, 3))
    F = np.zeros((nb, 3))
    vs, vhs = [], []
    for k in range(400):
        X, Vh = o.bead_kick_drift(X, V, F, cp, fp.h)
        F = o.coupling_force(Vh, np.zeros_like(Vh), cp, fp, k)
        V = o.bead_kick(Vh, F, cp, fp.h)
        if k >= 60:
            vs.append(V.copy())
            vhs.append(Vh.copy())
    alpha = fp.h * cp.zeta / (2 * cp.m)
    assert np.var(vs) == pytest.approx(fp.kT / cp.m, rel=0.015)
    assert np.var(vhs) == pytest.approx(fp.kT / (cp.m * (1 - alpha)), rel=0.015)


def _c1_like(L=8, N=8, seed=1, kT=1.0):
    fp = o.FluidParams(L=L, rho=1.0, eta=3.0, eta_b=3.0, kT=kT, h=0.01, a=1.0, seed=seed)
    cp = o.ChainParams(N=N, m=1.0, zeta=20.8, k_fene=30.0, R0=1.5, eps=1.0, sigma=1.0)
    X0 = inputs.chain_walk(N, L=L, bond=0.97, seed=seed, self_avoiding=True)
    return fp, cp, o.init_state(fp, cp, X0)


def test_mass_and_total_momentum_are_exactly_conserved():
    """Collision conserves mass and momentum (Sec. II B); the coupling subtracts from the
    fluid exactly the momentum it gives the beads; FENE/WCA forces are pairwise.  So
    a^3 sum j + sum m v + (h/2) sum F_c is invariant to round-off."""
    fp, cp, st = _c1_like()
    M0 = o.total_mass(st, fp)
    P0 = o.total_momentum(st, fp, cp)
    scale = fp.L ** 3 * fp.a ** 3 * fp.rho * fp.a / fp.h
    for _ in range(4):
        st = o.run(st, fp, cp, 25)
        assert o.total_mass(st, fp) == pytest.approx(M0, rel=1e-13)
        assert np.allclose(o.total_momentum(st, fp, cp), P0, rtol=0, atol=1e-13 * scale)
    assert np.abs(st.V).max() > 0.1  # the beads did move


def test_single_dragged_bead_reaches_stokes_velocity():
    """A constant force F on one bead, balanced by a uniform counter-force on the fluid:
    in steady state the friction balances F exactly (v - u_b = F / zeta_bare) and the bead
    moves through the fluid at F / zeta_eff with 1/zeta_eff = 1/zeta_bare + 1/(g eta a),
    g ~ 25 for linear interpolation (Eq. 7), corrected for the periodic images
    (Hasimoto: -2.837/(6 pi eta L))."""
    L = 10
    F = np.array([0.02, 0.0, 0.0])
    fp = o.FluidParams(L=L, rho=1.0, eta=3.0, eta_b=3.0, kT=0.0, h=0.01, noise_fluid=False,
                       body_force=tuple(-F / L ** 3))
    cp = o.ChainParams(N=1, m=1.0, zeta=20.8, noise_beads=False, ext_force=tuple(F))
    st = o.init_state(fp, cp, X0=np.array([[4.3, 5.6, 5.2]]))
    st = o.run(st, fp, cp, 1500)
    Vh = st.V - fp.h * st.F / (2 * cp.m)  # (F = F_cons + F_c of the last step)
    ub = o.interpolate_u(o.stream(st.n), fp, st.X)
    # force balance at the (quasi-)steady state, F_c = -F_ext; the bead drifts slowly
    # across its cell so the balance is approached to ~1e-6, not to round-off
    assert np.allclose(st.Fc[0], -F, rtol=1e-4, atol=1e-9)
    assert np.allclose(-cp.zeta * (Vh[0] - ub[0]), -F, rtol=1e-4, atol=1e-9)
    # mobility relative to the mean fluid velocity
    ubar = o.fluid_momentum(st, fp) / (fp.rho * L ** 3 * fp.a ** 3)
    v_rel = st.V[0, 0] - ubar[0]
    inv_zeta_eff = 1 / cp.zeta + 1 / (25 * fp.eta * fp.a) - 2.837 / (6 * math.pi * fp.eta * L * fp.a)
    assert v_rel == pytest.approx(F[0] * inv_zeta_eff, rel=0.10)


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_cell_index_edge_cases(dtype):
    """Cell of a coordinate = floor(x/a) mod L into [0, L), in the precision of the stored
    coordinate; checked against exact integer arithmetic."""
    L = 16
    one = dtype(1.0)
    cases = [0.0, -0.0, 1.0, 15.0, 16.0, -1.0, -16.0, 31.999, 1e4 * L, -1e4 * L - 0.5]
    xs = [dtype(v) for v in cases]
    for k in (1, 5, 15, 16, 17, -1, -16, 160000):
        xk = dtype(k)
        xs += [np.nextafter(xk, dtype(np.inf)), np.nextafter(xk, dtype(-np.inf))]
    xs = np.array(xs, dtype=dtype)
    got = o.cell_index(xs, one, L)
    for x, g in zip(xs, got):
        fl = math.floor(float(x))  # a = 1: x/a = x exactly
        assert g == fl % L and 0 <= g < L
    # general spacing: the quotient is rounded once in the stored precision
    a = dtype(0.7)
    q = (xs / a).astype(dtype)
    want = np.array([math.floor(float(v)) % L for v in q])
    assert np.array_equal(o.cell_index(xs, a, L), want)


def test_bead_in_fluctuating_fluid_is_at_the_fluid_temperature():
    """Fluctuation-dissipation of the coupled system (Sec. II B): a bead coupled to the
    thermalized fluid reaches <v^2>/3 = kT/m (statistical tolerance)."""
    fp = o.FluidParams(L=6, rho=1.0, eta=3.0, eta_b=3.0, kT=1.0, h=0.01, seed=3)
    cp = o.ChainParams(N=1, m=1.0, zeta=20.8)
    st = o.init_state(fp, cp, X0=np.array([[3.3, 2.2, 4.1]]))
    vs = []
    for k in range(4000):
        st = o.step(st, fp, cp)
        if k > 200:
            vs.append(st.V[0].copy())
    assert np.var(vs) == pytest.approx(fp.kT / cp.m, rel=0.08)


def test_md_substeps_conserve_mass_and_momentum():
    """Two MD steps per LB step (Sec. II E: dt = 0.01, dtau = 0.02): the fluid receives the
    reaction averaged over the LB step, so the invariant a^3 sum j + sum m v + (dt/2) sum F_c
    (dt the MD step) still holds to round-off."""
    fp = o.FluidParams(L=8, rho=0.864, eta=0.864 * 2.8, eta_b=0.864 * 2.8, kT=1.2, h=0.02, a=1.0, seed=4)
    cp = o.ChainParams(N=6, m=1.0, zeta=20.8, k_fene=7.0, R0=2.0, eps=1.0, sigma=1.0, substeps=2)
    st = o.init_state(fp, cp, inputs.chain_walk(6, L=8, bond=0.97, seed=4, self_avoiding=True))
    M0, P0 = o.total_mass(st, fp), o.total_momentum(st, fp, cp)
    st = o.run(st, fp, cp, 60)
    scale = fp.L ** 3 * fp.a ** 3 * fp.rho * fp.a / fp.h
    assert o.total_mass(st, fp) == pytest.approx(M0, rel=1e-13)
    assert np.allclose(o.total_momentum(st, fp, cp), P0, rtol=0, atol=1e-13 * scale)


def test_single_substep_is_the_plain_step():
    fp, cp, st = _c1_like(L=6, N=4, seed=2)
    cp1 = o.ChainParams(**{**cp.__dict__, "substeps": 1})
    a = o.run(st, fp, cp, 5)
    b = o.run(st, fp, cp1, 5)
    assert np.array_equal(a.n, b.n) and np.array_equal(a.X, b.X)


# ---------------------------------------------------------------------------------------
# Chain size observables (Sec. III A: R_g^2 = (1/2N^2) sum_ij r_ij^2, R_e^2 = (r_N - r_1)^2)
# ---------------------------------------------------------------------------------------
def _rotation(seed):
    q, r = np.linalg.qr(np.random.default_rng(seed).standard_normal((3, 3)))
    q = q * np.sign(np.diag(r))[None]
    return q if np.linalg.det(q) > 0 else -q


def _size_pin_failures(rg2, re2):
    """Names of the closed forms that rg2 / re2 miss (empty when all hold):
    - a straight rod of N beads at spacing b: R_g^2 = b^2 (N^2 - 1) / 12, R_e^2 = (N - 1)^2 b^2;
    - N beads equally spaced on a circle of radius R: R_g^2 = R^2, R_e^2 = (2 R sin(pi/N))^2;
    - a single bead: both zero;
    - any chain: R_g^2 equals the mean squared distance from the centre of mass (the identity
      (1/2N^2) sum_ij |r_i - r_j|^2 = (1/N) sum_i |r_i - r_cm|^2), and neither changes under a
      rotation plus a translation."""
    fails = []
    close = lambda a, b: abs(a - b) <= 1e-12 * max(abs(b), 1e-300)
    for N, b in ((2, 0.97), (3, 1.3), (8, 0.97), (33, 0.5)):
        d = np.array([0.36, -0.48, 0.8])
        X = np.array([2.0, -1.0, 0.5])[None] + b * np.arange(N)[:, None] * d[None]
        if not close(rg2(X), b * b * (N * N - 1) / 12.0):
            fails.append(f"rod R_g^2 N={N}")
        if not close(re2(X), ((N - 1) * b) ** 2):
            fails.append(f"rod R_e^2 N={N}")
    for N, R in ((5, 1.7), (12, 0.8)):
        ph = 2.0 * np.pi * np.arange(N) / N
        X = R * np.stack([np.cos(ph), np.sin(ph), np.zeros(N)], axis=1) @ _rotation(N).T + 3.0
        if not close(rg2(X), R * R):
            fails.append(f"ring R_g^2 N={N}")
        if not close(re2(X), (2.0 * R * np.sin(np.pi / N)) ** 2):
            fails.append(f"ring R_e^2 N={N}")
    one = np.array([[0.3, 0.2, -0.7]])
    if rg2(one) != 0.0 or re2(one) != 0.0:
        fails.append("single bead")
    X = inputs.chain_walk(24, L=12, bond=0.97, seed=11, self_avoiding=True)
    cm = X.mean(axis=0)
    if not close(rg2(X), float(((X - cm) ** 2).sum(axis=1).mean())):
        fails.append("centre-of-mass form")
    Y = X @ _rotation(5).T + np.array([40.0, -7.0, 3.0])
    if not (close(rg2(Y), rg2(X)) and close(re2(Y), re2(X))):
        fails.append("rigid motion")
    return fails


def test_chain_size_observables_match_closed_forms():
    assert _size_pin_failures(o.radius_of_gyration2, o.end_to_end2) == []


def _rg2_over_n2(X):  # planted: 1/N^2 instead of 1/(2N^2)
    d = X[:, None, :] - X[None, :, :]
    return float((d * d).sum() / (X.shape[0] ** 2))


def _rg2_over_pairs(X):  # planted: normalised by the number of distinct ordered pairs
    N = X.shape[0]
    d = X[:, None, :] - X[None, :, :]
    return float((d * d).sum() / (2.0 * N * max(N - 1, 1)))


def _rg2_about_first_bead(X):  # planted: distances from bead 1 instead of the centre of mass
    return float(((X - X[0]) ** 2).sum(axis=1).mean())


def _re2_second_bead(X):  # planted: r_N - r_2
    d = X[-1] - X[min(1, X.shape[0] - 1)]
    return float(d @ d)


def _re2_not_squared(X):  # planted: |r_N - r_1| instead of its square
    return float(np.linalg.norm(X[-1] - X[0]))


@pytest.mark.parametrize("rg2,re2", [
    (_rg2_over_n2, o.end_to_end2), (_rg2_over_pairs, o.end_to_end2), (_rg2_about_first_bead, o.end_to_end2),
    (o.radius_of_gyration2, _re2_second_bead), (o.radius_of_gyration2, _re2_not_squared),
], ids=["rg2_1/N^2", "rg2_pairs", "rg2_about_bead1", "re2_second_bead", "re2_not_squared"])
def test_planted_size_observable_mistakes_are_caught(rg2, re2):
    """Each planted normalisation, centre or index mistake fails at least one closed form."""
    assert _size_pin_failures(rg2, re2)


def test_mass_and_momentum_observables_match_closed_forms():
    """total_mass, fluid_momentum and total_momentum against their definitions on states with a
    closed form (Sec. II B: rho = sum_i n_i and j = sum_i n_i c_i per node, c_i = e_i a/h; the
    box holds L^3 nodes of volume a^3 each): a fluid at rest has mass rho0 L^3 a^3 and no
    momentum; the equilibrium populations of a uniform velocity u (Eq. 4) carry rho0 u L^3 a^3;
    beads add m sum v + (dt/2) sum F_c (dt the MD step)."""
    fp = o.FluidParams(L=5, rho=0.864, a=0.7, h=0.02)
    L, a, h = fp.L, fp.a, fp.h
    st = o.init_state(fp, None)
    assert o.total_mass(st, fp) == pytest.approx(fp.rho * L ** 3 * a ** 3, rel=1e-14)
    assert np.allclose(o.fluid_momentum(st, fp), 0.0, atol=1e-14)
    u = np.array([0.013, -0.021, 0.007])  # physical velocity
    U = u * h / a  # lattice velocity
    rho = np.full((L, L, L), fp.rho)
    st.n = o.n_eq(rho, np.broadcast_to(U[:, None, None, None], (3, L, L, L)))
    assert o.total_mass(st, fp) == pytest.approx(fp.rho * L ** 3 * a ** 3, rel=1e-13)
    assert np.allclose(o.fluid_momentum(st, fp), fp.rho * u * L ** 3 * a ** 3, rtol=1e-12, atol=0)
    cp = o.ChainParams(N=3, m=1.7, substeps=2)
    st.V = np.array([[0.1, 0.2, -0.3], [0.0, 0.5, 0.1], [-0.2, 0.1, 0.4]])
    st.Fc = np.array([[1.0, -2.0, 0.5], [0.3, 0.1, -0.2], [-0.4, 0.6, 0.9]])
    want = fp.rho * u * L ** 3 * a ** 3 + cp.m * st.V.sum(axis=0) + 0.5 * (h / 2) * st.Fc.sum(axis=0)
    assert np.allclose(o.total_momentum(st, fp, cp), want, rtol=1e-12, atol=0)
