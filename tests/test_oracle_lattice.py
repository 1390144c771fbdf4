"""Pins of the oracle's lattice, mode basis, equilibrium, streaming and collision against
what the paper prints (Sec. II B) and what the mathematics of the D3Q19 model fixes."""
import itertools
import os
from fractions import Fraction

import numpy as np
import pytest

from oracle import lbchain as o

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


def test_velocity_set_and_weights_match_paper():
    rows = _read_golden("d3q19_paper.txt")
    classes = {int(r[0]): (int(r[1]), Fraction(int(r[2]), int(r[3]))) for r in rows if r[0] != "cs2"}
    cs2 = [Fraction(int(r[1]), int(r[2])) for r in rows if r[0] == "cs2"][0]
    s = (o.E * o.E).sum(axis=1)
    for s2, (count, w) in classes.items():
        sel = s == s2
        assert sel.sum() == count
        assert np.allclose(o.W[sel], float(w), rtol=0, atol=1e-16)
    # the set is exactly the rest vector plus every nearest and next-nearest neighbour
    want = {v for v in itertools.product((-1, 0, 1), repeat=3) if sum(c * c for c in v) <= 2}
    assert {tuple(int(c) for c in e) for e in o.E} == want
    assert len(o.E) == 19
    assert o.CS2 == pytest.approx(float(cs2), abs=0)


def test_lattice_isotropy_identities():
    """sum w = 1, odd moments vanish, sum w e_a e_b = c_s^2 d_ab and the 4th moment is the
    isotropic tensor c_s^4 (d_ab d_cd + d_ac d_bd + d_ad d_bc)."""
    e = o.E.astype(float)
    w = o.W
    assert w.sum() == pytest.approx(1.0, abs=1e-15)
    d = np.eye(3)
    assert np.allclose(np.einsum("i,ia->a", w, e), 0, atol=1e-16)
    assert np.allclose(np.einsum("i,ia,ib->ab", w, e, e), d / 3, atol=1e-16)
    assert np.allclose(np.einsum("i,ia,ib,ic->abc", w, e, e, e), 0, atol=1e-16)
    iso = (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d)
           + np.einsum("ad,bc->abcd", d, d)) / 9.0
    assert np.allclose(np.einsum("i,ia,ib,ic,id->abcd", w, e, e, e, e), iso, atol=1e-16)


def test_mode_basis_orthogonal_with_listed_norms():
    """Exact (rational) orthogonality under the weights, and the norms b_k of the basis."""
    wq = [Fraction(1, 3)] + [Fraction(1, 18)] * 6 + [Fraction(1, 36)] * 12
    Mq = [[Fraction(int(round(v))) for v in row] for row in o.M]
    assert np.all(o.M == np.round(o.M))  # integer entries
    for k in range(19):
        for l in range(19):
            dot = sum(wq[i] * Mq[k][i] * Mq[l][i] for i in range(19))
            if k != l:
                assert dot == 0, (k, l)
    bk = [sum(wq[i] * Mq[k][i] ** 2 for i in range(19)) for k in range(19)]
    listed = ([Fraction(1)] + [Fraction(1, 3)] * 3 + [Fraction(2, 3), Fraction(4, 3), Fraction(4, 9)]
              + [Fraction(1, 9)] * 3 + [Fraction(2, 3)] * 3 + [Fraction(2, 9)] * 3
              + [Fraction(2), Fraction(4, 3), Fraction(4, 9)])
    assert bk == listed
    assert np.allclose(o.MINV @ o.M, np.eye(19), atol=1e-14)
    assert np.allclose(o.M @ o.MINV, np.eye(19), atol=1e-14)


def test_equilibrium_moments_are_the_hydrodynamic_ones():
    """Eq. 4: mass rho, momentum rho U and momentum flux rho (c_s^2 1 + U U) exactly; the
    kinetic (ghost) moments of the equilibrium vanish and the stress modes are the
    second-order ones."""
    rng = np.random.default_rng(3)
    rho = 0.5 + rng.random(50)
    U = 0.1 * (rng.random((3, 50)) - 0.5)
    neq = o.n_eq(rho, U)
    e = o.E.astype(float)
    assert np.allclose(neq.sum(axis=0), rho, rtol=1e-14)
    assert np.allclose(np.einsum("ia,in->an", e, neq), rho * U, rtol=1e-13, atol=1e-16)
    Pi = np.einsum("ia,ib,in->abn", e, e, neq)
    want = rho[None, None] * (np.eye(3)[:, :, None] / 3.0 + U[:, None] * U[None, :])
    assert np.allclose(Pi, want, rtol=1e-13, atol=1e-16)
    m = o.M @ neq
    u2 = (U * U).sum(axis=0)
    assert np.allclose(m[4], rho * u2, atol=1e-15)
    assert np.allclose(m[5], rho * (3 * U[0] ** 2 - u2), atol=1e-15)
    assert np.allclose(m[6], rho * (U[1] ** 2 - U[2] ** 2), atol=1e-15)
    assert np.allclose(m[7], rho * U[0] * U[1], atol=1e-15)
    assert np.allclose(m[8], rho * U[1] * U[2], atol=1e-15)
    assert np.allclose(m[9], rho * U[0] * U[2], atol=1e-15)
    assert np.allclose(m[10:], 0.0, atol=1e-15)


@pytest.mark.parametrize("L", [4, 5])
def test_streaming_moves_each_population_one_link(L):
    """Eq. 3: the population with velocity c_i leaves r and arrives at r + c_i dtau, with
    periodic wrap-around."""
    for i in range(19):
        n = np.zeros((19, L, L, L))
        x0, y0, z0 = L - 1, 0, 2  # at the faces so that the wrap is exercised
        n[i, z0, y0, x0] = 1.0
        s = o.stream(n)
        ex, ey, ez = o.E[i]
        assert s[i, (z0 + ez) % L, (y0 + ey) % L, (x0 + ex) % L] == 1.0
        assert s.sum() == 1.0


def test_collision_conserves_mass_and_momentum_per_node():
    """Sec. II B: the collision conserves rho and u at every node, noise and forcing-free."""
    L = 5
    fp = o.FluidParams(L=L, kT=1.0, seed=11)
    rng = np.random.default_rng(4)
    n = (o.W * fp.rho)[:, None, None, None] * (1 + 0.05 * (rng.random((19, L, L, L)) - 0.5))
    ns = o.collide(n, fp, step=3)
    m0, m1 = o.M @ n.reshape(19, -1), o.M @ ns.reshape(19, -1)
    assert np.allclose(m0[:4], m1[:4], rtol=0, atol=1e-15)
    assert not np.allclose(m0[4:], m1[4:])


def test_equilibrium_is_a_fixed_point_without_noise():
    L = 4
    fp = o.FluidParams(L=L, kT=0.0, noise_fluid=False)
    rng = np.random.default_rng(5)
    rho = 1 + 0.01 * rng.random((L, L, L))
    U = 0.02 * (rng.random((3, L, L, L)) - 0.5)
    neq = o.n_eq(rho, U)
    assert np.allclose(o.collide(neq, fp, step=0), neq, rtol=0, atol=1e-15)


def test_node_update_matches_whole_lattice_step():
    """The single-node update used for sampled checks equals stream + collide."""
    L = 5
    fp = o.FluidParams(L=L, kT=1.0, seed=9, body_force=(1e-3, -2e-3, 0.5e-3))
    rng = np.random.default_rng(6)
    n = (o.W * fp.rho)[:, None, None, None] * (1 + 0.05 * (rng.random((19, L, L, L)) - 0.5))
    full = o.collide(o.stream(n), fp, step=7)
    for node in [(0, 0, 0), (4, 3, 1), (2, 4, 4)]:
        x, y, z = node
        assert np.allclose(o.node_update(n, fp, 7, node), full[:, z, y, x], rtol=0, atol=1e-15)
