"""Tangent-linear (forward-mode) derivative of the oracle's coupled step, FP64.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or execute this
module.  It gives a second, independent derivative of the method to check the library's
reverse-mode (adjoint) gradient against: the adjoint runs the step backwards with
transposed Jacobians, this module pushes a direction forwards through the same step with the
ordinary chain rule, written here from the oracle's own expressions (``oracle.lbchain``).

The differentiated quantity is the chain's squared displacement after T coupled steps,
O = sum_b |x_b(T) - x_b(0)|^2, as a function of the initial bead positions x(0) and of the
bare friction coefficient zeta (Sec. II B).  The random numbers are held fixed: they are
functions of (seed, step, index) only, so the fluid noise enters the tangent only through
the density dependence of its amplitude (phi_k ~ sqrt(rho)) and the bead noise through the
zeta dependence of its amplitude (sqrt(2 kT zeta / dt)).

Every function here is pinned by ``tests/test_oracle_tangent.py`` against central finite
differences of the corresponding oracle function (force field, interpolation, spreading,
collision, whole trajectories with and without noise and with MD substeps).  The
derivative is one-sided across the kinks of the trilinear weights (a bead exactly on a cell
face) and of the WCA cut-off, as the adjoint is: both use the cell and the branch of the
unperturbed trajectory.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

from . import lbchain as o


@dataclasses.dataclass
class Tangent:
    """Directional derivatives of the State fields (same shapes)."""

    n: np.ndarray  # (19, L, L, L) post-collision populations
    X: np.ndarray  # (N, 3)
    V: np.ndarray
    F: np.ndarray


# ---------------------------------------------------------------------------------------
# Chain forces (Sec. II A, Eqs. 1-2): derivative of -grad(V_FENE + V_WCA) along dX.
# FENE pair force  f = -k d / (1 - r^2/R0^2)        (d = x_i - x_{i+1}, minimum image)
# WCA pair force   f = 24 eps / r^2 (2 s^2 - s) d,   s = (sigma^2 / r^2)^3,   r < 2^(1/6) sigma
# ---------------------------------------------------------------------------------------
def force_jvp(X: np.ndarray, dX: np.ndarray, cp: o.ChainParams, box: float) -> np.ndarray:
    N = X.shape[0]
    dF = np.zeros_like(X)
    R02 = cp.R0 * cp.R0
    for i in range(N - 1):
        d = o.min_image(X[i] - X[i + 1], box)
        dd = dX[i] - dX[i + 1]
        r2 = d @ d
        q = 1.0 - r2 / R02
        # d/dt [-k d / q] = -k dd / q - k d (2 d.dd / R0^2) / q^2
        dfi = -cp.k_fene * dd / q - cp.k_fene * d * (2.0 * (d @ dd) / R02) / (q * q)
        dF[i] += dfi
        dF[i + 1] -= dfi
    rc2 = 2.0 ** (1.0 / 3.0) * cp.sigma ** 2
    s2 = cp.sigma * cp.sigma
    for i in range(N):
        for j in range(i + 1, N):
            d = o.min_image(X[i] - X[j], box)
            r2 = d @ d
            if r2 < rc2:
                dd = dX[i] - dX[j]
                # f = g(r2) d with g(r2) = 24 eps (2 sigma^12 / r2^7 - sigma^6 / r2^4)
                g = 24.0 * cp.eps * (2.0 * s2 ** 6 / r2 ** 7 - s2 ** 3 / r2 ** 4)
                gp = 24.0 * cp.eps * (-14.0 * s2 ** 6 / r2 ** 8 + 4.0 * s2 ** 3 / r2 ** 5)
                dfi = gp * 2.0 * (d @ dd) * d + g * dd
                dF[i] += dfi
                dF[j] -= dfi
    return dF


# ---------------------------------------------------------------------------------------
# Coupling geometry (Sec. II B, last paragraph): trilinear weights of the 8 corner nodes and
# their derivatives along dx; the cell (floor of x/a) is that of the unperturbed position.
# ---------------------------------------------------------------------------------------
def corner_weights_jvp(x: np.ndarray, dx: np.ndarray, a: float, L: int):
    """(nodes (8, 3), weights (8,), weight derivatives (8,)) in the corner order of
    ``lbchain.corner_weights``."""
    nodes, wts = o.corner_weights(x, a, L)
    s = x / a
    d = s - np.floor(s)
    dd = dx / a
    dw = np.zeros(8)
    c = 0
    for dz in (0, 1):
        for dy in (0, 1):
            for dx_ in (0, 1):
                off = (dx_, dy, dz)
                fac = [d[al] if off[al] == 1 else 1.0 - d[al] for al in range(3)]
                dfac = [dd[al] if off[al] == 1 else -dd[al] for al in range(3)]
                dw[c] = (dfac[0] * fac[1] * fac[2] + fac[0] * dfac[1] * fac[2]
                         + fac[0] * fac[1] * dfac[2])
                c += 1
    return nodes, wts, dw


def velocity_field_jvp(n_ps: np.ndarray, dn_ps: np.ndarray, fp: o.FluidParams):
    """u = (J / rho) a / h at every node and its derivative
    du = (dJ - (J / rho) drho) / rho * a / h, shapes (3, L, L, L)."""
    Et = o.E.T.astype(float)
    rho = n_ps.sum(axis=0)
    J = np.tensordot(Et, n_ps, axes=(1, 0))
    drho = dn_ps.sum(axis=0)
    dJ = np.tensordot(Et, dn_ps, axes=(1, 0))
    U = J / rho[None]
    u = U * fp.a / fp.h
    du = (dJ - U * drho[None]) / rho[None] * fp.a / fp.h
    return u, du


def interp_field_jvp(field, dfield, X, dX, fp: o.FluidParams):
    """Trilinear interpolation of (field, dfield) at (X, dX): value and derivative (N, 3)."""
    val = np.zeros((X.shape[0], field.shape[0]))
    dval = np.zeros_like(val)
    for b in range(X.shape[0]):
        nodes, wts, dw = corner_weights_jvp(X[b], dX[b], fp.a, fp.L)
        for c in range(8):
            x, y, z = nodes[c]
            val[b] += wts[c] * field[:, z, y, x]
            dval[b] += dw[c] * field[:, z, y, x] + wts[c] * dfield[:, z, y, x]
    return val, dval


def spread_jvp(Fc, dFc, X, dX, fp: o.FluidParams):
    """Force density f(r) = -sum_b w_b(r) Fc_b / a^3 and its derivative."""
    L = fp.L
    f = np.zeros((3, L, L, L))
    df = np.zeros_like(f)
    a3 = fp.a ** 3
    for b in range(X.shape[0]):
        nodes, wts, dw = corner_weights_jvp(X[b], dX[b], fp.a, L)
        for c in range(8):
            x, y, z = nodes[c]
            f[:, z, y, x] -= wts[c] * Fc[b] / a3
            df[:, z, y, x] -= (dw[c] * Fc[b] + wts[c] * dFc[b]) / a3
    return f, df


# ---------------------------------------------------------------------------------------
# Collision (Sec. II B, Eqs. 3-4) with the second-order forcing: derivative of the
# post-collision populations along (dn, df).
# ---------------------------------------------------------------------------------------
def n_eq_jvp(rho, U, drho, dU):
    """Derivative of lbchain.n_eq(rho, U) = rho w (1 + cu/cs2 + cu^2/(2 cs2^2) - uu/(2 cs2))
    along (drho, dU); cu = e.U, uu = U.U."""
    E = o.E.astype(float)
    cs2 = o.CS2
    cu = np.tensordot(E, U, axes=(1, 0))
    dcu = np.tensordot(E, dU, axes=(1, 0))
    uu = (U * U).sum(axis=0)
    duu = 2.0 * (U * dU).sum(axis=0)
    w = o.W.reshape((o.Q,) + (1,) * np.ndim(rho))
    poly = 1.0 + cu / cs2 + cu * cu / (2.0 * cs2 * cs2) - uu[None] / (2.0 * cs2)
    dpoly = dcu / cs2 + cu * dcu / (cs2 * cs2) - duu[None] / (2.0 * cs2)
    return w * (drho[None] * poly + rho[None] * dpoly)


def force_moment_increment_jvp(rho, J, dJf, drho, dJ, ddJf, gam):
    """Derivative of lbchain.force_moment_increment(rho, J, dJf, gam) along
    (drho, dJ, ddJf): the increment is dm_1..3 = dJf and the stress increment
    P_ab = (1+g_s)/2 (U'_a dJf_b + U'_b dJf_a) + c delta_ab U'.dJf,
    c = (1+g_b)/3 - (1+g_s)/3, U' = (J + dJf/2) / rho, mapped on the modes 4..9."""
    gs, gb = gam[5], gam[4]
    Up = (J + 0.5 * dJf) / rho[None]
    dUp = (dJ + 0.5 * ddJf - Up * drho[None]) / rho[None]
    dud = (dUp * dJf).sum(axis=0) + (Up * ddJf).sum(axis=0)
    c = (1.0 + gb) / 3.0 - (1.0 + gs) / 3.0
    dP = np.empty((3, 3) + rho.shape)
    for al in range(3):
        for be in range(3):
            dP[al, be] = 0.5 * (1.0 + gs) * (dUp[al] * dJf[be] + Up[al] * ddJf[be]
                                             + dUp[be] * dJf[al] + Up[be] * ddJf[al])
            if al == be:
                dP[al, be] += c * dud
    ddm = np.zeros((o.Q,) + rho.shape)
    ddm[1:4] = ddJf
    ddm[4] = dP[0, 0] + dP[1, 1] + dP[2, 2]
    ddm[5] = 2.0 * dP[0, 0] - dP[1, 1] - dP[2, 2]
    ddm[6] = dP[1, 1] - dP[2, 2]
    ddm[7] = dP[0, 1]
    ddm[8] = dP[1, 2]
    ddm[9] = dP[0, 2]
    return ddm


def collide_jvp(n: np.ndarray, dn: np.ndarray, fp: o.FluidParams, step: int, force_density=None,
                dforce_density=None, replica: int = 0) -> np.ndarray:
    """Derivative of lbchain.collide(n, fp, step, force_density) along (dn, dforce_density):
    relaxation m*_k = m_eq,k + gamma_k (m_k - m_eq,k) of the non-conserved modes, the noise
    phi_k(rho) g_k with phi_k ~ sqrt(rho) and fixed g_k, and the forcing increment."""
    L = fp.L
    m = o.M @ n.reshape(o.Q, -1)
    dm = o.M @ dn.reshape(o.Q, -1)
    rho, J = m[0], m[1:4]
    drho, dJ = dm[0], dm[1:4]
    U = J / rho[None]
    dU = (dJ - U * drho[None]) / rho[None]
    dmeq = o.M @ n_eq_jvp(rho, U, drho, dU)
    gam = o.relaxation(fp)
    dms = dm.copy()
    for k in range(4, o.Q):
        dms[k] = dmeq[k] + gam[k] * (dm[k] - dmeq[k])
    if fp.noise_fluid and fp.kT > 0.0:
        mu = o.mu_thermal(fp)
        g = o.fluid_gaussians(fp.seed, o.TAG_FLUID, replica, step, np.arange(L ** 3))
        pos = rho > 0.0
        kmax = 10 if fp.stress_only else o.Q
        for k in range(4, kmax):
            # phi = sqrt(mu rho b_k (1 - gamma_k^2)): dphi = phi drho / (2 rho)
            phi = np.sqrt(mu * np.where(pos, rho, 0.0) * o.B[k] * (1.0 - gam[k] ** 2))
            dphi = np.where(pos, phi * drho / (2.0 * np.where(pos, rho, 1.0)), 0.0)
            dms[k] += dphi * g[k - 4]
    f = np.zeros((3, L ** 3))
    df = np.zeros((3, L ** 3))
    if force_density is not None:
        f += force_density.reshape(3, -1)
    if dforce_density is not None:
        df += dforce_density.reshape(3, -1)
    f += np.asarray(fp.body_force, dtype=float)[:, None]
    # the increment is a smooth function of the node's momentum input that vanishes with it,
    # so its derivative is taken wherever the input or its derivative is non-zero
    sel = np.any(f != 0.0, axis=0) | np.any(df != 0.0, axis=0)
    if np.any(sel):
        s = fp.h * fp.h / fp.a
        dms[:, sel] += force_moment_increment_jvp(rho[sel], J[:, sel], f[:, sel] * s, drho[sel],
                                                  dJ[:, sel], df[:, sel] * s, gam)
    return (o.MINV @ dms).reshape(o.Q, L, L, L)


# ---------------------------------------------------------------------------------------
# Coupled step (the same order as lbchain.step) with its tangent.
# ---------------------------------------------------------------------------------------
def init_tangent(st: o.State, fp: o.FluidParams, cp: o.ChainParams, dX0: np.ndarray) -> Tangent:
    """Tangent of the initial state for a displacement dX0 of the initial positions: the fluid
    and the velocities do not move; the initial force F0 = F_cons(x0) changes by its
    Jacobian times dX0."""
    dX0 = np.asarray(dX0, dtype=np.float64).reshape(st.X.shape)
    return Tangent(np.zeros_like(st.n), dX0.copy(), np.zeros_like(st.V),
                   force_jvp(st.X, dX0, cp, fp.L * fp.a))


def step_jvp(st: o.State, tg: Tangent, fp: o.FluidParams, cp: o.ChainParams, dzeta: float = 0.0,
             replica: int = 0):
    """One coupled step of the state and of its tangent; dzeta is the direction's component
    along zeta.  Returns (State, Tangent); the State equals lbchain.step's."""
    k = st.step
    n_ps = o.stream(st.n)
    dn_ps = o.stream(tg.n)
    X, V, F = st.X, st.V, st.F
    dX, dV, dF = tg.X, tg.V, tg.F
    box = fp.L * fp.a
    nsub = max(1, int(cp.substeps))
    dt = fp.h / nsub
    u, du = velocity_field_jvp(n_ps, dn_ps, fp)
    f = np.zeros((3, fp.L, fp.L, fp.L))
    df = np.zeros_like(f)
    Fc = st.Fc
    for sub in range(nsub):
        X, Vh = o.bead_kick_drift(X, V, F, cp, dt)
        dVh = dV + dt * dF / (2.0 * cp.m)
        dX = dX + dt * dVh
        Fcons = o.chain_forces(X, cp, box) + np.asarray(cp.ext_force, dtype=float)[None]
        dFcons = force_jvp(X, dX, cp, box)
        ub, dub = interp_field_jvp(u, du, X, dX, fp)
        Fc = o.coupling_force(Vh, ub, cp, fp, k * nsub + sub, replica, dt=dt)
        # Fc = -zeta (v_half - u_b) + sqrt(2 kT zeta / dt) g: d/dzeta of the noise term is
        # the noise term / (2 zeta)
        dzterm = -(Vh - ub)
        if cp.noise_beads and fp.kT > 0.0:
            amp = math.sqrt(2.0 * fp.kT * cp.zeta / dt)
            dzterm = dzterm + amp * o.bead_gaussians(fp.seed, replica, k * nsub + sub,
                                                     Vh.shape[0]) / (2.0 * cp.zeta)
        dFc = -cp.zeta * (dVh - dub) + dzeta * dzterm
        fs, dfs = spread_jvp(Fc, dFc, X, dX, fp)
        f += (dt / fp.h) * fs
        df += (dt / fp.h) * dfs
        F = Fcons + Fc
        dF = dFcons + dFc
        V = o.bead_kick(Vh, F, cp, dt)
        dV = dVh + dt * dF / (2.0 * cp.m)
    n_new = o.collide(n_ps, fp, k, force_density=f, replica=replica)
    dn_new = collide_jvp(n_ps, dn_ps, fp, k, force_density=f, dforce_density=df, replica=replica)
    return o.State(n_new, X, V, F, Fc, k + 1), Tangent(dn_new, dX, dV, dF)


def displacement_jvp(fp: o.FluidParams, cp: o.ChainParams, X0: np.ndarray, T: int,
                     dX0: np.ndarray, dzeta: float = 0.0, replica: int = 0):
    """O = sum_b |x_b(T) - x_b(0)|^2 from the fluid at rest and v(0) = 0, and its directional
    derivative dO = grad_x0 O . dX0 + dO/dzeta * dzeta."""
    X0 = np.asarray(X0, dtype=np.float64).reshape(cp.N, 3)
    st = o.init_state(fp, cp, X0)
    tg = init_tangent(st, fp, cp, dX0)
    for _ in range(T):
        st, tg = step_jvp(st, tg, fp, cp, dzeta=dzeta, replica=replica)
    D = st.X - X0
    O = float((D * D).sum())
    dO = float(2.0 * (D * (tg.X - np.asarray(dX0, dtype=np.float64).reshape(cp.N, 3))).sum())
    return O, dO
