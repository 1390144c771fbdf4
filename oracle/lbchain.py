"""Plain FP64 CPU oracle for the fluctuating D3Q19 lattice Boltzmann fluid coupled to a
FENE+WCA bead-spring chain (Pham, Schiller, Prakash, Duenweg, arXiv:0903.5067, Sec. II).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or execute this
module; it exists so that the tests, the smoke check and the CPU-baseline leg of the
benchmark can check the CUDA library against an obviously correct restatement of the
method.  It shares no code with the CUDA path: its random numbers, lattice tables and
arithmetic are written here from their definitions.

Everything is float64 numpy; every array over the lattice has the node axes (z, y, x) so
that the flat node index is ``x + L*(y + L*z)``.  Populations are partial mass densities
(Sec. II B: each n_i is a partial mass density of the fluid at its node).  Where the paper is silent
(mode basis, relaxation rates, noise amplitudes, forcing, integrator, random numbers) the
module follows the readings listed in the design notes; each function says which.

Pins: every function here is pinned by a ``-m "not gpu"`` test against what the paper or
the mathematics fixes (lattice isotropy, exact conservation, shear/sound-wave decay,
equipartition, Stokes drag, force = -grad V, Philox against an independent library
implementation, ...).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

# ---------------------------------------------------------------------------------------
# D3Q19 velocity set and weights (Sec. II B: rest particle, 6 nearest and 12 next-nearest
# neighbours of the simple cubic lattice; weights 1/3, 1/18, 1/36; c_s^2 = (1/3)(a/dtau)^2).
# The ORDER of the 19 velocities is a convention of this library (ABI order).
# ---------------------------------------------------------------------------------------
E = np.array(
    [
        (0, 0, 0),
        (1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1),
        (1, 1, 0), (-1, -1, 0), (1, -1, 0), (-1, 1, 0),
        (1, 0, 1), (-1, 0, -1), (1, 0, -1), (-1, 0, 1),
        (0, 1, 1), (0, -1, -1), (0, 1, -1), (0, -1, 1),
    ],
    dtype=np.int64,
)
Q = 19
W = np.array([1.0 / 3.0] + [1.0 / 18.0] * 6 + [1.0 / 36.0] * 12)
CS2 = 1.0 / 3.0  # speed of sound squared in lattice units (a = dtau = 1)


def mode_matrix() -> np.ndarray:
    """Rows e_k(c_i) of the D3Q19 moment basis (reading: the orthogonal basis of Duenweg,
    Schiller & Ladd 2007, which the paper cites for the fully thermalized model, Sec. II B).

    k=0 density; 1..3 momentum; 4 bulk stress (s-1); 5,6 shear-normal; 7..9 shear-off
    diagonal; 10..18 kinetic ("ghost") modes.  s = |e|^2.
    """
    ex, ey, ez = (E[:, 0].astype(float), E[:, 1].astype(float), E[:, 2].astype(float))
    s = ex * ex + ey * ey + ez * ez
    rows = [
        np.ones(Q),
        ex, ey, ez,
        s - 1.0,
        3.0 * ex * ex - s,
        ey * ey - ez * ez,
        ex * ey, ey * ez, ex * ez,
        (3.0 * s - 5.0) * ex, (3.0 * s - 5.0) * ey, (3.0 * s - 5.0) * ez,
        (ey * ey - ez * ez) * ex, (ez * ez - ex * ex) * ey, (ex * ex - ey * ey) * ez,
        3.0 * s * s - 6.0 * s + 1.0,
        (2.0 * s - 3.0) * (3.0 * ex * ex - s),
        (2.0 * s - 3.0) * (ey * ey - ez * ez),
    ]
    return np.array(rows)


M = mode_matrix()
B = (M * M * W[None, :]).sum(axis=1)  # norms b_k = sum_i w_i e_k(c_i)^2
MINV = (W[:, None] * M.T) / B[None, :]  # n_i = w_i sum_k e_k(c_i) m_k / b_k


# ---------------------------------------------------------------------------------------
# Parameters
# ---------------------------------------------------------------------------------------
@dataclasses.dataclass
class FluidParams:
    """Fluid parameters of Sec. II B / Sec. II E in physical (MD) units."""

    L: int
    rho: float = 1.0  # rho_0, background mass density
    eta: float = 3.0  # shear viscosity
    eta_b: float = 3.0  # bulk viscosity
    kT: float = 1.0
    h: float = 0.01  # LB time step (= MD time step in this library)
    a: float = 1.0  # lattice spacing
    seed: int = 1
    noise_fluid: bool = True
    stress_only: bool = False  # original Ahlrichs-Duenweg thermalization (Table 1, note b)
    body_force: tuple = (0.0, 0.0, 0.0)  # uniform force density on every node


@dataclasses.dataclass
class ChainParams:
    """Bead-spring chain of Sec. II A with the dissipative coupling of Sec. II B."""

    N: int
    m: float = 1.0
    zeta: float = 20.8  # zeta_bare
    k_fene: float = 30.0
    R0: float = 1.5
    eps: float = 1.0
    sigma: float = 1.0
    noise_beads: bool = True
    ext_force: tuple = (0.0, 0.0, 0.0)  # constant external force on every bead
    substeps: int = 1  # MD steps per LB step (Sec. II E: dt_MD = 0.01, dtau_LB = 0.02 -> 2)


def relaxation(fp: FluidParams) -> np.ndarray:
    """Eigenvalues gamma_k of the linearised collision, per mode (reading, DSL07):
    gamma_b for the bulk mode 4, gamma_s for the shear modes 5..9, 0 for the kinetic modes.
    The conserved modes 0..3 are not relaxed (their entries are unused)."""
    nu = fp.eta * fp.h / (fp.rho * fp.a * fp.a)
    nub = fp.eta_b * fp.h / (fp.rho * fp.a * fp.a)
    gs = 1.0 - 2.0 / (6.0 * nu + 1.0)
    gb = 1.0 - 2.0 / (9.0 * nub + 1.0)
    g = np.zeros(Q)
    g[4] = gb
    g[5:10] = gs
    g[10:] = 0.0
    return g


def mu_thermal(fp: FluidParams) -> float:
    """Mass of the 'thermal particle' per a^3: mu = kT / (c_s^2 a^3) with c_s^2 = a^2/(3 h^2)."""
    return 3.0 * fp.kT * fp.h * fp.h / fp.a ** 5


# ---------------------------------------------------------------------------------------
# Equilibrium (Sec. II B, Eq. 4): second-order expansion of the Maxwell-Boltzmann
# distribution, here in lattice units (U = u h / a, c_s^2 = 1/3).
# ---------------------------------------------------------------------------------------
def n_eq(rho: np.ndarray, U: np.ndarray) -> np.ndarray:
    """rho: (...), U: (3, ...) lattice velocity -> (19, ...) equilibrium populations."""
    cu = np.tensordot(E.astype(float), U, axes=(1, 0))  # (19, ...)
    uu = (U * U).sum(axis=0)
    wshape = (Q,) + (1,) * np.ndim(rho)
    return rho[None] * W.reshape(wshape) * (
        1.0 + cu / CS2 + cu * cu / (2.0 * CS2 * CS2) - uu[None] / (2.0 * CS2)
    )


# ---------------------------------------------------------------------------------------
# Counter-based random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random
# numbers: as easy as 1, 2, 3", SC'11).  Written from that definition.
# ---------------------------------------------------------------------------------------
_MASK = np.uint64(0xFFFFFFFF)
PHILOX_M0 = 0xD2511F53
PHILOX_M1 = 0xCD9E8D57
PHILOX_W0 = 0x9E3779B9
PHILOX_W1 = 0xBB67AE85

TAG_FLUID = 0
TAG_BEAD = 1


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Ten Philox rounds on the 128-bit counter (c0..c3) under the 64-bit key (k0, k1).
    Each round multiplies c0 and c2 by the two round constants, swaps the halves of the
    products into the other lanes and xors in the key; the key is bumped by the Weyl
    constants between rounds.  Inputs: uint32-valued arrays (broadcastable)."""
    c = [np.asarray(v, dtype=np.uint64) & _MASK for v in (c0, c1, c2, c3)]
    k0 = np.uint64(k0) & _MASK
    k1 = np.uint64(k1) & _MASK
    for r in range(10):
        if r > 0:
            k0 = (k0 + np.uint64(PHILOX_W0)) & _MASK
            k1 = (k1 + np.uint64(PHILOX_W1)) & _MASK
        p0 = np.uint64(PHILOX_M0) * c[0]
        p1 = np.uint64(PHILOX_M1) * c[2]
        hi0, lo0 = p0 >> np.uint64(32), p0 & _MASK
        hi1, lo1 = p1 >> np.uint64(32), p1 & _MASK
        c = [hi1 ^ c[1] ^ k0, lo1, hi0 ^ c[3] ^ k1, lo0]
    return [v.astype(np.uint32) for v in c]


def philox_key(seed: int, tag: int, replica: int = 0):
    return (int(seed) & 0xFFFFFFFF, (int(tag) | (int(replica) << 8)) & 0xFFFFFFFF)


def uniform01(x: np.ndarray) -> np.ndarray:
    """uint32 -> u in (0, 1): u = ((x >> 9) + 1/2) * 2^-23 (23 random bits; exact in FP32
    and FP64)."""
    return ((np.asarray(x, dtype=np.uint32) >> np.uint32(9)).astype(np.float64) + 0.5) * 2.0 ** -23


def box_muller(u0: np.ndarray, u1: np.ndarray):
    """Box & Muller (1958): two independent standard normals from two uniforms, the angle
    taken in (-pi, pi): r = sqrt(-2 ln u0), theta = 2 pi (u1 - 1/2)."""
    r = np.sqrt(-2.0 * np.log(u0))
    theta = 2.0 * np.pi * (u1 - 0.5)
    return r * np.cos(theta), r * np.sin(theta)


FLUID_CALLS = 2


def fluid_uniforms(seed, tag, replica, step, index, ncalls=FLUID_CALLS):
    """Uniform pairs of the fluid noise, shape (2, 4 ncalls, ...): call c (counter
    (step, index, c, 0)) gives four 32-bit words; word j is Box-Muller pair p = 4c + j.  Its 21
    high bits k_r = w >> 11 give the radius uniform u0 = (k_r + 1/2) 2^-21 (row 0), its 11 low
    bits k_a = w mod 2^11 the angle uniform u1 = (k_a + 1/2) 2^-11 (row 1): 2048 equally
    spaced angles, offset by half a step (reading of the noise layout; the paper asks only for
    Gaussian fluctuations of unit variance on the non-conserved modes, Sec. II B)."""
    k0, k1 = philox_key(seed, tag, replica)
    index = np.asarray(index, dtype=np.uint64)
    u0, u1 = [], []
    for call in range(ncalls):
        w = philox4x32_10(np.uint64(step) & _MASK, index, np.uint64(call), np.uint64(0), k0, k1)
        for j in range(4):
            wj = w[j].astype(np.uint64)
            u0.append(((wj >> np.uint64(11)).astype(np.float64) + 0.5) * 2.0 ** -21)
            u1.append(((wj & np.uint64(0x7FF)).astype(np.float64) + 0.5) * 2.0 ** -11)
    return np.array([u0, u1])


def fluid_gaussians(seed, tag, replica, step, index):
    """16 standard normals per index: pair p = 0..7 is Box-Muller on (u0[p], u1[p]) of
    fluid_uniforms, giving g[2p], g[2p+1].  Mode k = 4..18 takes g[k - 4] (g[15] is unused);
    the stress modes 4..9 thus depend on words 0..2 of the first call only."""
    u = fluid_uniforms(seed, tag, replica, step, index)
    out = []
    for p in range(8):
        g0, g1 = box_muller(u[0, p], u[1, p])
        out += [g0, g1]
    return np.array(out)


def bead_gaussians(seed, replica, step, N):
    """3 standard normals per bead b from one Philox call with counter (step, b, 0, 0)."""
    k0, k1 = philox_key(seed, TAG_BEAD, replica)
    x = philox4x32_10(np.uint64(step), np.arange(N, dtype=np.uint64), 0, 0, k0, k1)
    u = [uniform01(v) for v in x]
    g0, g1 = box_muller(u[0], u[1])
    g2, _ = box_muller(u[2], u[3])
    return np.stack([g0, g1, g2], axis=1)  # (N, 3)


# ---------------------------------------------------------------------------------------
# Streaming (Sec. II B, Eq. 3: n_i(r + c_i dtau, t + dtau) = post-collision n_i(r, t)),
# periodic L^3 box.  Populations are kept in "pull" storage: after a step the array holds
# the post-collision values at the node that produced them; streaming gathers
# n_i(r) = n*_i(r - e_i).
# ---------------------------------------------------------------------------------------
def stream(npost: np.ndarray) -> np.ndarray:
    out = np.empty_like(npost)
    for i in range(Q):
        ex, ey, ez = E[i]
        # axes of npost[i] are (z, y, x); np.roll(a, s)[j] = a[j - s]
        out[i] = np.roll(npost[i], shift=(ez, ey, ex), axis=(0, 1, 2))
    return out


# ---------------------------------------------------------------------------------------
# Collision (Sec. II B, Eq. 3): linear relaxation of the non-equilibrium moments plus the
# fluctuating term n'_i on every non-conserved mode (full thermalization), optional
# momentum input from a force density (second-order forcing, reading).
# ---------------------------------------------------------------------------------------
def force_moment_increment(rho, J, dJ, gam):
    """Moment increments dm (19, ...) for a force that adds lattice momentum dJ at a node of
    density rho and (pre-collision) lattice momentum J: dm_1..3 = dJ, and the stress
    increment dPi = (1+g_s)/2 (U' dJ + dJ U' - 2/3 1 U'.dJ) + (1+g_b)/3 1 U'.dJ with
    U' = (J + dJ/2) / rho, mapped on the stress modes 4..9."""
    gs, gb = gam[5], gam[4]
    Up = (J + 0.5 * dJ) / rho[None]
    ud = (Up * dJ).sum(axis=0)
    P = np.empty((3, 3) + rho.shape)
    for al in range(3):
        for be in range(3):
            P[al, be] = 0.5 * (1.0 + gs) * (Up[al] * dJ[be] + Up[be] * dJ[al])
            if al == be:
                P[al, be] += (-(2.0 / 3.0) * 0.5 * (1.0 + gs) + (1.0 + gb) / 3.0) * ud
    dm = np.zeros((Q,) + rho.shape)
    dm[1:4] = dJ
    dm[4] = P[0, 0] + P[1, 1] + P[2, 2]
    dm[5] = 2.0 * P[0, 0] - P[1, 1] - P[2, 2]
    dm[6] = P[1, 1] - P[2, 2]
    dm[7] = P[0, 1]
    dm[8] = P[1, 2]
    dm[9] = P[0, 2]
    return dm


def collide(n: np.ndarray, fp: FluidParams, step: int, force_density=None, replica: int = 0,
            stats: dict | None = None) -> np.ndarray:
    """Post-stream populations n (19, L, L, L) -> post-collision populations.

    force_density: (3, L, L, L) force per volume acting during this step, or None.
    """
    L = fp.L
    nf = n.reshape(Q, -1)
    m = M @ nf
    rho = m[0]
    J = m[1:4]
    U = J / rho[None]
    meq = M @ n_eq(rho, U)
    gam = relaxation(fp)
    mstar = m.copy()
    for k in range(4, Q):
        mstar[k] = meq[k] + gam[k] * (m[k] - meq[k])
    if fp.noise_fluid and fp.kT > 0.0:
        mu = mu_thermal(fp)
        g = fluid_gaussians(fp.seed, TAG_FLUID, replica, step, np.arange(L ** 3))
        rho_pos = np.where(rho > 0.0, rho, 0.0)
        if stats is not None:
            stats["nonpositive_rho"] = stats.get("nonpositive_rho", 0) + int((rho <= 0.0).sum())
        kmax = 10 if fp.stress_only else Q
        for k in range(4, kmax):
            phi = np.sqrt(mu * rho_pos * B[k] * (1.0 - gam[k] ** 2))
            mstar[k] += phi * g[k - 4]
    f = np.zeros((3, L ** 3))
    if force_density is not None:
        f += force_density.reshape(3, -1)
    bf = np.asarray(fp.body_force, dtype=float)
    if np.any(bf != 0.0):
        f += bf[:, None]
    forced = np.any(f != 0.0, axis=0)
    if np.any(forced):
        dJ = f[:, forced] * fp.h * fp.h / fp.a  # lattice momentum added this step
        mstar[:, forced] += force_moment_increment(rho[forced], J[:, forced], dJ, gam)
    return (MINV @ mstar).reshape(Q, L, L, L)


# ---------------------------------------------------------------------------------------
# Bead-spring chain (Sec. II A, Eqs. 1-2): FENE bonds between neighbours along the chain,
# WCA (LJ cut at 2^(1/6) sigma, shifted by +1/4) between ALL monomers; minimum image.
# ---------------------------------------------------------------------------------------
class FeneBroken(RuntimeError):
    pass


def min_image(d: np.ndarray, box: float) -> np.ndarray:
    return d - box * np.round(d / box)


def v_fene(r, k, R0):
    return -0.5 * k * R0 * R0 * np.log(1.0 - (r / R0) ** 2)


def v_wca(r, eps, sigma):
    rc = 2.0 ** (1.0 / 6.0) * sigma
    sr6 = (sigma / r) ** 6
    return np.where(r <= rc, 4.0 * eps * (sr6 * sr6 - sr6 + 0.25), 0.0)


def chain_energy(X: np.ndarray, cp: ChainParams, box: float) -> float:
    N = X.shape[0]
    e = 0.0
    for i in range(N - 1):
        r = np.linalg.norm(min_image(X[i] - X[i + 1], box))
        if r >= cp.R0:
            raise FeneBroken(f"bond {i} stretched to {r} >= R0")
        e += v_fene(r, cp.k_fene, cp.R0)
    for i in range(N):
        for j in range(i + 1, N):
            r = np.linalg.norm(min_image(X[i] - X[j], box))
            e += float(v_wca(r, cp.eps, cp.sigma))
    return e


def chain_forces(X: np.ndarray, cp: ChainParams, box: float) -> np.ndarray:
    """Conservative forces -grad(V_FENE + V_WCA) on every bead, (N, 3)."""
    N = X.shape[0]
    F = np.zeros_like(X)
    rc2 = 2.0 ** (1.0 / 3.0) * cp.sigma ** 2
    for i in range(N - 1):
        d = min_image(X[i] - X[i + 1], box)
        r2 = d @ d
        if r2 >= cp.R0 * cp.R0:
            raise FeneBroken(f"bond {i} stretched to {math.sqrt(r2)} >= R0")
        fi = -cp.k_fene * d / (1.0 - r2 / (cp.R0 * cp.R0))
        F[i] += fi
        F[i + 1] -= fi
    for i in range(N):
        for j in range(i + 1, N):
            d = min_image(X[i] - X[j], box)
            r2 = d @ d
            if r2 < rc2:
                sr6 = (cp.sigma * cp.sigma / r2) ** 3
                fi = 24.0 * cp.eps / r2 * (2.0 * sr6 * sr6 - sr6) * d
                F[i] += fi
                F[j] -= fi
    return F


# ---------------------------------------------------------------------------------------
# Point-particle coupling (Sec. II B, last paragraph; Sec. II D, Eq. 7 context): linear
# interpolation of the flow velocity from the 8 surrounding nodes, Stokes friction
# -zeta_bare (v - u) plus a balancing Langevin force, and the reaction spread back onto the
# same 8 nodes with the same weights so that momentum is conserved.  Nodes sit at a*integer.
# ---------------------------------------------------------------------------------------
def cell_index(x, a, L):
    """Cell of a coordinate: floor(x/a) taken modulo L into [0, L).  Works on float32 or
    float64 input in its own precision (x/a rounded in that precision)."""
    x = np.asarray(x)
    s = x / np.asarray(a, dtype=x.dtype)
    f = np.floor(s).astype(np.int64)
    return f - L * np.floor_divide(f, L)


def corner_weights(x: np.ndarray, a: float, L: int):
    """For one position x (3,), return the 8 corner node triples (8, 3) and the trilinear
    weights (8,) in the order (dz, dy, dx) over {0,1}^3 with dx fastest."""
    s = x / a
    base = np.floor(s)
    d = s - base
    base = base.astype(np.int64)
    nodes, wts = [], []
    for dz in (0, 1):
        for dy in (0, 1):
            for dx in (0, 1):
                off = np.array([dx, dy, dz])
                node = np.mod(base + off, L)
                w = 1.0
                for al in range(3):
                    w *= d[al] if off[al] == 1 else 1.0 - d[al]
                nodes.append(node)
                wts.append(w)
    return np.array(nodes), np.array(wts)


def velocity_field(n_ps: np.ndarray, fp: FluidParams) -> np.ndarray:
    """Flow velocity u = sum_i n_i c_i / sum_i n_i (Sec. II B) at every node from the
    post-stream populations, physical units, shape (3, L, L, L)."""
    rho = n_ps.sum(axis=0)
    J = np.tensordot(E.T.astype(float), n_ps, axes=(1, 0))
    return J / rho[None] * fp.a / fp.h


def interp_field(field: np.ndarray, X: np.ndarray, fp: FluidParams) -> np.ndarray:
    """Trilinear interpolation of a nodal vector field (3, L, L, L) at positions X (N, 3)."""
    out = np.zeros((X.shape[0], field.shape[0]))
    for b in range(X.shape[0]):
        nodes, wts = corner_weights(X[b], fp.a, fp.L)
        for c in range(8):
            x, y, z = nodes[c]
            out[b] += wts[c] * field[:, z, y, x]
    return out


def interpolate_u(n_ps: np.ndarray, fp: FluidParams, X: np.ndarray) -> np.ndarray:
    return interp_field(velocity_field(n_ps, fp), X, fp)


def spread(Fc: np.ndarray, X: np.ndarray, fp: FluidParams) -> np.ndarray:
    """Force density on the fluid: f(r) = -sum_b w_b(r) Fc_b / a^3, shape (3, L, L, L)."""
    L = fp.L
    f = np.zeros((3, L, L, L))
    for b in range(X.shape[0]):
        nodes, wts = corner_weights(X[b], fp.a, L)
        for c in range(8):
            x, y, z = nodes[c]
            f[:, z, y, x] -= wts[c] * Fc[b] / fp.a ** 3
    return f


def bead_kick_drift(X, V, F, cp: ChainParams, h: float):
    """First half of velocity Verlet: v_half = v + h F / 2m, x' = x + h v_half."""
    Vh = V + h * F / (2.0 * cp.m)
    return X + h * Vh, Vh


def coupling_force(Vh, ub, cp: ChainParams, fp: FluidParams, step_k: int, replica: int = 0, dt=None):
    """Friction against the interpolated flow plus the Langevin force that balances it:
    F_c = -zeta_bare (v_half - u_b) + sqrt(2 kT zeta_bare / dt) g_b (dt: the MD step)."""
    dt = fp.h if dt is None else dt
    Fc = -cp.zeta * (Vh - ub)
    if cp.noise_beads and fp.kT > 0.0:
        amp = math.sqrt(2.0 * fp.kT * cp.zeta / dt)
        Fc = Fc + amp * bead_gaussians(fp.seed, replica, step_k, Vh.shape[0])
    return Fc


def bead_kick(Vh, F, cp: ChainParams, h: float):
    """Second half of velocity Verlet: v' = v_half + h F / 2m."""
    return Vh + h * F / (2.0 * cp.m)


# ---------------------------------------------------------------------------------------
# Coupled step (reading: velocity Verlet with the friction evaluated at the half-step
# velocity).  One LB step of length h carries n = substeps MD steps of length dt = h / n
# (the paper uses dt = 0.01, dtau = 0.02, Sec. II E).  State k -> k+1:
#   n_ps = stream(n*)                                   (the fluid the beads see, frozen)
#   for s = 0 .. n-1 (noise counter q = k n + s):
#     1. v_half = v + dt F/(2m);  x' = x + dt v_half
#     2. F_cons(x')  (FENE + WCA + optional constant external force)
#     3. u_b = trilinear interpolation of the post-stream flow velocity at x'
#     4. F_c = -zeta (v_half - u_b) + sqrt(2 kT zeta / dt) g_b;
#        f(r) += -(dt/h) sum_b w_b(r) F_c / a^3     (reaction averaged over the LB step)
#     5. F = F_cons + F_c;  v' = v_half + dt F / (2m)
#   collide every node with the force density f
# For n = 1 this is the plain step with LB step = MD step.
# ---------------------------------------------------------------------------------------
@dataclasses.dataclass
class State:
    n: np.ndarray  # (19, L, L, L) post-collision populations, pull storage
    X: np.ndarray  # (N, 3) unwrapped bead positions
    V: np.ndarray  # (N, 3)
    F: np.ndarray  # (N, 3) total force of the last step
    Fc: np.ndarray  # (N, 3) coupling force of the last step
    step: int = 0


def fluid_at_rest(fp: FluidParams) -> np.ndarray:
    L = fp.L
    return np.broadcast_to((W * fp.rho)[:, None, None, None], (Q, L, L, L)).copy()


def init_state(fp: FluidParams, cp: ChainParams | None, X0=None, V0=None, n0=None) -> State:
    n = fluid_at_rest(fp) if n0 is None else np.array(n0, dtype=np.float64)
    if cp is None or cp.N == 0:
        z = np.zeros((0, 3))
        return State(n, z, z.copy(), z.copy(), z.copy())
    X = np.array(X0, dtype=np.float64).reshape(cp.N, 3)
    V = np.zeros_like(X) if V0 is None else np.array(V0, dtype=np.float64).reshape(cp.N, 3)
    F = chain_forces(X, cp, fp.L * fp.a) + np.asarray(cp.ext_force, dtype=float)[None]
    return State(n, X, V, F, np.zeros_like(X))


def step(st: State, fp: FluidParams, cp: ChainParams | None, replica: int = 0,
         stats: dict | None = None) -> State:
    k = st.step
    n_ps = stream(st.n)
    f = None
    X, V, F, Fc = st.X, st.V, st.F, st.Fc
    if cp is not None and cp.N > 0:
        box = fp.L * fp.a
        nsub = max(1, int(cp.substeps))
        dt = fp.h / nsub
        f = np.zeros((3, fp.L, fp.L, fp.L))
        for sub in range(nsub):
            X, Vh = bead_kick_drift(X, V, F, cp, dt)
            Fcons = chain_forces(X, cp, box) + np.asarray(cp.ext_force, dtype=float)[None]
            ub = interpolate_u(n_ps, fp, X)
            Fc = coupling_force(Vh, ub, cp, fp, k * nsub + sub, replica, dt=dt)
            f += (dt / fp.h) * spread(Fc, X, fp)
            F = Fcons + Fc
            V = bead_kick(Vh, F, cp, dt)
    n_new = collide(n_ps, fp, k, force_density=f, replica=replica, stats=stats)
    return State(n_new, X, V, F, Fc, k + 1)


def run(st: State, fp: FluidParams, cp: ChainParams | None, nsteps: int, replica: int = 0,
        stats: dict | None = None) -> State:
    for _ in range(nsteps):
        st = step(st, fp, cp, replica=replica, stats=stats)
    return st


# ---------------------------------------------------------------------------------------
# Single-node update, for sampled checks on lattices too large to step whole: the
# post-collision populations at one node given the post-collision field of the previous
# step (its 19 pull neighbours) and the force density acting at that node.
# ---------------------------------------------------------------------------------------
def node_update(npost: np.ndarray, fp: FluidParams, step_k: int, node, force=None,
                replica: int = 0) -> np.ndarray:
    L = fp.L
    x, y, z = (int(v) for v in node)
    col = np.empty(Q)
    for i in range(Q):
        ex, ey, ez = E[i]
        col[i] = npost[i, (z - ez) % L, (y - ey) % L, (x - ex) % L]
    m = M @ col
    rho, J = m[0], m[1:4]
    meq = M @ n_eq(np.array(rho), J / rho)
    gam = relaxation(fp)
    ms = m.copy()
    for kk in range(4, Q):
        ms[kk] = meq[kk] + gam[kk] * (m[kk] - meq[kk])
    if fp.noise_fluid and fp.kT > 0.0:
        mu = mu_thermal(fp)
        idx = x + L * (y + L * z)
        g = fluid_gaussians(fp.seed, TAG_FLUID, replica, step_k, np.array([idx]))[:, 0]
        kmax = 10 if fp.stress_only else Q
        for kk in range(4, kmax):
            ms[kk] += math.sqrt(mu * max(rho, 0.0) * B[kk] * (1.0 - gam[kk] ** 2)) * g[kk - 4]
    f = np.zeros(3) if force is None else np.asarray(force, dtype=float).copy()
    f += np.asarray(fp.body_force, dtype=float)
    if np.any(f != 0.0):
        dJ = f * fp.h * fp.h / fp.a
        ms += force_moment_increment(np.array(rho), J, dJ, gam)
    return MINV @ ms


# ---------------------------------------------------------------------------------------
# Observables (Sec. III A: R_g^2 = (1/2N^2) sum_ij r_ij^2, R_e^2 = (r_N - r_1)^2; Sec. III B:
# centre of mass) and the exact invariants of the coupled step.
# ---------------------------------------------------------------------------------------
def total_mass(st: State, fp: FluidParams) -> float:
    return float(st.n.sum()) * fp.a ** 3


def fluid_momentum(st: State, fp: FluidParams) -> np.ndarray:
    """a^3 sum_r j(r) of the stored (post-collision) populations, physical units."""
    J = np.tensordot(E.T.astype(float), st.n.reshape(Q, -1).sum(axis=1), axes=(1, 0))
    return J * fp.a / fp.h * fp.a ** 3


def total_momentum(st: State, fp: FluidParams, cp: ChainParams | None) -> np.ndarray:
    """Fluid + beads + (dt/2) sum_b F_c (dt: the MD step): exactly conserved by the coupled
    step when no external force acts."""
    P = fluid_momentum(st, fp)
    if cp is not None and cp.N > 0:
        dt = fp.h / max(1, int(cp.substeps))
        P = P + cp.m * st.V.sum(axis=0) + 0.5 * dt * st.Fc.sum(axis=0)
    return P


def radius_of_gyration2(X: np.ndarray) -> float:
    N = X.shape[0]
    d = X[:, None, :] - X[None, :, :]
    return float((d * d).sum() / (2.0 * N * N))


def end_to_end2(X: np.ndarray) -> float:
    d = X[-1] - X[0]
    return float(d @ d)
