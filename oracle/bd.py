"""Plain FP64 CPU oracle of the Brownian-dynamics (BD) chain of Sec. II C (arXiv:0903.5067):
the Ito-Euler update of the bead positions with the Rotne-Prager-Yamakawa diffusion tensor and
the noise B.W obtained by Fixman's truncated Chebyshev expansion of the square root of D.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or execute this
module; the tests compare the CUDA BD kernels with it.  It shares no code with the CUDA path.

Units: the MD/LB units of the paper (energy epsilon, length sigma, time tau); the BD friction
zeta is the long-time friction zeta_eff of the coupled model (Sec. II D) and the Stokes radius
d = zeta / (6 pi eta_s).

Readings (where the paper points to its references):
- the regularised RPY tensor: for r >= 2d the Rotne-Prager form, for r < 2d Yamakawa's
  overlap form; both are mobilities (D / kT);
- the excluded volume and springs are the chain model of Sec. II A (FENE on bonds, WCA between
  all pairs), in an infinite medium (no periodic images);
- Fixman's expansion: sqrt(x) is expanded in Chebyshev polynomials on [lam_min, lam_max] with
  `degree` + 1 terms (coefficients from the Chebyshev nodes); the bounds come from `power_iters`
  power iterations on D from the normalised all-ones vector (lam_max = 1.05 x the Rayleigh
  quotient) and the same number on lam_max I - D (lam_min = 0.5 x (lam_max - its Rayleigh
  quotient), at least lam_max / 1000: that iteration converges slowly, so its estimate of the
  smallest eigenvalue is high and needs the wide margin);
- noise: 3 standard normals per bead per step from one Philox4x32-10 call with key
  (seed, 3 | replica << 8) and counter (step, bead, 0, 0), as for the LB bead noise.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

from . import lbchain as lbo

TAG_BD = 3


@dataclasses.dataclass(frozen=True)
class BDParams:
    N: int
    kT: float = 1.2
    zeta: float = 15.48  # long-time friction zeta_eff (Sec. II D) for the production model
    eta_s: float = 0.864 * 2.8
    dt: float = 0.005 * 15.48 / 28.0  # 0.005 tau_k, tau_k = zeta / (4 k_FENE)
    k_fene: float = 7.0
    R0: float = 2.0
    eps: float = 1.0
    sigma: float = 1.0
    hi: bool = True  # RPY hydrodynamic interaction; False: free draining (diagonal D)
    degree: int = 20
    power_iters: int = 20
    seed: int = 1


def zeta_eff(zeta_bare: float, eta_s: float, a: float = 1.0, g: float = 25.0) -> float:
    """Long-time friction of a coupled point particle (Sec. II D): 1/zeta_eff = 1/zeta_bare
    + 1/(g eta_s a), g ~ 25 for linear interpolation to the nearest nodes."""
    return 1.0 / (1.0 / zeta_bare + 1.0 / (g * eta_s * a))


def rpy_block(d_vec: np.ndarray, radius: float, eta: float) -> np.ndarray:
    """3x3 mobility block of two beads at separation d_vec (regularised RPY)."""
    r = float(np.linalg.norm(d_vec))
    rr = np.outer(d_vec, d_vec) / (r * r)
    I = np.eye(3)
    if r >= 2.0 * radius:
        a2 = radius * radius / (r * r)
        return (1.0 / (8.0 * math.pi * eta * r)) * ((1.0 + 2.0 * a2 / 3.0) * I + (1.0 - 2.0 * a2) * rr)
    q = r / radius
    return (1.0 / (6.0 * math.pi * eta * radius)) * ((1.0 - 9.0 * q / 32.0) * I + (3.0 * q / 32.0) * rr)


def mobility(X: np.ndarray, p: BDParams) -> np.ndarray:
    """D / kT as a (3N, 3N) matrix: zeta^-1 on the diagonal blocks, RPY off the diagonal."""
    N = X.shape[0]
    M = np.zeros((3 * N, 3 * N))
    radius = p.zeta / (6.0 * math.pi * p.eta_s)
    for i in range(N):
        M[3 * i:3 * i + 3, 3 * i:3 * i + 3] = np.eye(3) / p.zeta
        if not p.hi:
            continue
        for j in range(N):
            if j != i:
                M[3 * i:3 * i + 3, 3 * j:3 * j + 3] = rpy_block(X[i] - X[j], radius, p.eta_s)
    return M


def forces(X: np.ndarray, p: BDParams) -> np.ndarray:
    """-grad(V_FENE + V_WCA) on every bead, infinite medium (Sec. II A)."""
    N = X.shape[0]
    F = np.zeros_like(X)
    rc2 = 2.0 ** (1.0 / 3.0) * p.sigma ** 2
    for i in range(N - 1):
        d = X[i] - X[i + 1]
        r2 = d @ d
        if r2 >= p.R0 * p.R0:
            raise lbo.FeneBroken(f"bond {i} stretched to {math.sqrt(r2)} >= R0")
        f = -p.k_fene * d / (1.0 - r2 / (p.R0 * p.R0))
        F[i] += f
        F[i + 1] -= f
    for i in range(N):
        for j in range(i + 1, N):
            d = X[i] - X[j]
            r2 = d @ d
            if r2 < rc2:
                sr6 = (p.sigma * p.sigma / r2) ** 3
                f = 24.0 * p.eps / r2 * (2.0 * sr6 * sr6 - sr6) * d
                F[i] += f
                F[j] -= f
    return F


def eigen_bounds(D: np.ndarray, iters: int):
    """[lam_min, lam_max] of the symmetric positive definite D by power iterations (reading
    listed in the module header)."""
    n = D.shape[0]
    v = np.ones(n) / math.sqrt(n)
    for _ in range(iters):
        w = D @ v
        v = w / np.linalg.norm(w)
    lam_max = 1.05 * float(v @ (D @ v))
    S = lam_max * np.eye(n) - D
    v = np.ones(n) / math.sqrt(n)
    for _ in range(iters):
        w = S @ v
        v = w / np.linalg.norm(w)
    lam_min = 0.5 * (lam_max - float(v @ (S @ v)))
    return max(lam_min, lam_max / 1000.0), lam_max


def chebyshev_sqrt_coeffs(lo: float, hi: float, degree: int) -> np.ndarray:
    """c_0..c_degree of sqrt(x) on [lo, hi] from the degree+1 Chebyshev nodes; c_0 halved, so
    that sqrt(x) ~ sum_k c_k T_k(y), y = (2x - lo - hi)/(hi - lo)."""
    K = degree + 1
    j = np.arange(K)
    th = math.pi * (j + 0.5) / K
    x = 0.5 * (hi + lo) + 0.5 * (hi - lo) * np.cos(th)
    f = np.sqrt(x)
    c = np.array([2.0 / K * float(np.sum(f * np.cos(k * th))) for k in range(K)])
    c[0] *= 0.5
    return c


def chebyshev_sqrt_apply(D: np.ndarray, w: np.ndarray, degree: int, iters: int) -> np.ndarray:
    """B.w with B B^T = D (Fixman): sum_k c_k T_k(Dt) w, Dt = (2D - (lo+hi) I)/(hi - lo),
    by the three-term recurrence T_{k+1} = 2 Dt T_k - T_{k-1}."""
    lo, hi = eigen_bounds(D, iters)
    c = chebyshev_sqrt_coeffs(lo, hi, degree)
    s, t = 2.0 / (hi - lo), (hi + lo) / (hi - lo)
    t_prev = w.copy()
    t_cur = s * (D @ w) - t * w
    y = c[0] * t_prev + c[1] * t_cur
    for k in range(2, degree + 1):
        t_next = 2.0 * (s * (D @ t_cur) - t * t_cur) - t_prev
        y = y + c[k] * t_next
        t_prev, t_cur = t_cur, t_next
    return y


def noise(p: BDParams, replica: int, step: int) -> np.ndarray:
    """3 standard normals per bead: one Philox call with counter (step, bead, 0, 0)."""
    k0, k1 = lbo.philox_key(p.seed, TAG_BD, replica)
    x = lbo.philox4x32_10(np.uint64(step), np.arange(p.N, dtype=np.uint64), 0, 0, k0, k1)
    u = [lbo.uniform01(v) for v in x]
    g0, g1 = lbo.box_muller(u[0], u[1])
    g2, _ = lbo.box_muller(u[2], u[3])
    return np.stack([g0, g1, g2], axis=1).reshape(-1)


def step(X: np.ndarray, p: BDParams, replica: int, k: int) -> np.ndarray:
    """One Ito-Euler step (Sec. II C): r += (D/kT) F dt + sqrt(2 dt) B W."""
    M = mobility(X, p)
    F = forces(X, p).reshape(-1)
    W = noise(p, replica, k)
    if p.hi:
        BW = chebyshev_sqrt_apply(p.kT * M, W, p.degree, p.power_iters)
    else:
        BW = math.sqrt(p.kT / p.zeta) * W
    return X + (M @ F * p.dt + math.sqrt(2.0 * p.dt) * BW).reshape(-1, 3)


def run(X: np.ndarray, p: BDParams, steps: int, replica: int = 0, k0: int = 0) -> np.ndarray:
    for k in range(k0, k0 + steps):
        X = step(X, p, replica, k)
    return X
