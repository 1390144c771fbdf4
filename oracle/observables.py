"""Plain FP64 CPU definitions of the chain observables of Sec. III B (arXiv:0903.5067):
monomer and centre-of-mass mean-square displacements g1, g2, g3; Rouse modes X_p and their
time correlation; static and dynamic structure factors S(k), S(k, t).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or execute this
module; the tests compare the CUDA analysis kernels with it.  It shares no code with the
CUDA path.

A trajectory is an array ``traj[t, n, 3]`` of unwrapped bead positions at T equally spaced
frames (frame spacing = the recording stride times the time step).  Time averages run over
every origin t0 with t0 + lag inside the trajectory, as written out below; nothing is
blocked, windowed or reordered beyond the definitions.

Readings (where the paper leaves a choice):
- g1 and g2 average over the two monomers at the middle of the chain (Sec. III B): for N beads numbered
  0..N-1, the monomers floor((N-1)/2) and ceil((N-1)/2) (the same bead twice when N is
  odd); the caller may pass another pair.
- The Rouse correlation is normalised by <X_p^2> averaged over all frames.
- S(k) and S(k, t) are the isotropic averages over the directions of the wave vector, so
  exp(i k.r) becomes sin(kr)/(kr) (and 1 at r = 0), as the paper writes for S(k); S(k, t)
  uses the same average of exp(i k.[r_i(t0+t) - r_j(t0)]).
"""
from __future__ import annotations

import math

import numpy as np


def inner_pair(N: int) -> tuple[int, int]:
    """The two innermost monomers of a chain of N beads (0-based)."""
    return (N - 1) // 2, N // 2


def centre_of_mass(traj: np.ndarray) -> np.ndarray:
    """R_CM(t) = (1/N) sum_n r_n(t) (equal masses), shape (T, 3)."""
    return traj.mean(axis=1)


def msd(traj: np.ndarray, max_lag: int, pair: tuple[int, int] | None = None):
    """g1, g2, g3 at lags 0..max_lag (Sec. III B, Eqs. for g1, g2, g3).

    g1(lag) = < |r_i(t0+lag) - r_i(t0)|^2 >, i over the pair, averaged over origins t0;
    g2 the same with the centre of mass subtracted at both times; g3 for the centre of mass.
    """
    T, N, _ = traj.shape
    i0, i1 = inner_pair(N) if pair is None else pair
    cm = centre_of_mass(traj)
    g1 = np.zeros(max_lag + 1)
    g2 = np.zeros(max_lag + 1)
    g3 = np.zeros(max_lag + 1)
    for lag in range(max_lag + 1):
        norig = T - lag
        if norig <= 0:
            continue
        s1 = s2 = s3 = 0.0
        for t0 in range(norig):
            dcm = cm[t0 + lag] - cm[t0]
            s3 += float(dcm @ dcm)
            for i in (i0, i1):
                d = traj[t0 + lag, i] - traj[t0, i]
                s1 += float(d @ d)
                dr = d - dcm
                s2 += float(dr @ dr)
        g1[lag] = s1 / (2 * norig)
        g2[lag] = s2 / (2 * norig)
        g3[lag] = s3 / norig
    return g1, g2, g3


def rouse_modes(traj: np.ndarray, P: int | None = None) -> np.ndarray:
    """X_p(t) = (1/N) sum_{n=1..N} r_n(t) cos[(p pi / N)(n - 1/2)], p = 1..P (default N-1)
    (Sec. III B, Rouse-mode definition).  Shape (T, P, 3); row p-1 holds mode p."""
    T, N, _ = traj.shape
    P = N - 1 if P is None else P
    X = np.zeros((T, P, 3))
    for p in range(1, P + 1):
        c = np.array([math.cos(p * math.pi / N * (n - 0.5)) for n in range(1, N + 1)])
        X[:, p - 1, :] = np.einsum("n,tnd->td", c, traj) / N
    return X


def rouse_correlation(X: np.ndarray, max_lag: int):
    """c_p(lag) = < X_p(t0+lag) . X_p(t0) > over origins, and <X_p^2> over all frames;
    the normalised correlation of Sec. III B is c_p(lag) / <X_p^2>.  Shapes (P, max_lag+1), (P,)."""
    T, P, _ = X.shape
    c = np.zeros((P, max_lag + 1))
    for lag in range(max_lag + 1):
        norig = T - lag
        if norig <= 0:
            continue
        for p in range(P):
            s = 0.0
            for t0 in range(norig):
                s += float(X[t0 + lag, p] @ X[t0, p])
            c[p, lag] = s / norig
    x2 = np.array([float(np.mean(np.sum(X[:, p] ** 2, axis=1))) for p in range(P)])
    return c, x2


def sinc_k(k: float, r: float) -> float:
    """Isotropic average of exp(i k.r) over the directions of k: sin(kr)/(kr), 1 at kr = 0."""
    x = k * r
    return 1.0 if x == 0.0 else math.sin(x) / x


def static_structure_factor(traj: np.ndarray, ks) -> np.ndarray:
    """S(k) = (1/N) sum_{i,j} < sin(k r_ij) / (k r_ij) > over frames (Sec. III A, S(k))."""
    T, N, _ = traj.shape
    out = np.zeros(len(ks))
    for a, k in enumerate(ks):
        s = 0.0
        for t in range(T):
            for i in range(N):
                for j in range(N):
                    d = traj[t, i] - traj[t, j]
                    s += sinc_k(k, math.sqrt(float(d @ d)))
        out[a] = s / (N * T)
    return out


def dynamic_structure_factor(traj: np.ndarray, ks, max_lag: int, origin_stride: int = 1) -> np.ndarray:
    """S(k, lag) = (1/N) sum_{i,j} < sin(k |r_i(t0+lag) - r_j(t0)|) / (k |...|) > over the
    origins t0 = 0, s, 2s, ... with t0 + lag < T (Sec. III B, S(k, t)).  Shape (nk, max_lag+1)."""
    T, N, _ = traj.shape
    out = np.zeros((len(ks), max_lag + 1))
    for a, k in enumerate(ks):
        for lag in range(max_lag + 1):
            origins = list(range(0, T - lag, origin_stride))
            if not origins:
                continue
            s = 0.0
            for t0 in origins:
                for i in range(N):
                    for j in range(N):
                        d = traj[t0 + lag, i] - traj[t0, j]
                        s += sinc_k(k, math.sqrt(float(d @ d)))
            out[a, lag] = s / (N * len(origins))
    return out


def inverse_hydrodynamic_radius(traj: np.ndarray) -> float:
    """<1/R_H> = (1/N^2) sum_{i != j} <1/r_ij>, averaged over the frames (Sec. III A, the
    infinite-medium hydrodynamic radius of the chain)."""
    T, N, _ = traj.shape
    s = 0.0
    for t in range(T):
        for i in range(N):
            for j in range(N):
                if i != j:
                    d = traj[t, i] - traj[t, j]
                    s += 1.0 / math.sqrt(float(d @ d))
    return s / (N * N * T)


def rouse_chain_trajectory(N: int, T: int, dt: float, b: float, zeta: float, kT: float, seed: int):
    """A Gaussian Rouse chain (harmonic springs of constant 3kT/b^2, no hydrodynamic or
    excluded-volume interaction, friction zeta per bead) sampled exactly: in its normal
    modes the overdamped Langevin equation decouples into independent Ornstein-Uhlenbeck
    processes, advanced here with their exact one-step transition.

    For the discrete chain with free ends the cosine basis diagonalises the spring forces:
    zeta dX_p/dt = -lam_p X_p + f_p with lam_p = 4 k_s sin^2(p pi / 2N), k_s = 3kT/b^2, and
    the projected noise f_p has variance kT zeta / N per component (p >= 1).  So X_p relaxes
    with tau_p = zeta / lam_p, its stationary variance per component is kT / (2 N lam_p),
    and the centre of mass X_0 diffuses with D = kT / (N zeta).  Returns (traj, tau, var),
    tau and var for p = 1..N-1.
    """
    rng = np.random.default_rng(seed)
    ks = 3.0 * kT / b ** 2
    n = np.arange(1, N + 1)
    # orthogonal DCT-II basis: r_n = X_0 + 2 sum_p X_p cos(p pi (n - 1/2) / N)
    C = np.array([[math.cos(p * math.pi * (m - 0.5) / N) for p in range(N)] for m in n])  # (N, N)
    lam = np.array([4.0 * ks * math.sin(p * math.pi / (2 * N)) ** 2 for p in range(N)])
    # equations of motion of X_p (p >= 1): zeta dX_p/dt = -lam_p X_p + f_p, with
    # f_p = (1/N) sum_n f_n cos(...) of white noise of variance 2 kT zeta per bead component:
    # <f_p f_p> = 2 kT zeta * (1/N^2) sum_n cos^2 = 2 kT zeta / (2N)  (p >= 1)
    tau = np.zeros(N)
    var = np.zeros(N)
    for p in range(1, N):
        tau[p] = zeta / lam[p]
        # stationary variance of dX = -X/tau dt + sqrt(2 D_p) dW with D_p = kT / (2 N zeta)
        var[p] = (kT / (2.0 * N * zeta)) * tau[p]
    X = np.zeros((N, 3))
    for p in range(1, N):
        X[p] = rng.standard_normal(3) * math.sqrt(var[p])
    traj = np.zeros((T, N, 3))
    D0 = kT / (N * zeta)
    for t in range(T):
        traj[t] = X[0] + 2.0 * (C[:, 1:] @ X[1:])
        X[0] = X[0] + rng.standard_normal(3) * math.sqrt(2.0 * D0 * dt)
        for p in range(1, N):
            a = math.exp(-dt / tau[p])
            X[p] = a * X[p] + rng.standard_normal(3) * math.sqrt(var[p] * (1.0 - a * a))
    return traj, tau[1:], var[1:]
