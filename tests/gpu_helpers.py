"""Shared helpers of the GPU tests: run the same seeded workload through the CUDA library
(C ABI via the ctypes binding) and through the oracle."""
from __future__ import annotations

import dataclasses
import functools

import numpy as np

from oracle import lbchain as o
from paper_0903_5067_gb300 import inputs


@dataclasses.dataclass(frozen=True)
class Case:
    L: int
    N: int
    steps: int
    seed: int = 1
    rho: float = 1.0
    eta: float = 3.0
    eta_b: float = 3.0
    kT: float = 1.0
    h: float = 0.01
    a: float = 1.0
    noise_fluid: bool = True
    noise_beads: bool = True
    stress_only: bool = False
    ext: tuple = (0.0, 0.0, 0.0)
    counter: bool = False
    perturb: float = 0.0  # relative perturbation of the initial populations
    m: float = 1.0
    zeta: float = 20.8
    k_fene: float = 30.0
    R0: float = 1.5
    eps: float = 1.0
    sigma: float = 1.0
    chain_seed: int = 0
    substeps: int = 1

    def fluid(self):
        body = (0.0, 0.0, 0.0)
        if self.counter and self.N > 0:
            vol = (self.L * self.a) ** 3
            body = tuple(-self.N * e / vol for e in self.ext)
        return o.FluidParams(L=self.L, rho=self.rho, eta=self.eta, eta_b=self.eta_b, kT=self.kT, h=self.h,
                             a=self.a, seed=self.seed, noise_fluid=self.noise_fluid,
                             stress_only=self.stress_only, body_force=body)

    def chain(self):
        if self.N == 0:
            return None
        return o.ChainParams(N=self.N, m=self.m, zeta=self.zeta, k_fene=self.k_fene, R0=self.R0, eps=self.eps,
                             sigma=self.sigma, noise_beads=self.noise_beads, ext_force=self.ext,
                             substeps=self.substeps)

    def x0(self):
        return inputs.chain_walk(self.N, L=self.L, a=self.a, bond=0.97, seed=self.chain_seed or self.seed,
                                 self_avoiding=True, sigma=self.sigma)

    def n0(self):
        if self.perturb == 0.0:
            return None
        rest = o.fluid_at_rest(self.fluid())
        return rest * (1.0 + inputs.perturbation(self.L, amplitude=self.perturb, seed=self.seed))


@functools.lru_cache(maxsize=32)
def oracle_run(case: Case):
    fp, cp = case.fluid(), case.chain()
    st = o.init_state(fp, cp, case.x0() if cp else None, n0=case.n0())
    st = o.run(st, fp, cp, case.steps)
    return st


def gpu_sim(lb, case: Case, precision: int):
    sim = lb.Simulation(L=case.L, rho=case.rho, eta=case.eta, eta_b=case.eta_b, kT=case.kT, h=case.h, a=case.a,
                        seed=case.seed, precision=precision)
    if case.N > 0:
        sim.add_chain(case.N, m=case.m, zeta=case.zeta, k_fene=case.k_fene, R0=case.R0, eps=case.eps,
                      sigma=case.sigma, x0=case.x0())
        if case.substeps > 1:
            sim.set_md_substeps(case.substeps)
    sim.set_options(noise_fluid=int(case.noise_fluid), noise_beads=int(case.noise_beads),
                    stress_only=int(case.stress_only), ext_bead_force=list(case.ext),
                    counter_force_fluid=int(case.counter))
    n0 = case.n0()
    if n0 is not None:
        sim.set_populations(n0)
    return sim


def gpu_run(lb, case: Case, precision: int, steps: int | None = None):
    sim = gpu_sim(lb, case, precision)
    sim.step(case.steps if steps is None else steps)
    sim.sync()
    n = sim.populations()
    x, v = sim.beads()
    obs = sim.observables()
    sim.close()
    return n, x, v, obs


def pop_rel_err(n_gpu, n_ref):
    """max over populations of |n_gpu - n_ref| / |n_ref|."""
    return float(np.max(np.abs(n_gpu - n_ref) / np.abs(n_ref)))


def bead_errs(x, v, st, case: Case):
    """position error relative to the box length and velocity error relative to the thermal
    velocity sqrt(kT/m) (or to max |v| when kT = 0)."""
    if case.N == 0:
        return 0.0, 0.0
    ex = float(np.max(np.abs(x - st.X))) / (case.L * case.a)
    vs = np.sqrt(case.kT / case.m) if case.kT > 0 else max(float(np.abs(st.V).max()), 1e-30)
    ev = float(np.max(np.abs(v - st.V))) / vs
    return ex, ev
