"""Hydrodynamic pins of the oracle's noise-free LB: the closed forms of linear hydrodynamics
(shear-wave decay at rate nu k^2, sound attenuation (4 eta/3 + eta_b) k^2 / 2 rho, forced
Kolmogorov flow F0/(rho nu k^2)) and the exact momentum input of a uniform body force."""
import math

import numpy as np
import pytest

from oracle import lbchain as o


def _run_fluid(n, fp, nsteps, force=None, every=1, probe=None):
    out = []
    for k in range(nsteps):
        n = o.collide(o.stream(n), fp, step=k, force_density=force)
        if probe is not None and (k + 1) % every == 0:
            out.append(probe(n))
    return n, out


def test_shear_wave_decays_at_nu_k2():
    """A transverse wave u_x = A sin(k z) decays as exp(-nu k^2 t) (nu = eta/rho)."""
    L = 32
    fp = o.FluidParams(L=L, rho=1.0, eta=3.0, eta_b=3.0, kT=0.0, h=0.01, noise_fluid=False)
    z = np.arange(L)
    kz = 2 * np.pi / L
    U = np.zeros((3, L, L, L))
    U[0] = (1e-4 * np.sin(kz * z))[:, None, None]
    n = o.n_eq(np.ones((L, L, L)), U)
    sinz = np.sin(kz * z)

    def amp(nn):
        jx = np.einsum("i,izyx->z", o.E[:, 0].astype(float), nn)
        return 2.0 / L * (jx * sinz).sum()

    _, a = _run_fluid(n, fp, 300, probe=amp)
    a = np.array(a)
    t = np.arange(1, 301)
    sel = t >= 80
    rate = -np.polyfit(t[sel], np.log(a[sel]), 1)[0]  # per step
    want = fp.eta / fp.rho * (kz / fp.a) ** 2 * fp.h
    assert rate == pytest.approx(want, rel=5e-3)


def test_sound_wave_attenuation():
    """A longitudinal wave oscillates at c_s k and its energy decays at 2 Gamma with
    Gamma = (4 eta/3 + eta_b) k^2 / (2 rho); this pins the bulk relaxation rate."""
    L = 32
    fp = o.FluidParams(L=L, rho=1.0, eta=3.0, eta_b=1.5, kT=0.0, h=0.01, noise_fluid=False)
    z = np.arange(L)
    kz = 2 * np.pi / L
    rho = (1.0 + 1e-4 * np.cos(kz * z))[:, None, None] * np.ones((L, L, L))
    n = o.n_eq(rho, np.zeros((3, L, L, L)))
    cosz, sinz = np.cos(kz * z), np.sin(kz * z)
    ez = o.E[:, 2].astype(float)

    def energy(nn):
        r = nn.sum(axis=(0, 2, 3))
        jz = np.einsum("i,izyx->z", ez, nn) / (L * L)
        dr = 2.0 / L * ((r / (L * L)) * cosz).sum()
        dj = 2.0 / L * (jz * sinz).sum()
        return o.CS2 * dr * dr + dj * dj

    nsteps = 5 * 111  # ten sound periods (period = L sqrt(3) steps)
    _, e = _run_fluid(n, fp, nsteps, probe=energy)
    e = np.array(e)
    t = np.arange(1, nsteps + 1)
    sel = t >= 56
    rate = -np.polyfit(t[sel], np.log(e[sel]), 1)[0]
    gamma = (4.0 / 3.0 * fp.eta + fp.eta_b) * (kz / fp.a) ** 2 / (2.0 * fp.rho) * fp.h
    assert rate == pytest.approx(2 * gamma, rel=0.03)


def test_uniform_body_force_adds_exact_momentum():
    """A uniform force density f adds exactly L^3 a^3 f h of momentum per step."""
    L = 6
    f = np.array([1e-3, -2e-3, 0.5e-3])
    fp = o.FluidParams(L=L, kT=0.0, noise_fluid=False, h=0.01, a=0.7, body_force=tuple(f))
    st = o.init_state(fp, None)
    P0 = o.fluid_momentum(st, fp)
    st = o.run(st, fp, None, 5)
    dP = o.fluid_momentum(st, fp) - P0
    want = 5 * L ** 3 * fp.a ** 3 * f * fp.h
    # round-off of the population sums, scaled by the momentum of the whole box moving at
    # one lattice unit of velocity
    scale = L ** 3 * fp.a ** 3 * fp.rho * fp.a / fp.h
    assert np.allclose(dP, want, rtol=0, atol=1e-13 * scale)
    assert np.all(np.abs(dP - want) < 1e-6 * np.abs(want))


def test_kolmogorov_flow_steady_profile():
    """A sinusoidal force density f_x = F0 sin(k z) drives the steady flow
    u_x = F0 sin(k z) / (rho nu k^2) (Stokes flow, lattice corrections O(k^2))."""
    L = 16
    fp = o.FluidParams(L=L, rho=1.0, eta=3.0, eta_b=3.0, kT=0.0, h=0.05, noise_fluid=False)
    z = np.arange(L)
    kz = 2 * np.pi / L
    F0 = 1e-4
    force = np.zeros((3, L, L, L))
    force[0] = (F0 * np.sin(kz * z))[:, None, None]
    st = o.fluid_at_rest(fp)
    nu = fp.eta / fp.rho
    relax_steps = int(12.0 / (nu * kz * kz * fp.h))
    n, _ = _run_fluid(st, fp, relax_steps, force=force)
    nps = o.stream(n)
    rho = nps.sum(axis=0)
    jx = np.einsum("i,izyx->zyx", o.E[:, 0].astype(float), nps)
    # velocity of the forced step: (J + dJ/2)/rho in lattice units, times a/h
    ux = (jx + 0.5 * force[0] * fp.h * fp.h / fp.a) / rho * fp.a / fp.h
    amp = 2.0 / L * (ux.mean(axis=(1, 2)) * np.sin(kz * z)).sum()
    want = F0 / (fp.rho * nu * kz * kz)
    assert amp == pytest.approx(want, rel=0.02)


def test_uniformly_forced_fluid_stress_follows_the_forcing_recurrence():
    """On a uniform state streaming is the identity, so the stress tensor of a uniformly
    forced fluid obeys a closed recurrence.  With the second-order forcing reading
    (momentum + dJ, stress + (1+Gamma)/2 D with D = U' dJ + dJ U', U' = (J + dJ/2)/rho and
    Gamma = gamma_s on the traceless part, gamma_b on the trace), the non-equilibrium stress
    x = Pi - (rho/3 1 + J J / rho) evolves as x' = Gamma x - (1 - Gamma)/2 D, and the kinetic
    modes stay zero.  Checks the mode-space implementation of the forcing term."""
    L = 3
    f = np.array([2e-2, -1e-2, 3e-2])
    fp = o.FluidParams(L=L, rho=1.1, eta=3.0, eta_b=1.5, kT=0.0, h=0.01, a=1.0,
                       noise_fluid=False, body_force=tuple(f))
    gam = o.relaxation(fp)
    gs, gb = gam[5], gam[4]
    U0 = np.array([0.01, 0.02, -0.005])
    n = o.n_eq(np.full((L, L, L), 1.1), np.broadcast_to(U0[:, None, None, None], (3, L, L, L)).copy())
    e = o.E.astype(float)
    dJ = f * fp.h * fp.h / fp.a
    I3 = np.eye(3)

    def Gamma(A):
        tr = np.trace(A) / 3.0
        return gs * (A - tr * I3) + gb * tr * I3

    x_pred = np.zeros((3, 3))
    for t in range(60):
        nps = o.stream(n)
        col = nps[:, 0, 0, 0]
        rho, J = col.sum(), e.T @ col
        Pi = np.einsum("i,ia,ib->ab", col, e, e)
        x = Pi - (rho / 3.0 * I3 + np.outer(J, J) / rho)
        assert np.allclose(x, x_pred, rtol=0, atol=1e-15), t
        assert np.allclose((o.M @ col)[10:], 0.0, atol=1e-15)
        Up = (J + 0.5 * dJ) / rho
        D = np.outer(Up, dJ) + np.outer(dJ, Up)
        x_pred = Gamma(x_pred) - 0.5 * (D - Gamma(D))
        n = o.collide(nps, fp, step=t)
    assert np.abs(x_pred).max() > 1e-8  # the recurrence was exercised
