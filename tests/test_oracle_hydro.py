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


def _linear_operator(fp, kvec):
    """One step of the LB linearised about the fluid at rest, for a Fourier mode exp(i k.r):
    pull streaming multiplies population i by exp(-i k.e_i); the collision keeps the
    conserved moments 0..3 and multiplies moment k >= 4 by gamma_k (the equilibrium moments
    beyond momentum are quadratic in U and drop out at linear order).  Step = collide after
    stream: n_{t+1} = M^-1 diag(lambda) M S(k) n_t."""
    lam = o.relaxation(fp).copy()
    lam[:4] = 1.0
    C = o.MINV @ np.diag(lam) @ o.M
    S = np.diag(np.exp(-1j * (o.E.astype(float) @ kvec)))
    return C @ S


def test_small_perturbation_follows_the_linearised_operator_exactly():
    """A small plane-wave perturbation with an arbitrary population profile, along a wave
    vector that is not a lattice axis, evolves under the oracle's nonlinear stream + collide
    as powers of the 19 x 19 linear operator.  The odd part in the amplitude (runs at +eps and
    -eps) removes the quadratic terms of the equilibrium; what is left is O(eps^2) relative
    (checked: a tenfold smaller amplitude shrinks it a hundredfold) down to round-off."""
    L = 8
    fp = o.FluidParams(L=L, rho=1.0, eta=3.0, eta_b=1.5, kT=0.0, h=0.01, noise_fluid=False)
    kvec = 2 * np.pi / L * np.array([1.0, 1.0, 2.0])
    rng = np.random.default_rng(9)
    v = rng.standard_normal(o.Q) + 1j * rng.standard_normal(o.Q)
    z, y, x = np.meshgrid(np.arange(L), np.arange(L), np.arange(L), indexing="ij")
    phase = np.exp(1j * (kvec[0] * x + kvec[1] * y + kvec[2] * z))  # (z, y, x)
    base = o.fluid_at_rest(fp)
    T = 12
    vT = np.linalg.matrix_power(_linear_operator(fp, kvec), T) @ v

    def misfit(eps):
        runs = []
        for sgn in (1.0, -1.0):
            n = base + sgn * eps * np.real(v[:, None, None, None] * phase[None])
            for k in range(T):
                n = o.collide(o.stream(n), fp, step=k)
            runs.append(n)
        odd = 0.5 * (runs[0] - runs[1])
        want = eps * np.real(vT[:, None, None, None] * phase[None])
        assert np.abs(want).max() > 1e-3 * eps  # the mode has not decayed away
        return np.abs(odd - want).max() / np.abs(want).max(), odd, want

    r4, _, _ = misfit(1e-4)
    r5, _, _ = misfit(1e-5)
    assert 60.0 < r4 / r5 < 160.0  # the misfit is the cubic term of the equilibrium
    r6, odd, want = misfit(1e-6)
    assert r6 < 3e-9
    eps = 1e-6
    # streaming the other way (push instead of pull) would not match
    wrong = np.linalg.matrix_power(_linear_operator(fp, -kvec), T) @ v
    wrong = eps * np.real(wrong[:, None, None, None] * phase[None])
    assert np.abs(odd - wrong).max() > 1e-3 * np.abs(want).max()


@pytest.mark.parametrize("L,tol", [(16, 0.009), (32, 0.0022)])
def test_shear_eigenvalue_of_the_linear_operator_approaches_hydrodynamics(L, tol):
    """For k along z the two transverse-momentum eigenvalues of the linear operator are the
    shear modes; their magnitude approaches exp(-nu k^2 h) as k -> 0 (lattice corrections of
    relative order k^2), and the oracle's shear wave decays at exactly that eigenvalue."""
    fp = o.FluidParams(L=L, rho=1.0, eta=3.0, eta_b=3.0, kT=0.0, h=0.01, noise_fluid=False)
    kz = 2 * np.pi / L
    Lk = _linear_operator(fp, np.array([0.0, 0.0, kz]))
    w, V = np.linalg.eig(Lk)
    # eigenvectors carrying x-momentum
    jx = np.abs(o.E[:, 0].astype(float) @ V)
    i = int(np.argmax(jx))
    lam = w[i]
    assert abs(lam.imag) < 1e-12
    want = math.exp(-fp.eta / fp.rho * kz * kz * fp.h)
    assert abs(lam.real) == pytest.approx(want, rel=tol)
    # the oracle's shear wave: amplitude ratio over 100 steps once the non-hydrodynamic
    # transients (|gamma_s|^t) have died out
    z = np.arange(L)
    U = np.zeros((3, L, L, L))
    U[0] = (1e-6 * np.sin(kz * z))[:, None, None]
    n = o.n_eq(np.ones((L, L, L)), U)
    sinz = np.sin(kz * z)
    amps = []
    for k in range(160):
        n = o.collide(o.stream(n), fp, step=k)
        jx_z = np.einsum("i,izyx->z", o.E[:, 0].astype(float), n)
        amps.append(2.0 / L * (jx_z * sinz).sum())
    assert (amps[159] / amps[59]) ** 0.01 == pytest.approx(lam.real, rel=1e-11)


@pytest.mark.parametrize("L,tol_damp,tol_freq", [(16, 5e-4, 5e-3), (32, 1.5e-4, 1.25e-3)])
def test_sound_eigenvalues_of_the_linear_operator(L, tol_damp, tol_freq):
    """For k along z the two density-carrying eigenvalues of largest magnitude are the sound
    pair exp(-Gamma h +- i c_s k h), Gamma = (4 eta/3 + eta_b) k^2 / (2 rho), c_s = a/(h sqrt 3):
    the damping pins the bulk relaxation rate (eta_b != eta here), the frequency the speed of
    sound; both approach the closed forms as k^2."""
    fp = o.FluidParams(L=L, rho=1.0, eta=3.0, eta_b=1.5, kT=0.0, h=0.01, noise_fluid=False)
    kz = 2 * np.pi / L
    w, V = np.linalg.eig(_linear_operator(fp, np.array([0.0, 0.0, kz])))
    carries_rho = np.abs(np.ones(o.Q) @ V)
    pair = np.argsort(-carries_rho * np.abs(w))[:2]
    gamma = (4.0 / 3.0 * fp.eta + fp.eta_b) * kz * kz / (2.0 * fp.rho) * fp.h
    for j in pair:
        assert -math.log(abs(w[j])) == pytest.approx(gamma, rel=tol_damp)
        assert abs(np.angle(w[j])) == pytest.approx(kz / math.sqrt(3.0), rel=tol_freq)
    assert np.angle(w[pair[0]]) == pytest.approx(-np.angle(w[pair[1]]), rel=1e-12)


def test_collision_projects_out_the_kinetic_modes():
    """Reading of the kinetic-mode rate (gamma = 0 for modes 10..18, the paper being silent):
    with the noise off, one collision of an arbitrary non-equilibrium state leaves every
    kinetic moment at zero, keeps rho and J, and relaxes the stress modes by gamma_b, gamma_s
    about their equilibrium values."""
    L = 3
    fp = o.FluidParams(L=L, rho=1.0, eta=3.0, eta_b=1.5, kT=0.0, h=0.01, noise_fluid=False)
    rng = np.random.default_rng(4)
    n = o.fluid_at_rest(fp) * (1.0 + 0.2 * rng.random((o.Q, L, L, L)))
    out = o.collide(n, fp, step=0)
    m_in = o.M @ n.reshape(o.Q, -1)
    m_out = o.M @ out.reshape(o.Q, -1)
    assert np.abs(m_out[10:]).max() < 1e-15
    assert np.allclose(m_out[:4], m_in[:4], rtol=0, atol=1e-15)
    rho, J = m_in[0], m_in[1:4]
    meq = o.M @ o.n_eq(rho, J / rho[None])
    # eta = rho c_s^2 h (1 + g) / (2 (1 - g)) and eta_b = rho c_s^2 h (1 + g_b) / (3 (1 - g_b))
    # with c_s^2 = a^2 / (3 h^2): solve for the stress eigenvalues
    x = 6.0 * fp.eta * fp.h / (fp.rho * fp.a ** 2)
    gs = (x - 1.0) / (x + 1.0)
    xb = 9.0 * fp.eta_b * fp.h / (fp.rho * fp.a ** 2)
    gb = (xb - 1.0) / (xb + 1.0)
    assert np.allclose(m_out[4], meq[4] + gb * (m_in[4] - meq[4]), rtol=0, atol=1e-15)
    for k in range(5, 10):
        assert np.allclose(m_out[k], meq[k] + gs * (m_in[k] - meq[k]), rtol=0, atol=1e-15)


def test_plane_wave_force_response_follows_the_linearised_operator():
    """From the fluid at rest, a force density f = F0 Re(v e^{i k.r}) (arbitrary direction,
    k not along an axis) adds the lattice momentum f h^2 / a to modes 1..3 of every node after
    each relaxation.  To linear order in F0 the populations after T steps are therefore
    sum_{t<T} (C S)^t M^-1 e_J (f h^2/a): the odd part in F0 of the oracle's run matches it
    (the forcing's stress terms, U'.dJ, are even in F0 and drop out)."""
    L, T = 8, 15
    fp = o.FluidParams(L=L, rho=1.0, eta=3.0, eta_b=1.5, kT=0.0, h=0.01, noise_fluid=False)
    kvec = 2 * np.pi / L * np.array([1.0, -1.0, 2.0])
    rng = np.random.default_rng(13)
    vf = rng.standard_normal(3) + 1j * rng.standard_normal(3)
    z, y, x = np.meshgrid(np.arange(L), np.arange(L), np.arange(L), indexing="ij")
    phase = np.exp(1j * (kvec[0] * x + kvec[1] * y + kvec[2] * z))
    F0 = 1e-3
    base = o.fluid_at_rest(fp)
    runs = []
    for sgn in (1.0, -1.0):
        force = sgn * F0 * np.real(vf[:, None, None, None] * phase[None])
        n = base.copy()
        for k in range(T):
            n = o.collide(o.stream(n), fp, step=k, force_density=force)
        runs.append(n - base)
    odd = 0.5 * (runs[0] - runs[1])
    A = _linear_operator(fp, kvec)
    dm = np.zeros(o.Q, dtype=complex)
    dm[1:4] = F0 * vf * fp.h * fp.h / fp.a
    g = o.MINV @ dm
    acc = np.zeros(o.Q, dtype=complex)
    P = np.eye(o.Q, dtype=complex)
    for _ in range(T):
        acc += P @ g
        P = A @ P
    want = np.real(acc[:, None, None, None] * phase[None])
    assert np.abs(want).max() > 0.0
    assert np.abs(odd - want).max() < 1e-8 * np.abs(want).max()
    # the momentum entering before streaming instead of after the collision would not match
    wrong = np.real((A @ acc)[:, None, None, None] * phase[None])
    assert np.abs(odd - wrong).max() > 1e-3 * np.abs(want).max()
