"""Pins of the oracle's force evaluation, integrator, cosmology and P(k) (CPU)."""
import math

import numpy as np
import pytest

from oracle import cosmology, mesh, power, step


def test_dt_eds_closed_form():
    a0, a1 = 0.02, 0.2
    assert cosmology.dt_supercomoving(a0, a1, 1.0, 0.0) == pytest.approx(2 * (a0 ** -0.5 - a1 ** -0.5), rel=1e-12)


def test_growth_eds_and_lcdm(golden):
    a = np.array([0.01, 0.1, 1.0])
    D, E, f1, f2 = cosmology.growth_factors(a, 1.0, 0.0)
    assert D / a == pytest.approx(np.ones(3), rel=1e-6)
    assert E / D ** 2 == pytest.approx(np.full(3, golden["growth_eds"]["D2_over_D1sq"]), rel=1e-5)
    # LCDM growing mode: D proportional to E(a) * int_0^a da' / (a' E(a'))^3
    Om, OL = 0.3, 0.7
    a = np.array([0.1, 0.5, 1.0])
    D, _, _, _ = cosmology.growth_factors(a, Om, OL)
    from scipy.integrate import quad
    heath = np.array([cosmology.hubble_E(x, Om, OL) * quad(lambda y: (y * cosmology.hubble_E(y, Om, OL)) ** -3,
                                                           0, x, epsrel=1e-12)[0] for x in a])
    assert D / D[-1] == pytest.approx(heath / heath[-1], rel=1e-6)


def test_momentum_conservation_and_no_self_force():
    prm = step.PMParams(n=16, Om=1.0, OL=0.0)
    pos = np.random.default_rng(9).random((300, 3))
    acc, _, _ = step.accelerations(pos, 0.5, prm)
    assert np.abs(acc.sum(axis=0)).max() < 1e-11 * np.abs(acc).sum()
    one = np.array([[0.3141, 0.5926, 0.5358]])
    acc1, _, _ = step.accelerations(one, 0.5, prm)
    assert np.abs(acc1).max() < 1e-14


def test_kdk_time_reversible():
    prm = step.PMParams(n=16, Om=1.0, OL=0.0)
    rng = np.random.default_rng(10)
    pos0 = rng.random((200, 3))
    vel0 = 1e-3 * rng.standard_normal((200, 3))
    a = list(np.linspace(0.1, 0.3, 6))
    pos1, vel1 = step.run_kdk(pos0, vel0, a, prm)
    pos2, vel2 = step.run_kdk(pos1, vel1, a[::-1], prm)
    d = (pos2 - pos0 + 0.5) % 1.0 - 0.5
    assert np.abs(d).max() < 1e-12
    assert np.abs(vel2 - vel0).max() < 1e-12


def _plane_wave_growth(n, m=1):
    """EdS Zel'dovich plane wave along x, amplitude chosen pre-shell-crossing;
    returns the growth of the displacement amplitude divided by a_end/a_start."""
    a0, a1, steps = 0.02, 0.2, 20
    A1 = 0.3 / (2 * np.pi * m)                  # D |dPsi/dq| = 0.3 at a1
    A0 = A1 * a0 / a1
    q = (np.arange(n) + 0.5) / n
    qx, qy, qz = np.meshgrid(q, q, q, indexing="ij")
    psi = A0 * np.sin(2 * np.pi * m * qx)
    pos = np.stack([(qx + psi).ravel(), qy.ravel(), qz.ravel()], axis=1)
    vel = np.zeros_like(pos)
    vel[:, 0] = (psi * math.sqrt(a0)).ravel()
    prm = step.PMParams(n=n, Om=1.0, OL=0.0)
    pos, _ = step.run_kdk(pos, vel, list(np.linspace(a0, a1, steps + 1)), prm)
    dx = (pos[:, 0] - qx.ravel() + 0.5) % 1.0 - 0.5
    amp = 2 * np.mean(dx * np.sin(2 * np.pi * m * qx.ravel()))
    return (amp / A0) / (a1 / a0)


@pytest.mark.slow
def test_zeldovich_growth_eds():
    """D = a in Einstein-de Sitter before shell crossing (§3.3 / Appendix A);
    the PM deficit comes from the discrete operators (TSC window, 7-point
    Laplacian, 5-point gradient) and from 20 leapfrog steps, and shrinks with
    resolution."""
    g16, g32, g64 = (_plane_wave_growth(n) for n in (16, 32, 64))
    assert abs(g64 - 1.0) < 0.01
    assert (1.0 - g16) > (1.0 - g32) > (1.0 - g64) > 0.0


def test_power_spectrum_plane_wave_total():
    n, L, A, m = 32, 100.0, 0.1, 3
    i = np.arange(n)
    delta = A * np.cos(2 * np.pi * m * i / n)[:, None, None] * np.ones((1, n, n))
    k, P, cnt = power.power_spectrum(1.0 + delta, L)
    total = P * cnt
    assert total[m - 1] == pytest.approx(L ** 3 * A ** 2 / 2, rel=1e-12)
    assert np.abs(np.delete(total, m - 1)).max() < 1e-20
    assert abs(k[m - 1] - 2 * np.pi * m / L) < 0.5 * 2 * np.pi / L   # mode-averaged shell wavenumber


def test_parametrised_coupling_closed_forms():
    from oracle.cosmology import mu_parametrised
    # today mu = 1 + mu0 (Omega_Lambda(1) = Omega_Lambda,0); early times mu -> 1
    assert abs(mu_parametrised(1.0, 0.3, 0.7, 0.4) - 1.4) < 1e-14
    assert abs(mu_parametrised(1e-3, 0.3, 0.7, 0.4) - 1.0) < 1e-8
    # Omega_Lambda(a) / Omega_Lambda,0 = 1 / E(a)^2
    a = 0.5
    assert abs(mu_parametrised(a, 0.3, 0.7, -0.5) - (1.0 - 0.5 / (0.3 / a ** 3 + 0.7))) < 1e-14


def test_parametrised_accelerations_scale_with_mu():
    """The parametrised source only rescales the Poisson equation, so the
    accelerations are mu(a) times the Newtonian ones."""
    from oracle.cosmology import mu_parametrised
    rng = np.random.Generator(np.random.PCG64(7))
    pos = rng.random((500, 3))
    base = step.PMParams(n=16, Om=0.3, OL=0.7)
    acc_n, _, _ = step.accelerations(pos, 0.6, base)
    acc_m, _, _ = step.accelerations(pos, 0.6, step.PMParams(n=16, Om=0.3, OL=0.7, gravity="mu", mu0=0.3))
    np.testing.assert_allclose(acc_m, mu_parametrised(0.6, 0.3, 0.7, 0.3) * acc_n, rtol=1e-12, atol=1e-15)


def _eds_a_after(a, dt):
    """EdS: t~(a) = -2 a^(-1/2) + const, so a after dt is (a^(-1/2) - dt/2)^(-2)."""
    return (a ** -0.5 - 0.5 * dt) ** -2


def test_next_timestep_eds_closed_forms():
    """Each §3.4 criterion alone, in Einstein-de Sitter where the supercomoving
    time has the closed form t~ = -2 a^(-1/2): the 2% growth of a, the free
    fall over one cell and the cell crossing, times the Courant factor, and
    the clip at a_end."""
    from oracle.step import next_timestep
    a, n, C, da = 0.1, 32, 0.8, 0.02
    dt_a = 2.0 * (a ** -0.5 - (a * (1 + da)) ** -0.5)
    dt, an = next_timestep(a, 1.0, 0.0, n, 0.0, 0.0, C, da)               # growth of a only
    assert dt == pytest.approx(C * dt_a, rel=1e-12)
    assert an == pytest.approx(_eds_a_after(a, dt), rel=1e-12)
    big_acc = 10.0 / (n * dt_a ** 2)                                      # free fall: sqrt(h / acc) < dt_a
    dt, an = next_timestep(a, 1.0, 0.0, n, big_acc, 0.0, C, da)
    assert dt == pytest.approx(C * np.sqrt(1.0 / n / big_acc), rel=1e-12)
    assert an == pytest.approx(_eds_a_after(a, dt), rel=1e-12)
    big_v = 10.0 / (n * dt_a)                                             # crossing: h / v < dt_a
    dt, an = next_timestep(a, 1.0, 0.0, n, big_acc * 1e-6, big_v, C, da)
    assert dt == pytest.approx(C / (n * big_v), rel=1e-12)
    dt, an = next_timestep(0.995, 1.0, 0.0, n, 0.0, 0.0, C, da, a_end=1.0)  # clipped at a_end
    assert an == 1.0 and dt == pytest.approx(2.0 * (0.995 ** -0.5 - 1.0), rel=1e-12)
