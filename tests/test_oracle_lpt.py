"""Pins of the LPT initial-conditions oracle (CPU): closed forms of single and
crossed plane waves, and the input generator's statistics."""
import numpy as np

from oracle import lpt


def _plane(n, axis, m, amp=1e-2, phase=0.0):
    i = np.arange(n)
    c = (i + 0.5) / n
    shape = [1, 1, 1]
    shape[axis] = n
    return amp * np.cos(2 * np.pi * m * c + phase).reshape(shape) * np.ones((n, n, n)), c


def test_first_order_plane_wave_and_no_second_order():
    """delta = A cos(2 pi m x): Psi1_x = -A sin(2 pi m x)/(2 pi m), other
    components 0; a single plane wave has phi_ii phi_jj = phi_ij^2, so Psi2 = 0."""
    n, m = 16, 3
    delta, c = _plane(n, 0, m)
    ones = np.ones((n, n, n // 2 + 1))
    psi1, psi2 = lpt.displacements(delta, ones)
    q = lpt.lattice(n)
    np.testing.assert_allclose(psi1[0], -1e-2 * np.sin(2 * np.pi * m * q[0]) / (2 * np.pi * m), atol=1e-15)
    np.testing.assert_allclose(psi1[1:], 0.0, atol=1e-15)
    np.testing.assert_allclose(psi2, 0.0, atol=1e-15)


def test_second_order_crossed_plane_waves_closed_form():
    """delta = A cos(kx x) + B cos(ky y): phi1 = -A cos/kx^2 - B cos/ky^2,
    phi_xx phi_yy = A B cos(kx x) cos(ky y), phi_xy = 0, so
    phi2 = -A B cos(kx x) cos(ky y) / (kx^2 + ky^2) and Psi2 = grad phi2."""
    n, mx, my, A, B = 16, 2, 3, 1e-2, 2e-2
    dx, c = _plane(n, 0, mx, A)
    dy, _ = _plane(n, 1, my, B)
    psi1, psi2 = lpt.displacements(dx + dy, np.ones((n, n, n // 2 + 1)))
    q = lpt.lattice(n)
    kx, ky = 2 * np.pi * mx, 2 * np.pi * my
    den = kx ** 2 + ky ** 2
    np.testing.assert_allclose(psi2[0], A * B * kx * np.sin(kx * q[0]) * np.cos(ky * q[1]) / den, atol=1e-14)
    np.testing.assert_allclose(psi2[1], A * B * ky * np.cos(kx * q[0]) * np.sin(ky * q[1]) / den, atol=1e-14)
    np.testing.assert_allclose(psi2[2], 0.0, atol=1e-14)
    np.testing.assert_allclose(psi1[1], -B * np.sin(ky * q[1]) / ky, atol=1e-14)


def test_matches_the_input_generator():
    """The input generator's 2LPT (torch, on its own code) gives the same
    particles for the same noise and spectrum."""
    import math
    import torch
    from paper_2410_20501_gb300 import inputs
    n, L, Om, a = 16, 64.0, 0.3, 1 / 31
    X, V = inputs.lpt_ics(n, L, Om, 1 - Om, a, 7, order=2)
    D, E, f1, f2 = inputs.growth([a, 1.0], Om, 1 - Om)
    amp = inputs.lpt_amplitude(n, L, Om)
    vfac = a * a * inputs.hubble_E(a, Om, 1 - Om)
    d1, e2 = D[0] / D[1], E[0] / D[1] ** 2
    x, v = lpt.lpt2(inputs.white_noise(n, 7), amp, d1, e2, vfac * d1 * f1[0], vfac * e2 * f2[0])
    dx = (X.astype(np.float64) / 2 ** 32 - x + 0.5) % 1.0 - 0.5
    assert np.abs(dx).max() < 1e-9
    np.testing.assert_allclose(V, v, rtol=1e-9, atol=1e-12 * np.abs(v).max())
