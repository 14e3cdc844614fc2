"""Pins of the differentiable FP64 oracle (oracle/adjoint.py) to things other
than itself: the numpy oracle's forward step, closed forms, the defining
property of the Poisson solve, and central finite differences of the
forward map."""
import math

import numpy as np
import pytest
import torch

from oracle import adjoint as adj
from oracle import cosmology, mesh, step
from paper_2410_20501_gb300 import inputs

T = torch.float64


def _particles(n_part, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.random((n_part, 3))


def test_forward_matches_numpy_oracle():
    # deposit, interp and the whole force evaluation equal the numpy oracle's
    n = 16
    pos = _particles(700, 11)
    rho_t = adj.deposit(torch.from_numpy(pos), n).numpy()
    np.testing.assert_allclose(rho_t, mesh.deposit_tsc(pos, n), rtol=0, atol=1e-12)
    prm = step.PMParams(n=n, Om=0.3, OL=0.7, solver="fft7", grad_order=5)
    acc_np, _, _ = step.accelerations(pos, 0.5, prm)
    acc_t = adj.accelerations(torch.from_numpy(pos), 0.5, 0.3, n, 5).numpy()
    np.testing.assert_allclose(acc_t, acc_np, rtol=0, atol=1e-12 * np.abs(acc_np).max())


def test_poisson_definition_and_self_adjoint():
    n, h = 16, 1.0 / 16
    rng = np.random.Generator(np.random.PCG64(3))
    f = torch.from_numpy(rng.standard_normal((n, n, n)))
    g = torch.from_numpy(rng.standard_normal((n, n, n)))
    phi = adj.solve_fft7(f, h)
    # (L(phi) - 6 phi)/h^2 = f - <f> and <phi> = 0
    torch.testing.assert_close(adj.laplacian7(phi, h), f - f.mean(), rtol=0, atol=1e-10)
    assert abs(float(phi.mean())) < 1e-14
    # the inverse of a symmetric operator on zero-mean fields is symmetric
    lhs = float((adj.solve_fft7(f, h) * (g - g.mean())).sum())
    rhs = float(((f - f.mean()) * adj.solve_fft7(g, h)).sum())
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_lpt_plane_wave_closed_form():
    # delta = eps cos(2 pi m x)  =>  Psi_x = -eps sin(2 pi m x) / (2 pi m), Psi_y = Psi_z = 0
    n, m, eps = 16, 3, 0.01
    c = (np.arange(n) + 0.5) / n
    noise = eps * np.cos(2 * math.pi * m * c)[:, None, None] * np.ones((n, n, n))
    amp = torch.ones((n, n, n // 2 + 1), dtype=T)
    pos, vel = adj.lpt1(torch.from_numpy(noise), amp, 0.5, 2.0)
    q = np.stack(np.meshgrid(c, c, c, indexing="ij"), -1).reshape(-1, 3)
    psi_x = -eps * np.sin(2 * math.pi * m * q[:, 0]) / (2 * math.pi * m)
    np.testing.assert_allclose(pos[:, 0].numpy(), (q[:, 0] + 0.5 * psi_x) % 1.0, atol=1e-14)
    np.testing.assert_allclose(pos[:, 1:].numpy(), q[:, 1:], atol=1e-14)
    np.testing.assert_allclose(vel[:, 0].numpy(), 2.0 * psi_x, atol=1e-14)
    np.testing.assert_allclose(vel[:, 1:].numpy(), 0.0, atol=1e-14)


def test_step_vjp_matches_finite_differences():
    # <x_bar, dx'> + <v_bar, dv'> along random directions, central differences in FP64
    n = 8
    rng = np.random.Generator(np.random.PCG64(21))
    pos = rng.random((300, 3))
    vel = 0.05 * rng.standard_normal((300, 3))
    xb, vb = rng.standard_normal((300, 3)), rng.standard_normal((300, 3))
    a, dtk, dtd = 0.4, 0.3, 0.2
    gx, gv = adj.step_vjp(pos, vel, a, 1.0, n, dtk, dtd, xb, vb)

    def L(p, v):
        x1, v1 = adj.kdk_step(torch.from_numpy(p), torch.from_numpy(v), a, 1.0, n, dtk, dtd)
        d = (x1 - torch.from_numpy(p) + 0.5) % 1.0 - 0.5        # unwrapped displacement
        return float((d * torch.from_numpy(xb)).sum() + (v1 * torch.from_numpy(vb)).sum())

    for k in range(3):
        dp, dv = rng.standard_normal((300, 3)), rng.standard_normal((300, 3))
        eps = 1e-6
        fd = (L(pos + eps * dp, vel + eps * dv) - L(pos - eps * dp, vel - eps * dv)) / (2 * eps)
        fd += float((dp * xb).sum())       # the unwrapped displacement dropped the identity term
        an = float((gx.numpy() * dp).sum() + (gv.numpy() * dv).sum())
        assert abs(fd - an) <= 1e-6 * (abs(an) + 1.0), (k, fd, an)


def _schedule(a_steps, Om, OL):
    """Fused-kick leapfrog coefficients (a_i, (dt_{i-1} + dt_i)/2, dt_i)."""
    dts = [cosmology.dt_supercomoving(a0, a1, Om, OL) for a0, a1 in zip(a_steps[:-1], a_steps[1:])]
    return [(a_steps[i], 0.5 * ((dts[i - 1] if i else 0.0) + dts[i]), dts[i]) for i in range(len(dts))]


@pytest.mark.slow
def test_density_loss_gradient_matches_finite_differences():
    n = 8
    w = inputs.c4_workload(n, boxsize=200.0 * n / 128, steps=3)
    steps = _schedule(w["a_steps"], w["Om"], w["OL"])
    amp = torch.from_numpy(w["amp"])
    with torch.no_grad():
        target = adj.density_model(torch.from_numpy(w["target_noise"]), amp, w["d_ratio"], w["vfac"], steps,
                                   w["Om"], n)
    loss, grad = adj.density_loss_grad(w["noise"], target, w["amp"], w["d_ratio"], w["vfac"], steps, w["Om"], n)
    rng = np.random.Generator(np.random.PCG64(6))

    def L(noise):
        with torch.no_grad():
            rho = adj.density_model(torch.from_numpy(noise), amp, w["d_ratio"], w["vfac"], steps, w["Om"], n)
        return float(((rho - target) ** 2).sum())

    for _ in range(4):
        u = rng.standard_normal((n, n, n))
        u /= np.linalg.norm(u)
        eps = 1e-5
        fd = (L(w["noise"] + eps * u) - L(w["noise"] - eps * u)) / (2 * eps)
        an = float((grad.numpy() * u).sum())
        assert abs(fd - an) <= 1e-5 * abs(an) + 1e-9 * loss, (fd, an)
