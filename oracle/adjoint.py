"""Reverse-mode derivatives of the Newtonian PM step (oracle; test infrastructure only).

The forward operators of §3.3-§3.7 (first-order LPT displacement, TSC
assignment, Poisson solve by the exact discrete inverse of the 7-point
Laplacian (FFT_7pt), Table 1 finite-difference gradient, inverse TSC and the
kick-drift update of the leapfrog) written with plain torch float64 CPU
operations, so that torch.autograd supplies their derivatives.  Nothing here is
blocked, fused or reordered: each function is the plain definition, and the
derivatives are whatever autograd makes of it.

Positions are float64 box fractions [N, 3].  The periodic wrap x mod 1 has
derivative 1 almost everywhere and is applied as such.  The floor that picks a
particle's nearest cell is piecewise constant (derivative 0); the TSC kernel is
C1, so the weights and their first derivatives are continuous across it.
"""
import math

import torch

from .mesh import GRADIENT_COEFFS

DT = torch.float64


def w_tsc(x):
    """TSC kernel of §3.4 (0.75 - x^2 for |x| < 1/2, (1.5 - |x|)^2 / 2 for
    1/2 <= |x| < 3/2, 0 beyond), x in cells."""
    ax = x.abs()
    return torch.where(ax < 0.5, 0.75 - x * x, torch.where(ax < 1.5, 0.5 * (1.5 - ax) ** 2, torch.zeros_like(x)))


def tsc_stencil(pos, n):
    """The 27 periodic cell indices [27, N] (int64, flat (i n + j) n + k) and
    weights [27, N] of each particle, weights differentiable in pos."""
    s = pos * n - 0.5
    i0 = torch.floor(s.detach() + 0.5)
    idx, wts = [], []
    for ox in (-1, 0, 1):
        for oy in (-1, 0, 1):
            for oz in (-1, 0, 1):
                c = i0 + torch.tensor([ox, oy, oz], dtype=DT)
                w = w_tsc(s[:, 0] - c[:, 0]) * w_tsc(s[:, 1] - c[:, 1]) * w_tsc(s[:, 2] - c[:, 2])
                ci = torch.remainder(c, n).to(torch.int64)
                idx.append((ci[:, 0] * n + ci[:, 1]) * n + ci[:, 2])
                wts.append(w)
    return torch.stack(idx), torch.stack(wts)


def deposit(pos, n):
    """rho~_c = (n^3 / N) sum_p W(x_p - x_c) (§3.4), [n, n, n]."""
    N = pos.shape[0]
    idx, wts = tsc_stencil(pos, n)
    rho = torch.zeros(n ** 3, dtype=DT).index_add(0, idx.reshape(-1), wts.reshape(-1))
    return (rho * (n ** 3 / N)).reshape(n, n, n)


def interp(fields, pos):
    """Inverse TSC (§3.4): [N, len(fields)] values at the particles."""
    n = fields[0].shape[0]
    idx, wts = tsc_stencil(pos, n)
    return torch.stack([(wts * f.reshape(-1)[idx]).sum(0) for f in fields], dim=-1)


def solve_fft7(f, h):
    """Zero-mean phi with (L(phi) - 6 phi) / h^2 = f - <f>: division by the
    7-point Laplacian's Fourier symbol -(4/h^2) sum_d sin^2(pi m_d / n) (§3.7)."""
    n = f.shape[0]
    m = torch.fft.fftfreq(n, dtype=DT) * n
    mz = torch.fft.rfftfreq(n, dtype=DT) * n
    s2 = lambda mm: torch.sin(math.pi * mm / n) ** 2
    lam = -(4.0 / h ** 2) * (s2(m)[:, None, None] + s2(m)[None, :, None] + s2(mz)[None, None, :])
    lam[0, 0, 0] = 1.0
    fk = torch.fft.rfftn(f)
    phik = fk / lam
    keep = torch.ones_like(lam)
    keep[0, 0, 0] = 0.0
    return torch.fft.irfftn(phik * keep, s=f.shape)


def laplacian7(u, h):
    """(sum of the six face neighbours - 6 u) / h^2 (Eq. 7pt-laplacian)."""
    nb = sum(torch.roll(u, s, dims=a) for a in range(3) for s in (1, -1))
    return (nb - 6.0 * u) / (h * h)


def derivative(u, axis, h, order=5):
    """(1/h) sum_q c_q u_{i+q} with the Table 1 coefficients."""
    out = torch.zeros_like(u)
    for off, c in GRADIENT_COEFFS[order].items():
        out = out + c * torch.roll(u, -off, dims=axis)
    return out / h


def accelerations(pos, a, Om, n, order=5):
    """Newtonian PM accelerations [N, 3] (§3.4-§3.7): deposit, source
    3/2 a Omega_m (rho~ - <rho~>), exact 7-point Poisson solve, g = -grad phi,
    inverse TSC."""
    h = 1.0 / n
    rho = deposit(pos, n)
    f = 1.5 * a * Om * (rho - rho.mean())
    phi = solve_fft7(f, h)
    g = [-derivative(phi, ax, h, order) for ax in range(3)]
    return interp(g, pos)


def kdk_step(pos, vel, a, Om, n, dt_kick, dt_drift, order=5):
    """One fused-kick leapfrog update (§3.4 Integrator): force at the input
    positions, v' = v + dt_kick acc, x' = (x + dt_drift v') mod 1."""
    acc = accelerations(pos, a, Om, n, order)
    v1 = vel + dt_kick * acc
    return torch.remainder(pos + dt_drift * v1, 1.0), v1


def lpt1(noise, amp, d_ratio, vfac):
    """First-order LPT (§3.3) on an n^3 lattice of cell centres from real-space
    white noise [n, n, n]: delta_k = amp_k * FFT(noise)_k (amp = sqrt(P(k) n^3 / L^3),
    zero at k = 0 and on Nyquist planes), Psi solves div Psi = -delta,
    i.e. Psi_k = i k delta_k / k^2, x = q + d_ratio Psi, v = vfac Psi
    (vfac = a^2 E(a) d_ratio f(a)).  Returns (pos [N, 3], vel [N, 3])."""
    n = noise.shape[0]
    m = torch.fft.fftfreq(n, dtype=DT) * n
    mz = torch.fft.rfftfreq(n, dtype=DT) * n
    k = [2 * math.pi * m[:, None, None], 2 * math.pi * m[None, :, None], 2 * math.pi * mz[None, None, :]]
    k2 = k[0] ** 2 + k[1] ** 2 + k[2] ** 2
    k2[0, 0, 0] = 1.0
    dk = torch.fft.rfftn(noise) * amp
    psi = torch.stack([torch.fft.irfftn(1j * kd * dk / k2, s=(n, n, n)).reshape(-1) for kd in k], dim=-1)
    c = (torch.arange(n, dtype=DT) + 0.5) / n
    q = torch.stack(torch.meshgrid(c, c, c, indexing="ij"), dim=-1).reshape(-1, 3)
    return torch.remainder(q + d_ratio * psi, 1.0), vfac * psi


def density_model(noise, amp, d_ratio, vfac, steps, Om, n, order=5):
    """White noise -> LPT -> the fused-kick steps (a, dt_kick, dt_drift) ->
    final TSC density [n, n, n]."""
    pos, vel = lpt1(noise, amp, d_ratio, vfac)
    for a, dtk, dtd in steps:
        pos, vel = kdk_step(pos, vel, a, Om, n, dtk, dtd, order)
    return deposit(pos, n)


def density_loss_grad(noise, target, amp, d_ratio, vfac, steps, Om, n, order=5):
    """(loss, d loss / d noise) of loss = sum_c (rho~_c - target_c)^2."""
    w = torch.as_tensor(noise, dtype=DT).clone().requires_grad_(True)
    rho = density_model(w, torch.as_tensor(amp, dtype=DT), d_ratio, vfac, steps, Om, n, order)
    loss = ((rho - torch.as_tensor(target, dtype=DT)) ** 2).sum()
    loss.backward()
    return float(loss.detach()), w.grad.detach()


def step_vjp(pos, vel, a, Om, n, dt_kick, dt_drift, pos_bar, vel_bar, order=5):
    """Cotangents (pos_bar_in, vel_bar_in) [N, 3] of one kdk_step given the
    output cotangents, by reverse-mode differentiation."""
    x = torch.as_tensor(pos, dtype=DT).clone().requires_grad_(True)
    v = torch.as_tensor(vel, dtype=DT).clone().requires_grad_(True)
    x1, v1 = kdk_step(x, v, a, Om, n, dt_kick, dt_drift, order)
    (x1 * torch.as_tensor(pos_bar, dtype=DT)).sum().add((v1 * torch.as_tensor(vel_bar, dtype=DT)).sum()).backward()
    return x.grad.detach(), v.grad.detach()
