"""Poisson solvers for the 7-point Laplacian (oracle; test infrastructure only).

``solve_fft7`` is the definition of the converged result: the unique zero-mean
phi with (L(phi) - 6 phi)/h^2 = f - <f> (FFT_7pt of §3.7).  ``mg_solve`` is the
paper's linear multigrid written out step by step (§3.5, §3.6.1), used to pin
cycle-by-cycle behaviour.
"""
from dataclasses import dataclass

import numpy as np

from .mesh import neighbour_sum, laplacian7


def solve_fft7(f, h):
    """FFT_7pt (§3.7): phi_k = f_k / lambda_k with the Fourier symbol of the
    7-point Laplacian, lambda_k = -(4/h^2) sum_d sin^2(k_d h / 2)  (the paper's
    printed kernel has a misplaced h; this is its intended reading).  The k = 0
    mode is set to zero, which also removes any mean of f."""
    n = f.shape[0]
    fk = np.fft.rfftn(f)
    m = np.fft.fftfreq(n) * n
    mz = np.fft.rfftfreq(n) * n
    s2 = lambda mm: np.sin(np.pi * mm / n) ** 2
    lam = -(4.0 / h ** 2) * (s2(m)[:, None, None] + s2(m)[None, :, None] + s2(mz)[None, None, :])
    lam[0, 0, 0] = 1.0
    phik = fk / lam
    phik[0, 0, 0] = 0.0
    return np.fft.irfftn(phik, s=f.shape, axes=(0, 1, 2))


def solve_fft_tsc(f, h):
    """FFT solver of §3.7 with the exact Laplacian kernel and the TSC window
    deconvolved: phi_k = -f_k / (k^2 W_TSC(k)^2), k = 2 pi m / (n h) (box
    units for h = 1/n), W_TSC = prod_d sinc(pi m_d / n)^3 (p = 3 of the
    mass-assignment filter), sinc(x) = sin(x)/x; the k = 0 mode is set to zero."""
    n = f.shape[0]
    fk = np.fft.rfftn(f)
    m = np.fft.fftfreq(n) * n
    mz = np.fft.rfftfreq(n) * n
    L = n * h
    k2 = (2.0 * np.pi / L) ** 2 * (m[:, None, None] ** 2 + m[None, :, None] ** 2 + mz[None, None, :] ** 2)
    w = lambda mm: np.sinc(mm / n) ** 3          # numpy sinc(x) = sin(pi x) / (pi x)
    W = w(m)[:, None, None] * w(m)[None, :, None] * w(mz)[None, None, :]
    k2[0, 0, 0] = 1.0
    phik = -fk / (k2 * W * W)
    phik[0, 0, 0] = 0.0
    return np.fft.irfftn(phik, s=f.shape, axes=(0, 1, 2))


def parity(n):
    """(i + j + k) mod 2 on an n^3 grid; red cells are the even ones (§3.5)."""
    i = np.arange(n)
    return (i[:, None, None] + i[None, :, None] + i[None, None, :]) % 2


def rbgs_sweep(u, f, h, omega):
    """One red-black Gauss-Seidel sweep with over-relaxation (§3.5,
    Eq. jacobi_sweep_laplacian, then u = omega u_GS + (1 - omega) u_old),
    red cells first.  In place."""
    par = parity(u.shape[0])
    for colour in (0, 1):
        u_gs = (neighbour_sum(u) - h * h * f) / 6.0
        m = par == colour
        u[m] = omega * u_gs[m] + (1.0 - omega) * u[m]
    return u


def residual(u, f, h):
    """d_h = f_h - L_h u_h (§3.6)."""
    return f - laplacian7(u, h)


def restrict(d):
    """Restriction by averaging the 8 children (§3.6.1)."""
    n = d.shape[0] // 2
    return d.reshape(n, 2, n, 2, n, 2).mean(axis=(1, 3, 5))


# Prolongation weights of §3.6.1, by how many of the three per-axis separations
# (fine-cell centre to coarse-cell centre, in fine cells) are the near one.
PROLONG_WEIGHT_BY_NEAR_AXES = {3: 27.0 / 64.0, 2: 9.0 / 64.0, 1: 3.0 / 64.0, 0: 1.0 / 64.0}


def prolong(vH):
    """Cell-centred prolongation of §3.6.1.  For every fine cell and every
    coarse cell of the 3x3x3 block around its parent, the per-axis separation
    between centres (in fine cells) is 0.5 (near), 1.5 (far) or 2.5; the
    weight is 27/64, 9/64, 3/64 or 1/64 for 3, 2, 1 or 0 near axes and zero if
    any axis is beyond 1.5."""
    nH = vH.shape[0]
    n = 2 * nH
    i = np.arange(n)
    I = i // 2
    out = np.zeros((n, n, n))
    for ox in (-1, 0, 1):
        for oy in (-1, 0, 1):
            for oz in (-1, 0, 1):
                seps = [np.abs((i + 0.5) - (2.0 * (I + o) + 1.0)) for o in (ox, oy, oz)]
                near = [(s == 0.5).astype(int) for s in seps]
                ok = [s <= 1.5 for s in seps]
                nnear = near[0][:, None, None] + near[1][None, :, None] + near[2][None, None, :]
                valid = ok[0][:, None, None] & ok[1][None, :, None] & ok[2][None, None, :]
                table = np.array([PROLONG_WEIGHT_BY_NEAR_AXES[k] for k in range(4)])
                w = table[nnear] * valid
                src = vH[((I + ox) % nH)][:, ((I + oy) % nH)][:, :, ((I + oz) % nH)]
                out += w * src
    return out


@dataclass
class MGParams:
    """Multigrid knobs (§3.6.1): Npre/Npost smoothing sweeps, SOR factor,
    coarsest level size, stopping rule and the coarsest-level sweep rule."""
    npre: int = 2
    npost: int = 2
    omega: float = 1.25
    coarsest: int = 16
    tol: float = 1e-8            # relative residual ||d|| / ||f||
    max_cycles: int = 60
    coarse_drop: float = 1e-3     # coarsest level: sweep until ||d|| drops by this
    coarse_max_sweeps: int = 200
    coarse_omega: float = 0.0     # coarsest-level SOR factor; 0: optimal_sor_omega(coarsest)


def optimal_sor_omega(n):
    """Young's optimal SOR factor 2 / (1 + sqrt(1 - mu^2)) for red-black
    ordering of the periodic 7-point Laplacian on n^3 cells, mu = (2 + cos(2 pi / n)) / 3
    being the Jacobi iteration's largest eigenvalue below 1 (the constant mode,
    mu = 1, is absent from a zero-mean problem)."""
    mu = (2.0 + np.cos(2.0 * np.pi / n)) / 3.0
    return 2.0 / (1.0 + np.sqrt(1.0 - mu * mu))


def coarse_solve(u, f, h, prm):
    """Coarsest level: red-black SOR sweeps (factor ``coarse_omega``, by default
    the optimal one for this grid) until the level residual has dropped by
    ``coarse_drop`` or ``coarse_max_sweeps`` sweeps have run.  §3.6.1 fixes the
    coarsest size (16^3) but not how that level is solved; this is the reading
    used throughout."""
    r0 = np.linalg.norm(residual(u, f, h))
    omega = prm.coarse_omega if prm.coarse_omega > 0 else optimal_sor_omega(u.shape[0])
    for _ in range(prm.coarse_max_sweeps):
        rbgs_sweep(u, f, h, omega)
        if np.linalg.norm(residual(u, f, h)) <= prm.coarse_drop * r0:
            break
    return u


def sweep_omegas(count, omega, first_plain, last_plain):
    """SOR factors for ``count`` sweeps: omega = 1 on the first pre-sweep and on
    the last post-sweep of a cycle, omega elsewhere (§3.6.1, "omit SOR on the
    first and last iterations")."""
    w = [omega] * count
    if count and first_plain:
        w[0] = 1.0
    if count and last_plain:
        w[-1] = 1.0
    return w


def v_cycle(u, f, h, prm):
    """One V-cycle (§3.6.1): pre-smooth, residual, restrict, recurse on the
    error equation with a zero initial guess, prolong, correct, post-smooth.
    In place on u."""
    n = u.shape[0]
    if n <= prm.coarsest:
        return coarse_solve(u, f, h, prm)
    for w in sweep_omegas(prm.npre, prm.omega, True, False):
        rbgs_sweep(u, f, h, w)
    fH = restrict(residual(u, f, h))
    vH = np.zeros_like(fH)
    v_cycle(vH, fH, 2.0 * h, prm)
    u += prolong(vH)
    for w in sweep_omegas(prm.npost, prm.omega, False, True):
        rbgs_sweep(u, f, h, w)
    return u


def jacobi_first_guess(f, h):
    """One Jacobi step from u = 0 (Eq. multigrid_initial_guess): -h^2 f / 6."""
    return -h * h * f / 6.0


def mg_solve(f, h, u0=None, prm=None, cycles=None):
    """Linear multigrid solve of (L(u) - 6u)/h^2 = f - <f>.  Starts from u0 or
    the Jacobi first guess; runs V-cycles until ||d|| <= tol ||f|| (or exactly
    ``cycles`` V-cycles when given).  Returns (u, [||d|| after each cycle])."""
    prm = prm or MGParams()
    f = f - f.mean()
    u = jacobi_first_guess(f, h) if u0 is None else np.array(u0, dtype=np.float64)
    nf = np.linalg.norm(f)
    hist = [np.linalg.norm(residual(u, f, h))]
    ncyc = prm.max_cycles if cycles is None else cycles
    for _ in range(ncyc):
        if cycles is None and hist[-1] <= prm.tol * nf:
            break
        v_cycle(u, f, h, prm)
        hist.append(np.linalg.norm(residual(u, f, h)))
    return u, hist


def truncation_error(u, f, h):
    """tau~_h = L_H(R u_h) - R L_h u_h (§3.6.1, the paper's estimate of the
    truncation error used by the stopping rule |d_h| < alpha tau~_h)."""
    return laplacian7(restrict(u), 2.0 * h) - restrict(laplacian7(u, h))
