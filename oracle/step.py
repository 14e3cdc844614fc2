"""Force evaluation and kick-drift-kick leapfrog (oracle; test infrastructure only)."""
from dataclasses import dataclass, field

import numpy as np

from . import fr as frmod
from .cosmology import dt_supercomoving, growth_factors, mu_parametrised
from .mesh import deposit_tsc, force_from_potential, interp_tsc
from .poisson import MGParams, mg_solve, solve_fft7


@dataclass
class PMParams:
    n: int = 32
    Om: float = 1.0
    OL: float = 0.0
    boxsize: float = 64.0
    gravity: str = "newton"          # "newton", "fr" or "mu" (parametrised)
    fR0: float = -1e-5
    mu0: float = 0.0                 # parametrised gravity: coupling today
    fr_n: int = 1                    # Hu-Sawicki exponent (1 or 2)
    grad_order: int = 5
    solver: str = "fft7"             # "fft7" (exact discrete inverse) or "mg"
    mg: MGParams = field(default_factory=MGParams)
    fr_cycles: int = 1


def poisson_source(rho, a, Om):
    """Right-hand side 3/2 a Omega_m (rho~ - <rho~>) of the supercomoving
    Poisson equation (§3.1)."""
    return 1.5 * a * Om * (rho - rho.mean())


def accelerations(pos, a, prm, phi_guess=None, u_guess=None):
    """One PM force evaluation (§3.4-§3.10): TSC deposit, Poisson solve (exact
    discrete inverse, or the paper's multigrid from ``phi_guess``), for f(R) the
    scalaron (one F-cycle from ``u_guess``) combined as
    F = -grad(phi) + (c~^2/2) grad f~_R, finite-difference gradient and
    inverse-TSC interpolation.  Returns (acc [N,3], phi, u or None)."""
    n = prm.n
    h = 1.0 / n
    rho = deposit_tsc(pos, n)
    f = poisson_source(rho, a, prm.Om)
    if prm.gravity == "mu":      # nabla^2 psi = 4 pi G mu(a) a^2 delta rho (Eq. parametrized_newtonian_equation)
        f = f * mu_parametrised(a, prm.Om, prm.OL, prm.mu0)
    if prm.solver == "fft7":
        phi = solve_fft7(f, h)
    else:
        phi, _ = mg_solve(f, h, u0=phi_guess, prm=prm.mg)
    Phi = phi
    u = None
    if prm.gravity == "fr":
        model = frmod.FRModel(Om=prm.Om, OL=prm.OL, fR0=prm.fR0, boxsize=prm.boxsize, n=prm.fr_n)
        u, _ = frmod.fr_solve(rho, a, model, u0=u_guess, cycles=prm.fr_cycles)
        Phi = phi + frmod.scalaron_potential(u, a, model)
    g = force_from_potential(Phi, h, prm.grad_order)
    return interp_tsc(g, pos), phi, u


def run_kdk(pos, vel, a_steps, prm, warm_start=True):
    """Kick-drift-kick leapfrog (§3.4 Integrator) through the scale factors
    a_steps[0] -> a_steps[-1]: v += a dt/2; x += v dt; v += a dt/2, with
    dt = t~(a_{i+1}) - t~(a_i) (supercomoving time, §3.1) and periodic wrap.
    With the multigrid solver the previous potential, rescaled by
    a1 D1 / (a0 D0), is the first guess (Eq. rescaming_newtonian_potential as
    read for the supercomoving potential).  Returns (pos, vel)."""
    pos = np.array(pos, dtype=np.float64) % 1.0
    vel = np.array(vel, dtype=np.float64)
    D = growth_factors(np.asarray(a_steps), prm.Om, prm.OL)[0]
    acc, phi, u = accelerations(pos, a_steps[0], prm)
    for i in range(len(a_steps) - 1):
        a0, a1 = a_steps[i], a_steps[i + 1]
        dt = dt_supercomoving(a0, a1, prm.Om, prm.OL)
        vel += 0.5 * dt * acc
        pos = (pos + dt * vel) % 1.0
        guess = phi * (a1 * D[i + 1]) / (a0 * D[i]) if warm_start else None
        acc, phi, u = accelerations(pos, a1, prm, phi_guess=guess, u_guess=u)
        vel += 0.5 * dt * acc
    return pos, vel


def next_timestep(a, Om, OL, n, max_acc, max_vel, courant=0.8, da_max=0.02, a_end=1.0):
    """The adaptive time step of §3.4 (Integrator), in supercomoving time:
    the smallest of (i) the time over which a grows by the fraction da_max,
    (ii) the free-fall time sqrt(h / max|a|) and (iii) the cell-crossing time
    h / max|v| (h = 1/n; a criterion with a zero maximum does not apply),
    times the Courant factor; a step that would pass a_end stops there.
    Returns (dt, a reached after dt), the latter by root finding on the
    monotone t(a)."""
    from scipy.optimize import brentq
    h = 1.0 / n
    limits = [dt_supercomoving(a, a * (1.0 + da_max), Om, OL)]
    if max_acc > 0.0:
        limits.append(np.sqrt(h / max_acc))
    if max_vel > 0.0:
        limits.append(h / max_vel)
    dt = courant * min(limits)
    to_end = dt_supercomoving(a, a_end, Om, OL)
    if to_end <= dt:
        return to_end, a_end
    a_next = brentq(lambda x: dt_supercomoving(a, x, Om, OL) - dt, a, a_end, xtol=1e-16, rtol=1e-15, maxiter=500)
    return dt, a_next
