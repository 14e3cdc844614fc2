"""Hu-Sawicki f(R) scalaron (n = 1 and n = 2) in supercomoving units (oracle; test infrastructure only).

Units (§3.1, §3.10): f~_R = a^2 f_R; the background curvature in simulation units
is R~ = 3 Omega_m (a^-3 + 4 Omega_L / Omega_m) (the 3 m^2 (...) of §2.x with
m^2 L^2 = Omega_m / c~^2, the 1/c~^2 written explicitly in the equations); the
background scalaron is f~_R = a^2 (R0/R)^(n+1) f_R0.  With u = (f~_R / fbar)^(1/(n+1))
the field equation Eq. fr_sim_2 discretised with the 7-point Laplacian is

    N_h(u) = (fbar / h^2) (L(u^(n+1)) - 6 u^(n+1)) - kappa (1/u - 1) = b,
    kappa = a^4 R~ / (3 c~^2),   b = -(Omega_m a / c~^2) (rho~ - <rho~>)

whose per-cell Gauss-Seidel update (multiply by h^2 u / (6 fbar)) is
u^(n+2) + p u + q = 0 with p = h^2 (b - kappa) / (6 fbar) - L(u^(n+1))/6 and
q = h^2 kappa / (6 fbar): the depressed cubic for n = 1 (Eq. cubic_equation)
and the quartic for n = 2 (§3.10).  Eq. fr_depressed_equation prints the
exponent as n + 1; both special cases the paper then solves have n + 2, which
is what the algebra gives, and that is the reading used here.
"""
from dataclasses import dataclass

import numpy as np

from .cosmology import c_tilde
from .mesh import neighbour_sum
from .poisson import parity, restrict, prolong


@dataclass
class FRModel:
    Om: float = 0.3
    OL: float = 0.7
    fR0: float = -1e-5
    boxsize: float = 512.0   # Mpc/h
    n: int = 1               # Hu-Sawicki exponent (1 or 2)


def background(a, model):
    """(fbar, kappa, c~^2) at scale factor a (§2.x R-bar and f_R-bar; §3.10
    units).  fbar < 0."""
    Rbar = 3.0 * model.Om * (a ** -3.0 + 4.0 * model.OL / model.Om)
    Rbar0 = 3.0 * model.Om * (1.0 + 4.0 * model.OL / model.Om)
    fbar = a * a * model.fR0 * (Rbar0 / Rbar) ** (model.n + 1)
    c2 = c_tilde(model.boxsize) ** 2
    kappa = a ** 4 * Rbar / (3.0 * c2)
    return fbar, kappa, c2


def depressed_cubic_root(p, q):
    """Root of u^3 + p u + q = 0 by the closed form of Eq. cubic_equation
    (four branches on the sign of p and of Delta_1^2 - 4 Delta_0^3, with
    Delta_0 = -3p, Delta_1 = 27q).  For q < 0 this is the unique positive root.
    Only defined here for q < 0, which holds for n = 1 (q = h^2 kappa/(6 fbar))."""
    p, q = np.broadcast_arrays(np.asarray(p, dtype=np.float64), np.asarray(q, dtype=np.float64))
    d0 = -3.0 * p
    d1 = 27.0 * q
    disc = d1 * d1 - 4.0 * d0 ** 3
    out = np.empty(p.shape)
    zero = p == 0.0
    cardano = (p > 0.0) | ((p < 0.0) & (disc > 0.0))
    trig = ~zero & ~cardano
    out[zero] = np.cbrt(-q[zero])
    # C^3 = (Delta_1 + sqrt(disc)) / 2, evaluated as the algebraically equal
    # 2 Delta_0^3 / (Delta_1 - sqrt(disc)): for q < 0 (Delta_1 < 0) the printed
    # sum cancels catastrophically when |p| is small, the quotient does not.
    C = np.cbrt(2.0 * d0[cardano] ** 3 / (d1[cardano] - np.sqrt(disc[cardano])))
    out[cardano] = -(C + d0[cardano] / C) / 3.0
    cos_t = d1[trig] / (2.0 * d0[trig] ** 1.5)
    theta = np.arccos(np.clip(cos_t, -1.0, 1.0))
    out[trig] = -2.0 * np.sqrt(d0[trig]) * np.cos(theta / 3.0 + 2.0 * np.pi / 3.0) / 3.0
    return out


def depressed_quartic_root(p, q):
    """Root of u^4 + p u + q = 0 by the closed form of §3.10 (n = 2):
    Delta_0 = 12 q, Delta_1 = 27 p^2, Q = [(Delta_1 + sqrt(Delta_1^2 - 4 Delta_0^3))/2]^(1/3),
    S = (1/2) sqrt((Q + Delta_0/Q)/3); u = -S + sqrt(-4S^2 + p/S)/2 for p > 0,
    S + sqrt(-4S^2 - p/S)/2 for p < 0, (-q)^(1/4) for p = 0 and wherever
    Delta_1^2 - 4 Delta_0^3 < 0 or Q + Delta_0/Q <= 0 (the paper's rule).
    For q < 0 the root is the unique positive one.  Q + Delta_0/Q is formed as
    (Q^3 - |Delta_0|^(3/2)) (Q + |Delta_0|^(1/2)) / (Q (Q^2 + Q |Delta_0|^(1/2) + |Delta_0|))
    with Q^3 - |Delta_0|^(3/2) = (Delta_1 + Delta_1^2 / (sqrt(Delta_1^2 + 4|Delta_0|^3)
    + 2 |Delta_0|^(3/2))) / 2: algebraically the printed expression, without the
    cancellation it suffers for small p when Delta_0 < 0."""
    p, q = np.broadcast_arrays(np.asarray(p, dtype=np.float64), np.asarray(q, dtype=np.float64))
    out = np.power(-np.minimum(q, 0.0), 0.25)
    d0 = 12.0 * q
    d1 = 27.0 * p * p
    disc = d1 * d1 - 4.0 * d0 ** 3
    ok = (p != 0.0) & (disc >= 0.0) & (q < 0.0)
    A = -d0[ok]                                              # |Delta_0| (Delta_0 < 0 for q < 0)
    sq = np.sqrt(disc[ok])
    Q3 = 0.5 * (d1[ok] + sq)
    Q = np.cbrt(Q3)
    rA = np.sqrt(A)
    diff3 = 0.5 * (d1[ok] + d1[ok] ** 2 / (sq + 2.0 * A * rA))    # Q^3 - A^(3/2)
    s_arg = diff3 * (Q + rA) / (Q * (Q * Q + Q * rA + A))         # Q + Delta_0 / Q
    good = s_arg > 0.0
    S = 0.5 * np.sqrt(np.where(good, s_arg, 1.0) / 3.0)
    pp = p[ok]
    r = np.where(pp > 0.0, -S + 0.5 * np.sqrt(np.maximum(-4.0 * S * S + pp / S, 0.0)),
                 S + 0.5 * np.sqrt(np.maximum(-4.0 * S * S - pp / S, 0.0)))
    sub = out[ok]
    sub[good] = r[good]
    out[ok] = sub
    return out


def operator(u, h, fbar, kappa, n=1):
    """N_h(u) (module docstring)."""
    un = u ** (n + 1)
    return (fbar / (h * h)) * (neighbour_sum(un) - 6.0 * un) - kappa * (1.0 / u - 1.0)


def gs_sweep(u, b, h, fbar, kappa, n=1):
    """One red-black non-linear Gauss-Seidel sweep: each cell takes the root of
    its cubic (n = 1) or quartic (n = 2) given its neighbours (§3.10; no
    over-relaxation for the non-linear solver, Appendix C).  In place."""
    par = parity(u.shape[0])
    beta = h * h / (6.0 * fbar)
    q = beta * kappa
    root = depressed_cubic_root if n == 1 else depressed_quartic_root
    for colour in (0, 1):
        p = beta * (b - kappa) - neighbour_sum(u ** (n + 1)) / 6.0
        m = par == colour
        u[m] = root(p[m], q)
    return u


@dataclass
class FASParams:
    npre: int = 2
    npost: int = 2
    coarsest: int = 16
    coarse_drop: float = 1e-3
    coarse_max_sweeps: int = 200


def _coarse(u, b, h, fbar, kappa, prm, n=1):
    """Coarsest level: non-linear Gauss-Seidel sweeps until the residual has
    dropped by ``coarse_drop`` or ``coarse_max_sweeps`` sweeps have run (the
    paper leaves the coarsest-level method open; same reading as the linear
    solver's)."""
    r0 = np.linalg.norm(b - operator(u, h, fbar, kappa, n))
    for _ in range(prm.coarse_max_sweeps):
        gs_sweep(u, b, h, fbar, kappa, n)
        if np.linalg.norm(b - operator(u, h, fbar, kappa, n)) <= prm.coarse_drop * r0:
            break
    return u


def _to_coarse(u, b, h, fbar, kappa, prm, n=1):
    """Pre-smooth, then the FAS coarse problem (§3.6.2):
    u_H = R u_h, b_H = N_H(R u_h) + R d_h."""
    for _ in range(prm.npre):
        gs_sweep(u, b, h, fbar, kappa, n)
    d = b - operator(u, h, fbar, kappa, n)
    uH = restrict(u)
    bH = operator(uH, 2.0 * h, fbar, kappa, n) + restrict(d)
    return uH, uH.copy(), bH


def fas_v_cycle(u, b, h, fbar, kappa, prm, n=1):
    """FAS V-cycle (§3.6.2): coarse problem as in _to_coarse, recurse,
    u_h += P(u_H - R u_h), post-smooth.  In place."""
    if u.shape[0] <= prm.coarsest:
        return _coarse(u, b, h, fbar, kappa, prm, n)
    uH, RuH, bH = _to_coarse(u, b, h, fbar, kappa, prm, n)
    fas_v_cycle(uH, bH, 2.0 * h, fbar, kappa, prm, n)
    u += prolong(uH - RuH)
    for _ in range(prm.npost):
        gs_sweep(u, b, h, fbar, kappa, n)
    return u


def fas_f_cycle(u, b, h, fbar, kappa, prm, n=1):
    """FAS F-cycle: pre-smooth, restrict, F-cycle on the coarse level, prolong
    and correct, then one V-cycle on this level (the paper names F-cycles
    without defining them; this is the reading used throughout).  In place."""
    if u.shape[0] <= prm.coarsest:
        return _coarse(u, b, h, fbar, kappa, prm, n)
    uH, RuH, bH = _to_coarse(u, b, h, fbar, kappa, prm, n)
    fas_f_cycle(uH, bH, 2.0 * h, fbar, kappa, prm, n)
    u += prolong(uH - RuH)
    return fas_v_cycle(u, b, h, fbar, kappa, prm, n)


def source(rho, a, model):
    """b = -(Omega_m a / c~^2)(rho~ - <rho~>) (Eq. fr_sim_2, density term)."""
    c2 = c_tilde(model.boxsize) ** 2
    return -(model.Om * a / c2) * (rho - rho.mean())


def fr_solve(rho, a, model, u0=None, prm=None, cycles=1, cycle="F", tol=None, max_cycles=100):
    """Scalaron u on the grid of rho.  Starts from u0 (the previous step's u,
    no rescaling, §3.10) or the background u = 1, then runs ``cycles`` cycles of
    type ``cycle`` (one F-cycle is the paper's default) or, when ``tol`` is
    given, cycles until ||b - N(u)|| <= tol ||b||.  Returns (u, residual norms)."""
    prm = prm or FASParams()
    n = rho.shape[0]
    h = 1.0 / n
    fbar, kappa, _ = background(a, model)
    b = source(rho, a, model)
    u = np.ones_like(rho) if u0 is None else np.array(u0, dtype=np.float64)
    step = fas_f_cycle if cycle == "F" else fas_v_cycle
    nh = model.n
    hist = [np.linalg.norm(b - operator(u, h, fbar, kappa, nh))]
    nb = np.linalg.norm(b)
    ncyc = max_cycles if tol is not None else cycles
    for _ in range(ncyc):
        if tol is not None and hist[-1] <= tol * nb:
            break
        step(u, b, h, fbar, kappa, prm, nh)
        hist.append(np.linalg.norm(b - operator(u, h, fbar, kappa, nh)))
    return u, hist


def scalaron_potential(u, a, model):
    """-(c~^2/2) f~_R with f~_R = fbar u^(n+1): the term that, added to the
    Newtonian potential, gives F = F_N + (c~^2/2) grad f~_R (§3.10)."""
    fbar, _, c2 = background(a, model)
    return -0.5 * c2 * fbar * u ** (model.n + 1)
