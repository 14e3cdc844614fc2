"""Pins of the oracle's f(R) scalaron solver (CPU)."""
import numpy as np
import pytest

from oracle import fr, mesh, poisson
from oracle.cosmology import c_tilde


def test_cubic_root_all_branches_vs_numpy_roots():
    rng = np.random.default_rng(0)
    p = np.concatenate([[0.0], rng.uniform(0.01, 3, 50), rng.uniform(-3, -0.01, 200), rng.uniform(-1e-4, 1e-4, 20)])
    q = -rng.uniform(1e-6, 2.0, p.size)
    u = fr.depressed_cubic_root(p, q)
    d0, d1 = -3 * p, 27 * q
    disc = d1 ** 2 - 4 * d0 ** 3
    assert np.any((p < 0) & (disc > 0)) and np.any((p < 0) & (disc <= 0)) and np.any(p > 0)
    for pi, qi, ui in zip(p, q, u):
        r = np.roots([1.0, 0.0, pi, qi])
        pos = r[(np.abs(r.imag) < 1e-9) & (r.real > 0)].real
        assert pos.size == 1
        assert ui == pytest.approx(pos[0], rel=1e-9, abs=1e-12)


def test_cubic_root_vs_bisection_operating_range():
    """The f(R) regime: p close to -1, small negative q."""
    rng = np.random.default_rng(1)
    p = -1.0 + rng.uniform(-0.05, 0.05, 100)
    q = -rng.uniform(1e-4, 1e-2, 100)
    u = fr.depressed_cubic_root(p, q)
    lo, hi = np.zeros_like(p), np.full_like(p, 10.0)
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        neg = mid ** 3 + p * mid + q < 0
        lo = np.where(neg, mid, lo)
        hi = np.where(neg, hi, mid)
    assert np.abs(u - 0.5 * (lo + hi)).max() < 1e-13


def test_q_negative(golden):
    for a in (0.05, 0.3, 1.0):
        fbar, kappa, _ = fr.background(a, fr.FRModel())
        assert fbar < 0 and (1.0 / 64) ** 2 * kappa / (6 * fbar) < 0


def test_background_today_is_fR0():
    m = fr.FRModel(fR0=-3e-6)
    fbar, _, _ = fr.background(1.0, m)
    assert fbar == pytest.approx(-3e-6, rel=1e-15)


def test_uniform_density_fixed_point():
    n = 8
    m = fr.FRModel(boxsize=8.0)
    fbar, kappa, _ = fr.background(0.5, m)
    u = np.ones((n, n, n))
    assert np.abs(fr.operator(u, 1.0 / n, fbar, kappa)).max() == 0.0
    fr.gs_sweep(u, np.zeros_like(u), 1.0 / n, fbar, kappa)
    assert np.abs(u - 1.0).max() < 1e-13


def _yukawa_prediction(delta, a, model, n):
    """Linearised field equation: (lambda_k - mu^2) df_k = -(Om a / c~^2) delta_k,
    mu^2 = a^4 R~ / (6 c~^2 |fbar|), lambda_k the 7-point Laplacian symbol."""
    h = 1.0 / n
    Rbar = 3 * model.Om * (a ** -3 + 4 * model.OL / model.Om)
    Rbar0 = 3 * model.Om * (1 + 4 * model.OL / model.Om)
    fbar = a * a * model.fR0 * (Rbar0 / Rbar) ** 2
    c2 = c_tilde(model.boxsize) ** 2
    mu2 = a ** 4 * Rbar / (6 * c2 * abs(fbar))
    m = np.fft.fftfreq(n) * n
    mz = np.fft.rfftfreq(n) * n
    lam = -(4 / h ** 2) * (np.sin(np.pi * m / n)[:, None, None] ** 2 + np.sin(np.pi * m / n)[None, :, None] ** 2
                            + np.sin(np.pi * mz / n)[None, None, :] ** 2)
    dk = np.fft.rfftn(delta)
    dfk = -(model.Om * a / c2) * dk / (lam - mu2)
    return np.fft.irfftn(dfk, s=delta.shape, axes=(0, 1, 2)), fbar, mu2


def test_linear_regime_matches_yukawa_closed_form():
    n = 16
    a = 0.6
    model = fr.FRModel(boxsize=16.0)
    i = np.arange(n)
    delta = 1e-4 * (np.cos(2 * np.pi * 2 * i / n)[:, None, None] + np.sin(2 * np.pi * 5 * i / n)[None, None, :])
    delta = np.broadcast_to(delta, (n, n, n)).copy()
    rho = 1.0 + delta
    u, hist = fr.fr_solve(rho, a, model, prm=fr.FASParams(coarsest=4), tol=1e-11)
    df_pred, fbar, mu2 = _yukawa_prediction(delta, a, model, n)
    df = fbar * (u * u - 1.0)
    assert np.abs(df - df_pred).max() < 2e-3 * np.abs(df_pred).max()


def test_force_enhancement_limits():
    """Fifth force: the combined potential phi - (c~^2/2) f~_R is 4/3 of the
    Newtonian one for k^2 >> mu^2 and equal to it for k^2 << mu^2 (§2.x / §3.10)."""
    n = 16
    i = np.arange(n)
    for boxsize, m, lo, hi in ((1.0, 1, 1.30, 1.34), (1000.0, 1, 1.0, 1.02)):
        model = fr.FRModel(boxsize=boxsize)
        a = 1.0
        delta = np.broadcast_to(1e-5 * np.cos(2 * np.pi * m * i / n)[:, None, None], (n, n, n)).copy()
        u, _ = fr.fr_solve(1.0 + delta, a, model, prm=fr.FASParams(coarsest=4), tol=1e-9)
        phiN = poisson.solve_fft7(1.5 * a * model.Om * delta, 1.0 / n)
        Phi = phiN + fr.scalaron_potential(u, a, model)
        gN = mesh.force_from_potential(phiN, 1.0 / n)[0]
        g = mesh.force_from_potential(Phi, 1.0 / n)[0]
        ratio = np.abs(g).max() / np.abs(gN).max()
        assert lo < ratio < hi, (boxsize, ratio)


def test_fas_f_cycle_rate(golden):
    n = 32
    model = fr.FRModel(boxsize=32.0)
    rng = np.random.default_rng(1)
    rho = np.exp(0.8 * rng.standard_normal((n, n, n)))
    rho /= rho.mean()
    u, hist = fr.fr_solve(rho, 0.5, model, prm=fr.FASParams(coarsest=4), cycles=3)
    rate = (hist[0] / hist[-1]) ** (1 / 3)
    assert rate > golden["multigrid_convergence"]["f_cycle"] / 2
    assert u.min() > 0


# ------------------------------------------------------------------ n = 2 --

def test_quartic_root_vs_numpy_roots():
    """u^4 + p u + q = 0, q < 0: the closed form of §3.10 gives the unique
    positive root for either sign of p, tiny |p| included."""
    rng = np.random.default_rng(2)
    p = np.concatenate([[0.0], rng.uniform(0.01, 3, 60), rng.uniform(-3, -0.01, 60), rng.uniform(-1e-4, 1e-4, 30),
                        -1.0 + rng.uniform(-0.05, 0.05, 30)])
    q = -rng.uniform(1e-6, 2.0, p.size)
    u = fr.depressed_quartic_root(p, q)
    for pi, qi, ui in zip(p, q, u):
        r = np.roots([1.0, 0.0, 0.0, pi, qi])
        pos = r[(np.abs(r.imag) < 1e-7) & (r.real > 0)].real
        assert pos.size == 1
        assert ui == pytest.approx(pos[0], rel=1e-9, abs=1e-12), (pi, qi)


def test_quartic_root_vs_bisection_operating_range():
    rng = np.random.default_rng(3)
    p = -1.0 + rng.uniform(-0.05, 0.05, 100)
    q = -rng.uniform(1e-4, 1e-2, 100)
    u = fr.depressed_quartic_root(p, q)
    lo, hi = np.zeros_like(p), np.full_like(p, 10.0)
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        neg = mid ** 4 + p * mid + q < 0
        lo = np.where(neg, mid, lo)
        hi = np.where(neg, hi, mid)
    assert np.abs(u - 0.5 * (lo + hi)).max() < 1e-13


def test_n2_background_and_fixed_point():
    m = fr.FRModel(fR0=-1e-5, n=2, boxsize=8.0)
    assert fr.background(1.0, m)[0] == pytest.approx(-1e-5, rel=1e-15)
    Rb = 3 * 0.3 * (0.5 ** -3 + 4 * 0.7 / 0.3)
    R0 = 3 * 0.3 * (1 + 4 * 0.7 / 0.3)
    assert fr.background(0.5, m)[0] == pytest.approx(0.25 * -1e-5 * (R0 / Rb) ** 3, rel=1e-14)
    fbar, kappa, _ = fr.background(0.5, m)
    u = np.ones((8, 8, 8))
    assert np.abs(fr.operator(u, 1.0 / 8, fbar, kappa, 2)).max() == 0.0
    fr.gs_sweep(u, np.zeros_like(u), 1.0 / 8, fbar, kappa, 2)
    assert np.abs(u - 1.0).max() < 1e-13


def test_n2_linear_regime_matches_yukawa_closed_form():
    """Linearised with f~_R = fbar (1 + x): (1 + x)^(-1/3) - 1 ~ -x/3, so the
    mass term is mu^2 = a^4 R~ / (9 c~^2 |fbar|) for n = 2."""
    n, a = 16, 0.6
    model = fr.FRModel(boxsize=16.0, n=2)
    i = np.arange(n)
    delta = 1e-4 * (np.cos(2 * np.pi * 2 * i / n)[:, None, None] + np.sin(2 * np.pi * 5 * i / n)[None, None, :])
    delta = np.broadcast_to(delta, (n, n, n)).copy()
    u, _ = fr.fr_solve(1.0 + delta, a, model, prm=fr.FASParams(coarsest=4), tol=1e-11)
    h = 1.0 / n
    fbar, _, c2 = fr.background(a, model)
    Rbar = 3 * model.Om * (a ** -3 + 4 * model.OL / model.Om)
    mu2 = a ** 4 * Rbar / (9 * c2 * abs(fbar))
    m = np.fft.fftfreq(n) * n
    mz = np.fft.rfftfreq(n) * n
    lam = -(4 / h ** 2) * (np.sin(np.pi * m / n)[:, None, None] ** 2 + np.sin(np.pi * m / n)[None, :, None] ** 2
                            + np.sin(np.pi * mz / n)[None, None, :] ** 2)
    pred = np.fft.irfftn(-(model.Om * a / c2) * np.fft.rfftn(delta) / (lam - mu2), s=delta.shape, axes=(0, 1, 2))
    df = fbar * (u ** 3 - 1.0)
    assert np.abs(df - pred).max() < 2e-3 * np.abs(pred).max()


def _fas_problem(n, seed, a=0.7):
    rng = np.random.Generator(np.random.PCG64(seed))
    g = rng.standard_normal((n, n, n))
    rho = np.exp(0.5 * g)
    rho /= rho.mean()
    model = fr.FRModel(Om=0.3, OL=0.7, fR0=-1e-5, boxsize=float(n))
    fbar, kappa, _ = fr.background(a, model)
    return fr.source(rho, a, model), fbar, kappa


@pytest.mark.parametrize("nh", [1, 2])
def test_gs_sweep_solves_each_cell_in_colour_order(nh):
    """One non-linear Gauss-Seidel sweep (§3.10), checked against the operator
    N_h rather than the root formulas: every cell with i + j + k even (red,
    updated first) satisfies N_h(u) = b exactly with the old values of its
    neighbours, and every odd cell with the new red values around it.  A swapped
    colour order, a wrong sign of b or kappa in p, or a missing 1/6 leaves a
    residual of order 0.1 of the operator's scale."""
    n, h = 8, 1.0 / 8
    rng = np.random.Generator(np.random.PCG64(7))
    rho = np.exp(0.5 * rng.standard_normal((n, n, n)))
    rho /= rho.mean()
    model = fr.FRModel(Om=0.3, OL=0.7, fR0=-1e-5, boxsize=float(n), n=nh)
    fbar, kappa, _ = fr.background(0.7, model)
    b = fr.source(rho, 0.7, model)
    u0 = 1.0 + 0.05 * rng.standard_normal((n, n, n))
    u = fr.gs_sweep(u0.copy(), b, h, fbar, kappa, n=nh)
    i, j, k = np.indices((n, n, n))
    red = (i + j + k) % 2 == 0
    scale = 6.0 * abs(fbar) / (h * h) * np.max(u ** (nh + 1))
    r_red_old = (b - fr.operator(np.where(red, u, u0), h, fbar, kappa, n=nh))[red]
    r_final = b - fr.operator(u, h, fbar, kappa, n=nh)
    assert np.max(np.abs(r_red_old)) < 1e-10 * scale
    assert np.max(np.abs(r_final[~red])) < 1e-10 * scale
    assert np.max(np.abs(r_final[red])) > 1e-3 * scale      # red cells saw the old black values
    assert np.all(u != u0)


def test_f_cycle_is_its_steps_in_order():
    """A three-level FAS F-cycle (16^3 over 8^3 over a 4^3 coarsest level)
    equals, bit for bit, the sequence written out here (§3.6.2 for the FAS
    coarse problem; the F-cycle reading: pre-smooth, FAS coarse problem,
    F-cycle on it, correction, then a V-cycle on this level).  Running the
    V-cycle first instead changes the result."""
    n, h = 16, 1.0 / 16
    b, fbar, kappa = _fas_problem(n, 41)
    prm = fr.FASParams(coarsest=4)
    got = fr.fas_f_cycle(np.ones((n, n, n)), b, h, fbar, kappa, prm)

    def smooth(u, bb, hh, k):
        for _ in range(k):
            fr.gs_sweep(u, bb, hh, fbar, kappa)

    def coarse_problem(u, bb, hh):
        smooth(u, bb, hh, 2)                                  # pre-smooth
        d = bb - fr.operator(u, hh, fbar, kappa)
        uH = poisson.restrict(u)
        return uH, uH.copy(), fr.operator(uH, 2 * hh, fbar, kappa) + poisson.restrict(d)

    def v8(u, bb):                                           # V-cycle on the 8^3 level
        u4, r4, b4 = coarse_problem(u, bb, 2 * h)
        fr._coarse(u4, b4, 4 * h, fbar, kappa, prm)
        u += poisson.prolong(u4 - r4)
        smooth(u, bb, 2 * h, 2)

    u = np.ones((n, n, n))
    u8, r8, b8 = coarse_problem(u, b, h)                     # 16: pre-smooth, FAS problem on 8
    u4, r4, b4 = coarse_problem(u8, b8, 2 * h)               # F-cycle on 8: FAS problem on 4,
    fr._coarse(u4, b4, 4 * h, fbar, kappa, prm)              # solved (coarsest),
    u8 += poisson.prolong(u4 - r4)                           # corrected,
    v8(u8, b8)                                               # then a V-cycle on 8
    u += poisson.prolong(u8 - r8)                            # correct 16
    v_u8, v_r8, v_b8 = coarse_problem(u, b, h)               # V-cycle on 16: FAS problem on 8,
    v8(v_u8, v_b8)                                           # V-cycle there,
    u += poisson.prolong(v_u8 - v_r8)                        # correct,
    smooth(u, b, h, 2)                                       # post-smooth
    assert np.array_equal(got, u)

    alt = np.ones((n, n, n))
    fr.fas_v_cycle(alt, b, h, fbar, kappa, prm)
    fr.fas_f_cycle(alt, b, h, fbar, kappa, fr.FASParams(coarsest=16))   # V first, then the smoother
    assert not np.allclose(got, alt, rtol=0, atol=1e-12)


def test_fas_coarsest_solve_reaches_its_drop_in_fp64():
    """The non-linear coarsest-level solve stops on the 1e-3 drop inside its
    sweep cap in float64, from the background u = 1."""
    n, h = 16, 1.0 / 16
    for seed in (1, 2):
        b, fbar, kappa = _fas_problem(n, seed)
        u = np.ones((n, n, n))
        r0 = np.linalg.norm(b - fr.operator(u, h, fbar, kappa))
        fr._coarse(u, b, h, fbar, kappa, fr.FASParams(coarse_max_sweeps=150))
        assert np.linalg.norm(b - fr.operator(u, h, fbar, kappa)) <= 1e-3 * r0
