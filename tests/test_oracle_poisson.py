"""Pins of the oracle's Poisson solvers (CPU)."""
import itertools

import numpy as np
import pytest

from oracle import mesh, poisson


def test_fft7_sine_plane_wave_closed_form():
    n = 16
    h = 1.0 / n
    i = np.arange(n)
    m = (2, 0, 3)
    f = np.sin(2 * np.pi * (m[0] * i[:, None, None] + m[2] * i[None, None, :]) / n) * np.ones((1, n, 1))
    lam = -(4.0 / h ** 2) * sum(np.sin(np.pi * mm / n) ** 2 for mm in m)
    assert np.abs(poisson.solve_fft7(f, h) - f / lam).max() < 1e-14 * np.abs(f / lam).max() * 10


def test_fft7_equals_dense_direct_solve_8cubed():
    """Dense 512 x 512 system assembled cell by cell from the 7-point stencil,
    solved with the zero-mean constraint by least squares."""
    n = 8
    h = 1.0 / n
    N = n ** 3
    A = np.zeros((N, N))
    idx = lambda i, j, k: ((i % n) * n + (j % n)) * n + (k % n)
    for i, j, k in itertools.product(range(n), repeat=3):
        r = idx(i, j, k)
        A[r, r] -= 6.0 / h ** 2
        for d in ((1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)):
            A[r, idx(i + d[0], j + d[1], k + d[2])] += 1.0 / h ** 2
    f = np.random.default_rng(0).standard_normal(N)
    f -= f.mean()
    Ac = np.vstack([A, np.ones((1, N))])
    u = np.linalg.lstsq(Ac, np.append(f, 0.0), rcond=None)[0]
    phi = poisson.solve_fft7(f.reshape(n, n, n), h).ravel()
    assert np.abs(u - phi).max() < 1e-12 * np.abs(phi).max()


def test_restrict_and_prolong_basic(golden):
    rng = np.random.default_rng(1)
    d = rng.standard_normal((8, 8, 8))
    assert poisson.restrict(d).mean() == pytest.approx(d.mean(), abs=1e-15)
    w = golden["prolongation_weights"]["by_near_axes"]
    assert [poisson.PROLONG_WEIGHT_BY_NEAR_AXES[k] for k in range(4)] == [w[str(k)] for k in range(4)]
    # weights of one fine cell sum to one: 27 + 3*9 + 3*3 + 1 = 64
    assert poisson.prolong(np.ones((4, 4, 4))) == pytest.approx(np.ones((8, 8, 8)), abs=1e-15)
    # a single coarse spike spreads exactly the printed weights to its children's neighbourhood
    vH = np.zeros((4, 4, 4))
    vH[1, 1, 1] = 1.0
    P = poisson.prolong(vH)
    assert P[2, 2, 2] == pytest.approx(27 / 64)     # child, all three axes near
    assert P[1, 2, 2] == pytest.approx(9 / 64)      # one axis far
    assert P[1, 1, 2] == pytest.approx(3 / 64)
    assert P[1, 1, 1] == pytest.approx(1 / 64)
    assert P[0, 2, 2] == 0.0                         # beyond 1.5 fine cells


def test_prolong_reproduces_linear_fields_in_interior():
    nH = 8
    I = np.arange(nH) + 0.5                          # coarse centres in coarse units
    vH = np.broadcast_to(3.0 * I[:, None, None] - 2.0 * I[None, None, :], (nH, nH, nH))
    P = poisson.prolong(np.ascontiguousarray(vH))
    i = (np.arange(2 * nH) + 0.5) / 2.0              # fine centres in coarse units
    exact = 3.0 * i[:, None, None] - 2.0 * i[None, None, :]
    sl = slice(2, 2 * nH - 2)
    assert np.abs(P[sl, :, sl] - np.broadcast_to(exact, P.shape)[sl, :, sl]).max() < 1e-12


def test_jacobi_first_guess(golden):
    f = np.random.default_rng(2).standard_normal((4, 4, 4))
    h = 0.25
    assert poisson.jacobi_first_guess(f, h) == pytest.approx(golden["jacobi_first_guess_factor"]["value"] * h * h * f)


def test_multigrid_converges_to_fft7():
    n = 32
    h = 1.0 / n
    f = np.random.default_rng(3).standard_normal((n, n, n))
    prm = poisson.MGParams(coarsest=4, tol=1e-12)
    u, hist = poisson.mg_solve(f, h, prm=prm)
    phi = poisson.solve_fft7(f, h)
    assert hist[-1] <= 1e-12 * np.linalg.norm(f - f.mean())
    assert np.abs((u - u.mean()) - phi).max() < 1e-10 * np.abs(phi).max()


@pytest.mark.parametrize("omega,key", [(1.0, "v_no_sor"), (1.25, "v_sor_1p25")])
def test_multigrid_convergence_rate(golden, omega, key):
    """Appendix C: a V-cycle cuts the residual by ~10x without SOR and 20-30x
    with omega = 1.25 (soft: within a factor 2 of the printed rate)."""
    n = 32
    h = 1.0 / n
    f = np.random.default_rng(4).standard_normal((n, n, n))
    prm = poisson.MGParams(coarsest=4, omega=omega)
    _, hist = poisson.mg_solve(f, h, prm=prm, cycles=5)
    rate = (hist[1] / hist[-1]) ** (1.0 / 4)
    assert rate > golden["multigrid_convergence"][key] / 2


def test_truncation_error_of_smooth_field_is_second_order():
    errs = []
    for n in (16, 32):
        h = 1.0 / n
        x = (np.arange(n) + 0.5) * h
        u = np.broadcast_to(np.sin(2 * np.pi * x)[:, None, None], (n, n, n)).copy()
        errs.append(np.abs(poisson.truncation_error(u, mesh.laplacian7(u, h), h)).max())
    assert np.log2(errs[0] / errs[1]) == pytest.approx(2.0, abs=0.15)


def test_fft_tsc_plane_wave_closed_form():
    """A cosine source along y: phi = -f / (k^2 W(k)^2) with k = 2 pi m and
    W = sinc(pi m / n)^3 (the other two axes contribute sinc(0) = 1)."""
    n, m = 16, 3
    c = (np.arange(n) + 0.5) / n
    f = np.cos(2 * np.pi * m * c)[None, :, None] * np.ones((n, n, n))
    phi = poisson.solve_fft_tsc(f, 1.0 / n)
    x = np.pi * m / n
    W = (np.sin(x) / x) ** 3
    np.testing.assert_allclose(phi, -f / ((2 * np.pi * m) ** 2 * W * W), atol=1e-13)


def test_fft_tsc_removes_the_mean_and_is_linear():
    rng = np.random.Generator(np.random.PCG64(4))
    f, g = rng.standard_normal((2, 8, 8, 8))
    a = poisson.solve_fft_tsc(f + 3.0, 1.0 / 8)
    assert abs(a.mean()) < 1e-14
    np.testing.assert_allclose(poisson.solve_fft_tsc(2 * f - g, 1.0 / 8),
                               2 * poisson.solve_fft_tsc(f, 1.0 / 8) - poisson.solve_fft_tsc(g, 1.0 / 8),
                               atol=1e-12)


def test_rbgs_sweep_point_source_by_hand():
    """One sweep from u = 0 with a unit source in red cell (0, 0, 0), h = 1 on a
    4^3 grid, worked by hand from Eq. jacobi_sweep_laplacian with SOR: the red
    pass sets u_000 = -omega/6 (its neighbours are still 0); the black pass then
    gives each of the six neighbours omega (u_000 / 6) and leaves the other
    black cells at 0.  A black-first sweep would leave the neighbours at 0."""
    for omega in (1.0, 1.25):
        f = np.zeros((4, 4, 4))
        f[0, 0, 0] = 1.0
        u = poisson.rbgs_sweep(np.zeros((4, 4, 4)), f, 1.0, omega)
        expect = np.zeros((4, 4, 4))
        expect[0, 0, 0] = -omega / 6.0
        for d in ((1, 0, 0), (3, 0, 0), (0, 1, 0), (0, 3, 0), (0, 0, 1), (0, 0, 3)):
            expect[d] = omega * (-omega / 6.0) / 6.0
        assert np.abs(u - expect).max() < 1e-15
    # a source in a black cell: the red pass sees only zeros, so only that cell moves
    f = np.zeros((4, 4, 4))
    f[1, 0, 0] = 1.0
    u = poisson.rbgs_sweep(np.zeros((4, 4, 4)), f, 1.0, 1.25)
    expect = np.zeros((4, 4, 4))
    expect[1, 0, 0] = -1.25 / 6.0
    assert np.abs(u - expect).max() < 1e-15


def test_sweep_omegas_reading():
    """§3.6.1 "omit SOR on the first and last iterations", read per level visit:
    omega = 1 on the first pre-sweep and on the last post-sweep only."""
    assert poisson.sweep_omegas(2, 1.25, True, False) == [1.0, 1.25]
    assert poisson.sweep_omegas(2, 1.25, False, True) == [1.25, 1.0]
    assert poisson.sweep_omegas(3, 1.25, True, False) == [1.0, 1.25, 1.25]
    assert poisson.sweep_omegas(1, 1.25, False, True) == [1.0]
    assert poisson.sweep_omegas(0, 1.25, True, False) == []


def test_v_cycle_is_its_steps_in_order():
    """A two-level V-cycle (8^3 over a 4^3 coarsest level) equals, bit for bit,
    the sequence written out here: sweeps with omega 1 then 1.25, residual,
    restriction, coarsest solve of the error from zero, prolongation and
    correction, sweeps with omega 1.25 then 1.  Swapping the SOR factors of the
    pre-sweeps changes the result."""
    n, h = 8, 1.0 / 8
    rng = np.random.Generator(np.random.PCG64(31))
    f = rng.standard_normal((n, n, n))
    f -= f.mean()
    u0 = 1e-3 * rng.standard_normal((n, n, n))
    prm = poisson.MGParams(coarsest=4)
    got = poisson.v_cycle(u0.copy(), f, h, prm)

    def written_out(w_pre):
        u = u0.copy()
        for w in w_pre:
            poisson.rbgs_sweep(u, f, h, w)
        fH = poisson.restrict(f - mesh.laplacian7(u, h))
        vH = poisson.coarse_solve(np.zeros_like(fH), fH, 2 * h, prm)
        u += poisson.prolong(vH)
        poisson.rbgs_sweep(u, f, h, 1.25)
        poisson.rbgs_sweep(u, f, h, 1.0)
        return u

    assert np.array_equal(got, written_out((1.0, 1.25)))
    assert not np.allclose(got, written_out((1.25, 1.0)), rtol=0, atol=1e-12)


def test_coarsest_solve_rate_is_youngs_optimum():
    """With Young's optimal factor the asymptotic residual reduction per
    red-black SOR sweep is omega_opt - 1 (0.634 at 16^3); a wrong Jacobi
    eigenvalue in the factor's formula moves the measured rate off it."""
    n = 16
    h = 1.0 / n
    w = poisson.optimal_sor_omega(n)
    assert w == pytest.approx(1.634, abs=5e-4)
    rng = np.random.Generator(np.random.PCG64(32))
    f = rng.standard_normal((n, n, n))
    f -= f.mean()
    u = np.zeros((n, n, n))
    r = []
    for _ in range(80):
        poisson.rbgs_sweep(u, f, h, w)
        u -= u.mean()
        r.append(np.linalg.norm(poisson.residual(u, f, h)))
    rate = (r[-1] / r[-21]) ** (1.0 / 20)
    assert rate == pytest.approx(w - 1.0, rel=0.1)
    for other in (1.25, 1.9):      # both converge more slowly
        v = np.zeros((n, n, n))
        for _ in range(40):
            poisson.rbgs_sweep(v, f, h, other)
        assert np.linalg.norm(poisson.residual(v, f, h)) > r[39]


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_coarsest_solve_reaches_its_drop_in_fp64(seed):
    """The coarsest-level solve stops on the 1e-3 drop well inside its
    200-sweep cap on 16^3 levels in float64 (no other stopping rule is
    needed at this precision)."""
    n = 16
    h = 1.0 / 16
    rng = np.random.Generator(np.random.PCG64(seed))
    f = rng.standard_normal((n, n, n))
    f -= f.mean()
    r0 = np.linalg.norm(f)
    prm = poisson.MGParams(coarse_max_sweeps=60)
    u = poisson.coarse_solve(np.zeros((n, n, n)), f, h, prm)
    assert np.linalg.norm(poisson.residual(u, f, h)) <= 1e-3 * r0
