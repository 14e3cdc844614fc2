"""Parity at the benchmark's full size (512^3 cells) and launch configuration,
on sampled outputs the oracle computes one by one, plus properties that hold
at any size."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import fr as ofr
from oracle import mesh, poisson
from paper_2410_20501_gb300 import inputs

pytestmark = pytest.mark.gpu

N = 512


@pytest.fixture(scope="module")
def pm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import os
    from paper_2410_20501_gb300 import build, pm as _pm
    if not os.path.exists(_pm.LIB_PATH):
        build.build()
    _pm.lib()
    return _pm


@pytest.fixture(scope="module")
def densities():
    """Two seeded lognormal densities: rho1 is rho0 after a small evolution
    (as between two time steps), both float32-representable."""
    g = inputs.random_field(N, 51)
    rho0 = np.exp(0.7 * g)
    rho0 /= rho0.mean()
    rho1 = rho0 * (1.0 + 0.01 * inputs.random_field(N, 52))
    return rho0.astype(np.float32), rho1.astype(np.float32)


@pytest.mark.parametrize("cycles", [2])
def test_fullsize_warm_start_accelerations_sampled(pm, densities, cycles):
    rho0, rho1 = densities
    a, Om = 0.5, 0.3
    s = 1.5 * a * Om
    f0 = torch.from_numpy(rho0).cuda() * s
    f1 = torch.from_numpy(rho1).cuda() * s
    phi, st0 = pm.mg_solve(f0, tol=1e-7, max_cycles=20)
    phi, st1 = pm.mg_solve(f1, phi=phi, fixed_cycles=cycles, first_guess=pm.MG_GUESS_SCALED, guess_scale=1.0)
    g = pm.gradient(phi)
    X = inputs.uniform_particles(10000, 53)
    acc = pm.interp(g, pm.positions_to_device(X)).cpu().numpy()
    del g, phi, f0, f1
    torch.cuda.empty_cache()
    f1_64 = s * rho1.astype(np.float64)
    ref_phi = poisson.solve_fft7(f1_64 - f1_64.mean(), 1.0 / N)
    ref_g = mesh.force_from_potential(ref_phi, 1.0 / N)
    ref = mesh.interp_tsc(ref_g, mesh.positions_from_fixed_point(X)).T
    err = np.linalg.norm(acc - ref) / np.linalg.norm(ref)
    assert err < 1e-5, err


def test_fullsize_deposit_sampled_cells(pm):
    """Displaced lattice (at most 0.45 cell): the particles that reach a cell
    are known by index, so the oracle sums them cell by cell."""
    rng = np.random.Generator(np.random.PCG64(54))
    disp = rng.uniform(-0.45, 0.45, (3, N ** 3)).astype(np.float64)
    X = inputs.to_fixed_point(inputs.lattice(N) + disp / N)
    rho = pm.deposit(pm.positions_to_device(X), N)
    cells = rng.integers(0, N, (200, 3))
    flat = torch.from_numpy((cells[:, 0] * N + cells[:, 1]) * N + cells[:, 2]).cuda()
    got = rho.reshape(-1)[flat].cpu().numpy()
    for c, v in zip(cells, got):
        idx = []
        for di in (-1, 0, 1):
            for dj in (-1, 0, 1):
                for dk in (-1, 0, 1):
                    i, j, k = (c[0] + di) % N, (c[1] + dj) % N, (c[2] + dk) % N
                    idx.append((i * N + j) * N + k)
        pos = mesh.positions_from_fixed_point(X[:, idx])
        d = pos * N - (c + 0.5)
        d -= N * np.rint(d / N)
        ref = np.prod(mesh.w_tsc(d), axis=1).sum()       # n^3 / N_p = 1
        assert abs(v - ref) <= 2e-6 * max(1.0, abs(ref))


def test_fullsize_fr_f_cycle_reduces_residual(pm, densities):
    """One FAS F-cycle at 512^3 from the background: the float64 residual of
    the discrete equation (oracle operator) drops by more than 10."""
    rho0, _ = densities
    model = ofr.FRModel(Om=0.3, OL=0.7, fR0=-1e-5, boxsize=512.0)
    a = 0.6
    eps, st = pm.fr_solve(torch.from_numpy(rho0).cuda(), a=a, Om=0.3, OL=0.7, fR0=-1e-5, boxsize=512.0, cycles=1)
    e = eps.cpu().numpy().astype(np.float64)
    fbar, kappa, _ = ofr.background(a, model)
    b = ofr.source(rho0.astype(np.float64), a, model)
    h = 1.0 / N
    r1 = np.linalg.norm(b - ofr.operator(1.0 + e, h, fbar, kappa))
    r0 = np.linalg.norm(b - ofr.operator(np.ones_like(e), h, fbar, kappa))
    assert np.isfinite(e).all() and e.min() > -1.0
    assert r1 < r0 / 10.0


def test_fullsize_fft7_accelerations_sampled(pm, densities):
    """The FFT_7pt path at 512^3 against the oracle's exact 7-point inverse,
    at 10^4 sampled particles."""
    _, rho1 = densities
    s = 1.5 * 0.5 * 0.3
    phi = pm.poisson_fft(torch.from_numpy(rho1).cuda(), scale=s, kind=pm.PM_POISSON_FFT7)
    g = pm.gradient(phi)
    X = inputs.uniform_particles(10000, 53)
    acc = pm.interp(g, pm.positions_to_device(X)).cpu().numpy()
    del g, phi
    torch.cuda.empty_cache()
    f1_64 = s * rho1.astype(np.float64)
    ref_phi = poisson.solve_fft7(f1_64 - f1_64.mean(), 1.0 / N)
    ref_g = mesh.force_from_potential(ref_phi, 1.0 / N)
    ref = mesh.interp_tsc(ref_g, mesh.positions_from_fixed_point(X)).T
    err = np.linalg.norm(acc - ref) / np.linalg.norm(ref)
    assert err < 1e-5, err

