"""The FFT Poisson path (pm_poisson_fft and pm_step with an FFT solver)
against the oracle's FFT_7pt and exact-kernel solvers, converged multigrid
and the oracle's step accelerations."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import mesh, poisson, step
from paper_2410_20501_gb300 import inputs

pytestmark = pytest.mark.gpu


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


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a, dtype=np.float64) - b) / np.linalg.norm(b))


def field(n, seed):
    """A lognormal density (float32-representable) with a spectrum like the
    runs' (large scales dominate)."""
    r = np.exp(0.7 * inputs.random_field(n, seed))
    return (r / r.mean()).astype(np.float32)


@pytest.mark.parametrize("n", [16, 32, 64, 128, 256])
def test_fft7_matches_oracle(pm, n):
    rho = field(n, 70 + n)
    phi = pm.poisson_fft(torch.from_numpy(rho).cuda(), scale=0.45, kind=pm.PM_POISSON_FFT7).cpu().numpy()
    f = 0.45 * rho.astype(np.float64)
    ref = poisson.solve_fft7(f - f.mean(), 1.0 / n)
    # float32 transforms: rounding of order eps32 log2(n^3) relative to |phi|
    err = rel_l2(phi, ref)
    print("fft7", n, err)
    assert err < 1e-7 * np.log2(n ** 3)
    assert abs(float(phi.astype(np.float64).mean())) < 1e-6 * np.abs(ref).max()


@pytest.mark.parametrize("n", [32, 64, 256])
def test_fft_exact_tsc_matches_oracle(pm, n):
    rho = field(n, 90 + n)
    phi = pm.poisson_fft(torch.from_numpy(rho).cuda(), scale=1.2, kind=pm.PM_POISSON_FFT).cpu().numpy()
    f = 1.2 * rho.astype(np.float64)
    ref = poisson.solve_fft_tsc(f, 1.0 / n)
    err = rel_l2(phi, ref)
    print("fft", n, err)
    assert err < 1e-7 * np.log2(n ** 3)


def test_fft7_plane_waves_every_axis(pm):
    """Single Fourier modes along x, y and z (one at the z Nyquist frequency,
    which the z packing treats apart): the transform pairs, the packing and
    the kernel's per-axis factors each exercised alone.  (A mode near the
    Nyquist frequency in x or y is no test at 1e-6: the float32 rounding it
    leaves in the low modes is amplified there by the kernel's 1/k^2, up to
    (k_mode / k_min)^2 = 400 times at m = 31 of 64.)"""
    n = 64
    i = np.arange(n)
    for axis, m in ((0, 5), (1, 3), (2, 32), (2, 1)):
        shape = [1, 1, 1]
        shape[axis] = n
        f = (np.cos(2 * np.pi * m * i / n + 0.3).reshape(shape) * np.ones((n, n, n))).astype(np.float32)
        phi = pm.poisson_fft(torch.from_numpy(f).cuda(), kind=pm.PM_POISSON_FFT7).cpu().numpy()
        ref = poisson.solve_fft7(f.astype(np.float64) - f.mean(dtype=np.float64), 1.0 / n)
        err = rel_l2(phi, ref)
        print("plane", axis, m, err)
        assert err < 2e-6, (axis, m)


def test_fft7_equals_converged_multigrid(pm):
    n = 128
    rho = torch.from_numpy(field(n, 11)).cuda()
    a = pm.poisson_fft(rho, scale=1.0).cpu().numpy().astype(np.float64)
    b, st = pm.mg_solve(rho - rho.mean(), tol=1e-9, max_cycles=40)
    b = b.cpu().numpy().astype(np.float64)
    assert rel_l2(b - b.mean(), a) < 1e-5


@pytest.mark.parametrize("kind", [1, 2])
def test_step_accelerations_with_fft_solvers(pm, kind):
    n = 64
    X, V = inputs.lpt_ics(n, float(n), 0.3, 0.7, 0.25, seed=9, order=2)
    sim = pm.Simulation(X, V, n, Om=0.3, OL=0.7, boxsize=float(n), track_ids=True, keep_acc=True, poisson=kind)
    sim.step(a=0.25, dt_kick=0.0, dt_drift=0.0)
    acc = np.empty((3, n ** 3))
    acc[:, sim.particle_ids()] = sim.acc.cpu().numpy()
    pos = mesh.positions_from_fixed_point(X)
    rho = mesh.deposit_tsc(pos, n)
    f = step.poisson_source(rho, 0.25, 0.3)
    phi = poisson.solve_fft7(f, 1.0 / n) if kind == 1 else poisson.solve_fft_tsc(f, 1.0 / n)
    ref = mesh.interp_tsc(mesh.force_from_potential(phi, 1.0 / n), pos)
    assert rel_l2(acc.T, ref) < 1e-5
