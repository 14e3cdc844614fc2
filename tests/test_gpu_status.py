"""Solver failure statuses, made on the host: a source with a NaN (PM_ENAN)
and a tolerance that one cycle cannot meet (PM_ENOCONV).  The solvers run a
bounded number of cycles and sweeps in both cases, so nothing waits on the
GPU; the library stays usable afterwards."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2410_20501_gb300 import inputs

pytestmark = pytest.mark.gpu

PM_ENOCONV, PM_ENAN = 3, 4


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


def _source(n, seed=3):
    return torch.from_numpy(inputs.random_field(n, seed).astype(np.float32)).cuda()


def _density(n, seed=4):
    r = np.exp(0.5 * inputs.random_field(n, seed))
    return torch.from_numpy((r / r.mean()).astype(np.float32)).cuda()


@pytest.mark.parametrize("n", [32, 128])
def test_mg_nan_source_reports_enan(pm, n):
    f = _source(n)
    f[n // 3, 1, 2] = float("nan")
    with pytest.raises(pm.PMError) as e:
        pm.mg_solve(f, tol=1e-7, max_cycles=5)
    assert e.value.code == PM_ENAN


def test_fr_nan_density_reports_enan(pm):
    n = 32
    rho = _density(n)
    rho[5, 6, 7] = float("nan")
    with pytest.raises(pm.PMError) as e:
        pm.fr_solve(rho, a=0.5, Om=0.3, OL=0.7, fR0=-1e-5, boxsize=float(n), tol=1e-6, max_cycles=3)
    assert e.value.code == PM_ENAN


@pytest.mark.parametrize("n", [32, 128])
def test_mg_unreachable_tolerance_reports_enoconv(pm, n):
    _, st = pm.mg_solve(_source(n), tol=1e-30, max_cycles=1, stall=0.0)
    assert st["status"] == PM_ENOCONV and st["cycles"] == 1
    assert np.isfinite(st["res"]) and st["res"] > 0.0


@pytest.mark.parametrize("n", [32, 128])
def test_fr_unreachable_tolerance_reports_enoconv(pm, n):
    _, st = pm.fr_solve(_density(n), a=0.5, Om=0.3, OL=0.7, fR0=-1e-5, boxsize=float(n), tol=1e-30,
                        max_cycles=1)
    assert st["status"] == PM_ENOCONV and st["cycles"] == 1


def test_library_usable_after_failures(pm):
    """A normal solve right after the failing ones converges."""
    _, st = pm.mg_solve(_source(32), tol=1e-6, max_cycles=20)
    assert st["status"] == 0
