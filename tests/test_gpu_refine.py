"""Mixed-precision iterative refinement of the Poisson solve (mg_solve_refine):
float32 multigrid corrections on float64 residuals of a float64 iterate reach
the exact inverse of the 7-point Laplacian (the oracle's FFT_7pt, §3.7) far
below the float32 solve's floor, and report the float64 residual."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import mesh, poisson
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


def rel_l2(x, y):
    return float(np.linalg.norm(x - y) / np.linalg.norm(y))


def centred(x):
    return x - x.mean()


@pytest.mark.parametrize("n", [32, 128])
def test_refined_solve_reaches_the_exact_inverse_below_float32(pm, n):
    f = inputs.random_field(n, 33).astype(np.float32)
    h = 1.0 / n
    exact = poisson.solve_fft7(f.astype(np.float64), h)          # zero mean
    ft = torch.from_numpy(f).cuda()
    phi32, st32 = pm.mg_solve(ft, tol=1e-9, max_cycles=40, coarsest=16)
    phi64, st = pm.mg_solve_refine(ft, outer=5, fixed_cycles=3, coarsest=16)
    e32 = rel_l2(centred(phi32.cpu().numpy().astype(np.float64)), exact)
    e64 = rel_l2(centred(phi64.cpu().numpy()), exact)
    assert st["status"] == 0
    assert e64 < 1e-11, (e32, e64)
    assert e64 < 1e-3 * e32, (e32, e64)
    assert st["res"] < 1e-5 * st["res0"]
    assert st["cycles"] == 5 * 3


def test_reported_residual_is_the_float64_residual(pm):
    n = 64
    f = inputs.random_field(n, 34).astype(np.float32)
    h = 1.0 / n
    phi64, st = pm.mg_solve_refine(torch.from_numpy(f).cuda(), outer=1, fixed_cycles=2)
    u = phi64.cpu().numpy()
    fd = f.astype(np.float64)
    r = (fd - fd.mean()) - mesh.laplacian7(u, h)
    assert st["res"] == pytest.approx(np.linalg.norm(r), rel=1e-9)
    assert st["norm_f"] == pytest.approx(np.linalg.norm(fd - fd.mean()), rel=1e-12)
    assert st["res0"] == pytest.approx(st["norm_f"], rel=1e-12)     # from phi = 0


def test_refinement_resumes_bitwise_from_its_own_result(pm):
    """Two calls of two steps (the second from the first's phi) equal one call
    of four: nothing but phi carries over between steps."""
    n = 64
    ft = torch.from_numpy(inputs.random_field(n, 35).astype(np.float32)).cuda()
    a, _ = pm.mg_solve_refine(ft, outer=2, fixed_cycles=2)
    a, _ = pm.mg_solve_refine(ft, a, outer=2, fixed_cycles=2)
    b, _ = pm.mg_solve_refine(ft, outer=4, fixed_cycles=2)
    assert torch.equal(a, b)
