"""The streaming red-black smoother (two sweeps per pass over HBM, levels with
n >= 128) against the colour-by-colour kernels and the oracle."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import fr as ofr
from oracle import poisson
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


@pytest.mark.parametrize("n,guess", [(128, "jacobi"), (256, "jacobi"), (128, "scaled")])
def test_streaming_poisson_bitwise_equals_colour_passes(pm, n, guess):
    f = torch.from_numpy(inputs.random_field(n, 3).astype(np.float32)).cuda()
    outs = []
    for smoother in (0, 1):
        if guess == "jacobi":
            phi, _ = pm.mg_solve(f, fixed_cycles=2, first_guess=pm.MG_GUESS_JACOBI, smoother=smoother)
        else:
            phi0 = torch.from_numpy(inputs.random_field(n, 4).astype(np.float32)).cuda()
            phi, _ = pm.mg_solve(f, phi=phi0, fixed_cycles=1, first_guess=pm.MG_GUESS_SCALED, guess_scale=1.07,
                                 smoother=smoother)
        outs.append(phi.cpu().numpy())
    assert np.array_equal(outs[0], outs[1])


def test_streaming_fr_matches_colour_passes(pm):
    n = 128
    rho = np.exp(0.8 * inputs.random_field(n, 8))
    rho = torch.from_numpy((rho / rho.mean()).astype(np.float32)).cuda()
    outs = []
    for smoother in (0, 1):
        eps, _ = pm.fr_solve(rho, a=0.7, Om=0.3, OL=0.7, fR0=-1e-5, boxsize=float(n), cycles=1, smoother=smoother)
        outs.append(eps.cpu().numpy())
    assert rel_l2(outs[0], outs[1].astype(np.float64)) < 1e-6


def test_streaming_mg_one_cycle_matches_oracle_128(pm):
    n = 128
    f = inputs.random_field(n, 6).astype(np.float32).astype(np.float64)
    phi, _ = pm.mg_solve(torch.from_numpy(f.astype(np.float32)).cuda(), fixed_cycles=1,
                         first_guess=pm.MG_GUESS_JACOBI, smoother=0)
    ref, _ = poisson.mg_solve(f, 1.0 / n, prm=poisson.MGParams(), cycles=1)
    # float32 against float64 after one cycle: bounded by eps32 times the
    # condition number (n / pi)^2 of the 7-point Laplacian
    assert rel_l2(phi.cpu().numpy(), ref) < 6e-8 * (n / np.pi) ** 2


def test_streaming_mg_converged_matches_fft7_256(pm):
    n = 256
    f = inputs.random_field(n, 7).astype(np.float32).astype(np.float64)
    phi, st = pm.mg_solve(torch.from_numpy(f.astype(np.float32)).cuda(), tol=1e-9, max_cycles=40, smoother=0)
    ref = poisson.solve_fft7(f, 1.0 / n)
    phi = phi.cpu().numpy().astype(np.float64)
    assert st["status"] == 0
    assert rel_l2(phi - phi.mean(), ref) < 5e-6
