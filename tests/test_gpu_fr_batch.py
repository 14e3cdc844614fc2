"""Batched f(R) scalaron (fr_solve_batch, §3.6.2, §3.10): B boxes in one launch
per kernel and level are bitwise the same boxes solved alone by fr_solve, and a
box of the batch matches the oracle's FAS F-cycle."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import fr as ofr
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


def densities(n, B, seed):
    """B lognormal densities of mean 1 with different seeds and contrasts."""
    out = np.empty((B, n, n, n), dtype=np.float32)
    for b in range(B):
        rho = np.exp((0.6 + 0.2 * b) * inputs.random_field(n, seed + b))
        out[b] = (rho / rho.mean()).astype(np.float32)
    return out


def rel_l2(x, y):
    return float(np.linalg.norm(x - y) / np.linalg.norm(y))


COMMON = dict(Om=0.3, OL=0.7, fR0=-1e-5, tol=0.0)


@pytest.mark.parametrize("n,B,nhs,cycle,smoother", [
    (32, 5, 1, 1, 2),     # every level below the fused kernel's; coarsest 16^3 one CTA per box
    (64, 3, 2, 0, 2),     # quartic per cell, V-cycles
    (64, 2, 1, 1, 1),     # colour passes everywhere
    (128, 2, 1, 1, 2),    # fused four-cell sweep on the finest level (ping-pong partner per box)
])
def test_batch_is_bitwise_the_boxes_solved_alone(pm, n, B, nhs, cycle, smoother):
    rho = densities(n, B, 40 + n)
    prm = dict(COMMON, a=0.6, boxsize=float(n), cycles=2, cycle=cycle, smoother=smoother, nhs=nhs)
    guess = np.zeros((B, n, n, n), dtype=np.float32)
    guess[B - 1] = 0.01 * inputs.random_field(n, 7).astype(np.float32)   # one box starts from a non-zero guess
    eps_b = pm.fr_solve_batch(torch.from_numpy(rho).cuda(), torch.from_numpy(guess.copy()).cuda(), **prm)
    torch.cuda.synchronize()
    eps_b = eps_b.cpu().numpy()
    for b in range(B):
        eps_s, _ = pm.fr_solve(torch.from_numpy(rho[b]).cuda(), torch.from_numpy(guess[b].copy()).cuda(), **prm)
        assert np.array_equal(eps_b[b], eps_s.cpu().numpy()), b
    assert not np.array_equal(eps_b[0], eps_b[1])


def test_batch_box_matches_oracle_one_f_cycle(pm):
    n, B, a = 32, 3, 0.5
    rho = densities(n, B, 90)
    eps = pm.fr_solve_batch(torch.from_numpy(rho).cuda(), a=a, boxsize=float(n), coarsest=16, cycles=1, cycle=1,
                            **COMMON)
    eps = eps.cpu().numpy()
    model = ofr.FRModel(Om=0.3, OL=0.7, fR0=-1e-5, boxsize=float(n))
    for b in (0, B - 1):
        u, _ = ofr.fr_solve(rho[b].astype(np.float64), a, model, prm=ofr.FASParams(coarsest=16), cycles=1)
        assert rel_l2(eps[b], u - 1.0) < 1e-4, b


def test_batch_reuses_its_workspace(pm):
    """Two calls on one workspace: the second starts from the first's result
    and equals one call of two cycles (nothing stale is read)."""
    n, B = 64, 2
    rho = torch.from_numpy(densities(n, B, 5)).cuda()
    ws = pm.fr_batch_workspace(n, B)
    prm = dict(COMMON, a=0.9, boxsize=float(n), cycle=1)
    e1 = pm.fr_solve_batch(rho, ws=ws, cycles=1, **prm)
    e1 = pm.fr_solve_batch(rho, e1, ws=ws, cycles=1, **prm)
    e2 = pm.fr_solve_batch(rho, cycles=2, **prm)
    assert torch.equal(e1, e2)
