"""Cells of more than four particles: their 27 TSC moments are summed before
the streaming deposit, by eight lanes per cell up to 13 particles, one warp
per cell up to 256 and one block per cell beyond, in fixed trees.
Deposit, the valued deposit of the interpolation adjoint and the step's
accelerations on clustered particles against the FP64 oracle, and reruns
bitwise equal."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import adjoint as oadj
from oracle import mesh, step
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


def clustered(n, counts, seed, background=0, spread=1.0):
    """counts[q] particles uniformly inside a cube of `spread` cells at cell
    q * 997 % n^3 (plus `background` uniform ones), in seeded random order."""
    rng = np.random.Generator(np.random.PCG64(seed))
    pos = [rng.uniform(0.0, 1.0, (3, background))]
    for q, m in enumerate(counts):
        c = (q * 997) % n ** 3
        ijk = np.array([c // (n * n), (c // n) % n, c % n], dtype=np.float64)[:, None]
        pos.append((ijk + spread * rng.uniform(0.0, 1.0, (3, m))) / n)
    pos = np.concatenate(pos, axis=1)
    return inputs.to_fixed_point(pos[:, rng.permutation(pos.shape[1])])


CASES = [(32, [13, 14, 20, 32, 33, 40, 100, 257, 1000, 5000, 20000], 30000),
         (32, [64, 65, 128, 129, 255, 256, 257, 258, 600], 30000),
         (32, [4, 5, 6, 7, 8, 9, 12, 13] + [5 + q % 9 for q in range(300)], 30000),
         (64, [14, 31, 33, 64, 500, 3000, 12000] + [14 + q % 19 for q in range(200)], 200000)]


@pytest.mark.parametrize("n,counts,background", CASES)
def test_crowded_deposit_matches_oracle(pm, n, counts, background):
    X = clustered(n, counts, 3 + n, background)
    rho = pm.deposit(pm.positions_to_device(X), n).cpu().numpy()
    ref = mesh.deposit_tsc(mesh.positions_from_fixed_point(X), n)
    assert np.abs(rho - ref).max() <= 4e-6 * np.abs(ref).max()
    assert np.array_equal(rho, pm.deposit(pm.positions_to_device(X), n).cpu().numpy())


def test_crowded_interp_adj_matches_oracle(pm):
    n = 32
    X = clustered(n, [5, 9, 13, 40, 700, 6000], 9, 20000)
    rng = np.random.Generator(np.random.PCG64(10))
    g32 = rng.standard_normal((3, n, n, n)).astype(np.float32)
    ab32 = rng.standard_normal((3, X.shape[1])).astype(np.float32)
    gbar, dX = pm.interp_adj(torch.from_numpy(g32).cuda(), pm.positions_to_device(X), torch.from_numpy(ab32).cuda())
    gt = torch.from_numpy(g32.astype(np.float64)).requires_grad_(True)
    pos = torch.from_numpy(mesh.positions_from_fixed_point(X)).requires_grad_(True)
    (oadj.interp([gt[0], gt[1], gt[2]], pos) * torch.from_numpy(ab32.astype(np.float64).T)).sum().backward()
    ref = gt.grad.numpy()
    assert np.linalg.norm(gbar.cpu().numpy() - ref) / np.linalg.norm(ref) < 1e-5


def test_crowded_step_accelerations_match_oracle(pm):
    """A halo-like clump of 20000 particles spread over 3 cells beside uniform
    ones: one step's accelerations against the oracle (exact Poisson)."""
    n = 32
    X = clustered(n, [20000, 3000, 500], 12, 32 ** 3, spread=3.0)
    V = np.zeros((3, X.shape[1]))
    sim = pm.Simulation(X, V, n, Om=0.3, OL=0.7, boxsize=float(n), track_ids=True, keep_acc=True,
                        mg=pm.default_mg(tol=1e-9))
    sim.step(a=0.5, dt_kick=0.0, dt_drift=0.0)
    acc = np.empty((3, X.shape[1]))
    acc[:, sim.particle_ids()] = sim.acc.cpu().numpy()
    ref, _, _ = step.accelerations(mesh.positions_from_fixed_point(X), 0.5,
                                   step.PMParams(n=n, Om=0.3, OL=0.7, boxsize=float(n)))
    assert np.linalg.norm(acc.T - ref) / np.linalg.norm(ref) < 1e-5


@pytest.fixture(scope="module")
def dyn_clustered(pm):
    """A state clustered by the dynamics themselves: 90 Newtonian steps of the
    100-step ln-a schedule from 2LPT at z = 30, 128^3 particles in a 128 Mpc/h
    box (the 1 Mpc/h cells of the 512^3 run).  Returns (n, positions)."""
    import bench
    n = 128
    a = bench.schedule()
    coeffs = bench.step_coefficients(0.3, 0.7, a)
    X, V = inputs.lpt_ics(n, float(n), 0.3, 0.7, a[0], 5, order=2, device="cuda")
    sim = pm.Simulation(X, V, n, 0.3, 0.7, float(n), mg=pm.default_mg(tol=1e-7, fixed_cycles=2))
    for i in range(90):
        sim.step(*coeffs[i])
    return n, sim.positions()


def test_gravitationally_clustered_deposit_matches_oracle(pm, dyn_clustered):
    """Every cell size class of the sort and the deposit occurs in the
    clustered state (walked cells of up to four particles, groups of eight and
    sixteen lanes, a warp); the density against the FP64 oracle."""
    n, Xh = dyn_clustered
    counts = np.bincount(mesh.cell_key(Xh, n).astype(np.int64), minlength=n ** 3)
    for lo, hi in ((5, 13), (14, 32), (33, 256)):
        assert ((counts >= lo) & (counts <= hi)).sum() > 0, (lo, hi)
    rho = pm.deposit(pm.positions_to_device(Xh), n).cpu().numpy()
    ref = mesh.deposit_tsc(mesh.positions_from_fixed_point(Xh), n)
    assert np.abs(rho - ref).max() <= 4e-6 * np.abs(ref).max()
    assert np.array_equal(rho, pm.deposit(pm.positions_to_device(Xh), n).cpu().numpy())


def test_gravitationally_clustered_sort_is_the_stable_order(pm, dyn_clustered):
    """The cell sort of the clustered state, shuffled so that every cell's run
    arrives in pieces: permutation and cell starts bit-exact against the
    oracle's stable order."""
    n, Xh = dyn_clustered
    rng = np.random.Generator(np.random.PCG64(21))
    Xs = np.ascontiguousarray(Xh[:, rng.permutation(Xh.shape[1])])
    perm, cs = pm.sort(pm.positions_to_device(Xs), n)
    ref = mesh.stable_cell_order(Xs, n)
    assert np.array_equal(perm.cpu().numpy().view(np.uint32), ref)
    keys = mesh.cell_key(Xs, n)[ref]
    ref_cs = np.searchsorted(keys, np.arange(n ** 3 + 1), side="left").astype(np.uint32)
    assert np.array_equal(cs.cpu().numpy().view(np.uint32), ref_cs)
