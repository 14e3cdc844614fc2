"""The stages' batched entry points (the `batch` argument of the boundary):
every box of pm_deposit_batch, mg_solve_batch, pm_gradient_batch and
pm_interp_batch equals, bit for bit, the single-box call on that box."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

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


def boxes_of_particles(n, B, np_box, seed):
    """B boxes: a displaced lattice, uniform particles and a clumped box
    (cells above the one-thread limits), np_box particles each."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for b in range(B):
        if b % 3 == 0:
            pos = inputs.lattice(n)[:, :np_box] + rng.uniform(-0.4, 0.4, (3, np_box)) / n
        elif b % 3 == 1:
            pos = rng.uniform(0, 1, (3, np_box))
        else:
            pos = np.concatenate([rng.uniform(0, 1, (3, np_box - 3000)), 0.5 + 0.01 * rng.uniform(0, 1, (3, 3000))], 1)
        out.append(inputs.to_fixed_point(pos))
    return np.concatenate(out, axis=1)


@pytest.mark.parametrize("n,B", [(32, 3), (64, 2)])
def test_deposit_batch_equals_single_boxes(pm, n, B):
    np_box = n ** 3
    X = boxes_of_particles(n, B, np_box, 7 + n)
    rho = pm.deposit_batch(pm.positions_to_device(X), n, B).cpu().numpy()
    for b in range(B):
        one = pm.deposit(pm.positions_to_device(np.ascontiguousarray(X[:, b * np_box:(b + 1) * np_box])), n)
        assert np.array_equal(rho[b], one.cpu().numpy()), b


@pytest.mark.parametrize("n,B", [(32, 3), (64, 3)])
def test_mg_solve_batch_equals_single_boxes(pm, n, B):
    f = torch.from_numpy(np.stack([inputs.random_field(n, 40 + b) for b in range(B)]).astype(np.float32)).cuda()
    phi = pm.mg_solve_batch(f, fixed_cycles=2).cpu().numpy()
    for b in range(B):
        one, _ = pm.mg_solve(f[b].contiguous(), fixed_cycles=2, first_guess=pm.MG_GUESS_JACOBI)
        assert np.array_equal(phi[b], one.cpu().numpy()), b


def test_gradient_and_interp_batch_equal_single_boxes(pm):
    n, B, np_box = 32, 3, 5000
    phi = torch.from_numpy(np.stack([inputs.random_field(n, 60 + b) for b in range(B)]).astype(np.float32)).cuda()
    g = pm.gradient_batch(phi, order=5)
    X = inputs.uniform_particles(B * np_box, 61)
    acc = pm.interp_batch(g, pm.positions_to_device(X)).cpu().numpy()
    for b in range(B):
        gb = pm.gradient(phi[b].contiguous(), order=5)
        assert torch.equal(g[b], gb), b
        Xb = pm.positions_to_device(np.ascontiguousarray(X[:, b * np_box:(b + 1) * np_box]))
        assert np.array_equal(acc[:, b * np_box:(b + 1) * np_box], pm.interp(gb, Xb).cpu().numpy()), b
