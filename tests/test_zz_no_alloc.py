"""pm_deposit_noalloc, the deposit for callers that cannot allocate device
memory (a host application whose pool owns the device, a path that must not
pay cudaMalloc's implicit synchronisation, a binding with no device
allocator): it takes its scratch from a static array inside the library
instead of a caller workspace.  Checked through the C ABI against pm_deposit
on two calls in a row, so the second call also shows that contents left in
the shared array by the first do not leak into its result.  This file is
collected last on purpose."""
import ctypes

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


def _noalloc(pm, X, n):
    rho = torch.empty((n, n, n), dtype=torch.float32, device="cuda")
    code = pm.lib().pm_deposit_noalloc(ctypes.c_void_p(X.data_ptr()), X.shape[1], n,
                                       ctypes.c_void_p(rho.data_ptr()), pm._stream())
    assert code == 0, pm.STATUS.get(code, code)
    return rho.cpu().numpy()


def _crowded(n, seed):
    """Uniform particles plus clumps of 100 to 20000 inside single cells: the
    cells whose moments a block sums."""
    rng = np.random.Generator(np.random.PCG64(seed))
    pos = [rng.uniform(0.0, 1.0, (3, 100000))]
    for q, m in enumerate((100, 1000, 20000)):
        c = rng.integers(0, n, 3).astype(np.float64)[:, None]
        pos.append((c + rng.uniform(0.0, 1.0, (3, m))) / n)
    return inputs.to_fixed_point(np.concatenate(pos, axis=1))


def test_noalloc_deposit_matches_pm_deposit_twice(pm):
    """Both entry points run the same sort, permutation and deposit kernels on
    the same buffer layout, so their densities agree bit for bit.  The cases
    run back to back: the first (n = 64, np = 2^18, the largest accepted
    layout) fills the shared array, the later smaller ones run over what it
    left there."""
    cases = [(64, inputs.uniform_particles(1 << 18, 40)),
             (64, inputs.uniform_particles(200000, 41)),
             (32, inputs.to_fixed_point(inputs.lattice(32) + 0.004 * inputs.random_field(32, 2).reshape(1, -1))),
             (64, _crowded(64, 42))]
    for n, Xh in cases:
        X = pm.positions_to_device(Xh)
        got = _noalloc(pm, X, n)
        ref = pm.deposit(X, n).cpu().numpy()
        assert np.array_equal(got, ref)


def test_noalloc_rejects_sizes_beyond_the_limit(pm):
    X = torch.zeros((3, 10), dtype=torch.int32, device="cuda")
    rho = torch.empty(128 ** 3, dtype=torch.float32, device="cuda")
    L = pm.lib()
    assert L.pm_deposit_noalloc(ctypes.c_void_p(X.data_ptr()), 10, 128, ctypes.c_void_p(rho.data_ptr()),
                                pm._stream()) == 1
    assert L.pm_deposit_noalloc(ctypes.c_void_p(X.data_ptr()), (1 << 18) + 1, 64,
                                ctypes.c_void_p(rho.data_ptr()), pm._stream()) == 1
