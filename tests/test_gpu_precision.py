"""Precision of the multigrid residual.  The solver keeps the iterate in
float32 and forms the finest-level residual f - L(phi) with compensated
float32 arithmetic (every difference and partial sum kept exactly by
TwoSum), accumulating its norm in float64.  That residual is what an outer
refinement loop would compute in float64: the norm the solver reports
matches the float64 residual of the float32 iterate it returns, cycle after
cycle down to the float32 floor, where a plain float32 evaluation of the
same residual is off by orders of magnitude."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import mesh
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


def test_compensated_residual_is_the_fp64_residual_256(pm):
    n = 256
    h = 1.0 / n
    f32 = inputs.random_field(n, 81).astype(np.float32)
    mean32 = np.float32(f32.astype(np.float64).mean())
    src = (f32 - mean32).astype(np.float64)                 # the float32 source the kernels see, exactly
    ws = pm.workspace(n, 0, pm.PM_WS_MG)
    f_t = torch.from_numpy(f32).cuda()
    rows = []
    for k in (1, 2, 4, 8, 16):
        phi, st = pm.mg_solve(f_t, ws=ws, tol=1e-30, max_cycles=k, stall=0.0)
        p32 = phi.cpu().numpy()
        r64 = np.linalg.norm(src - mesh.laplacian7(p32.astype(np.float64), h))
        nb32 = sum(np.roll(p32, s, ax) for ax in range(3) for s in (1, -1)).astype(np.float32)
        r32 = np.linalg.norm((src.astype(np.float32) - (nb32 - np.float32(6) * p32) * np.float32(n * n))
                             .astype(np.float64))
        rows.append((k, st["res"], r64, r32))
        assert st["res"] == pytest.approx(r64, rel=1e-4), rows
    # at the float32 floor (the last cycles) a plain float32 residual is far off
    k, res, r64, r32 = rows[-1]
    assert abs(r32 - r64) > 100 * abs(res - r64), rows
    assert rows[-1][2] < 1e-5 * np.linalg.norm(src)
