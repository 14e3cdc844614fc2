"""The GPU initial conditions (pm_lpt2) against the LPT oracle."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import lpt
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


@pytest.mark.parametrize("n,order", [(16, 2), (32, 1), (32, 2), (64, 2)])
def test_lpt_matches_oracle(pm, n, order):
    L, Om, a = 2.0 * n, 0.3, 1 / 31
    noise = inputs.white_noise(n, 40 + n).astype(np.float32)
    amp = inputs.lpt_amplitude(n, L, Om).astype(np.float32)
    D, E, f1, f2 = inputs.growth([a, 1.0], Om, 1 - Om)
    vfac = a * a * inputs.hubble_E(a, Om, 1 - Om)
    d1 = D[0] / D[1]
    e2 = E[0] / D[1] ** 2 if order == 2 else 0.0
    v1, v2 = vfac * d1 * f1[0], (vfac * e2 * f2[0] if order == 2 else 0.0)
    X, V = pm.lpt2(torch.from_numpy(noise).cuda(), torch.from_numpy(amp).cuda(), d1, e2, v1, v2)
    x_ref, v_ref = lpt.lpt2(noise.astype(np.float64), amp.astype(np.float64), d1, e2, v1, v2)
    q = lpt.lattice(n)
    disp = (X.cpu().numpy().view(np.uint32).astype(np.float64) / 2 ** 32 - q + 0.5) % 1.0 - 0.5
    disp_ref = (x_ref - q + 0.5) % 1.0 - 0.5
    assert rel_l2(disp, disp_ref) < 1e-5
    assert rel_l2(V.cpu().numpy(), v_ref) < 1e-5
