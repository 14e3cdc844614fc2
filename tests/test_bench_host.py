"""Host logic of bench.py without a GPU: the CPU leg that scores the GPU's
results against the oracle."""
import numpy as np

import bench


def test_refine_probe_errors_against_the_exact_inverse():
    """The bench's CPU leg for the Poisson precision forms: a potential equal
    to the oracle's exact inverse up to a constant scores 0, and one off by a
    known relative amount scores that amount."""
    from oracle import poisson
    n = 16
    rng = np.random.Generator(np.random.PCG64(3))
    f = rng.standard_normal((n, n, n)).astype(np.float32)
    exact = poisson.solve_fft7(f.astype(np.float64), 1.0 / n)
    noise = rng.standard_normal((n, n, n))
    noise -= noise.mean()
    noise *= 1e-3 * np.linalg.norm(exact) / np.linalg.norm(noise)
    probe = {"kind": "refine", "n": n, "f": f, "phi32": (exact + noise).astype(np.float32),
             "phi64": exact + 0.25}
    out = bench.oracle_errors({"p": probe})["p"]
    assert out["refined_rel_l2"] < 1e-14
    assert 0.99e-3 < out["plain_rel_l2"] < 1.01e-3


def test_patch_probe_scoring_equals_the_full_grid_oracle():
    """The bench scores sampled accelerations with the oracle's Table 1
    gradient and inverse TSC evaluated on the 7^3 cells around each particle
    only.  On a random potential that local evaluation must equal the oracle
    on the whole grid (gradient everywhere, then interpolation), and a known
    relative perturbation of the accelerations must score as that amount."""
    from oracle import mesh
    n, P = 16, 300
    rng = np.random.Generator(np.random.PCG64(5))
    phi = rng.standard_normal((n, n, n))
    pos = rng.uniform(0.0, 1.0, (P, 3))
    full = mesh.interp_tsc(mesh.force_from_potential(phi, 1.0 / n, 5), pos)
    i0 = np.floor(pos * n).astype(np.int64)
    d = np.arange(-3, 4)
    ii, jj, kk = ((i0[:, ax, None] + d) % n for ax in range(3))
    patches = phi[ii[:, :, None, None], jj[:, None, :, None], kk[:, None, None, :]]
    probe = {"kind": "patch", "n": n, "a": 0.5, "step": 0, "pos": pos, "phi": patches, "eps": None}
    exact = bench.oracle_errors({"p": dict(probe, acc=full)})["p"]["rel_l2_acc"]
    off = bench.oracle_errors({"p": dict(probe, acc=full * (1.0 + 1e-3))})["p"]["rel_l2_acc"]
    assert exact < 1e-13
    assert abs(off - 1e-3) < 1e-9
