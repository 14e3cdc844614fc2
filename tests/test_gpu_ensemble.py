"""Batched ensembles (pm_step_batch): B boxes in one launch per kernel are
bitwise the same boxes run alone, a captured CUDA graph replays bitwise the
eager steps, and the batched accelerations match the oracle box by box."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

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


@pytest.fixture(scope="module")
def small():
    # 5 boxes of 32^3 (a non power of two batch), different cosmologies and seeds
    return inputs.ensemble_workload(n=32, B=5, boxsize=64.0, steps=6)


def run(pm, w, boxes, steps, graph=False):
    X, V = w["X"][boxes], w["V"][boxes]
    ens = pm.Ensemble(X, V, w["n"], w["Om"][boxes], w["boxsize"], cold_cycles=8)
    coef = ens.coefficients(w["a_steps"][: steps + 1])
    for i in range(steps):
        if graph and i >= 2:
            if ens.graph is None:
                ens.capture()
            ens.replay_step(coef[i])
        else:
            ens.step(coef[i])
    torch.cuda.synchronize()
    return ens.positions(), ens.velocities()


def test_batch_is_bitwise_the_boxes_run_alone(pm, small):
    Xb, Vb = run(pm, small, list(range(5)), 4)
    for b in range(5):
        Xs, Vs = run(pm, small, [b], 4)
        assert np.array_equal(Xb[b], Xs[0]) and np.array_equal(Vb[b], Vs[0]), b


def test_graph_replay_is_bitwise_the_eager_steps(pm, small):
    Xe, Ve = run(pm, small, list(range(5)), 6)
    Xg, Vg = run(pm, small, list(range(5)), 6, graph=True)
    assert np.array_equal(Xe, Xg) and np.array_equal(Ve, Vg)


def test_batched_accelerations_match_the_oracle(pm, small):
    """One cold step from rest with no drift: V' = acc dt_kick, box by box,
    against the oracle's exact-Poisson accelerations with each box's Omega_m."""
    B, n = 3, 32
    X, Om = small["X"][:B], small["Om"][:B]
    ens = pm.Ensemble(X, np.zeros((B, 3, n ** 3)), n, Om, small["boxsize"], cold_cycles=14)
    a, dtk = 0.1, 1e-2
    row = torch.zeros((4, ens.coef.shape[1]), dtype=torch.float32, device="cuda")
    row[0, :B] = torch.from_numpy((1.5 * a * Om).astype(np.float32))
    row[1, :B] = dtk
    row[3, :B] = 1.0
    ens.step(row)
    Vs = ens.velocities()
    for b in range(B):
        perm = mesh.stable_cell_order(X[b], n)
        acc = np.empty((3, n ** 3))
        acc[:, perm] = Vs[b].astype(np.float64) / np.float32(dtk)
        ref, _, _ = step.accelerations(mesh.positions_from_fixed_point(X[b]), a,
                                       step.PMParams(n=n, Om=float(Om[b]), OL=1.0 - float(Om[b])))
        err = np.linalg.norm(acc.T - ref) / np.linalg.norm(ref)
        assert err < 1e-5, (b, err)
    # no drift: the positions are the inputs, reordered into cell order
    Xo = ens.positions()
    for b in range(B):
        assert np.array_equal(Xo[b], X[b][:, mesh.stable_cell_order(X[b], n)])


def test_batch_of_eight_64cubed_is_bitwise_the_boxes_run_alone(pm):
    """With 8 or more boxes the 64^3 levels take the fused sweep (a single
    box takes the colour passes): still bitwise the boxes run alone."""
    w = inputs.ensemble_workload(n=64, B=8, boxsize=128.0, steps=3)
    Xb, Vb = run(pm, w, list(range(8)), 3)
    for b in (0, 5):
        Xs, Vs = run(pm, w, [b], 3)
        assert np.array_equal(Xb[b], Xs[0]) and np.array_equal(Vb[b], Vs[0]), b


def test_autotuned_tilings_are_bitwise_the_fixed_ones(pm):
    """The online autotuner tries each candidate tiling of the batched force
    pass (x chunk) and of the 64^3 smoothing (colour passes or fused sweeps,
    and the fused sweep's x chunk) on real steps and keeps the fastest: the
    particles are bitwise those of the fixed default tilings, and after ten
    steps every site it opened for this shape has chosen."""
    w = inputs.ensemble_workload(n=64, B=4, boxsize=128.0, steps=10)
    try:
        pm.autotune(0)
        Xf, Vf = run(pm, w, list(range(4)), 10)
        pm.autotune(2)
        Xt, Vt = run(pm, w, list(range(4)), 10)
        rep = [r for r in pm.autotune_report() if r["n"] == 64 and r["B"] == 4]
    finally:
        pm.autotune(1)
    assert np.array_equal(Xf, Xt) and np.array_equal(Vf, Vt)
    sites = {r["site"]: r for r in rep}
    assert "force_chunk" in sites and "mg_smoother" in sites, rep
    assert all(r["chosen"] is not None and r["samples"] >= 4 for r in rep), rep
    assert sites["force_chunk"]["chosen"] in (16, 32, 64)
    assert sites["mg_smoother"]["chosen"] in (0, 1)
