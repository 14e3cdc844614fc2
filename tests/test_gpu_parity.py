"""Parity of the CUDA path (through the C ABI) with the FP64 oracle, stage by
stage, on seeded inputs spanning several tiles and ragged sizes."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import fr as ofr
from oracle import mesh, poisson, step
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


def displaced_lattice(n, seed, amp=0.3):
    """n^3 particles at cell centres displaced by up to amp cells (seeded)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    pos = inputs.lattice(n) + rng.uniform(-amp, amp, (3, n ** 3)) / n
    return inputs.to_fixed_point(pos)


# ------------------------------------------------------------------ sort ---

@pytest.mark.parametrize("n,N", [(16, 0), (16, 1), (32, 5000), (32, 32 ** 3 + 777), (64, 100003)])
def test_sort_bit_exact(pm, n, N):
    X = inputs.uniform_particles(N, 100 + N)
    perm, cs = pm.sort(pm.positions_to_device(X), n)
    ref = mesh.stable_cell_order(X, n)
    assert np.array_equal(perm.cpu().numpy().view(np.uint32), ref)
    keys = mesh.cell_key(X, n)[ref]
    ref_cs = np.searchsorted(keys, np.arange(n ** 3 + 1), side="left").astype(np.uint32)
    assert np.array_equal(cs.cpu().numpy().view(np.uint32), ref_cs)


def test_sort_nearly_sorted_with_many_ties(pm):
    n = 32
    X = displaced_lattice(n, 7, amp=0.49)
    X = np.concatenate([X, X[:, ::3]], axis=1)      # duplicates: ties must keep input order
    perm, _ = pm.sort(pm.positions_to_device(X), n)
    assert np.array_equal(perm.cpu().numpy().view(np.uint32), mesh.stable_cell_order(X, n))


def clustered(n, counts, seed, background=0):
    """Particles piled into a few cells: counts[q] particles uniformly inside
    cell q * 37 % n^3 (plus `background` uniform ones), in seeded random order."""
    rng = np.random.Generator(np.random.PCG64(seed))
    pos = [rng.uniform(0.0, 1.0, (3, background))]
    for q, m in enumerate(counts):
        c = (q * 37) % n ** 3
        ijk = np.array([c // (n * n), (c // n) % n, c % n], dtype=np.float64)[:, None]
        pos.append((ijk + rng.uniform(0.0, 1.0, (3, m))) / n)
    pos = np.concatenate(pos, axis=1)
    return inputs.to_fixed_point(pos[:, rng.permutation(pos.shape[1])])


@pytest.mark.parametrize("counts,background", [
    ([12, 13, 14, 15, 20, 31, 32, 33], 3000),   # around the one-thread and one-warp limits
    ([32, 33, 34, 64, 100], 3000),              # around the one-warp limit
    ([63, 64, 65, 127, 128, 129, 255, 256, 257, 1379], 20000),   # the warp kernel's tiers and its limit
    ([4095, 4096, 4097, 8193], 20000),          # one and several shared-memory chunks
    ([150000, 999, 2], 50000),                  # a long run merged over several passes
])
def test_sort_long_runs(pm, counts, background):
    """Cells holding long runs of particles in shuffled order: the stable
    order (ties by input index) is restored inside every cell."""
    n = 16
    X = clustered(n, counts, 5 + len(counts), background)
    perm, cs = pm.sort(pm.positions_to_device(X), n)
    ref = mesh.stable_cell_order(X, n)
    assert np.array_equal(perm.cpu().numpy().view(np.uint32), ref)
    keys = mesh.cell_key(X, n)[ref]
    ref_cs = np.searchsorted(keys, np.arange(n ** 3 + 1), side="left").astype(np.uint32)
    assert np.array_equal(cs.cpu().numpy().view(np.uint32), ref_cs)


def test_sort_of_sorted_input_is_identity(pm):
    """Particles already in stable cell order (as the step leaves them) sort to
    the identity, long runs included."""
    n = 16
    X = clustered(n, [5000, 40, 3], 11, 30000)
    X = np.ascontiguousarray(X[:, mesh.stable_cell_order(X, n)])
    perm, _ = pm.sort(pm.positions_to_device(X), n)
    assert np.array_equal(perm.cpu().numpy().view(np.uint32), np.arange(X.shape[1], dtype=np.uint32))


# --------------------------------------------------------------- deposit ---

@pytest.mark.parametrize("n,kind", [(8, "lattice"), (32, "lattice"), (64, "lattice"), (32, "random"),
                                    (16, "single")])
def test_deposit_parity(pm, n, kind):
    if kind == "lattice":
        X = displaced_lattice(n, 11)
    elif kind == "random":
        X = inputs.uniform_particles(12345, 3)
    else:
        X = inputs.to_fixed_point(np.array([[0.31], [0.5 / n], [0.999]]))
    rho = pm.deposit(pm.positions_to_device(X), n).cpu().numpy()
    ref = mesh.deposit_tsc(mesh.positions_from_fixed_point(X), n)
    assert np.abs(rho - ref).max() <= 2e-6 * np.abs(ref).max()
    rho2 = pm.deposit(pm.positions_to_device(X), n).cpu().numpy()
    assert np.array_equal(rho, rho2)                  # deterministic


def test_deposit_empty(pm):
    rho = pm.deposit(torch.zeros((3, 0), dtype=torch.int32, device="cuda"), 16)
    assert float(rho.abs().max()) == 0.0


# ------------------------------------------------------------ multigrid ---

def random_source(n, seed):
    return inputs.random_field(n, seed)


@pytest.mark.parametrize("n", [16, 32, 64])
def test_mg_converged_matches_fft7(pm, n):
    f = random_source(n, 21)
    h = 1.0 / n
    phi, st = pm.mg_solve(torch.from_numpy(f.astype(np.float32)).cuda(), tol=1e-9, max_cycles=40,
                          coarsest=8 if n == 16 else 16)
    phi = phi.cpu().numpy().astype(np.float64)
    ref = poisson.solve_fft7(f.astype(np.float32).astype(np.float64), h)
    assert st["status"] == 0
    assert rel_l2(phi - phi.mean(), ref) < 2e-6
    g = mesh.force_from_potential(phi, h)
    gr = mesh.force_from_potential(ref, h)
    assert rel_l2(np.stack(g), np.stack(gr)) < 1e-5


@pytest.mark.parametrize("n,cycles", [(32, 1), (32, 2), (64, 1)])
def test_mg_fixed_cycles_match_oracle_multigrid(pm, n, cycles):
    """Same algorithm steps (Jacobi first guess, V-cycles with omega = 1 on the
    first pre- and last post-sweep, coarsest 16) in float32 vs float64."""
    f = random_source(n, 5).astype(np.float32).astype(np.float64)
    h = 1.0 / n
    phi, _ = pm.mg_solve(torch.from_numpy(f.astype(np.float32)).cuda(), fixed_cycles=cycles,
                         first_guess=pm.MG_GUESS_JACOBI)
    ref, _ = poisson.mg_solve(f, h, prm=poisson.MGParams(), cycles=cycles)
    assert rel_l2(phi.cpu().numpy(), ref) < 1e-5


def test_mg_warm_start_scaled_guess(pm):
    n = 32
    f = random_source(n, 9).astype(np.float32).astype(np.float64)
    h = 1.0 / n
    guess = 0.9 * poisson.solve_fft7(f, h)
    phi_t = torch.from_numpy((guess / 1.1).astype(np.float32)).cuda()
    phi, _ = pm.mg_solve(torch.from_numpy(f.astype(np.float32)).cuda(), phi=phi_t, fixed_cycles=1,
                         first_guess=pm.MG_GUESS_SCALED, guess_scale=1.1)
    ref, _ = poisson.mg_solve(f, h, u0=(guess / 1.1).astype(np.float32).astype(np.float64) * 1.1,
                              prm=poisson.MGParams(), cycles=1)
    assert rel_l2(phi.cpu().numpy(), ref) < 1e-5


# -------------------------------------------------------------- gradient ---

@pytest.mark.parametrize("order,n", [(3, 32), (5, 32), (7, 32), (3, 64), (5, 128), (7, 64)])
def test_gradient_parity(pm, order, n):
    phi = random_source(n, 4).astype(np.float32)
    g = pm.gradient(torch.from_numpy(phi).cuda(), order).cpu().numpy()
    ref = np.stack(mesh.force_from_potential(phi.astype(np.float64), 1.0 / n, order))
    assert np.abs(g - ref).max() <= 1e-5 * np.abs(ref).max()


# ----------------------------------------------------------------- interp ---

@pytest.mark.parametrize("n,N", [(32, 20000), (64, 1000)])
def test_interp_parity(pm, n, N):
    g = np.stack([random_source(n, 30 + d) for d in range(3)]).astype(np.float32)
    X = inputs.uniform_particles(N, 77)
    acc = pm.interp(torch.from_numpy(g).cuda(), pm.positions_to_device(X)).cpu().numpy()
    pos = mesh.positions_from_fixed_point(X)
    ref = mesh.interp_tsc([g[d].astype(np.float64) for d in range(3)], pos).T
    assert np.abs(acc - ref).max() <= 2e-6 * np.abs(ref).max()


# ------------------------------------------------------------------ f(R) ---

def lognormal_density(n, seed, sigma=0.8):
    rho = np.exp(sigma * inputs.random_field(n, seed))
    return rho / rho.mean()


@pytest.mark.parametrize("a", [0.3, 1.0])
def test_fr_one_f_cycle_matches_oracle(pm, a):
    n = 32
    rho = lognormal_density(n, 8).astype(np.float32).astype(np.float64)
    model = ofr.FRModel(Om=0.3, OL=0.7, fR0=-1e-5, boxsize=float(n))
    eps, _ = pm.fr_solve(torch.from_numpy(rho.astype(np.float32)).cuda(), a=a, Om=0.3, OL=0.7, fR0=-1e-5,
                         boxsize=float(n), coarsest=16, cycles=1)
    u, _ = ofr.fr_solve(rho, a, model, prm=ofr.FASParams(coarsest=16), cycles=1)
    assert rel_l2(eps.cpu().numpy(), u - 1.0) < 1e-4


def test_fr_converged_matches_oracle(pm):
    n = 32
    rho = lognormal_density(n, 12, 1.2).astype(np.float32).astype(np.float64)
    model = ofr.FRModel(Om=0.3, OL=0.7, fR0=-1e-5, boxsize=float(n))
    eps, st = pm.fr_solve(torch.from_numpy(rho.astype(np.float32)).cuda(), a=0.8, Om=0.3, OL=0.7, fR0=-1e-5,
                          boxsize=float(n), coarsest=8, tol=1e-6, max_cycles=20)
    u, _ = ofr.fr_solve(rho, 0.8, model, prm=ofr.FASParams(coarsest=8), tol=1e-10)
    assert st["status"] == 0
    assert rel_l2(eps.cpu().numpy(), u - 1.0) < 2e-5


# ------------------------------------------------------------------ step ---

def gpu_accelerations(pm, X, V, n, a, gravity="newton", boxsize=64.0, Om=1.0, OL=0.0, **kw):
    sim = pm.Simulation(X, V, n, Om=Om, OL=OL, boxsize=boxsize, gravity=gravity, track_ids=True, keep_acc=True,
                        **kw)
    sim.step(a=a, dt_kick=0.0, dt_drift=0.0)
    out = np.empty((3, X.shape[1]))
    out[:, sim.particle_ids()] = sim.acc.cpu().numpy()
    return out, sim


def test_step_accelerations_c1(pm):
    n = 32
    X, V = inputs.zeldovich_powerlaw_ics(n, seed=1)
    acc, _ = gpu_accelerations(pm, X, V, n, 0.02)
    ref, _, _ = step.accelerations(mesh.positions_from_fixed_point(X), 0.02,
                                   step.PMParams(n=n, Om=1.0, OL=0.0, boxsize=64.0))
    assert rel_l2(acc.T, ref) < 1e-5


def test_step_accelerations_fr(pm):
    n = 32
    X = displaced_lattice(n, 13, amp=0.45)
    V = np.zeros((3, n ** 3))
    mgp = pm.default_mg(tol=1e-9)
    frp = pm.default_fr(coarsest=16, cycles=1)
    acc, _ = gpu_accelerations(pm, X, V, n, 0.7, gravity="fr", boxsize=float(n), Om=0.3, OL=0.7, mg=mgp, fr=frp)
    prm = step.PMParams(n=n, Om=0.3, OL=0.7, boxsize=float(n), gravity="fr", fR0=-1e-5)
    ref, _, _ = step.accelerations(mesh.positions_from_fixed_point(X), 0.7, prm)
    assert rel_l2(acc.T, ref) < 1e-5


def test_step_fr_and_poisson_to_tolerance_together(pm):
    """Both solvers iterating to a tolerance in one step (the scalaron on its
    side stream, each reducing its residual norms in its own buffer): the
    step reports both converged and the forces match the oracle."""
    n = 32
    X = displaced_lattice(n, 17, amp=0.45)
    V = np.zeros((3, n ** 3))
    mgp = pm.default_mg(tol=1e-9)
    frp = pm.default_fr(coarsest=16, tol=1e-4, max_cycles=20)
    sim = pm.Simulation(X, V, n, Om=0.3, OL=0.7, boxsize=float(n), gravity="fr", track_ids=True, keep_acc=True,
                        mg=mgp, fr=frp)
    st = sim.step(a=0.7, dt_kick=0.0, dt_drift=0.0)
    acc = np.empty((3, X.shape[1]))
    acc[:, sim.particle_ids()] = sim.acc.cpu().numpy()
    assert st["fr"]["status"] == 0 and st["fr"]["cycles"] > 1
    assert st["mg"]["status"] == 0 and st["mg"]["cycles"] > 1
    # the oracle's scalaron from ten F-cycles (converged far below 1e-4)
    prm = step.PMParams(n=n, Om=0.3, OL=0.7, boxsize=float(n), gravity="fr", fR0=-1e-5, fr_cycles=10)
    ref, _, _ = step.accelerations(mesh.positions_from_fixed_point(X), 0.7, prm)
    assert rel_l2(acc.T, ref) < 1e-4


def test_step_fr_serial_equals_side_stream(pm):
    """The scalaron solve on the caller's stream (serial) and on the side
    stream beside the Poisson solve give bitwise-equal particles over three
    kick-drift-kick steps (same kernels, same reductions, own norm buffers)."""
    import torch
    n = 64
    X, V = inputs.lpt_ics(n, float(n), 0.3, 0.7, 0.25, seed=21, order=2)
    out = []
    for serial in (False, True):
        sim = pm.Simulation(X, V, n, Om=0.3, OL=0.7, boxsize=float(n), gravity="fr", track_ids=True,
                            mg=pm.default_mg(tol=1e-7), fr=pm.default_fr(tol=1e-3, max_cycles=4))
        sim.serial = serial
        for a in (0.25, 0.26, 0.27):
            sim.step(a=a, dt_kick=0.02, dt_drift=0.02)
        torch.cuda.synchronize()
        ids = sim.particle_ids()
        Xs = np.empty((3, n ** 3), dtype=np.int64)
        Vs = np.empty((3, n ** 3), dtype=np.float32)
        Xs[:, ids] = sim.X.cpu().numpy()
        Vs[:, ids] = sim.V.cpu().numpy()
        out.append((Xs, Vs))
    assert np.array_equal(out[0][0], out[1][0])
    assert np.array_equal(out[0][1], out[1][1])


@pytest.mark.parametrize("gravity", ["newton", "fr"])
def test_step_accelerations_64_lcdm(pm, gravity):
    """64^3 LCDM 2LPT particles (the float4 gradient / interpolation path of
    pm_step for n >= 64)."""
    n = 64
    X, V = inputs.lpt_ics(n, float(n), 0.3, 0.7, 0.25, seed=9, order=2)
    mgp = pm.default_mg(tol=1e-9)
    acc, _ = gpu_accelerations(pm, X, V, n, 0.25, gravity=gravity, boxsize=float(n), Om=0.3, OL=0.7, mg=mgp)
    prm = step.PMParams(n=n, Om=0.3, OL=0.7, boxsize=float(n), gravity=gravity, fR0=-1e-5)
    ref, _, _ = step.accelerations(mesh.positions_from_fixed_point(X), 0.25, prm)
    assert rel_l2(acc.T, ref) < 1e-5


@pytest.mark.parametrize("order", [3, 5, 7])
def test_step_force_in_shared_memory_equals_gradient_then_interpolation(pm, order):
    """For n >= 32 the step computes the force next to the particles (shared
    memory); it equals, bitwise, the force field of pm_gradient interpolated
    by pm_interp at the same positions."""
    n = 64
    X, V = inputs.lpt_ics(n, float(n), 0.3, 0.7, 0.25, seed=5, order=2)
    acc, sim = gpu_accelerations(pm, X, V, n, 0.25, boxsize=float(n), Om=0.3, OL=0.7, grad_order=order,
                                 mg=pm.default_mg(tol=1e-7))
    g = pm.gradient(sim.phi, order=order)
    ref = pm.interp(g, pm.positions_to_device(X)).cpu().numpy()
    assert np.array_equal(acc.astype(np.float32), ref)


def test_step_is_deterministic(pm):
    n = 32
    X, V = inputs.zeldovich_powerlaw_ics(n, seed=2)
    outs = []
    for _ in range(2):
        sim = pm.Simulation(X, V, n, Om=1.0, OL=0.0, boxsize=64.0, track_ids=True)
        sim.run([0.02, 0.03, 0.04])
        outs.append((sim.positions(), sim.velocities(), sim.particle_ids()))
    for a, b in zip(outs[0], outs[1]):
        assert np.array_equal(a, b)


def test_c1_twenty_steps_positions_and_power(pm):
    """The 32^3 Einstein-de Sitter workload: Zel'dovich ICs at a = 0.02, 20
    KDK steps uniform in a to 0.2.  Accuracy bars: final positions RMS <= 1e-4 cell,
    P(k) within 0.1% below half Nyquist."""
    from oracle import power
    n = 32
    X, V = inputs.zeldovich_powerlaw_ics(n, seed=1)
    a_steps = list(np.linspace(0.02, 0.2, 21))
    sim = pm.Simulation(X, V, n, Om=1.0, OL=0.0, boxsize=64.0, track_ids=True, mg=pm.default_mg(tol=1e-9))
    sim.run(a_steps)
    ids = sim.particle_ids()
    Xg = np.empty_like(X)
    Xg[:, ids] = sim.positions()
    pos_ref, _ = step.run_kdk(mesh.positions_from_fixed_point(X), V.T, a_steps,
                              step.PMParams(n=n, Om=1.0, OL=0.0, boxsize=64.0))
    d = (mesh.positions_from_fixed_point(Xg) - pos_ref + 0.5) % 1.0 - 0.5
    rms_cells = np.sqrt((d ** 2).sum(axis=1).mean()) * n
    assert rms_cells <= 1e-4
    k, P, _ = power.power_spectrum(mesh.deposit_tsc(mesh.positions_from_fixed_point(Xg), n), 64.0)
    kr, Pr, _ = power.power_spectrum(mesh.deposit_tsc(pos_ref, n), 64.0)
    sel = k < 0.5 * np.pi * n / 64.0
    assert np.abs(P[sel] / Pr[sel] - 1.0).max() < 1e-3


@pytest.mark.parametrize("mu0,poisson", [(0.5, 0), (-0.5, 0), (0.5, 1)])
def test_step_accelerations_parametrised_gravity(pm, mu0, poisson):
    """Parametrised gravity (mu(a) = 1 + mu0 Omega_L(a)/Omega_L,0) with the
    multigrid and the FFT_7pt solvers."""
    n = 64
    X, V = inputs.lpt_ics(n, float(n), 0.3, 0.7, 0.8, seed=9, order=2)
    mgp = pm.default_mg(tol=1e-9)
    acc, _ = gpu_accelerations(pm, X, V, n, 0.8, gravity="mu", boxsize=float(n), Om=0.3, OL=0.7, mg=mgp,
                               mu0=mu0, poisson=poisson)
    prm = step.PMParams(n=n, Om=0.3, OL=0.7, boxsize=float(n), gravity="mu", mu0=mu0)
    ref, _, _ = step.accelerations(mesh.positions_from_fixed_point(X), 0.8, prm)
    assert rel_l2(acc.T, ref) < 1e-5


def test_adaptive_steps_match_oracle_on_their_schedule(pm):
    """The 32^3 Einstein-de Sitter workload with the §3.4 adaptive time step
    (free fall, velocity, 2% in a; Courant factor 0.8) on the FFT_7pt solver: the final positions after the
    GPU-chosen schedule against the oracle's KDK on the same schedule."""
    n = 32
    X, V = inputs.zeldovich_powerlaw_ics(n, seed=1)
    sim = pm.Simulation(X, V, n, Om=1.0, OL=0.0, boxsize=64.0, track_ids=True, poisson=pm.PM_POISSON_FFT7)
    a_steps = sim.run_adaptive(0.02, 0.2, courant=0.8, da_max=0.02)
    assert len(a_steps) > 20 and a_steps[-1] == 0.2
    assert all(a1 <= 1.02 * a0 * (1 + 1e-12) for a0, a1 in zip(a_steps[:-1], a_steps[1:]))
    out = np.empty((3, n ** 3))
    out[:, sim.particle_ids()] = mesh.positions_from_fixed_point(sim.positions()).T
    ref, _ = step.run_kdk(mesh.positions_from_fixed_point(X), np.asarray(V, dtype=np.float32).T.astype(np.float64),
                          a_steps, step.PMParams(n=n, Om=1.0, OL=0.0, boxsize=64.0), warm_start=False)
    d = (out.T - ref + 0.5) % 1.0 - 0.5
    assert np.sqrt((d ** 2).sum(1).mean()) * n < 1e-4


# ---------------------------------------------------------- f(R), n = 2 ---

@pytest.mark.parametrize("a", [0.3, 1.0])
def test_fr_n2_one_f_cycle_matches_oracle(pm, a):
    """Hu-Sawicki n = 2 (the quartic per cell, §3.10): one F-cycle from u = 1."""
    n = 32
    rho = lognormal_density(n, 8).astype(np.float32).astype(np.float64)
    model = ofr.FRModel(Om=0.3, OL=0.7, fR0=-1e-5, boxsize=float(n), n=2)
    eps, _ = pm.fr_solve(torch.from_numpy(rho.astype(np.float32)).cuda(), a=a, Om=0.3, OL=0.7, fR0=-1e-5,
                         boxsize=float(n), coarsest=16, cycles=1, nhs=2)
    u, _ = ofr.fr_solve(rho, a, model, prm=ofr.FASParams(coarsest=16), cycles=1)
    assert rel_l2(eps.cpu().numpy(), u - 1.0) < 1e-4


def test_fr_n2_converged_matches_oracle(pm):
    n = 32
    rho = lognormal_density(n, 12, 1.2).astype(np.float32).astype(np.float64)
    model = ofr.FRModel(Om=0.3, OL=0.7, fR0=-1e-5, boxsize=float(n), n=2)
    eps, st = pm.fr_solve(torch.from_numpy(rho.astype(np.float32)).cuda(), a=0.8, Om=0.3, OL=0.7, fR0=-1e-5,
                          boxsize=float(n), coarsest=8, tol=1e-6, max_cycles=20, nhs=2)
    u, _ = ofr.fr_solve(rho, 0.8, model, prm=ofr.FASParams(coarsest=8), tol=1e-10)
    assert st["status"] == 0
    assert rel_l2(eps.cpu().numpy(), u - 1.0) < 2e-5


def test_step_accelerations_fr_n2(pm):
    n = 32
    X = displaced_lattice(n, 13, amp=0.45)
    V = np.zeros((3, n ** 3))
    mgp = pm.default_mg(tol=1e-9)
    frp = pm.default_fr(coarsest=16, cycles=1, nhs=2)
    acc, _ = gpu_accelerations(pm, X, V, n, 0.7, gravity="fr", boxsize=float(n), Om=0.3, OL=0.7, mg=mgp, fr=frp)
    prm = step.PMParams(n=n, Om=0.3, OL=0.7, boxsize=float(n), gravity="fr", fR0=-1e-5, fr_n=2)
    ref, _, _ = step.accelerations(mesh.positions_from_fixed_point(X), 0.7, prm)
    assert rel_l2(acc.T, ref) < 1e-5


@pytest.mark.parametrize("gravity", ["newton", "fr"])
def test_step_host_equals_device_step(pm, gravity):
    """pm_step_host (positions in before the sort, velocities in on a second
    stream beside the sort and the solvers, both out on two streams) gives
    bitwise the particles of pm_step on device-resident arrays, over three
    steps, with in-place host buffers."""
    import torch
    n = 64
    X, V = inputs.lpt_ics(n, float(n), 0.3, 0.7, 0.25, seed=23, order=2)
    mk = lambda: pm.Simulation(X, V, n, Om=0.3, OL=0.7, boxsize=float(n), gravity=gravity,
                               mg=pm.default_mg(tol=1e-7), fr=pm.default_fr(tol=1e-3, max_cycles=4))
    steps = [(0.25, 0.02, 0.02), (0.26, 0.02, 0.02), (0.27, 0.02, 0.02)]
    dev = mk()
    for a, k, d in steps:
        dev.step(a=a, dt_kick=k, dt_drift=d)
    torch.cuda.synchronize()
    host = mk()
    Xh = torch.empty((3, n ** 3), dtype=torch.int32).pin_memory()
    Vh = torch.empty((3, n ** 3), dtype=torch.float32).pin_memory()
    Xh.copy_(host.X)
    Vh.copy_(host.V)
    for a, k, d in steps:
        host.step_host(a, k, d, Xh, Vh, Xh, Vh)
    assert torch.equal(Xh, dev.X.cpu())
    assert torch.equal(Vh, dev.V.cpu())


@pytest.mark.parametrize("N", [0, 1, 1000, 300001])
def test_max_speed_matches_host(pm, N):
    """pm_max_speed: the largest |v| over the particles (the velocity
    criterion's input before the first step), against numpy."""
    rng = np.random.Generator(np.random.PCG64(N + 3))
    V = rng.standard_normal((3, N)).astype(np.float32)
    n = 32
    ws = pm.workspace(n, N, pm.PM_WS_STEP)
    got = pm.max_speed(torch.from_numpy(V).cuda(), n, ws, pm.PM_WS_STEP)
    ref = float(np.sqrt((V.astype(np.float64) ** 2).sum(0)).max()) if N else 0.0
    assert got == pytest.approx(ref, rel=1e-6, abs=0.0)


@pytest.mark.parametrize("gravity", ["newton", "fr"])
def test_checkpoint_resume_is_bitwise_the_uninterrupted_run(pm, tmp_path, gravity):
    """pm_state_save after three steps, pm_state_load into a fresh state, two
    more steps: bitwise the particles (and ids, potentials) of five steps
    without the interruption."""
    n = 32
    X, V = inputs.lpt_ics(n, float(n), 0.3, 0.7, 0.2, seed=31, order=2)
    mk = lambda: pm.Simulation(X, V, n, Om=0.3, OL=0.7, boxsize=float(n), gravity=gravity, track_ids=True,
                               mg=pm.default_mg(tol=1e-7, fixed_cycles=2), fr=pm.default_fr(cycles=1))
    steps = [(0.2 + 0.01 * i, 0.01, 0.01) for i in range(5)]
    ref = mk()
    for s in steps:
        ref.step(*s)
    first = mk()
    for s in steps[:3]:
        first.step(*s)
    path = str(tmp_path / "state.ckpt")
    first.save(path)
    resumed = mk()
    resumed.load(path)
    assert resumed.state.have_prev == 1
    for s in steps[3:]:
        resumed.step(*s)
    assert np.array_equal(resumed.positions(), ref.positions())
    assert np.array_equal(resumed.velocities(), ref.velocities())
    assert np.array_equal(resumed.particle_ids(), ref.particle_ids())
    assert torch.equal(resumed.phi, ref.phi)
    if gravity == "fr":
        assert torch.equal(resumed.eps, ref.eps)


def test_checkpoint_mismatch_is_an_io_error(pm, tmp_path):
    n = 16
    X = inputs.uniform_particles(1000, 5)
    a = pm.Simulation(X, np.zeros((3, 1000)), n, Om=1.0, OL=0.0, boxsize=16.0)
    path = str(tmp_path / "a.ckpt")
    a.save(path)
    b = pm.Simulation(X[:, :999], np.zeros((3, 999)), n, Om=1.0, OL=0.0, boxsize=16.0)
    with pytest.raises(pm.PMError) as e:
        b.load(path)
    assert e.value.code == 7
    with pytest.raises(pm.PMError) as e:
        a.load(str(tmp_path / "missing.ckpt"))
    assert e.value.code == 7
