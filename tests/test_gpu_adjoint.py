"""Adjoint entry points (pm_*_adj, mg_solve_adj, pm_step_adj) and the
differentiable PM built on them, against the FP64 autograd oracle
(oracle/adjoint.py), dot-product identities and finite differences."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import adjoint as oadj
from oracle import cosmology, mesh
from paper_2410_20501_gb300 import inputs

pytestmark = pytest.mark.gpu
T = torch.float64


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
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def rng_of(seed):
    return np.random.Generator(np.random.PCG64(seed))


def displaced_lattice(n, seed, amp=0.3):
    pos = inputs.lattice(n) + rng_of(seed).uniform(-amp, amp, (3, n ** 3)) / n
    return inputs.to_fixed_point(pos)


def f32(a):
    """float32 copy (the GPU's input) and its exact float64 value (the oracle's)."""
    a32 = np.ascontiguousarray(a, dtype=np.float32)
    return a32, a32.astype(np.float64)


# ------------------------------------------------------------- gradient ---

@pytest.mark.parametrize("n,order", [(16, 3), (32, 5), (64, 7), (64, 5)])
def test_gradient_adj_matches_oracle_and_transposes(pm, n, order):
    phi32, phi = f32(rng_of(n + order).standard_normal((n, n, n)))
    gb32, gb = f32(rng_of(7 * n + order).standard_normal((3, n, n, n)))
    out = pm.gradient_adj(torch.from_numpy(gb32).cuda(), order).cpu().numpy()
    p = torch.from_numpy(phi).requires_grad_(True)
    g = [-oadj.derivative(p, ax, 1.0 / n, order) for ax in range(3)]
    sum((g[d] * torch.from_numpy(gb[d])).sum() for d in range(3)).backward()
    assert rel_l2(out, p.grad.numpy()) < 1e-6
    # <G phi, g_bar> = <phi, G^T g_bar> with the forward kernel
    fwd = pm.gradient(torch.from_numpy(phi32).cuda(), order).cpu().numpy().astype(np.float64)
    lhs, rhs = float((fwd * gb).sum()), float((phi * out).sum())
    assert abs(lhs - rhs) <= 1e-5 * np.sqrt(float((fwd ** 2).sum()) * float((gb ** 2).sum()))


# -------------------------------------------------------------- deposit ---

def oracle_deposit_vjp(X, n, rho_bar):
    pos = torch.from_numpy(mesh.positions_from_fixed_point(X)).requires_grad_(True)
    (oadj.deposit(pos, n) * torch.from_numpy(rho_bar)).sum().backward()
    return pos.grad.numpy().T


@pytest.mark.parametrize("n,N,kind", [(16, 1, "uniform"), (32, 32 ** 3, "lattice"), (32, 20011, "uniform"),
                                      (64, 64 ** 3, "lattice")])
def test_deposit_adj_matches_oracle(pm, n, N, kind):
    X = displaced_lattice(n, 3, 0.45) if kind == "lattice" else inputs.uniform_particles(N, 5 + N)
    rb32, rb = f32(rng_of(N).standard_normal((n, n, n)))
    out = pm.deposit_adj(pm.positions_to_device(X), n, torch.from_numpy(rb32).cuda()).cpu().numpy()
    ref = oracle_deposit_vjp(X, n, rb)
    assert rel_l2(out, ref) < 1e-5
    assert np.abs(out - ref).max() <= 1e-5 * np.abs(ref).max()


def test_deposit_adj_empty(pm):
    X = np.zeros((3, 0), dtype=np.uint32)
    out = pm.deposit_adj(pm.positions_to_device(X), 16, torch.zeros((16, 16, 16), device="cuda"))
    assert out.shape == (3, 0)


def test_deposit_adj_matches_finite_difference_of_forward(pm):
    # directional derivative of <deposit(X), rho_bar> along random particle moves of 1e-3 cell
    n = 32
    X = displaced_lattice(n, 8, 0.45)
    rb32, rb = f32(rng_of(9).standard_normal((n, n, n)))
    out = pm.deposit_adj(pm.positions_to_device(X), n, torch.from_numpy(rb32).cuda()).cpu().numpy()
    d = rng_of(10).standard_normal((3, n ** 3))
    step = 1e-3 / n
    Xp = inputs.to_fixed_point(X.astype(np.float64) / 2 ** 32 + step * d)
    Xm = inputs.to_fixed_point(X.astype(np.float64) / 2 ** 32 - step * d)
    rp = pm.deposit(pm.positions_to_device(Xp), n).cpu().numpy().astype(np.float64)
    rm = pm.deposit(pm.positions_to_device(Xm), n).cpu().numpy().astype(np.float64)
    fd = float(((rp - rm) * rb).sum()) / (2 * step)
    an = float((out.astype(np.float64) * d).sum())
    assert abs(fd - an) <= 2e-3 * abs(an)


# --------------------------------------------------------------- interp ---

@pytest.mark.parametrize("n,N,kind", [(16, 333, "uniform"), (32, 32 ** 3, "lattice"), (64, 100003, "uniform")])
def test_interp_adj_matches_oracle(pm, n, N, kind):
    X = displaced_lattice(n, 4, 0.45) if kind == "lattice" else inputs.uniform_particles(N, 50 + N)
    g32, g = f32(rng_of(n).standard_normal((3, n, n, n)))
    ab32, ab = f32(rng_of(N + 1).standard_normal((3, X.shape[1])))
    gbar, dX = pm.interp_adj(torch.from_numpy(g32).cuda(), pm.positions_to_device(X), torch.from_numpy(ab32).cuda())
    gt = torch.from_numpy(g).requires_grad_(True)
    pos = torch.from_numpy(mesh.positions_from_fixed_point(X)).requires_grad_(True)
    (oadj.interp([gt[0], gt[1], gt[2]], pos) * torch.from_numpy(ab.T)).sum().backward()
    assert rel_l2(gbar.cpu().numpy(), gt.grad.numpy()) < 1e-5
    assert rel_l2(dX.cpu().numpy(), pos.grad.numpy().T) < 1e-5
    # <interp(g), a_bar> = <g, g_bar> with the forward kernel
    acc = pm.interp(torch.from_numpy(g32).cuda(), pm.positions_to_device(X)).cpu().numpy().astype(np.float64)
    lhs, rhs = float((acc * ab).sum()), float((g * gbar.cpu().numpy()).sum())
    assert abs(lhs - rhs) <= 1e-5 * abs(lhs) + 1e-6 * np.linalg.norm(acc) * np.linalg.norm(ab)


# -------------------------------------------------------------- poisson ---

def test_mg_solve_adj_self_adjoint_and_exact(pm):
    n = 64
    f32a, f = f32(rng_of(31).standard_normal((n, n, n)))
    g32a, g = f32(rng_of(32).standard_normal((n, n, n)))
    uf = pm.mg_solve_adj(torch.from_numpy(f32a).cuda(), tol=1e-7).cpu().numpy().astype(np.float64)
    ug = pm.mg_solve_adj(torch.from_numpy(g32a).cuda(), tol=1e-7).cpu().numpy().astype(np.float64)
    ref = oadj.solve_fft7(torch.from_numpy(f), 1.0 / n).numpy()
    assert rel_l2(uf - uf.mean(), ref) < 1e-5
    lhs = float((uf * (g - g.mean())).sum())
    rhs = float(((f - f.mean()) * ug).sum())
    assert abs(lhs - rhs) <= 1e-5 * abs(lhs)


# ----------------------------------------------------------------- step ---

def step_case(pm, X, V, n, a, Om, OL, boxsize, dtk, dtd, seed, order=5, saved_phi=False):
    """GPU and oracle cotangents of one fused-kick step; returns
    ((xbar_in_gpu, vbar_in_gpu), (xbar_in_ref, vbar_in_ref)) in input order.
    saved_phi: hand pm_step_adj the potential of a (cold-started) forward
    step instead of letting it recompute the solve."""
    mg = pm.default_mg(tol=1e-7)
    phi = None
    if saved_phi:
        fwd = pm.Simulation(X, V, n, Om=Om, OL=OL, boxsize=boxsize, grad_order=order, mg=mg)
        fwd.step(a, dtk, dtd)
        phi = fwd.phi.clone()
    sim = pm.Simulation(X, V, n, Om=Om, OL=OL, boxsize=boxsize, grad_order=order, adjoint=True, mg=mg)
    N = X.shape[1]
    xo32, xo = f32(rng_of(seed).standard_normal((3, N)))
    vo32, vo = f32(rng_of(seed + 1).standard_normal((3, N)))
    xb, vb = sim.step_adjoint(a, dtk, dtd, torch.from_numpy(xo32).cuda(), torch.from_numpy(vo32).cuda(), phi=phi)
    # output slot p of the step holds input particle perm[p] (stable cell order)
    perm = mesh.stable_cell_order(X, n)
    xo_in, vo_in = np.empty_like(xo), np.empty_like(vo)
    xo_in[:, perm], vo_in[:, perm] = xo, vo
    pos = mesh.positions_from_fixed_point(X)
    vel = np.asarray(V, dtype=np.float32).astype(np.float64).T
    rx, rv = oadj.step_vjp(pos, vel, a, Om, n, dtk, dtd, xo_in.T, vo_in.T, order)
    return (xb.cpu().numpy(), vb.cpu().numpy()), (rx.numpy().T, rv.numpy().T)


def test_step_adj_c1(pm):
    n = 32
    X, V = inputs.zeldovich_powerlaw_ics(n, seed=1)
    a = 0.02
    dt = cosmology.dt_supercomoving(0.02, 0.029, 1.0, 0.0)
    (xb, vb), (rx, rv) = step_case(pm, X, V, n, a, 1.0, 0.0, 64.0, 0.5 * dt, dt, 40)
    assert rel_l2(vb, rv) < 1e-6
    # the force part of x_bar alone (x_bar_in - x_bar_out, measured against the oracle's)
    xo = np.empty_like(rx)
    xo[:, mesh.stable_cell_order(X, n)] = rng_of(40).standard_normal((3, n ** 3)).astype(np.float32)
    assert rel_l2(xb - xo, rx - xo) < 1e-4
    assert rel_l2(xb, rx) < 1e-6


@pytest.mark.parametrize("order", [3, 5, 7])
def test_step_adj_64_lcdm(pm, order):
    n = 64
    X, V = inputs.lpt_ics(n, float(n), 0.3, 0.7, 0.25, seed=9, order=2)
    dt = cosmology.dt_supercomoving(0.25, 0.27, 0.3, 0.7)
    (xb, vb), (rx, rv) = step_case(pm, X, V, n, 0.25, 0.3, 0.7, float(n), dt, dt, 41, order)
    xo = np.empty_like(rx)
    xo[:, mesh.stable_cell_order(X, n)] = rng_of(41).standard_normal((3, n ** 3)).astype(np.float32)
    assert rel_l2(vb, rv) < 1e-6
    assert rel_l2(xb - xo, rx - xo) < 1e-4


def test_step_adj_saved_potential_is_bitwise_the_recomputed_one(pm):
    n = 32
    X, V = inputs.zeldovich_powerlaw_ics(n, seed=2)
    dt = cosmology.dt_supercomoving(0.02, 0.03, 1.0, 0.0)
    (xb1, vb1), _ = step_case(pm, X, V, n, 0.02, 1.0, 0.0, 64.0, dt, dt, 50)
    (xb2, vb2), _ = step_case(pm, X, V, n, 0.02, 1.0, 0.0, 64.0, dt, dt, 50, saved_phi=True)
    assert np.array_equal(xb1, xb2) and np.array_equal(vb1, vb2)


# ------------------------------------------------------- differentiable ---

def schedule(a_steps, Om, OL):
    """Oracle-side fused-kick leapfrog coefficients (a_i, (dt_{i-1} + dt_i)/2, dt_i)."""
    dts = [cosmology.dt_supercomoving(a0, a1, Om, OL) for a0, a1 in zip(a_steps[:-1], a_steps[1:])]
    return [(a_steps[i], 0.5 * ((dts[i - 1] if i else 0.0) + dts[i]), dts[i]) for i in range(len(dts))]


def test_density_loss_gradient_vs_oracle_32(pm):
    """The differentiable configuration at 32^3 (box 50 Mpc/h, the 128^3 / 200
    Mpc/h resolution), 10 steps from z = 20: d loss / d noise from the CUDA
    adjoint chain against the FP64 autograd oracle."""
    from paper_2410_20501_gb300 import diffpm
    n = 32
    w = inputs.c4_workload(n, boxsize=50.0)
    steps = schedule(w["a_steps"], w["Om"], w["OL"])
    amp = torch.from_numpy(w["amp"])
    with torch.no_grad():
        target = oadj.density_model(torch.from_numpy(w["target_noise"]), amp, w["d_ratio"], w["vfac"], steps,
                                    w["Om"], n)
    loss_ref, grad_ref = oadj.density_loss_grad(w["noise"], target, w["amp"], w["d_ratio"], w["vfac"], steps,
                                                w["Om"], n)
    st = diffpm.Stepper(n, n ** 3, w["Om"], w["OL"], w["boxsize"])
    noise = torch.from_numpy(w["noise"]).cuda().requires_grad_(True)
    loss = diffpm.density_loss(noise, target.cuda(), st, w["amp"], w["d_ratio"], w["vfac"],
                               diffpm.schedule_coefficients(w["a_steps"], w["Om"], w["OL"]))
    loss.backward()
    grad = noise.grad.cpu().numpy()
    # FP32 fields and uint32 positions through 10 steps: measured 2e-7 (loss) and 1e-6 (gradient)
    assert abs(float(loss.detach()) - loss_ref) <= 2e-6 * loss_ref
    assert rel_l2(grad, grad_ref.numpy()) < 1e-5


def test_density_loss_gradient_matches_central_differences(pm):
    """The CUDA adjoint chain against central differences of the same CUDA
    forward model (32^3, box 50 Mpc/h, 10 steps from z = 20) along 6 random
    unit directions of the noise, eps = 1.  The forward runs in float32 fields
    and uint32 positions and TSC is only C1 in the positions, so the
    difference quotient carries rounding (~1e-6 of the loss over eps) and a
    truncation term; both stay far below the bounds asserted."""
    from paper_2410_20501_gb300 import diffpm
    n = 32
    w = inputs.c4_workload(n, boxsize=50.0)
    coef = diffpm.schedule_coefficients(w["a_steps"], w["Om"], w["OL"])
    st = diffpm.Stepper(n, n ** 3, w["Om"], w["OL"], w["boxsize"])
    args = (st, w["amp"], w["d_ratio"], w["vfac"], coef)
    with torch.no_grad():
        target = diffpm.forward_model(torch.from_numpy(w["target_noise"]).cuda(), *args).to(torch.float64)
    noise0 = torch.from_numpy(w["noise"]).cuda()
    noise = noise0.clone().requires_grad_(True)
    diffpm.density_loss(noise, target, *args).backward()
    grad = noise.grad.detach()

    def loss(x):
        with torch.no_grad():
            return float(diffpm.density_loss(x, target, *args))

    rng = np.random.Generator(np.random.PCG64(6))
    errs = []
    for _ in range(6):
        u = torch.from_numpy(rng.standard_normal((n, n, n))).cuda()
        u /= torch.linalg.vector_norm(u)
        fd = (loss(noise0 + u) - loss(noise0 - u)) / 2.0
        an = float((grad * u).sum())
        errs.append(abs(fd - an) / abs(an))
    assert float(np.median(errs)) < 2e-3 and max(errs) < 2e-2, errs
