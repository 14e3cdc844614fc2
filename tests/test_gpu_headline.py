"""Parity of the kernels that dominate the 512^3 f(R) step with the FP64
oracle, at the sizes where those kernels run.

- The fused red-black f(R) sweep (levels n >= 128) inside one FAS F-cycle
  (§3.6.2, §3.10, Eq. fr_sim_2): element by element against the oracle's own
  F-cycle at 128^3 and 256^3, and the float64 residual of the result against
  the oracle's residual after that cycle.
- The fused force pass of the 512^3 step (the force computed in shared memory
  from phi and eps, Table 1 gradient, inverse TSC, §3.4): the accelerations of
  a warm-started step of the benchmark's workload, in its launch
  configuration, at 10^4 sampled particles, against the oracle's gradient and
  interpolation of the same phi and eps on the 7^3 cells around each one.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import fr as ofr
from oracle import mesh
from paper_2410_20501_gb300 import inputs

pytestmark = pytest.mark.gpu

OM, OL, FR0 = 0.3, 0.7, -1e-5


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


def lognormal(n, seed, sigma=0.8):
    rho = np.exp(sigma * inputs.random_field(n, seed))
    return (rho / rho.mean()).astype(np.float32).astype(np.float64)


def linear_condition(a, n, model):
    """Condition number of the f(R) operator linearised about u = 1: the
    eigenvalues of d N_h / d eps run from kappa (the constant mode) to
    kappa + 24 |fbar| / h^2 (the 7-point Laplacian's largest, 12 / h^2, times
    the factor 2 of d(u^2)/du)."""
    fbar, kappa, _ = ofr.background(a, model)
    return 1.0 + 24.0 * abs(fbar) * n * n / kappa


EPS32 = 6e-8     # float32 rounding unit (2^-24)


@pytest.fixture(scope="module")
def fcycle_cases(pm):
    """(n, a, rho, GPU eps, oracle u, oracle residual history) for one F-cycle
    from the background on a lognormal density at the 1 Mpc/h cells of the
    512^3 run (L = n Mpc/h)."""
    out = []
    for n, a in ((128, 0.6), (256, 0.45)):
        rho = lognormal(n, 70 + n)
        eps, _ = pm.fr_solve(torch.from_numpy(rho.astype(np.float32)).cuda(), a=a, Om=OM, OL=OL, fR0=FR0,
                             boxsize=float(n), cycles=1)
        e = eps.cpu().numpy().astype(np.float64)
        model = ofr.FRModel(Om=OM, OL=OL, fR0=FR0, boxsize=float(n))
        u, hist = ofr.fr_solve(rho, a, model, cycles=1)
        out.append((n, a, rho, e, u, hist))
    return out


@pytest.mark.parametrize("case", [0, 1], ids=["128", "256"])
def test_fused_fr_f_cycle_matches_oracle_elementwise(fcycle_cases, case):
    """One F-cycle with the fused sweep on the 256^3 / 128^3 levels against
    the FP64 F-cycle, cell by cell.  Bound: float32 rounding amplified by the
    condition number of the linearised operator (the way the Poisson one-cycle
    test bounds its error by eps32 (n/pi)^2)."""
    n, a, rho, e, u, _ = fcycle_cases[case]
    model = ofr.FRModel(Om=OM, OL=OL, fR0=FR0, boxsize=float(n))
    tol = EPS32 * linear_condition(a, n, model)
    ref = u - 1.0
    assert np.isfinite(e).all() and e.min() > -1.0
    err = np.linalg.norm(e - ref) / np.linalg.norm(ref)
    assert err < tol, (err, tol)
    # and cell by cell: no cell is off by more than the bound times the largest |eps|
    assert np.abs(e - ref).max() <= 10 * tol * np.abs(ref).max()


def test_fused_fr_f_cycle_residual_against_oracle_256(fcycle_cases):
    """The float64 residual ||b - N_h(1 + eps)|| of the GPU's one-F-cycle result
    at 256^3 is within 1.5 times the oracle's own residual after one F-cycle,
    plus the float32 floor of the stored iterate: (kappa + 24|fbar|/h^2)
    eps32 ||eps||, the residual that rounding eps to float32 alone causes."""
    n, a, rho, e, u, hist = fcycle_cases[1]
    model = ofr.FRModel(Om=OM, OL=OL, fR0=FR0, boxsize=float(n))
    fbar, kappa, _ = ofr.background(a, model)
    b = ofr.source(rho, a, model)
    h = 1.0 / n
    r_gpu = np.linalg.norm(b - ofr.operator(1.0 + e, h, fbar, kappa))
    floor = (kappa + 24.0 * abs(fbar) / h ** 2) * EPS32 * np.linalg.norm(e)
    assert hist[1] < hist[0] / 100.0                 # the oracle's cycle itself converges
    assert r_gpu <= 1.5 * hist[1] + floor, (r_gpu, hist[1], floor)


def _schedule():
    a0 = 1.0 / 31.0
    return list(np.exp(np.linspace(np.log(a0), 0.0, 101)))


def test_fullsize_force_pass_accelerations_sampled(pm):
    """The 512^3 f(R) step of the benchmark (2LPT at z = 30, L = 512 Mpc/h,
    one F-cycle and two warm-started V-cycles): after the cold first step, the
    accelerations of the second step computed by the fused force pass at 10^4
    sampled particles, against the oracle's 5-point gradient of
    Phi = phi - (c~^2/2) fbar u^2 (§3.10) and its inverse TSC, both from the
    GPU's own phi and eps.  Bar: relative L2 <= 1e-5."""
    n, L = 512, 512.0
    a = _schedule()
    X, V = inputs.lpt_ics(n, L, OM, OL, a[0], 5, order=2, device="cuda")
    sim = pm.Simulation(X, V, n, OM, OL, L, gravity="fr", fR0=FR0, track_ids=True, keep_acc=True,
                        mg=pm.default_mg(tol=1e-7, stall=0.5, max_cycles=12, fixed_cycles=2),
                        fr=pm.default_fr(cycle=1, cycles=1))
    del X, V
    dt = [pm.dt_supercomoving(OM, OL, a[i], a[i + 1]) for i in range(2)]
    aD = [x * pm.growth_D(OM, OL, x) for x in a[:2]]
    sim.step(a[0], 0.5 * dt[0], dt[0])
    X_in, id_in = sim.X.clone(), sim.ids.clone().long()
    sim.step(a[1], 0.5 * (dt[0] + dt[1]), dt[1], aD[1] / aD[0])
    torch.cuda.synchronize()
    rng = np.random.Generator(np.random.PCG64(91))
    ranks = torch.from_numpy(rng.choice(n ** 3, 10000, replace=False)).cuda()
    where_in = torch.empty_like(id_in)
    where_in[id_in] = torch.arange(id_in.numel(), device="cuda")
    src = where_in[sim.ids[ranks].long()]
    acc = sim.acc[:, ranks].double().cpu().numpy().T
    Xs = X_in[:, src].cpu().numpy().view(np.uint32)
    pos = mesh.positions_from_fixed_point(Xs)                      # [N, 3]
    i0 = np.floor(pos * n).astype(np.int64)                        # nearest cell centre
    d = np.arange(-3, 4)
    ii = (i0[:, 0, None] + d) % n
    jj = (i0[:, 1, None] + d) % n
    kk = (i0[:, 2, None] + d) % n
    flat = (ii[:, :, None, None] * n + jj[:, None, :, None]) * n + kk[:, None, None, :]
    flat_t = torch.from_numpy(flat.reshape(-1)).cuda()
    phi = sim.phi.reshape(-1)[flat_t].double().cpu().numpy().reshape(flat.shape)
    eps = sim.eps.reshape(-1)[flat_t].double().cpu().numpy().reshape(flat.shape)
    del sim, X_in, id_in, where_in
    torch.cuda.empty_cache()
    model = ofr.FRModel(Om=OM, OL=OL, fR0=FR0, boxsize=L)
    Phi = phi + ofr.scalaron_potential(1.0 + eps, a[1], model)
    h = 1.0 / n
    g = [-mesh.derivative(Phi, ax + 1, h, 5) for ax in range(3)]   # valid on the central 3^3 cells
    off = pos * n - 0.5 - i0                                      # offset from the nearest centre
    w = [np.stack([mesh.w_tsc(off[:, ax] - o) for o in (-1, 0, 1)], axis=1) for ax in range(3)]
    ref = np.zeros((pos.shape[0], 3))
    for ox in range(3):
        for oy in range(3):
            for oz in range(3):
                wt = w[0][:, ox] * w[1][:, oy] * w[2][:, oz]
                for ax in range(3):
                    ref[:, ax] += wt * g[ax][:, 2 + ox, 2 + oy, 2 + oz]
    err = np.linalg.norm(acc - ref) / np.linalg.norm(ref)
    assert err < 1e-5, err
