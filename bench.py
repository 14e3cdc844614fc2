"""Throughput of the PM step (particle-steps/s) on the 512^3 Hu-Sawicki f(R)
configuration: 512^3 particles on a 512^3 grid, L = 512 Mpc/h, Omega_m = 0.3,
sigma8 = 0.8, f_R0 = -1e-5, 2LPT initial conditions at z = 30 (seed 5), 100
steps uniform in ln a to z = 0.  One step = cell sort, TSC deposit, one FAS
F-cycle for the scalaron beside two warm-started Poisson V-cycles (the cold
first step iterates to a relative residual of 1e-7), gradient of the combined
potential, inverse TSC, kick and drift.

The headline times steps W .. W+K-1 (--warmup W, --steps K) of one run of the
whole schedule, which is timed in segments: the line also gives the late
window (steps 90-99, z < 0.1) and the mean over all 100 steps.  Beside it,
each from a fresh start over the same window: per-kernel-class CUDA-event
times with both solvers on one stream (the roofline of the dominant class),
the same step through the C ABI with host buffers (e2e), and the Newtonian,
FFT_7pt, n = 2 and parametrised-gravity steps; then the differentiable 128^3
run, the 64-box ensemble (eager and graph replay over the same steps), and
the CPU leg: the FP64 oracle on a bounded sample (median of 5 single-core
runs and an all-core run) and the error of the GPU results against it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints one JSON line.  N > 1 (under torchrun) runs N independent replicas, one
per GPU: the step has no exchange between boxes.  ``--impl reference`` times
the FP64 CPU oracle on a bounded sample of the same workload instead.
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_GRID = 512
BOX = 512.0
OM, OL = 0.3, 0.7
FR0 = -1e-5
MU0 = -0.2      # parametrised-gravity amplitude of the variant line (mu(a) = 1 + mu0 Omega_L(a)/Omega_L0)
Z_INI = 30.0
SEED = 5
N_STEPS_RUN = 100
METRIC = "particle-steps/s at 512^3 (Hu-Sawicki f(R) PM step)"


def schedule():
    a0 = 1.0 / (1.0 + Z_INI)
    return list(np.exp(np.linspace(math.log(a0), 0.0, N_STEPS_RUN + 1)))


def dist_env():
    return int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")), \
        int(os.environ.get("LOCAL_RANK", "0"))


def init_dist(world, backend):
    import torch.distributed as dist
    if world > 1 and not dist.is_initialized():
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group(backend=backend)
    return dist


def max_over_ranks(value, world, device="cpu"):
    """Max of a float over ranks (the timing rule: slowest rank)."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


class ClockSampler:
    """nvidia-smi sampling during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        rows = []
        if self.path and os.path.exists(self.path):
            for line in open(self.path):
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
            os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(rows)}


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def kernel_digest(relpath, kernel):
    """Short sha256 of a kernel's definition text (from its __global__ line to
    the closing brace at column 0)."""
    import hashlib
    src = open(os.path.join(ROOT, relpath)).read()
    i = src.find(kernel + "(")
    if i < 0:
        return None
    start, end = src.rfind("__global__", 0, i), src.find("\n}\n", i)
    return hashlib.sha256(src[start:end].encode()).hexdigest()[:16]


def parts_digest(parts):
    """Short sha256 of source excerpts: for each [file, begin, end], the text
    from the first occurrence of ``begin`` to the next ``end`` after it (the
    kernel, its update functor, the instantiation that is launched).  None if
    an excerpt is missing."""
    import hashlib
    h = hashlib.sha256()
    for rel, begin, end in parts:
        src = open(os.path.join(ROOT, rel)).read()
        i = src.find(begin)
        j = src.find(end, i + len(begin)) if i >= 0 else -1
        if i < 0 or j < 0:
            return None
        h.update(src[i:j + len(end)].encode())
    return h.hexdigest()[:16]


def load_ncu_traffic():
    """Per timing class: DRAM bytes per launch from an ncu capture, kept only
    while the captured kernel's source is unchanged (same digest: of the
    kernel's definition text, or of the source excerpts its launch depends on)."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    if not os.path.exists(path):
        return {}
    out = {}
    for cls, e in json.load(open(path)).items():
        try:
            d = parts_digest(e["parts"]) if "parts" in e else kernel_digest(e["source"], e["kernel"])
            if d == e["digest"]:
                out[cls] = e
        except OSError:
            pass
    return out


# --------------------------------------------------------------- oracle arm --

ORACLE_N = 64   # oracle sample: 64^3 particles on a 64^3 grid (a few seconds of one core per step)


def _oracle_setup(steps, n=ORACLE_N):
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ.setdefault(v, "1")
    from oracle import mesh, step
    from paper_2410_20501_gb300 import inputs
    X, V = inputs.lpt_ics(n, float(n), OM, OL, 1.0 / (1.0 + Z_INI), SEED, order=2)
    prm = step.PMParams(n=n, Om=OM, OL=OL, boxsize=float(n), gravity="fr", fR0=FR0)
    a = schedule()[:steps + 1]
    return lambda: step.run_kdk(mesh.positions_from_fixed_point(X), V.T, a, prm, warm_start=False)


def oracle_sample(steps, n=ORACLE_N):
    """The FP64 oracle, unchanged, on a bounded sample of the workload: n^3
    particles on an n^3 grid in an n Mpc/h box (the 1 Mpc/h cells of the
    512^3 run), same cosmology, f_R0 and 2LPT start at z = 30, advanced through
    the first ``steps`` steps of the same schedule with f(R) forces (exact
    discrete Poisson inverse, one FAS F-cycle) and kick-drift-kick.  Returns
    (particle-steps/s, seconds, sample description)."""
    run = _oracle_setup(steps, n)
    t0 = time.perf_counter()
    run()
    dt = time.perf_counter() - t0
    return n ** 3 * steps / dt, dt, (f"FP64 oracle, {steps} f(R) PM steps (deposit, exact 7-point Poisson "
                                     f"inverse, one FAS F-cycle, 5-point gradient, inverse TSC, KDK) of {n}^3 "
                                     f"particles on a {n}^3 grid with the 1 Mpc/h cells of the 512^3 run")


def _oracle_core(steps, start, queue):
    """One core of the all-core baseline: set up, wait for the others, run."""
    run = _oracle_setup(steps)
    start.wait()
    t0 = time.time()
    run()
    queue.put((t0, time.time()))


def cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo, else platform)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.processor() or platform.machine()


def cpu_baseline(steps=6, runs=5):
    """The oracle on the host cores: the median of ``runs`` single-core runs of
    the bounded sample, and one all-core run (one independent sample per core,
    in spawned processes that set up, meet at a barrier and then run; timed
    from the first start to the last finish).  Returns the cpu_baseline
    object."""
    single = [oracle_sample(steps) for _ in range(runs)]
    secs = sorted(r[1] for r in single)
    med = secs[len(secs) // 2]
    ncores = os.cpu_count() or 1
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    start, queue = ctx.Barrier(ncores), ctx.Queue()
    procs = [ctx.Process(target=_oracle_core, args=(steps, start, queue)) for _ in range(ncores)]
    for p in procs:
        p.start()
    spans = [queue.get() for _ in procs]
    for p in procs:
        p.join()
    wall = max(t1 for _, t1 in spans) - min(t0 for t0, _ in spans)
    per = ORACLE_N ** 3 * steps
    return {"value": per / med, "unit": "particle-steps/s", "cores": 1, "kind": "oracle",
            "sample": single[0][2], "runs": runs, "seconds_median": med, "seconds_all_runs": secs,
            "all_cores": {"value": ncores * per / wall, "cores": ncores, "seconds": wall,
                          "what": f"{ncores} independent samples at once, one per core (spawned processes)"},
            "nproc": ncores, "cpu_model": cpu_model()}


def oracle_errors(probes):
    """Error of the GPU results against the FP64 oracle, from the probes the
    GPU passes saved (plain arrays): sampled accelerations of the 512^3 steps
    (the oracle's Table 1 gradient and inverse TSC of the GPU's own phi and
    eps on the 7^3 cells around each sampled particle), and the accelerations
    of two ensemble boxes in a warm batched step (the oracle's exact-Poisson
    accelerations at the same positions)."""
    from oracle import fr as ofr
    from oracle import mesh, step
    out = {}
    for name, p in probes.items():
        if p["kind"] == "patch":
            n = p["n"]
            Phi = p["phi"]
            if p["eps"] is not None:
                model = ofr.FRModel(Om=OM, OL=OL, fR0=FR0, boxsize=BOX)
                Phi = Phi + ofr.scalaron_potential(1.0 + p["eps"], p["a"], model)
            h = 1.0 / n
            g = [-mesh.derivative(Phi, ax + 1, h, 5) for ax in range(3)]
            pos = p["pos"]
            i0 = np.floor(pos * n)
            off = pos * n - 0.5 - i0
            w = [np.stack([mesh.w_tsc(off[:, ax] - o) for o in (-1, 0, 1)], axis=1) for ax in range(3)]
            ref = np.zeros_like(p["acc"])
            for ox in range(3):
                for oy in range(3):
                    for oz in range(3):
                        wt = w[0][:, ox] * w[1][:, oy] * w[2][:, oz]
                        for ax in range(3):
                            ref[:, ax] += wt * g[ax][:, 2 + ox, 2 + oy, 2 + oz]
            out[name] = {"rel_l2_acc": float(np.linalg.norm(p["acc"] - ref) / np.linalg.norm(ref)),
                         "what": f"{p['acc'].shape[0]} sampled particles of step {p['step']}, oracle gradient and "
                                 "inverse TSC of the GPU's own potential(s)"}
        elif p["kind"] == "adjoint":
            import torch
            from oracle import adjoint as oadj
            from oracle import cosmology
            from paper_2410_20501_gb300 import inputs
            w = inputs.c4_workload(p["n"], boxsize=50.0)
            a = w["a_steps"]
            dts = [cosmology.dt_supercomoving(a0, a1, w["Om"], w["OL"]) for a0, a1 in zip(a[:-1], a[1:])]
            steps = [(a[i], 0.5 * ((dts[i - 1] if i else 0.0) + dts[i]), dts[i]) for i in range(len(dts))]
            loss_ref, grad_ref = oadj.density_loss_grad(w["noise"], torch.from_numpy(p["target"]), w["amp"],
                                                        w["d_ratio"], w["vfac"], steps, w["Om"], p["n"])
            g = grad_ref.numpy()
            out[name] = {"rel_l2_grad": float(np.linalg.norm(p["grad"] - g) / np.linalg.norm(g)),
                         "rel_loss": abs(p["loss"] - loss_ref) / abs(loss_ref),
                         "what": "d loss / d noise of the 10-step density loss at 32^3 (L = 50 Mpc/h) against "
                                 "the FP64 autograd oracle, same target"}
        elif p["kind"] == "boxes":
            errs = []
            for b, (pos, acc, Om_b) in enumerate(zip(p["pos"], p["acc"], p["Om"])):
                ref, _, _ = step.accelerations(pos, p["a"], step.PMParams(n=p["n"], Om=Om_b, OL=1.0 - Om_b,
                                                                         boxsize=p["boxsize"]))
                errs.append(float(np.linalg.norm(acc - ref) / np.linalg.norm(ref)))
            out[name] = {"rel_l2_acc": errs, "boxes": p["boxes"],
                         "what": "accelerations of a warm batched step (2 V-cycles) against the exact-Poisson "
                                 "oracle at the same positions"}
        elif p["kind"] == "refine":
            from oracle import poisson
            exact = poisson.solve_fft7(p["f"].astype(np.float64), 1.0 / p["n"])

            def err(x):
                x = x.astype(np.float64)
                return float(np.linalg.norm((x - x.mean()) - exact) / np.linalg.norm(exact))
            out[name] = {"plain_rel_l2": err(p["phi32"]), "refined_rel_l2": err(p["phi64"]),
                         "what": f"potential of the {p['n']}^3 Poisson solve, float32 multigrid and float64 "
                                 "iterative refinement, against the exact 7-point inverse (FFT_7pt)"}
    return out


def headline_config(world):
    """The headline workload (both arms print it: the reference arm times a
    bounded sample of it, stated in its cpu_baseline)."""
    return {"workload": "hu-sawicki f(R) n=1 pm step, 512^3 particles, 512^3 grid, L=512 Mpc/h, 2LPT z=30",
            "global_batch": world * N_GRID ** 3, "n_grid": N_GRID, "boxsize_mpc_h": BOX, "fR0": FR0,
            "parallelism": f"replicas{world}", "l2": "inputs larger than L2 (every array >= 537 MB)",
            "poisson": "2 warm-started V-cycles per step (first step: to relative residual 1e-7)",
            "fr": "one FAS F-cycle per step"}


def run_reference(args):
    world, rank, _ = dist_env()
    if world > 1:
        init_dist(world, "gloo")
    if rank != 0:
        return 0
    value, secs, sample = oracle_sample(max(1, args.steps))
    line = {"metric": METRIC, "value": value, "unit": "particle-steps/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / max(1, args.steps),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": headline_config(args.gpus),
            "cpu_baseline": {"value": value, "unit": "particle-steps/s", "cores": 1, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "particle-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# ------------------------------------------------------------------ GPU arm --

LATE = 90   # the late window: steps 90-99 of the schedule (z < 0.1)


def step_coefficients(Om, OL, a):
    """Per step i of the schedule: (a_i, kick, drift, potential rescale), with
    the two half kicks around a_i merged: kick_i = (dt_{i-1} + dt_i)/2."""
    from paper_2410_20501_gb300 import pm
    dts = [pm.dt_supercomoving(Om, OL, a[i], a[i + 1]) for i in range(len(a) - 1)]
    D = [pm.growth_D(Om, OL, x) for x in a]
    out = []
    for i in range(len(a) - 1):
        prev = dts[i - 1] if i > 0 else 0.0
        resc = (a[i] * D[i]) / (a[i - 1] * D[i - 1]) if i > 0 else 1.0
        out.append((a[i], 0.5 * (prev + dts[i]), dts[i], resc))
    return out


def timed_steps(sim, coeffs, first, count, host_buffers=None, world=1):
    """Runs steps first .. first+count-1 between a barrier and a device
    synchronisation on both sides; returns (device ms from CUDA events on the
    launching stream, per-step stats)."""
    import torch
    s = torch.cuda.current_stream()
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    stats = []
    torch.cuda.synchronize()
    barrier(world)
    start.record(s)
    for i in range(first, first + count):
        a, kick, drift, resc = coeffs[i]
        if host_buffers is None:
            stats.append(sim.step(a, kick, drift, resc))
        else:
            Xh, Vh = host_buffers
            stats.append(sim.step_host(a, kick, drift, Xh, Vh, Xh, Vh, resc))
    end.record(s)
    torch.cuda.synchronize()
    barrier(world)
    return start.elapsed_time(end), stats


def make_sim(pm, X, V, variant, **kw):
    n = N_GRID
    mg = pm.default_mg(tol=1e-7, stall=0.5, max_cycles=12, fixed_cycles=2)
    fr = pm.default_fr(cycle=1, cycles=1, nhs=2 if variant == "fr_n2" else 1)
    gravity = {"fr": "fr", "fr_n2": "fr", "mu": "mu"}.get(variant, "newton")
    return pm.Simulation(X, V, n, OM, OL, BOX, gravity=gravity, fR0=FR0, mg=mg, fr=fr,
                         poisson=pm.PM_POISSON_FFT7 if variant == "newton_fft7" else pm.PM_POISSON_MG,
                         mu0=MU0 if variant == "mu" else 0.0, **kw)


def patch_probe(pm, X, V, variant, coeffs, at, count=10000):
    """A fresh run of ``variant`` to step ``at`` (untimed), keeping ids and
    accelerations: the accelerations of step ``at`` at ``count`` sampled
    particles, their positions, and the 7^3 cells of phi (and eps) around each
    (plain arrays for the oracle comparison of the CPU leg)."""
    import torch
    n = N_GRID
    sim = make_sim(pm, X, V, variant, track_ids=True, keep_acc=True)
    for i in range(at):
        sim.step(*coeffs[i])
    X_in, id_in = sim.X.clone(), sim.ids.clone().long()
    sim.step(*coeffs[at])
    torch.cuda.synchronize()
    rng = np.random.Generator(np.random.PCG64(91))
    ranks = torch.from_numpy(rng.choice(n ** 3, count, replace=False)).cuda()
    where_in = torch.empty_like(id_in)
    where_in[id_in] = torch.arange(id_in.numel(), device="cuda")
    src = where_in[sim.ids[ranks].long()]
    acc = sim.acc[:, ranks].double().cpu().numpy().T
    pos = (X_in[:, src].cpu().numpy().view(np.uint32).astype(np.float64) * 2.0 ** -32).T
    i0 = np.floor(pos * n).astype(np.int64)
    d = np.arange(-3, 4)
    ii, jj, kk = ((i0[:, ax, None] + d) % n for ax in range(3))
    flat = (ii[:, :, None, None] * n + jj[:, None, :, None]) * n + kk[:, None, None, :]
    ft = torch.from_numpy(flat.reshape(-1)).cuda()
    phi = sim.phi.reshape(-1)[ft].double().cpu().numpy().reshape(flat.shape)
    eps = None if sim.eps is None else sim.eps.reshape(-1)[ft].double().cpu().numpy().reshape(flat.shape)
    del sim, X_in, id_in, where_in
    torch.cuda.empty_cache()
    return {"kind": "patch", "n": n, "a": coeffs[at][0], "step": at, "acc": acc, "pos": pos, "phi": phi, "eps": eps}


def run_adjoint(n=128, fd_dirs=16, reps=3, eps=1.0):
    """The differentiable-PM workload: 128^3 white noise (seed 4) -> 1LPT at
    z = 20 in a 200 Mpc/h box -> 10 fused-kick PM steps to a = 1 -> TSC
    density; loss = sum (rho - rho_target)^2 with the target the same model
    from seed 5.  Times the forward pass and the backward pass (pm_step_adj
    per step, recomputing that step's forces) with CUDA events, and checks the
    gradient against central differences along ``fd_dirs`` random unit
    directions (seed 6)."""
    import torch
    from paper_2410_20501_gb300 import diffpm, inputs
    w = inputs.c4_workload(n)
    steps = diffpm.schedule_coefficients(w["a_steps"], w["Om"], w["OL"])
    st = diffpm.Stepper(n, n ** 3, w["Om"], w["OL"], w["boxsize"])
    args = (st, w["amp"], w["d_ratio"], w["vfac"], steps)
    with torch.no_grad():
        target = diffpm.forward_model(torch.from_numpy(w["target_noise"]).cuda(), *args).to(torch.float64)
    noise0 = torch.from_numpy(w["noise"]).cuda()
    s = torch.cuda.current_stream()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    fwd, bwd = [], []
    for _ in range(reps + 1):
        noise = noise0.clone().requires_grad_(True)
        torch.cuda.synchronize()
        ev[0].record(s)
        loss = diffpm.density_loss(noise, target, *args)
        ev[1].record(s)
        loss.backward()
        ev[2].record(s)
        torch.cuda.synchronize()
        fwd.append(ev[0].elapsed_time(ev[1]))
        bwd.append(ev[1].elapsed_time(ev[2]))
    fwd, bwd = statistics.median(fwd[1:]), statistics.median(bwd[1:])
    grad = noise.grad.detach()
    rng = np.random.Generator(np.random.PCG64(6))
    errs = []

    def L(x):
        with torch.no_grad():
            return float(diffpm.density_loss(x, target, *args))

    for _ in range(fd_dirs):
        u = torch.from_numpy(rng.standard_normal((n, n, n))).cuda()
        u /= torch.linalg.vector_norm(u)
        fd = (L(noise0 + eps * u) - L(noise0 - eps * u)) / (2 * eps)
        an = float((grad * u).sum())
        errs.append(abs(fd - an) / max(abs(an), 1e-30))
    # the same chain at 32^3 (the 200 Mpc/h / 128 resolution: L = 50 Mpc/h),
    # kept for the CPU leg's comparison with the FP64 autograd oracle
    ws = inputs.c4_workload(32, boxsize=50.0)
    st32 = diffpm.Stepper(32, 32 ** 3, ws["Om"], ws["OL"], ws["boxsize"])
    steps32 = diffpm.schedule_coefficients(ws["a_steps"], ws["Om"], ws["OL"])
    args32 = (st32, ws["amp"], ws["d_ratio"], ws["vfac"], steps32)
    with torch.no_grad():
        target32 = diffpm.forward_model(torch.from_numpy(ws["target_noise"]).cuda(), *args32).to(torch.float64)
    noise32 = torch.from_numpy(ws["noise"]).cuda().requires_grad_(True)
    loss32 = diffpm.density_loss(noise32, target32, *args32)
    loss32.backward()
    probe = {"kind": "adjoint", "n": 32, "target": target32.cpu().numpy(), "grad": noise32.grad.cpu().numpy(),
             "loss": float(loss32.detach())}
    return ({"workload": f"{n}^3 particles/grid, L=200 Mpc/h, 1LPT z=20 from white noise, 10 PM steps to z=0, "
                         "density-difference loss", "forward_ms": fwd, "backward_ms": bwd,
             "adjoint_over_forward": bwd / fwd, "loss": float(loss.detach()),
             "fd_check": {"directions": fd_dirs, "eps": eps,
                          "median_rel_err": statistics.median(errs) if errs else None,
                          "max_rel_err": max(errs) if errs else None}}, probe)


def run_refine(n=256, outer=4, cycles=3, reps=3):
    """The precision forms of the Poisson solve on a seeded 256^3 random source:
    mg_solve to its float32 floor (tol 1e-7) against mg_solve_refine (float64
    residuals of a float64 iterate, ``outer`` steps of ``cycles`` float32
    V-cycles).  CUDA-event times on the launching stream, median of ``reps``;
    both include their host synchronisations (one per cycle, one per step)."""
    import torch
    from paper_2410_20501_gb300 import inputs, pm
    f = torch.from_numpy(inputs.random_field(n, 36).astype(np.float32)).cuda()
    ws32 = pm.workspace(n, 0, pm.PM_WS_MG)
    ws64 = pm.workspace(n, 0, pm.PM_WS_MG | pm.PM_WS_REFINE)

    def timed(fn):
        times, out = [], None
        for _ in range(reps):
            t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            t0.record()
            out = fn()
            t1.record()
            torch.cuda.synchronize()
            times.append(t0.elapsed_time(t1))
        return out, float(np.median(times))

    (phi32, st32), ms32 = timed(lambda: pm.mg_solve(f, ws=ws32, tol=1e-7, max_cycles=40))
    (phi64, st64), ms64 = timed(lambda: pm.mg_solve_refine(f, ws=ws64, outer=outer, fixed_cycles=cycles))
    line = {"n": n,
            "plain": {"ms": ms32, "cycles": st32["cycles"], "rel_res": st32["res"] / st32["norm_f"],
                      "what": "mg_solve, float32 iterate, to tol 1e-7"},
            "refined": {"ms": ms64, "outer": outer, "cycles": st64["cycles"],
                        "rel_res": st64["res"] / st64["norm_f"],
                        "what": f"mg_solve_refine, float64 iterate, {outer} steps of {cycles} V-cycles"}}
    probe = {"kind": "refine", "n": n, "f": f.cpu().numpy(), "phi32": phi32.cpu().numpy(),
             "phi64": phi64.cpu().numpy()}
    return line, probe


def run_ensemble(n=64, B=64, steps=50):
    """The ensemble workload: 64 boxes of 64^3 particles on 64^3 grids,
    L = 128 Mpc/h, Omega_m ~ U[0.25, 0.35], sigma8 ~ U[0.7, 0.9] (PCG64 seed 3),
    box seeds 1000 + b, 2LPT at z = 30, 50 steps uniform in ln a, stepped
    together by pm_step_batch (2 fixed V-cycles per warm step, 8 on the first).
    Times the warm steps 2..49 eagerly and, from a fresh start, as CUDA-graph
    replays of one captured warm step (the same window); then a probe step 4
    (positions unchanged, velocities zeroed, so V = acc dt_kick) whose
    accelerations of two boxes the CPU leg compares with the oracle."""
    import torch
    from paper_2410_20501_gb300 import inputs, pm
    w = inputs.ensemble_workload(n=n, B=B, steps=steps, device="cuda")
    s = torch.cuda.current_stream()
    out = {}
    for mode in ("eager", "graph"):
        ens = pm.Ensemble(w["X"], w["V"], n, w["Om"], w["boxsize"], cold_cycles=8)
        coef = ens.coefficients(w["a_steps"])
        ens.step(coef[0])
        ens.step(coef[1])
        if mode == "graph":
            ens.capture()
        torch.cuda.synchronize()
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0.record(s)
        for i in range(2, steps):
            if mode == "graph":
                ens.replay_step(coef[i])
            else:
                ens.step(coef[i])
        t1.record(s)
        torch.cuda.synchronize()
        ms = t0.elapsed_time(t1) / (steps - 2)
        out[mode] = {"ms_per_step": ms, "value": B * n ** 3 / (ms / 1e3), "steps_timed": f"2..{steps - 1}"}
        del ens
    tuned = [{k: r[k] for k in ("site", "n", "chosen", "samples")} for r in pm.autotune_report() if r["B"] == B]
    # probe: steps 0..3, then step 4 with no drift from zeroed velocities
    ens = pm.Ensemble(w["X"], w["V"], n, w["Om"], w["boxsize"], cold_cycles=8)
    coef = ens.coefficients(w["a_steps"])
    for i in range(4):
        ens.step(coef[i])
    dtk = 1e-2
    row = coef[4].clone()
    row[1, :B] = dtk
    row[2, :B] = 0.0
    ens.V.zero_()
    ens.step(row)
    Xp, Vp = ens.positions(), ens.velocities()
    boxes = [0, B - 1]
    probe = {"kind": "boxes", "n": n, "a": float(w["a_steps"][4]), "boxsize": w["boxsize"], "boxes": boxes,
             "Om": [float(w["Om"][b]) for b in boxes],
             "pos": [(Xp[b].astype(np.float64) * 2.0 ** -32).T for b in boxes],
             "acc": [(Vp[b].astype(np.float64) / np.float32(dtk)).T for b in boxes]}
    del ens
    return ({"workload": f"{B} boxes x {n}^3 particles/grid, L=128 Mpc/h, Om~U[0.25,0.35], s8~U[0.7,0.9], "
                         "2LPT z=30, 50 steps in ln a", "unit": "particle-steps/s", **out,
             "graph_over_eager": out["graph"]["ms_per_step"] / out["eager"]["ms_per_step"],
             "autotune": {"what": "tilings the online tuner chose for this batch (eager steps; the graph "
                                  "replays the choices)", "sites": tuned}}, probe)


def run_lpt(n, reps=3):
    """2LPT initial conditions of n^3 particles (L = n Mpc/h, z = 30) by
    pm_lpt2: device time per generation."""
    import torch
    from paper_2410_20501_gb300 import inputs, pm
    a = 1.0 / (1.0 + Z_INI)
    D, E, f1, f2 = inputs.growth([a, 1.0], OM, OL)
    vfac = a * a * inputs.hubble_E(a, OM, OL)
    d1, e2 = D[0] / D[1], E[0] / D[1] ** 2
    noise = torch.from_numpy(inputs.white_noise(n, SEED).astype(np.float32)).cuda()
    amp = torch.from_numpy(inputs.lpt_amplitude(n, float(n), OM).astype(np.float32)).cuda()
    ws = pm.workspace(n, 0, pm.PM_WS_LPT)
    pm.lpt2(noise, amp, d1, e2, vfac * d1 * f1[0], vfac * e2 * f2[0], ws)
    s = torch.cuda.current_stream()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record(s)
    for _ in range(reps):
        pm.lpt2(noise, amp, d1, e2, vfac * d1 * f1[0], vfac * e2 * f2[0], ws)
    t1.record(s)
    torch.cuda.synchronize()
    return {"stage": "lpt", "n": n, "ms_per_generation": t0.elapsed_time(t1) / reps}


def run_gpu(args):
    import torch
    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    init_dist(world, "nccl")
    from paper_2410_20501_gb300 import build, inputs, pm
    if not os.path.exists(pm.LIB_PATH):
        if rank == 0:
            build.build()
        barrier(world)
    pm.lib()
    a = schedule()
    coeffs = step_coefficients(OM, OL, a)
    n = N_GRID
    X, V = inputs.lpt_ics(n, BOX, OM, OL, a[0], SEED + rank, order=2, device="cuda")
    npart = X.shape[1]
    W, K = args.warmup, args.steps
    probes = {}

    # f(R), the headline: the whole 100-step schedule in timed segments --
    # warm-up [0, W), the headline window [W, W+K), the middle and the late
    # window [90, 100) -- each between barriers and synchronisations
    sim = make_sim(pm, X, V, "fr")
    seg = {}
    seg["warmup"], _ = timed_steps(sim, coeffs, 0, W, world=world)
    launches0 = pm.launch_count()
    with ClockSampler(local) as clk:
        seg["window"], fr_stats = timed_steps(sim, coeffs, W, K, world=world)
    launches = pm.launch_count() - launches0
    fr_clocks = clk.summary()
    seg["middle"], _ = timed_steps(sim, coeffs, W + K, LATE - W - K, world=world)
    with ClockSampler(local) as clk_late:
        seg["late"], _ = timed_steps(sim, coeffs, LATE, N_STEPS_RUN - LATE, world=world)
    seg = {k: max_over_ranks(v, world, "cuda") for k, v in seg.items()}
    del sim
    torch.cuda.empty_cache()

    # per-kernel classes on the same window, from a fresh start, with both
    # solvers on one stream (CUDA events would time kernels sharing the GPU)
    sim = make_sim(pm, X, V, "fr")
    sim.serial = True
    timed_steps(sim, coeffs, 0, W, world=world)
    pm.timing_enable(True)
    ms_serial, _ = timed_steps(sim, coeffs, W, K, world=world)
    kern = pm.timing_collect()
    pm.timing_enable(False)
    del sim
    torch.cuda.empty_cache()

    # end to end through the C ABI with host buffers, same window: H2D of X, V
    # and D2H of X, V every step
    e2e_ms, e2e_bytes = None, None
    if not args.lean:
        sim = make_sim(pm, X, V, "fr")
        timed_steps(sim, coeffs, 0, W, world=world)
        Xh = torch.empty((3, npart), dtype=torch.int32).pin_memory()
        Vh = torch.empty((3, npart), dtype=torch.float32).pin_memory()
        Xh.copy_(sim.X)
        Vh.copy_(sim.V)
        e2e_ms, _ = timed_steps(sim, coeffs, W, K, host_buffers=(Xh, Vh), world=world)
        e2e_ms = max_over_ranks(e2e_ms, world, "cuda")
        e2e_bytes = int(Xh.numel() * 4 + Vh.numel() * 4)
        del sim, Xh, Vh
        torch.cuda.empty_cache()

    # the other gravity and solver forms on the same window
    variants = {}
    if not args.lean:
        for variant in ("newton", "newton_fft7", "fr_n2", "mu"):
            sim = make_sim(pm, X, V, variant)
            timed_steps(sim, coeffs, 0, W, world=world)
            l0 = pm.launch_count()
            ms, st = timed_steps(sim, coeffs, W, K, world=world)
            variants[variant] = {"ms": max_over_ranks(ms, world, "cuda"), "stats": st,
                                 "launches": pm.launch_count() - l0}
            del sim
            torch.cuda.empty_cache()
    if rank == 0 and not args.lean and not args.no_cpu_baseline:
        for variant in ("fr", "newton", "newton_fft7"):
            probes[variant] = patch_probe(pm, X, V, variant, coeffs, W)
    if rank != 0:
        return 0

    total = world * npart * K
    value = total / (seg["window"] / 1e3)
    peak, peak_kind = load_peaks()
    dom = max(kern.items(), key=lambda kv: kv[1][0])
    dname, (dms, dcount, dbytes) = dom
    traffic = load_ncu_traffic().get(dname)
    achieved = (dbytes / dcount) / (dms / dcount / 1e3) / 1e9 if dcount else None
    roof = {"bound": "hbm", "kernel": dname, "timed": f"per-class CUDA events, steps {W}..{W + K - 1} with both "
            "solvers on one stream", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak if achieved else None,
            "traffic": traffic.get("bytes_per_launch") if traffic else None,
            "peak_source": peak_kind,
            "launches": dcount, "avg_launch_ms": dms / dcount if dcount else None,
            "share_of_step": dms / ms_serial if ms_serial else None}
    mg_classes = [k for k in kern if k.startswith("mg_")]
    mg_ms = sum(kern[k][0] for k in mg_classes)
    mg_bytes = sum(kern[k][2] for k in mg_classes)
    vcycle = {"achieved": mg_bytes / (mg_ms / 1e3) / 1e9 if mg_ms else None, "unit": "GB/s",
              "ms_per_step": mg_ms / K, "frac": (mg_bytes / (mg_ms / 1e3) / 1e9) / peak if mg_ms else None,
              "what": "algorithmic bytes of every Poisson multigrid kernel (all levels, smoothing, transfers, "
                      "coarsest solve) / their CUDA-event time, 512^3"}
    per_kernel = {k: {"ms": round(v[0], 4), "launches": v[1],
                      "GB/s": round(v[2] / (v[0] / 1e3) / 1e9, 1) if v[0] > 0 else None,
                      "share_of_step": round(v[0] / ms_serial, 4) if ms_serial else None}
                  for k, v in kern.items() if v[1] > 0}

    def vline(key, what):
        r = variants.get(key)
        if r is None:
            return None
        out = {"value": total / (r["ms"] / 1e3), "ms_per_step": r["ms"] / K, "gpu_launches": r["launches"],
               "what": what}
        if key == "newton":
            out["mg_cycles"] = [s["mg"]["cycles"] for s in r["stats"]]
        return out

    late_n = N_STEPS_RUN - LATE
    full_ms = sum(seg.values())
    line = {
        "metric": METRIC, "value": value, "unit": "particle-steps/s", "n_gpus": world, "steps": K,
        "warmup": W, "ms_per_step": seg["window"] / K, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": headline_config(world),
        "window": {"steps": f"{W}..{W + K - 1}", "z": [1.0 / a[W] - 1.0, 1.0 / a[W + K - 1] - 1.0],
                   "what": "the headline's steps of the 100-step schedule uniform in ln a from z = 30"},
        "late": {"steps": f"{LATE}..{N_STEPS_RUN - 1}", "z": [1.0 / a[LATE] - 1.0, 1.0 / a[N_STEPS_RUN - 1] - 1.0],
                 "ms_per_step": seg["late"] / late_n, "value": world * npart * late_n / (seg["late"] / 1e3),
                 "clocks": clk_late.summary()},
        "full_run_ms_per_step": full_ms / N_STEPS_RUN,
        "full_run": {"value": world * npart * N_STEPS_RUN / (full_ms / 1e3), "seconds": full_ms / 1e3,
                     "what": "all 100 steps of the schedule (the first iterates the Poisson solve to 1e-7 from "
                             "the Jacobi guess)"},
        "newton": vline("newton", "Newtonian step, multigrid, same window"),
        "newton_fft7": vline("newton_fft7", "Newtonian step with the FFT_7pt Poisson solve (the exact 7-point "
                                            "inverse) instead of multigrid, same window"),
        "fr_n2": vline("fr_n2", "the same step with the Hu-Sawicki n = 2 scalaron (quartic per cell)"),
        "mu": vline("mu", f"the Newtonian step with parametrised gravity, mu0 = {MU0}"),
        "mg_cycles": [s["mg"]["cycles"] for s in fr_stats],
        "serial_ms_per_step": ms_serial / K,
        "e2e": None if e2e_ms is None else {
            "value": total / (e2e_ms / 1e3), "unit": "particle-steps/s",
            "h2d_bytes_per_step": e2e_bytes, "d2h_bytes_per_step": e2e_bytes},
        "gpu_launches": launches,
        "roofline": roof,
        "vcycle_hbm": vcycle,
        "kernels": per_kernel,
        "clocks": fr_clocks,
    }
    if world == 1 and not args.lean:
        line["adjoint"], probes["adjoint"] = run_adjoint()
        line["ensemble"], probes["ensemble"] = run_ensemble()
        line["poisson_precision"], probes["poisson_precision"] = run_refine()
    if world == 1 and not args.no_cpu_baseline and not args.lean:
        line["cpu_baseline"] = cpu_baseline()
        line["oracle_error"] = oracle_errors(probes)
    print(json.dumps(line))
    return 0


def run_step_stage(n, steps, warmup):
    """The f(R) step of the bench workload at n^3 particles on an n^3 grid
    (same 1 Mpc/h cells, cosmology, schedule and solver settings): a small
    case of every step kernel for profilers.  Returns the device time per
    step."""
    import torch
    from paper_2410_20501_gb300 import build, inputs, pm
    if not os.path.exists(pm.LIB_PATH):
        build.build()
    box = BOX * n / N_GRID
    a = schedule()
    coeffs = step_coefficients(OM, OL, a)
    X, V = inputs.lpt_ics(n, box, OM, OL, a[0], SEED, order=2, device="cuda")
    sim = pm.Simulation(X, V, n, OM, OL, box, gravity="fr", fR0=FR0,
                        mg=pm.default_mg(tol=1e-7, stall=0.5, max_cycles=12, fixed_cycles=2),
                        fr=pm.default_fr(cycle=1, cycles=1))
    timed_steps(sim, coeffs, 0, warmup)
    ms, _ = timed_steps(sim, coeffs, warmup, steps)
    return {"stage": "step", "n": n, "steps": steps, "ms_per_step": ms / steps}


def run_stage(args):
    """One stage alone on seeded synthetic inputs at size n (for profilers:
    a few GB on the device at most).  Prints one JSON line with the
    device time per repetition."""
    import torch
    from paper_2410_20501_gb300 import build, inputs, pm
    if not os.path.exists(pm.LIB_PATH):
        build.build()
    n = args.n
    X = None
    if args.stage in ("sort", "deposit"):
        # nearly cell-ordered, as a step receives the particles the previous
        # step wrote back: lattice order, displaced by up to 0.7 cells
        rng = np.random.Generator(np.random.PCG64(61))
        X = pm.positions_to_device(inputs.to_fixed_point(inputs.lattice(n) + rng.uniform(-0.7, 0.7, (3, n ** 3)) / n))
    elif args.stage == "interp":   # cell-ordered particles, as pm_step interpolates them
        rng = np.random.Generator(np.random.PCG64(61))
        X = pm.positions_to_device(inputs.to_fixed_point(inputs.lattice(n) + rng.uniform(-0.45, 0.45, (3, n ** 3)) / n))
    rho = None
    if args.stage in ("mg", "refine", "fr", "fft"):
        g = inputs.random_field(n, 62)
        r = np.exp(0.7 * g)
        rho = torch.from_numpy((r / r.mean()).astype(np.float32)).cuda()
    elif args.stage == "fr_batch":   # eight boxes of n^3, different seeds
        r = np.exp(0.7 * np.stack([inputs.random_field(n, 62 + b) for b in range(8)]))
        rho = torch.from_numpy((r / r.mean(axis=(1, 2, 3), keepdims=True)).astype(np.float32)).cuda()
    ws = None

    def once():
        nonlocal ws
        if args.stage == "sort":
            ws = ws if ws is not None else pm.workspace(n, n ** 3, pm.PM_WS_SORT)
            pm.sort(X, n, ws)
        elif args.stage == "deposit":
            ws = ws if ws is not None else pm.workspace(n, n ** 3, pm.PM_WS_SORT)
            pm.deposit(X, n, ws)
        elif args.stage == "mg":
            ws = ws if ws is not None else pm.workspace(n, 0, pm.PM_WS_MG)
            pm.mg_solve(rho * 0.45, ws=ws, fixed_cycles=1, first_guess=pm.MG_GUESS_JACOBI, smoother=args.smoother)
        elif args.stage == "refine":
            ws = ws if ws is not None else pm.workspace(n, 0, pm.PM_WS_MG | pm.PM_WS_REFINE)
            pm.mg_solve_refine(rho * 0.45, ws=ws, outer=2, fixed_cycles=2)
        elif args.stage == "fr_batch":
            ws = ws if ws is not None else pm.fr_batch_workspace(n, rho.shape[0])
            pm.fr_solve_batch(rho, ws=ws, a=0.6, Om=OM, OL=OL, fR0=FR0, boxsize=float(n), cycles=1, tol=0.0,
                              smoother=args.smoother)
        elif args.stage == "fr":
            ws = ws if ws is not None else pm.workspace(n, 0, pm.PM_WS_FR)
            pm.fr_solve(rho, ws=ws, a=0.6, Om=OM, OL=OL, fR0=FR0, boxsize=float(n), cycles=1,
                        smoother=args.smoother)
        elif args.stage == "interp":
            gr = torch.randn((3, n, n, n), device="cuda")
            pm.interp(gr, X)
        elif args.stage == "fft":
            ws = ws if ws is not None else pm.workspace(n, 0, pm.PM_WS_FFT)
            pm.poisson_fft(rho, scale=0.45, kind=pm.PM_POISSON_FFT7, ws=ws)

    for _ in range(args.warmup):
        once()
    torch.cuda.synchronize()
    s = torch.cuda.current_stream()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record(s)
    for _ in range(args.steps):
        once()
    t1.record(s)
    torch.cuda.synchronize()
    print(json.dumps({"stage": args.stage, "n": n, "steps": args.steps, "ms_per_rep": t0.elapsed_time(t1) / args.steps}))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--lean", action="store_true",
                    help="f(R) device-timed steps only (no Newtonian line, e2e or CPU baseline): for profilers")
    ap.add_argument("--stage", choices=["sort", "deposit", "mg", "refine", "fr", "fr_batch", "fft", "interp",
                                        "adjoint", "ensemble", "lpt", "step"],
                    help="time one stage alone on synthetic inputs (for profilers)")
    ap.add_argument("--n", type=int, default=256, help="grid size for --stage")
    ap.add_argument("--smoother", type=int, default=2,
                    help="--stage mg/fr: 2 fused sweeps, 1 colour passes, 0 two-sweep streaming")
    args = ap.parse_args()
    if args.stage == "adjoint":
        print(json.dumps(run_adjoint(args.n, fd_dirs=args.steps)[0]))
        return 0
    if args.stage == "ensemble":
        print(json.dumps(run_ensemble()[0]))
        return 0
    if args.stage == "lpt":
        print(json.dumps(run_lpt(args.n, args.steps)))
        return 0
    if args.stage == "step":
        print(json.dumps(run_step_stage(args.n, args.steps, args.warmup)))
        return 0
    if args.stage:
        return run_stage(args)
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.warmup + args.steps > LATE:
        ap.error(f"--warmup + --steps must be <= {LATE} (the late window is steps {LATE}..{N_STEPS_RUN - 1})")
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
