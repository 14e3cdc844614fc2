"""The C ABI without a GPU: the library builds and loads, exports every function
declared in include/pm_api.h, validates arguments before touching the device,
and its host utilities agree with the oracle."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_2410_20501_gb300 import build, pm
    if not os.path.exists(pm.LIB_PATH):
        build.build()
    return pm.lib()


def header_functions():
    src = open(os.path.join(ROOT, "include", "pm_api.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^[A-Za-z_][\w\s\*]*?\b([A-Za-z_]\w*)\s*\([^;{]*\)\s*;", src, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = header_functions()
    for must in ("pm_deposit", "mg_solve", "fr_solve", "pm_gradient", "pm_interp", "pm_step", "pm_sort"):
        assert must in names


def test_every_declared_symbol_is_exported(L):
    missing = [f for f in header_functions() if not hasattr(L, f)]
    assert not missing, missing


def test_status_strings_and_version(L):
    assert L.pm_status_string(0) == b"PM_OK"
    assert b"EINVAL" in L.pm_status_string(1)
    assert L.pm_version().decode().count(".") == 2


def test_argument_errors_are_synchronous(L):
    from paper_2410_20501_gb300 import pm
    fake = ctypes.c_void_p(0x100000)      # never dereferenced: rejected before any CUDA call
    assert L.pm_deposit(fake, 10, 3, fake, fake, 1 << 20, None) == 1          # n not a power of two
    assert L.pm_deposit(fake, -1, 8, fake, fake, 1 << 20, None) == 1          # np < 0
    assert L.pm_deposit(fake, 10, 8, fake, fake, 16, None) == 2               # workspace too small
    assert L.pm_deposit(fake, 10, 8, fake, ctypes.c_void_p(0x100001), 1 << 30, None) == 1  # misaligned ws
    assert L.pm_gradient(fake, fake, 16, 4, None) == 1                        # bad stencil order
    prm = pm.default_mg(coarsest=32)
    assert L.mg_solve(fake, fake, 64, ctypes.byref(prm), None, fake, 1 << 30, None) == 1
    fr = pm.default_fr(fR0=1e-5)
    assert L.fr_solve(fake, fake, 64, ctypes.byref(fr), None, fake, 1 << 30, None) == 1


def test_misaligned_arrays_are_rejected_before_any_launch(L):
    """Every device array must start on a 16-byte boundary (kernels move grids
    as float2/float4): a view at an odd float offset is an argument error."""
    from paper_2410_20501_gb300 import pm
    ok, odd = ctypes.c_void_p(0x100000), ctypes.c_void_p(0x100004)
    prm = pm.default_mg()
    assert L.mg_solve(ok, odd, 64, ctypes.byref(prm), None, ok, 1 << 30, None) == 1
    assert L.mg_solve(odd, ok, 64, ctypes.byref(prm), None, ok, 1 << 30, None) == 1
    fr = pm.default_fr()
    assert L.fr_solve(ok, odd, 64, ctypes.byref(fr), None, ok, 1 << 30, None) == 1
    assert L.pm_deposit(odd, 10, 8, ok, ok, 1 << 30, None) == 1
    assert L.pm_sort(ok, 10, 8, odd, ok, ok, 1 << 30, None) == 1
    assert L.pm_gradient(ok, odd, 16, 5, None) == 1
    assert L.pm_interp(ok, ok, 10, 16, odd, None) == 1
    assert L.pm_deposit_adj(ok, 10, 16, ok, odd, None) == 1
    assert L.pm_gradient_adj(odd, ok, 16, 5, None) == 1
    assert L.pm_deposit_noalloc(ok, 10, 16, odd, None) == 1
    st = pm.pm_state(n=16, np=10, X=ok.value, V=odd.value, phi=ok.value, ws=ok.value, ws_bytes=1 << 30)
    sp = pm.pm_step_params(a=0.5, Om=0.3, OL=0.7, boxsize=16.0, grad_order=5, dt_kick=0.0, dt_drift=0.0,
                           phi_rescale=1.0, mg=pm.default_mg(), fr=pm.default_fr())
    assert L.pm_step(ctypes.byref(st), ctypes.byref(sp), None, None) == 1
    # the host-buffer step checks the same arguments before enqueuing any copy
    host = ctypes.c_void_p(0x200000)
    assert L.pm_step_host(ctypes.byref(st), ctypes.byref(sp), None, host, host, host, host, None) == 1
    st.V = ok.value
    st.ws_bytes = 1024
    assert L.pm_step_host(ctypes.byref(st), ctypes.byref(sp), None, host, host, host, host, None) == 2


def test_workspace_size_monotone(L):
    from paper_2410_20501_gb300 import pm
    a = pm.workspace_size(32, 32 ** 3, pm.PM_WS_STEP)
    b = pm.workspace_size(64, 64 ** 3, pm.PM_WS_STEP)
    assert 0 < a < b
    assert pm.workspace_size(64, 64 ** 3, pm.PM_WS_STEP | pm.PM_WS_IDS) > b


def test_host_cosmology_matches_oracle(L):
    from oracle import cosmology
    from paper_2410_20501_gb300 import pm
    for Om, OL in ((1.0, 0.0), (0.3, 0.7)):
        for a0, a1 in ((0.02, 0.03), (1 / 31, 0.5), (0.5, 1.0)):
            assert pm.dt_supercomoving(Om, OL, a0, a1) == pytest.approx(
                cosmology.dt_supercomoving(a0, a1, Om, OL), rel=1e-10)
        a = np.array([0.05, 0.3, 1.0])
        D = cosmology.growth_factors(a, Om, OL)[0]
        Dc = np.array([pm.growth_D(Om, OL, x) for x in a])
        assert Dc / Dc[-1] == pytest.approx(D / D[-1], rel=1e-7)


def test_batch_arguments_are_checked(L):
    from paper_2410_20501_gb300 import pm
    ok = ctypes.c_void_p(0x100000)
    size = ctypes.c_size_t()
    assert L.pm_batch_workspace_size(64, 64, 64 ** 3, ctypes.byref(size)) == 0 and size.value > 0
    big = ctypes.c_size_t()
    assert L.pm_batch_workspace_size(64, 128, 64 ** 3, ctypes.byref(big)) == 0 and big.value > size.value
    assert L.pm_batch_workspace_size(16, 4, 100, ctypes.byref(size)) == 1        # n < 32
    assert L.pm_batch_workspace_size(512, 64, 10, ctypes.byref(size)) == 1       # key bits 27 + 6 > 32
    st = pm.pm_batch_state(n=32, B=2, np_box=10, X=ok.value, V=ok.value, phi=ok.value, ws=ok.value,
                           ws_bytes=1 << 30)
    prm = pm.pm_batch_params(grad_order=5, src_scale=ok.value, dt_kick=ok.value, dt_drift=ok.value,
                             phi_rescale=ok.value, mg=pm.default_mg(fixed_cycles=0), cold_cycles=8)
    assert L.pm_step_batch(ctypes.byref(st), ctypes.byref(prm), None) == 1      # fixed cycles required
    prm.mg = pm.default_mg(fixed_cycles=2)
    prm.cold_cycles = 0
    assert L.pm_step_batch(ctypes.byref(st), ctypes.byref(prm), None) == 1      # cold cycles required
    prm.cold_cycles = 8
    st.ws_bytes = 16
    assert L.pm_step_batch(ctypes.byref(st), ctypes.byref(prm), None) == 2      # workspace too small


def test_refine_arguments_are_checked(L):
    """mg_solve_refine: its workspace adds exactly two float32 grids to the
    multigrid one; bad sizes, no refinement steps, a scaled first guess, a
    misaligned float64 iterate and a short workspace are rejected on the host."""
    from paper_2410_20501_gb300 import pm
    n = 64
    assert (pm.workspace_size(n, 0, pm.PM_WS_MG | pm.PM_WS_REFINE) - pm.workspace_size(n, 0, pm.PM_WS_MG)
            == 2 * 4 * n ** 3)
    ok = ctypes.c_void_p(0x100000)
    prm = pm.default_mg(fixed_cycles=2)
    st = pm.mg_stats()
    big = 1 << 30
    assert L.mg_solve_refine(ok, ok, 48, 2, ctypes.byref(prm), ctypes.byref(st), ok, big, None) == 1   # n
    assert L.mg_solve_refine(ok, ok, n, 0, ctypes.byref(prm), ctypes.byref(st), ok, big, None) == 1    # outer < 1
    assert L.mg_solve_refine(ok, ctypes.c_void_p(0x100008), n, 2, ctypes.byref(prm), ctypes.byref(st), ok, big,
                             None) == 1                                                                 # phi alignment
    assert L.mg_solve_refine(ok, ok, n, 2, ctypes.byref(prm), ctypes.byref(st), ok, 16, None) == 2     # workspace
    scaled = pm.default_mg(first_guess=pm.MG_GUESS_SCALED)
    assert L.mg_solve_refine(ok, ok, n, 2, ctypes.byref(scaled), ctypes.byref(st), ok, big, None) == 1


def test_fr_batch_arguments_are_checked(L):
    """fr_solve_batch: sizes, cycle count and workspace are checked on the host;
    its workspace holds B boxes' levels (more than one box's, less than B
    single-box workspaces plus nothing)."""
    from paper_2410_20501_gb300 import pm
    ok = ctypes.c_void_p(0x100000)
    one, four = ctypes.c_size_t(), ctypes.c_size_t()
    assert L.pm_fr_batch_workspace_size(64, 1, ctypes.byref(one)) == 0
    assert L.pm_fr_batch_workspace_size(64, 4, ctypes.byref(four)) == 0
    single = pm.workspace_size(64, 0, pm.PM_WS_FR)
    assert one.value == single and single < four.value <= 4 * single
    assert L.pm_fr_batch_workspace_size(16, 4, ctypes.byref(one)) == 1           # n < 32
    assert L.pm_fr_batch_workspace_size(64, 0, ctypes.byref(one)) == 1           # no boxes
    fr = pm.default_fr(cycles=1, tol=0.0)
    assert L.fr_solve_batch(ok, ok, 48, 2, ctypes.byref(fr), ok, 1 << 30, None) == 1   # n not a power of two
    assert L.fr_solve_batch(ok, ok, 64, 0, ctypes.byref(fr), ok, 1 << 30, None) == 1   # B < 1
    assert L.fr_solve_batch(ok, ok, 64, 2, ctypes.byref(fr), ok, 16, None) == 2        # workspace too small
    assert L.fr_solve_batch(ok, ctypes.c_void_p(0x100004), 64, 2, ctypes.byref(fr), ok, 1 << 30, None) == 1
    fr.cycles = 0
    assert L.fr_solve_batch(ok, ok, 64, 2, ctypes.byref(fr), ok, 1 << 30, None) == 1   # fixed cycles required
    fr = pm.default_fr(cycles=1, fR0=1e-5)
    assert L.fr_solve_batch(ok, ok, 64, 2, ctypes.byref(fr), ok, 1 << 30, None) == 1   # f_R0 >= 0



def test_adaptive_timestep_criteria(L):
    """The §3.4 time-step rule on the host (EdS: t~(a) = -2 a^(-1/2), so the
    scale factor a step reaches is known in closed form)."""
    from paper_2410_20501_gb300 import pm
    a, n = 0.05, 32
    dt, a1 = pm.next_timestep(a, 1.0, 0.0, n, 0.0, 0.0, courant=1.0, da_max=0.02)
    assert abs(a1 - 1.02 * a) < 1e-12 * a                                    # cosmological limit
    assert abs(dt - 2 * (a ** -0.5 - (1.02 * a) ** -0.5)) < 1e-12 * dt
    dt, a1 = pm.next_timestep(a, 1.0, 0.0, n, 1e6, 0.0, courant=0.5)
    assert abs(dt - 0.5 * (1.0 / n / 1e6) ** 0.5) < 1e-15                     # free fall
    assert abs(a1 - (a ** -0.5 - dt / 2) ** -2) < 1e-12 * a1
    dt, a1 = pm.next_timestep(a, 1.0, 0.0, n, 1e-6, 1e4, courant=0.5)
    assert abs(dt - 0.5 / n / 1e4) < 1e-18                                    # velocity
    dt, a1 = pm.next_timestep(a, 1.0, 0.0, n, 0.0, 0.0, courant=1.0, da_max=0.5, a_end=0.06)
    assert a1 == 0.06 and abs(dt - 2 * (a ** -0.5 - 0.06 ** -0.5)) < 1e-12 * dt   # clipped at a_end


def test_autotune_mode_is_checked_on_the_host(L):
    """pm_autotune rejects unknown modes before touching any device state; the
    report of a tuner that has seen no batched launch is empty."""
    assert L.pm_autotune(3) == 1 and L.pm_autotune(-1) == 1
    assert L.pm_autotune_report(None, 0) == 0
    assert L.pm_autotune(1) == 0


def test_next_timestep_matches_oracle(L):
    """pm_next_timestep (host code of the library) against the oracle's
    restatement of §3.4 on LCDM and EdS cases where each criterion wins."""
    from oracle.step import next_timestep as oracle_dt
    from paper_2410_20501_gb300 import pm
    cases = [(0.05, 0.3, 0.7, 512, 0.0, 0.0), (0.3, 0.3, 0.7, 512, 5e3, 0.0), (0.6, 0.3, 0.7, 256, 1e2, 40.0),
             (0.9, 0.3, 0.7, 64, 0.0, 1e3), (0.1, 1.0, 0.0, 32, 3.0, 0.5), (0.999, 0.3, 0.7, 512, 0.0, 0.0)]
    for a, Om, OL, n, acc, vel in cases:
        dt, an = pm.next_timestep(a, Om, OL, n, acc, vel, 0.8, 0.02, 1.0)
        rdt, ran = oracle_dt(a, Om, OL, n, acc, vel, 0.8, 0.02, 1.0)
        assert dt == pytest.approx(rdt, rel=1e-10) and an == pytest.approx(ran, rel=1e-12), (a, n, acc, vel)


def test_next_timestep_rejects_bad_arguments(L):
    out = ctypes.c_double()
    bad = [(0.0, 0.3, 0.7, 32, 0.0, 0.0, 0.8, 0.02, 1.0), (0.5, 0.3, 0.7, 32, 0.0, 0.0, 0.8, 0.02, 0.5),
           (0.5, 0.3, 0.7, 32, -1.0, 0.0, 0.8, 0.02, 1.0), (0.5, 0.3, 0.7, 32, 0.0, 0.0, 0.0, 0.02, 1.0)]
    for args in bad:
        assert L.pm_next_timestep(*args, ctypes.byref(out), ctypes.byref(out)) == 1
