"""Differentiable PM: autograd over the CUDA step and its hand-written adjoint.

Forward model: white noise w on an n^3 grid -> first-order LPT initial
conditions (§3.3: delta_k = sqrt(P(k) n^3 / L^3) w_k, div Psi = -delta,
x = q + D Psi, v~ = a^2 E(a) D f Psi) -> kick-drift-kick PM steps (pm_step)
-> TSC density -> loss.  The LPT transform is written with torch.fft so autograd follows it;
each PM step and the final deposit are autograd Functions whose backward calls
the library's adjoint entry points (pm_step_adj, pm_deposit_adj).  Each step
keeps its inputs (positions as uint32 fixed point, velocities: 24 B per
particle) and the potential it solved for (4 B per cell), so the backward pass
re-sorts the particles but solves only the adjoint Poisson problem.  Within a
forward pass each step's Poisson solve starts from the previous step's
potential rescaled by a D(a) (the first from the Jacobi guess) and runs to
the multigrid tolerance.

Positions flow through autograd as float64 box coordinates [3, np]; the step
converts them to uint32 fixed point (the rounding, 2^-32 of the box, is
treated as the identity for derivatives).
"""

import numpy as np
import torch

from . import inputs, pm

TWO32 = 4294967296.0


def to_bits(x):
    """float64 box positions -> int32 tensor holding the uint32 fixed point."""
    X = torch.floor(torch.remainder(x, 1.0) * TWO32 + 0.5).to(torch.int64)
    X = torch.where(X >= int(TWO32), X - int(TWO32), X)
    return torch.where(X >= 2 ** 31, X - 2 ** 32, X).to(torch.int32).contiguous()


def from_bits(X):
    """int32 fixed-point bits -> float64 box positions."""
    Xi = X.to(torch.int64)
    Xi = torch.where(Xi < 0, Xi + 2 ** 32, Xi)
    return Xi.to(torch.float64) / TWO32


class Stepper:
    """Owns the device state and workspace used by the step Functions."""

    def __init__(self, n, npart, Om, OL, boxsize, grad_order=5, mg=None, device="cuda"):
        dummyX = np.zeros((3, npart), dtype=np.uint32)
        dummyV = np.zeros((3, npart), dtype=np.float32)
        self.sim = pm.Simulation(dummyX, dummyV, n, Om, OL, boxsize, grad_order=grad_order,
                                 mg=mg if mg is not None else pm.default_mg(tol=1e-7, stall=0.5, max_cycles=20),
                                 adjoint=True, device=device)
        self.n, self.np, self.Om, self.OL = n, npart, Om, OL

    def load(self, Xbits, V):
        self.sim.X.copy_(Xbits)
        self.sim.V.copy_(V.to(torch.float32))


class _StepFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, v, stepper, a, dt_kick, dt_drift, rescale, first):
        Xb = to_bits(x.detach())
        Vin = v.detach().to(torch.float32).contiguous()
        stepper.load(Xb, Vin)
        if first:
            stepper.sim.state.have_prev = 0      # Jacobi first guess; later steps start from the last potential
        stepper.sim.step(a, dt_kick, dt_drift, rescale)
        ctx.save_for_backward(Xb, Vin, stepper.sim.phi.clone())
        ctx.stepper, ctx.coef = stepper, (a, dt_kick, dt_drift)
        return from_bits(stepper.sim.X.clone()), stepper.sim.V.clone().to(v.dtype)

    @staticmethod
    def backward(ctx, gx, gv):
        Xb, Vin, phi = ctx.saved_tensors
        st = ctx.stepper
        st.load(Xb, Vin)
        a, dtk, dtd = ctx.coef
        gx = torch.zeros((3, st.np), dtype=torch.float32, device=Xb.device) if gx is None else gx
        gv = torch.zeros((3, st.np), dtype=torch.float32, device=Xb.device) if gv is None else gv
        xb, vb = st.sim.step_adjoint(a, dtk, dtd, gx.to(torch.float32).contiguous(),
                                     gv.to(torch.float32).contiguous(), phi=phi)
        return xb.to(torch.float64), vb.to(gv.dtype), None, None, None, None, None, None


class _DepositFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, n):
        Xb = to_bits(x.detach())
        ctx.save_for_backward(Xb)
        ctx.n = n
        return pm.deposit(Xb, n)

    @staticmethod
    def backward(ctx, grho):
        (Xb,) = ctx.saved_tensors
        return pm.deposit_adj(Xb, ctx.n, grho.to(torch.float32).contiguous()).to(torch.float64), None


def pm_step(x, v, stepper, a, dt_kick, dt_drift, rescale=1.0, first=True):
    """One differentiable pm_step.  first: start the Poisson solve from the
    Jacobi guess; otherwise from the stepper's last potential times rescale."""
    return _StepFn.apply(x, v, stepper, a, dt_kick, dt_drift, rescale, first)


def deposit(x, n):
    return _DepositFn.apply(x, n)


def lpt1_from_noise(w, amp, d_ratio, vfac):
    """First-order LPT (§3.3) from real-space white noise w [n, n, n]
    (float64, differentiable): delta_k = amp_k FFT(w)_k, Psi_k = i k delta_k / k^2
    (so div Psi = -delta), x = q + d_ratio Psi on the cell-centre lattice q,
    v~ = vfac Psi.  ``amp`` is sqrt(P(k) n^3 / L^3) on the rfft grid (zero at
    k = 0 and on the Nyquist planes).  Returns (x [3, n^3], v [3, n^3]) float64."""
    n = w.shape[0]
    dev = w.device
    kx, ky, kz, _ = inputs._kgrid(n, dev)
    k2 = kx * kx + ky * ky + kz * kz
    k2[0, 0, 0] = 1.0
    delta_k = torch.fft.rfftn(w) * torch.as_tensor(amp, dtype=torch.float64, device=dev)
    psi = torch.stack([torch.fft.irfftn(1j * kd * delta_k / k2, s=(n, n, n)).reshape(-1) for kd in (kx, ky, kz)])
    q = torch.from_numpy(inputs.lattice(n)).to(dev)
    return q + d_ratio * psi, vfac * psi


def schedule_coefficients(a_steps, Om, OL):
    """(a_i, dt_kick_i, dt_drift_i, rescale_i) of the fused-kick leapfrog
    through a_steps that ends with the drift to a_steps[-1]: the force at a_i
    kicks by (dt_{i-1} + dt_i)/2 (dt_{-1} = 0), then the particles drift by
    dt_i; rescale_i = a_i D_i / (a_{i-1} D_{i-1}) scales the previous
    potential into the first guess.  The closing half kick at a_steps[-1]
    changes only velocities and is left out (a density loss does not see it)."""
    dts = [pm.dt_supercomoving(Om, OL, a_steps[i], a_steps[i + 1]) for i in range(len(a_steps) - 1)]
    aD = [a * pm.growth_D(Om, OL, a) for a in a_steps]
    return [(a_steps[i], 0.5 * ((dts[i - 1] if i > 0 else 0.0) + dts[i]), dts[i],
             aD[i] / aD[i - 1] if i > 0 else 1.0) for i in range(len(dts))]


def forward_model(w, stepper, amp, d_ratio, vfac, steps):
    """White noise -> LPT -> ``steps`` [(a, dt_kick, dt_drift, rescale)] ->
    final TSC density (differentiable in w)."""
    x, v = lpt1_from_noise(w, amp, d_ratio, vfac)
    for i, (a, dtk, dtd, resc) in enumerate(steps):
        x, v = pm_step(x, v, stepper, a, dtk, dtd, resc, first=(i == 0))
    return deposit(x, stepper.n)


def density_loss(w, target, stepper, amp, d_ratio, vfac, steps):
    """sum_c (rho~_c - target_c)^2 of the forward model's final density."""
    rho = forward_model(w, stepper, amp, d_ratio, vfac, steps)
    return ((rho.to(torch.float64) - target) ** 2).sum()
