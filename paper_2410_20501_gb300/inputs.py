"""Seeded synthetic inputs: particle states and fields shaped like the paper's runs.

This module only draws and shapes inputs; it holds none of the force-step
arithmetic (no mass assignment, no 7-point Laplacian or multigrid, no
finite-difference gradient, no leapfrog).  Both the CUDA path and the FP64
oracle take its outputs as inputs.

Initial conditions follow §3.3: Gaussian white noise (drawn in configuration
space from numpy's PCG64, which has the same statistics as the Fourier-space
Rayleigh-amplitude / uniform-phase draw of §3.3), coloured by sqrt(P(k)),
then first / second order Lagrangian displacements computed spectrally
(Psi1 = -grad phi1, grad^2 phi1 = delta; Psi2 = grad phi2,
grad^2 phi2 = 1/2 [phi1_ii phi1_jj - phi1_ij phi1_ij]) and placed on cell
centres (Appendix B.2).  Velocities in simulation units (§3.1) are
v~ = a^2 E(a) (D f1 Psi1 + E f2 Psi2).

The linear spectrum is the no-wiggle Eisenstein & Hu (1998) fitting formula
(their Eqs. 26, 28-31) standing in for the CAMB spectrum of §4, normalised to
sigma8; FFTs run through torch (CPU or GPU) in float64.
"""
import math

import numpy as np
import torch
from scipy.integrate import quad, solve_ivp

TWO32 = 2.0 ** 32


def white_noise(n, seed):
    """Unit Gaussian white noise on an n^3 grid from numpy PCG64(seed)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.standard_normal((n, n, n))


def to_fixed_point(pos):
    """float64 box positions [3, N] (any real value) -> uint32 fixed point
    x * 2^32 wrapped into [0, 2^32)."""
    x = np.mod(np.asarray(pos, dtype=np.float64), 1.0)
    X = np.floor(x * TWO32 + 0.5)
    X[X >= TWO32] -= TWO32
    return X.astype(np.uint32)


def lattice(n):
    """Cell-centre positions (i + 1/2)/n as float64 [3, n^3], C order."""
    g = (np.arange(n) + 0.5) / n
    x, y, z = np.meshgrid(g, g, g, indexing="ij")
    return np.stack([x.ravel(), y.ravel(), z.ravel()])


def uniform_particles(N, seed):
    """N uniformly random uint32 fixed-point positions [3, N]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.integers(0, 2 ** 32, size=(3, N), dtype=np.uint64).astype(np.uint32)


def random_field(n, seed, scale=1.0):
    """float64 white-noise field (e.g. a synthetic density contrast)."""
    return scale * white_noise(n, seed)


# ---------------------------------------------------------------- cosmology ---

def hubble_E(a, Om, OL):
    return math.sqrt(Om * a ** -3 + OL)


def growth(a_list, Om, OL):
    """(D, E, f1, f2) at the given scale factors from the Appendix A growth
    ODEs in ln a, started on the matter-dominated growing mode."""
    a_list = np.atleast_1d(np.asarray(a_list, dtype=np.float64))

    def rhs(lna, y):
        a = math.exp(lna)
        e2 = Om * a ** -3 + OL
        beta = 1.5 * Om * a ** -3 / e2
        gamma = 0.5 * (1.0 + 3.0 * OL / e2)
        D, dD, E, dE = y
        return [dD, -gamma * dD + beta * D, dE, -gamma * dE + beta * (E - D * D)]

    a0 = 1e-5
    y0 = [a0, a0, -3.0 / 7.0 * a0 ** 2, -6.0 / 7.0 * a0 ** 2]
    order = np.argsort(a_list)
    sol = solve_ivp(rhs, (math.log(a0), math.log(a_list.max())), y0,
                    t_eval=np.log(a_list[order]), rtol=1e-11, atol=1e-30, method="DOP853")
    out = np.empty((4, a_list.size))
    D, dD, E, dE = sol.y
    out[:, order] = np.stack([D, E, dD / D, dE / E])
    return out


def eh_nowiggle_transfer(k_h, Om, Ob, h, Tcmb=2.7255):
    """Eisenstein & Hu (1998) zero-baryon-oscillation transfer function,
    k in h/Mpc."""
    theta = Tcmb / 2.7
    om = Om * h * h
    fb = Ob / Om
    s = 44.5 * np.log(9.83 / om) / np.sqrt(1.0 + 10.0 * (Ob * h * h) ** 0.75)
    alpha = 1.0 - 0.328 * np.log(431.0 * om) * fb + 0.38 * np.log(22.3 * om) * fb * fb
    k_mpc = k_h * h
    gamma_eff = Om * h * (alpha + (1.0 - alpha) / (1.0 + (0.43 * k_mpc * s) ** 4))
    q = k_h * theta * theta / gamma_eff
    L0 = np.log(2.0 * math.e + 1.8 * q)
    C0 = 14.2 + 731.0 / (1.0 + 62.5 * q)
    return L0 / (L0 + C0 * q * q)


def linear_power(Om, Ob, h, ns, sigma8):
    """P(k, z=0) [(Mpc/h)^3], k in h/Mpc, normalised to sigma8 (top hat of
    8 Mpc/h)."""
    def shape(k):
        return k ** ns * eh_nowiggle_transfer(k, Om, Ob, h) ** 2

    def integrand(lnk):
        k = math.exp(lnk)
        x = 8.0 * k
        w = 3.0 * (math.sin(x) - x * math.cos(x)) / x ** 3
        return k ** 3 * shape(k) * w * w / (2.0 * math.pi ** 2)

    s2, _ = quad(integrand, math.log(1e-5), math.log(1e3), limit=500)
    amp = sigma8 ** 2 / s2
    return lambda k: amp * shape(k)


# ------------------------------------------------------------ displacements ---

def _kgrid(n, device):
    m = torch.fft.fftfreq(n, d=1.0 / n, dtype=torch.float64, device=device)
    mz = torch.fft.rfftfreq(n, d=1.0 / n, dtype=torch.float64, device=device)
    kx = 2.0 * math.pi * m[:, None, None]
    ky = 2.0 * math.pi * m[None, :, None]
    kz = 2.0 * math.pi * mz[None, None, :]
    nyq = (m.abs() == n // 2)
    bad = nyq[:, None, None] | nyq[None, :, None] | (mz == n // 2)[None, None, :]
    return kx, ky, kz, bad


def _lpt_potentials(delta_k, n, order, device):
    """Spectral phi1 (grad^2 phi1 = delta) and, for order 2, phi2; returned in
    Fourier space.  Box units (k = 2 pi m)."""
    kx, ky, kz, bad = _kgrid(n, device)
    k2 = kx * kx + ky * ky + kz * kz
    k2[0, 0, 0] = 1.0
    phi1 = -delta_k / k2
    phi1[0, 0, 0] = 0.0
    phi1 = torch.where(bad, torch.zeros_like(phi1), phi1)
    if order < 2:
        return phi1, None
    kk = [kx, ky, kz]
    d2 = {}
    for i in range(3):
        for j in range(i, 3):
            d2[(i, j)] = torch.fft.irfftn(-kk[i] * kk[j] * phi1, s=(n, n, n))
    src = (d2[(0, 0)] * d2[(1, 1)] + d2[(0, 0)] * d2[(2, 2)] + d2[(1, 1)] * d2[(2, 2)]
           - d2[(0, 1)] ** 2 - d2[(0, 2)] ** 2 - d2[(1, 2)] ** 2)
    del d2
    src_k = torch.fft.rfftn(src)
    phi2 = -src_k / k2
    phi2[0, 0, 0] = 0.0
    phi2 = torch.where(bad, torch.zeros_like(phi2), phi2)
    return phi1, phi2


def _grad(phi_k, n, device):
    kx, ky, kz, _ = _kgrid(n, device)
    return torch.stack([torch.fft.irfftn(1j * k * phi_k, s=(n, n, n)).reshape(-1)
                        for k in (kx, ky, kz)])


def lpt_ics(n, boxsize, Om, OL, a_ini, seed, order=2, h=0.7, Ob=0.05, ns=0.96,
            sigma8=0.8, device="cpu"):
    """LCDM initial conditions on a lattice of n^3 particles at cell centres:
    returns (X uint32 [3, N], V float64 [3, N]) in supercomoving units."""
    pk = linear_power(Om, Ob, h, ns, sigma8)
    D, E, f1, f2 = growth([a_ini, 1.0], Om, OL)
    d_ratio = D[0] / D[1]
    noise = torch.from_numpy(white_noise(n, seed)).to(device)
    wk = torch.fft.rfftn(noise)
    del noise
    kx, ky, kz, _ = _kgrid(n, device)
    kmag = torch.sqrt(kx * kx + ky * ky + kz * kz) / boxsize   # h/Mpc
    kmag[0, 0, 0] = 1.0
    kcpu = kmag.cpu().numpy()
    amp = torch.from_numpy(np.sqrt(pk(kcpu) * n ** 3 / boxsize ** 3)).to(device)
    amp[0, 0, 0] = 0.0
    delta_k = wk * amp          # z = 0 linear density contrast
    del wk, amp, kmag
    phi1, phi2 = _lpt_potentials(delta_k, n, order, device)
    psi1 = -_grad(phi1, n, device)
    a = a_ini
    vfac = a * a * hubble_E(a, Om, OL)
    D1 = d_ratio                                    # normalised D(a_ini)/D(1)
    E1 = E[0] / D[1] ** 2                           # second-order factor in the same normalisation
    pos = torch.from_numpy(lattice(n)).to(device) + D1 * psi1
    vel = vfac * D1 * f1[0] * psi1
    del psi1
    if order >= 2:
        psi2 = _grad(phi2, n, device)
        pos += E1 * psi2
        vel += vfac * E1 * f2[0] * psi2
    X = to_fixed_point(pos.cpu().numpy())
    return X, vel.cpu().numpy()


def zeldovich_powerlaw_ics(n=32, seed=1, a_ini=0.02, rms_cells=0.2):
    """Einstein-de Sitter Zel'dovich initial conditions with a density spectrum
    P(k) proportional to k^-2 (white noise times 1/k), scaled so that the RMS
    displacement 3-vector is ``rms_cells`` cells at a_ini; v~ = Psi a^(1/2)
    (EdS: D = a, f = 1, a^2 E(a) = a^(1/2)).  Returns (X uint32 [3,N],
    V float64 [3,N])."""
    noise = torch.from_numpy(white_noise(n, seed))
    wk = torch.fft.rfftn(noise)
    kx, ky, kz, bad = _kgrid(n, "cpu")
    k2 = kx * kx + ky * ky + kz * kz
    k2[0, 0, 0] = 1.0
    delta_k = wk / torch.sqrt(k2)
    delta_k[0, 0, 0] = 0.0
    delta_k = torch.where(bad, torch.zeros_like(delta_k), delta_k)
    phi1, _ = _lpt_potentials(delta_k, n, 1, "cpu")
    psi = -_grad(phi1, n, "cpu").numpy()
    rms = np.sqrt((psi ** 2).sum(axis=0).mean())
    psi *= (rms_cells / n) / rms
    X = to_fixed_point(lattice(n) + psi)
    V = psi * math.sqrt(a_ini)
    return X, V


# ------------------------------------------------------ differentiable runs ---

def lpt_amplitude(n, boxsize, Om=0.3, Ob=0.05, h=0.7, ns=0.96, sigma8=0.8):
    """sqrt(P(k) n^3 / L^3) on the rfft grid [n, n, n//2+1] (float64 numpy),
    zero at k = 0 and on the Nyquist planes: the factor that turns the FFT of
    unit white noise into the z = 0 linear density contrast."""
    pk = linear_power(Om, Ob, h, ns, sigma8)
    kx, ky, kz, bad = _kgrid(n, "cpu")
    kmag = torch.sqrt(kx * kx + ky * ky + kz * kz) / boxsize
    kmag[0, 0, 0] = 1.0
    amp = np.sqrt(pk(kmag.numpy()) * n ** 3 / boxsize ** 3)
    amp[0, 0, 0] = 0.0
    amp[bad.numpy()] = 0.0
    return amp


def lpt_growth(a_ini, Om, OL):
    """(D(a)/D(1), a^2 E(a) D(a)/D(1) f(a)): the displacement and velocity
    factors of first-order LPT at a_ini."""
    D, _, f1, _ = growth([a_ini, 1.0], Om, OL)
    d_ratio = D[0] / D[1]
    return d_ratio, a_ini * a_ini * hubble_E(a_ini, Om, OL) * d_ratio * f1[0]


def c4_workload(n, boxsize=200.0, Om=0.3, z_ini=20.0, steps=10, noise_seed=4, target_seed=5):
    """The differentiable-PM workload: unit white noise (seed 4), the target
    noise (seed 5), the spectrum amplitude, LPT factors and the scale factors
    of ``steps`` leapfrog steps uniform in a from 1/(1+z_ini) to 1."""
    a_ini = 1.0 / (1.0 + z_ini)
    d_ratio, vfac = lpt_growth(a_ini, Om, 1.0 - Om)
    return {"noise": white_noise(n, noise_seed), "target_noise": white_noise(n, target_seed),
            "amp": lpt_amplitude(n, boxsize, Om), "d_ratio": d_ratio, "vfac": vfac,
            "a_steps": list(np.linspace(a_ini, 1.0, steps + 1)), "Om": Om, "OL": 1.0 - Om, "boxsize": boxsize}


def ensemble_workload(n=64, B=64, boxsize=128.0, z_ini=30.0, steps=50, param_seed=3, box_seed0=1000,
                      device="cpu"):
    """The ensemble workload: B boxes of n^3 particles (2LPT at z_ini), box b
    from white-noise seed box_seed0 + b, with Omega_m ~ U[0.25, 0.35] and
    sigma8 ~ U[0.7, 0.9] drawn from PCG64(param_seed), flat; scale factors of
    ``steps`` steps uniform in ln a to a = 1.  Returns a dict with X uint32
    [B, 3, n^3], V float32 [B, 3, n^3], Om [B], sigma8 [B], a_steps."""
    rng = np.random.Generator(np.random.PCG64(param_seed))
    Om = rng.uniform(0.25, 0.35, B)
    s8 = rng.uniform(0.7, 0.9, B)
    a_ini = 1.0 / (1.0 + z_ini)
    X = np.empty((B, 3, n ** 3), dtype=np.uint32)
    V = np.empty((B, 3, n ** 3), dtype=np.float32)
    for b in range(B):
        X[b], V[b] = lpt_ics(n, boxsize, float(Om[b]), 1.0 - float(Om[b]), a_ini, box_seed0 + b, order=2,
                             sigma8=float(s8[b]), device=device)
    a_steps = list(np.exp(np.linspace(math.log(a_ini), 0.0, steps + 1)))
    return {"X": X, "V": V, "Om": Om, "sigma8": s8, "a_steps": a_steps, "n": n, "B": B, "boxsize": boxsize}
