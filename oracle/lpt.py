"""Lagrangian perturbation theory initial conditions, 1LPT and 2LPT (oracle;
test infrastructure only).

§3.3: delta = amp * FFT(noise) (amp = sqrt(P(k) n^3 / L^3) on the rfft grid),
phi1 = grad^-2 delta, Psi1 = -grad phi1,
phi2 = (1/2) grad^-2 [phi1_ii phi1_jj - phi1_ij phi1_ij] (sums over i, j),
Psi2 = grad phi2; particles start on the cell centres q and move to
x = q + d1 Psi1 + e2 Psi2 with velocities v = v1 Psi1 + v2 Psi2 (d1, e2 the
first- and second-order growth factors, v1, v2 the matching velocity factors).
Derivatives are spectral with k = 2 pi m (box units); every Fourier mode on a
Nyquist plane (|m_d| = n/2 on any axis) is set to zero, in phi1 and in phi2.
"""
import numpy as np


def _kgrid(n):
    m = np.fft.fftfreq(n) * n
    mz = np.fft.rfftfreq(n) * n
    k = [2 * np.pi * m[:, None, None], 2 * np.pi * m[None, :, None], 2 * np.pi * mz[None, None, :]]
    nyq = (np.abs(m) == n // 2)
    bad = nyq[:, None, None] | nyq[None, :, None] | (mz == n // 2)[None, None, :]
    return k, bad


def _inv_laplacian(fk, k, bad):
    k2 = k[0] ** 2 + k[1] ** 2 + k[2] ** 2
    k2[0, 0, 0] = 1.0
    out = -fk / k2
    out[0, 0, 0] = 0.0
    out[np.broadcast_to(bad, out.shape)] = 0.0
    return out


def potentials(noise, amp):
    """(phi1_k, phi2_k) on the rfft grid from real white noise [n, n, n]."""
    n = noise.shape[0]
    k, bad = _kgrid(n)
    delta_k = np.fft.rfftn(noise) * amp
    phi1 = _inv_laplacian(delta_k, k, bad)
    d2 = {}
    for i in range(3):
        for j in range(i, 3):
            d2[(i, j)] = np.fft.irfftn(-k[i] * k[j] * phi1, s=(n, n, n), axes=(0, 1, 2))
    diag = d2[(0, 0)] * d2[(1, 1)] + d2[(0, 0)] * d2[(2, 2)] + d2[(1, 1)] * d2[(2, 2)]
    off = d2[(0, 1)] ** 2 + d2[(0, 2)] ** 2 + d2[(1, 2)] ** 2
    # (1/2) sum_ij (phi_ii phi_jj - phi_ij phi_ij) = sum_{i<j} (phi_ii phi_jj - phi_ij^2)
    phi2 = _inv_laplacian(np.fft.rfftn(diag - off), k, bad)
    return phi1, phi2


def displacements(noise, amp):
    """(Psi1, Psi2), each [3, n^3] float64."""
    n = noise.shape[0]
    k, _ = _kgrid(n)
    phi1, phi2 = potentials(noise, amp)
    psi1 = np.stack([np.fft.irfftn(-1j * kd * phi1, s=(n, n, n), axes=(0, 1, 2)).reshape(-1) for kd in k])
    psi2 = np.stack([np.fft.irfftn(1j * kd * phi2, s=(n, n, n), axes=(0, 1, 2)).reshape(-1) for kd in k])
    return psi1, psi2


def lattice(n):
    c = (np.arange(n) + 0.5) / n
    return np.stack([g.reshape(-1) for g in np.meshgrid(c, c, c, indexing="ij")])


def lpt2(noise, amp, d1, e2, v1, v2):
    """Positions x = q + d1 Psi1 + e2 Psi2 (box units, wrapped into [0, 1))
    and velocities v1 Psi1 + v2 Psi2, each [3, n^3]."""
    n = noise.shape[0]
    psi1, psi2 = displacements(noise, amp)
    return (lattice(n) + d1 * psi1 + e2 * psi2) % 1.0, v1 * psi1 + v2 * psi2
