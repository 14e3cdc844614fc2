"""Power-spectrum estimator (oracle; test infrastructure only)."""
import numpy as np


def power_spectrum(rho, boxsize):
    """Simple estimator without dealiasing or shot-noise subtraction (§4):
    delta = rho~/<rho~> - 1, P(k) = (L^3 / n^6) |FFT(delta)|^2 averaged in
    shells of width k_f = 2 pi / L centred on integer multiples of k_f.
    Returns (k, P, modes) for shells 1 .. n/2."""
    n = rho.shape[0]
    delta = rho / rho.mean() - 1.0
    dk = np.fft.rfftn(delta)
    m = np.fft.fftfreq(n) * n
    mz = np.fft.rfftfreq(n) * n
    mag = np.sqrt(m[:, None, None] ** 2 + m[None, :, None] ** 2 + mz[None, None, :] ** 2)
    # modes on the kz = 0 and kz = Nyquist planes appear once in rfft; others twice
    weight = np.full(mag.shape, 2.0)
    weight[:, :, 0] = 1.0
    if n % 2 == 0:
        weight[:, :, -1] = 1.0
    shell = np.rint(mag).astype(int)
    p = (np.abs(dk) ** 2) * boxsize ** 3 / n ** 6
    nb = n // 2 + 1
    cnt = np.bincount(shell.ravel(), weights=weight.ravel(), minlength=nb)[:nb]
    pk = np.bincount(shell.ravel(), weights=(weight * p).ravel(), minlength=nb)[:nb]
    ks = np.bincount(shell.ravel(), weights=(weight * mag).ravel(), minlength=nb)[:nb]
    sel = slice(1, nb)
    kf = 2.0 * np.pi / boxsize
    return ks[sel] / cnt[sel] * kf, pk[sel] / cnt[sel], cnt[sel]
