"""Background cosmology for the oracle (test infrastructure only).

Flat LCDM / Einstein-de Sitter without radiation, as used by the hot-path
configurations.  Supercomoving units follow §3.1: positions in box units, the
time unit t_* = a^2 / H0, so that d(t~) = H0 dt / a^2 = da / (a^3 E(a)).
"""
import numpy as np
from scipy.integrate import quad, solve_ivp

C_KM_S = 299792.458  # speed of light [km/s]


def hubble_E(a, Om, OL):
    """E(a) = H(a)/H0 for a flat universe without radiation (§2.2, H(z) with
    Omega_r = 0 and a cosmological constant, w0 = -1, wa = 0)."""
    return np.sqrt(Om * a ** -3.0 + OL)


def dt_supercomoving(a0, a1, Om, OL):
    """Supercomoving time elapsed between a0 and a1 (§3.1: dt~ = dt / t_*,
    t_* = a^2/H0; with da/dt = a H0 E(a) this is the integral of
    da / (a^3 E(a)))."""
    val, _ = quad(lambda a: 1.0 / (a ** 3 * hubble_E(a, Om, OL)), a0, a1,
                  epsabs=0.0, epsrel=1e-13, limit=200)
    return val


def c_tilde(boxsize_mpc_h):
    """Speed of light in simulation units (§3.1: c~ = c t_* / (a x_*)).  With
    x_* = a L_box and t_* = a^2/H0 this is c / (H0 L_box); for L_box in Mpc/h
    and H0 = 100 h km/s/Mpc it is constant in time."""
    return C_KM_S / (100.0 * boxsize_mpc_h)


def omega_m_of_a(a, Om, OL):
    """Omega_m(a) = Omega_m a^-3 / E(a)^2."""
    return Om * a ** -3.0 / hubble_E(a, Om, OL) ** 2


def omega_l_of_a(a, Om, OL):
    """Omega_Lambda(a) = Omega_Lambda / E(a)^2 (w = -1)."""
    return OL / hubble_E(a, Om, OL) ** 2


def mu_parametrised(a, Om, OL, mu0):
    """Effective gravitational coupling of the parametrised model (§2.4,
    Eq. mu_parametrized_gravity): mu(a) = 1 + mu0 Omega_Lambda(a) / Omega_Lambda,0."""
    return 1.0 + mu0 * omega_l_of_a(a, Om, OL) / OL


def growth_factors(a_eval, Om, OL, a_start=1e-5):
    """First and second order growth factors D, E and rates f1 = D'/D,
    f2 = E'/E (Appendix A, the ODEs in ln a):

        D'' = -gamma D' + beta D
        E'' = -gamma E' + beta (E - D^2)

    with beta = 3/2 Omega_m(a) and gamma = 1/2 (1 - 3 Omega_L(a) w - Omega_r(a))
    for w = -1, Omega_r = 0.  Started deep in matter domination on the growing
    mode D = a, E = -3/7 a^2 (Appendix A, EdS limits).  D is not normalised.
    Returns arrays (D, E, f1, f2) at a_eval (scalar or increasing sequence).
    """
    a_eval = np.atleast_1d(np.asarray(a_eval, dtype=np.float64))

    def rhs(lna, y):
        a = np.exp(lna)
        D, dD, E, dE = y
        beta = 1.5 * omega_m_of_a(a, Om, OL)
        gamma = 0.5 * (1.0 + 3.0 * omega_l_of_a(a, Om, OL))
        return [dD, -gamma * dD + beta * D, dE, -gamma * dE + beta * (E - D * D)]

    y0 = [a_start, a_start, -3.0 / 7.0 * a_start ** 2, -6.0 / 7.0 * a_start ** 2]
    grid = np.unique(a_eval)
    sol = solve_ivp(rhs, (np.log(a_start), np.log(grid[-1])), y0,
                    t_eval=np.log(grid), rtol=1e-12, atol=1e-30, method="DOP853")
    at = np.searchsorted(grid, a_eval)
    D, dD, E, dE = (row[at] for row in sol.y)
    return D, E, dD / D, dE / E
