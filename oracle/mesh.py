"""Particle <-> mesh operators and finite differences (oracle; test infrastructure only).

Conventions (§3.2): a scalar grid is a C-ordered [n, n, n] array over cells
(i, j, k) whose centres sit at ((i + 1/2) h, (j + 1/2) h, (k + 1/2) h), h = 1/n,
periodic.  Positions are box fractions in [0, 1), given here as float64 [N, 3].
"""
import numpy as np

# Central-derivative coefficients c_n for n = -3..3 (Table 1).
GRADIENT_COEFFS = {
    3: {-1: -0.5, 1: 0.5},
    5: {-2: 1.0 / 12.0, -1: -2.0 / 3.0, 1: 2.0 / 3.0, 2: -1.0 / 12.0},
    7: {-3: -1.0 / 60.0, -2: 3.0 / 20.0, -1: -0.75, 1: 0.75, 2: -3.0 / 20.0, 3: 1.0 / 60.0},
}


def positions_from_fixed_point(X):
    """uint32 fixed-point box coordinates [3, N] -> float64 positions [N, 3]
    (x = X * 2^-32; exact in float64)."""
    X = np.asarray(X, dtype=np.uint32)
    return (X.astype(np.float64) * 2.0 ** -32).T.copy()


def w_tsc(x):
    """Triangular-shaped-cloud kernel W_TSC(x) of §3.4 (the piecewise form
    0.75 - x^2 for |x| < 0.5, (1.5 - |x|)^2 / 2 for 0.5 <= |x| < 1.5, else 0),
    x being the particle-to-cell-centre separation in units of h."""
    ax = np.abs(x)
    return np.where(ax < 0.5, 0.75 - x * x, np.where(ax < 1.5, 0.5 * (1.5 - ax) ** 2, 0.0))


def _tsc_stencil(pos, n):
    """For each particle: the 27 periodic cell flat indices and TSC weights
    (product of the per-axis W_TSC, §3.4), each a [27, N] array."""
    s = pos * n - 0.5                       # coordinate measured from cell centres
    i0 = np.floor(s + 0.5).astype(np.int64)  # nearest cell centre
    idx, wts = [], []
    for ox in (-1, 0, 1):
        for oy in (-1, 0, 1):
            for oz in (-1, 0, 1):
                c = i0 + np.array([ox, oy, oz])
                w = (w_tsc(s[:, 0] - c[:, 0]) * w_tsc(s[:, 1] - c[:, 1])
                     * w_tsc(s[:, 2] - c[:, 2]))
                c %= n
                idx.append((c[:, 0] * n + c[:, 1]) * n + c[:, 2])
                wts.append(w)
    return np.array(idx), np.array(wts)


def deposit_tsc(pos, n):
    """TSC mass assignment (§3.4): rho~_c = (n^3 / N_part) sum_p W(x_p - x_c),
    normalised so that the grid sums to n^3 (the mean density is 1; for
    N_part = n^3 this is the paper's sum rho~ = N_part)."""
    pos = np.asarray(pos, dtype=np.float64)
    N = pos.shape[0]
    rho = np.zeros(n ** 3)
    if N == 0:
        return rho.reshape(n, n, n)
    idx, wts = _tsc_stencil(pos, n)
    rho = np.bincount(idx.ravel(), weights=wts.ravel(), minlength=n ** 3)
    return (rho * (n ** 3 / N)).reshape(n, n, n)


def interp_tsc(field, pos):
    """Inverse TSC (§3.4, last paragraph): value at each particle =
    sum over the 27 cells of W(x_p - x_c) field_c.  ``field`` is [n,n,n] or a
    list of such grids (one per component); returns [N] or [N, ncomp]."""
    pos = np.asarray(pos, dtype=np.float64)
    fields = field if isinstance(field, (list, tuple)) else [field]
    n = fields[0].shape[0]
    idx, wts = _tsc_stencil(pos, n)
    out = np.stack([(wts * f.ravel()[idx]).sum(axis=0) for f in fields], axis=-1)
    return out if isinstance(field, (list, tuple)) else out[:, 0]


def cell_key(X, n):
    """Flat index (i n + j) n + k of the cell containing each particle, from
    uint32 fixed-point coordinates [3, N]: i = floor(x n).  For TSC this cell is
    also the one whose centre is nearest (§3.4)."""
    X = np.asarray(X, dtype=np.uint64)
    ijk = (X * n) >> 32
    return ((ijk[0] * n + ijk[1]) * n + ijk[2]).astype(np.uint32)


def stable_cell_order(X, n):
    """Permutation that sorts particles by cell key, ties kept in input order
    (the cell ordering that replaces the Morton reordering of §3.2)."""
    return np.argsort(cell_key(X, n), kind="stable").astype(np.uint32)


def neighbour_sum(u):
    """L_{i,j,k}(u): sum of the six face neighbours (Eq. 7pt-laplacian)."""
    return sum(np.roll(u, s, axis=a) for a in range(3) for s in (1, -1))


def laplacian7(u, h):
    """Seven-point Laplacian (L(u) - 6u) / h^2 (Eq. 7pt-laplacian)."""
    return (neighbour_sum(u) - 6.0 * u) / (h * h)


def derivative(u, axis, h, order=5):
    """Central derivative along ``axis`` with the Table 1 stencil:
    (1/h) sum_n c_n u_{i+n}."""
    out = np.zeros_like(u)
    for off, c in GRADIENT_COEFFS[order].items():
        out += c * np.roll(u, -off, axis=axis)
    return out / h


def force_from_potential(phi, h, order=5):
    """g = -grad(phi) with the Table 1 stencil (§3.5); returns [gx, gy, gz]."""
    return [-derivative(phi, a, h, order) for a in range(3)]
