"""Pins of the oracle's particle-mesh operators against the paper and mathematics (CPU)."""
import itertools

import numpy as np
import pytest

from oracle import mesh
from paper_2410_20501_gb300 import inputs


def test_tsc_kernel_printed_values(golden):
    g = golden["tsc_kernel"]
    for x, w in zip(g["x"], g["W"]):
        assert mesh.w_tsc(np.array([x, -x])) == pytest.approx([w, w], abs=1e-15)


def test_tsc_partition_of_unity():
    d = np.linspace(-0.5, 0.5, 1001, endpoint=False)
    s = sum(mesh.w_tsc(d - o) for o in (-1, 0, 1))
    assert np.abs(s - 1.0).max() < 1e-15


def test_deposit_lattice_is_uniform():
    n = 8
    rho = mesh.deposit_tsc(inputs.lattice(n).T, n)
    assert np.abs(rho - 1.0).max() < 1e-14


def test_deposit_mass_conservation_random():
    n = 16
    pos = np.random.default_rng(3).random((1000, 3))
    rho = mesh.deposit_tsc(pos, n)
    assert rho.sum() == pytest.approx(n ** 3, rel=1e-13)
    assert rho.min() >= 0.0


def test_point_mass_at_centre_and_edge(golden):
    g = golden["point_mass_cells"]
    n = 8
    rho = mesh.deposit_tsc(np.array([[3.5, 3.5, 3.5]]) / n, n) / n ** 3
    assert np.count_nonzero(rho) == g["centre_nonzero_cells"]
    w1 = np.array([mesh.w_tsc(1.0), mesh.w_tsc(0.0), mesh.w_tsc(1.0)])
    assert np.allclose(rho[2:5, 2:5, 2:5], np.einsum("i,j,k->ijk", w1, w1, w1), atol=1e-15)
    rho = mesh.deposit_tsc(np.array([[3.0, 3.0, 3.0]]) / n, n) / n ** 3
    nz = rho[rho > 1e-15]
    assert nz.size == g["edge_nonzero_cells"]
    assert np.allclose(nz, g["edge_fraction_per_cell"], atol=1e-15)


def test_deposit_matches_brute_force_n4():
    """All-cells x all-particles sum with minimal-image separations."""
    n = 4
    pos = np.random.default_rng(5).random((7, 3))
    rho = np.zeros((n, n, n))
    for i, j, k in itertools.product(range(n), repeat=3):
        c = (np.array([i, j, k]) + 0.5) / n
        for p in pos:
            s = (p - c) * n
            s -= n * np.rint(s / n)
            rho[i, j, k] += float(np.prod(mesh.w_tsc(s)))
    rho *= n ** 3 / len(pos)
    assert np.abs(mesh.deposit_tsc(pos, n) - rho).max() < 1e-13


def test_deposit_interp_adjoint():
    n = 16
    rng = np.random.default_rng(7)
    pos = rng.random((500, 3))
    G = rng.standard_normal((n, n, n))
    lhs = (mesh.deposit_tsc(pos, n) * G).sum()
    rhs = n ** 3 / len(pos) * mesh.interp_tsc(G, pos).sum()
    assert lhs == pytest.approx(rhs, rel=1e-12)


def test_interp_reproduces_linear_field_inside():
    """TSC is a symmetric quadratic B-spline: it reproduces affine fields."""
    n = 16
    i = np.arange(n) + 0.5
    F = np.broadcast_to(2.0 * i[:, None, None] + 0.5 * i[None, :, None] - i[None, None, :], (n, n, n))
    pos = np.random.default_rng(8).uniform(0.3, 0.7, (50, 3))
    exact = (2.0 * pos[:, 0] + 0.5 * pos[:, 1] - pos[:, 2]) * n
    assert np.abs(mesh.interp_tsc(np.ascontiguousarray(F), pos) - exact).max() < 1e-12


def test_cell_key_and_stable_order():
    n = 8
    X = inputs.uniform_particles(300, 11)
    key = mesh.cell_key(X, n)
    for p in range(300):
        ijk = [int(X[d, p]) * n // 2 ** 32 for d in range(3)]
        assert key[p] == (ijk[0] * n + ijk[1]) * n + ijk[2]
    perm = mesh.stable_cell_order(X, n)
    ks = key[perm]
    assert np.all(np.diff(ks.astype(np.int64)) >= 0)
    for a, b in zip(perm[:-1], perm[1:]):
        if key[a] == key[b]:
            assert a < b


@pytest.mark.parametrize("order", [3, 5, 7])
def test_gradient_coefficients_and_plane_wave(golden, order):
    coef = golden["gradient_coefficients"][str(order)]
    assert [mesh.GRADIENT_COEFFS[order].get(k, 0.0) for k in range(-3, 4)] == pytest.approx(coef, abs=1e-15)
    n = 32
    h = 1.0 / n
    m = 3
    theta = 2 * np.pi * m / n
    x = np.arange(n)
    u = np.broadcast_to(np.sin(theta * x)[None, :, None], (n, n, n)).copy()
    du = mesh.derivative(u, 1, h, order)
    # symbol of an antisymmetric stencil on sin: (1/h) sum_{k>0} 2 c_k sin(k theta) cos(theta x)
    sym = sum(2 * coef[3 + k] * np.sin(k * theta) for k in (1, 2, 3)) / h
    assert np.abs(du - sym * np.cos(theta * x)[None, :, None]).max() < 1e-11


@pytest.mark.parametrize("order", [3, 5, 7])
def test_gradient_accuracy_order(golden, order):
    """Truncation error of the Table 1 stencils scales as h^order_accuracy."""
    errs = []
    for n in (32, 64):
        h = 1.0 / n
        x = (np.arange(n) + 0.5) * h
        u = np.broadcast_to(np.sin(2 * np.pi * x)[:, None, None], (n, 1, 1)).copy()
        du = mesh.derivative(u, 0, h, order)[:, 0, 0]
        errs.append(np.abs(du - 2 * np.pi * np.cos(2 * np.pi * x)).max())
    p = np.log2(errs[0] / errs[1])
    assert p == pytest.approx(golden["gradient_coefficients"]["accuracy_order"][str(order)], abs=0.1)


def test_gradient_antisymmetric_and_zero_sum():
    n = 16
    phi = np.random.default_rng(2).standard_normal((n, n, n))
    g = mesh.force_from_potential(phi, 1.0 / n, 5)
    for c in g:
        assert abs(c.sum()) < 1e-9
    # <psi, D phi> = -<D psi, phi>
    psi = np.random.default_rng(4).standard_normal((n, n, n))
    lhs = (psi * mesh.derivative(phi, 2, 1.0 / n)).sum()
    rhs = -(mesh.derivative(psi, 2, 1.0 / n) * phi).sum()
    assert lhs == pytest.approx(rhs, rel=1e-12)


def test_laplacian_plane_wave_eigenvalue():
    n = 16
    h = 1.0 / n
    i = np.arange(n)
    mx, my, mz = 1, 2, 5
    u = np.cos(2 * np.pi * (mx * i[:, None, None] + my * i[None, :, None] + mz * i[None, None, :]) / n)
    lam = -(4 / h ** 2) * sum(np.sin(np.pi * m / n) ** 2 for m in (mx, my, mz))
    assert np.abs(mesh.laplacian7(u, h) - lam * u).max() < 1e-9 * abs(lam)
