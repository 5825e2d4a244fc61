"""Pins of the test-particle integrator of the oracle (Sec. III.D): the spectral derivative against
closed forms, the interpolation, free motion, and second-order convergence in dt."""
import numpy as np
import pytest

import twa_inputs as ti
from oracle import particles as pt
from oracle import sp, twa


def test_spectral_derivative_of_fourier_modes():
    L, shape = 2.0, (12, 16, 8)          # (z, y, x)
    z, y, x = np.meshgrid(*[np.arange(n) * L / n for n in shape], indexing="ij")
    kx, ky, kz = 2 * np.pi * 3 / L, 2 * np.pi * 2 / L, 2 * np.pi * 1 / L
    V = np.sin(kx * x) + np.cos(ky * y) * np.sin(kz * z)
    gx, gy, gz = pt.grad_on_grid(V, L, 3)
    assert np.allclose(gx, kx * np.cos(kx * x), atol=1e-12)
    assert np.allclose(gy, -ky * np.sin(ky * y) * np.sin(kz * z), atol=1e-12)
    assert np.allclose(gz, kz * np.cos(ky * y) * np.cos(kz * z), atol=1e-12)


def test_nyquist_component_has_no_derivative():
    n, L = 16, 1.0
    x = np.arange(n) * L / n
    V = np.cos(np.pi * n * x / L)                    # the Nyquist mode (+1, -1, ...)
    assert np.allclose(pt.grad_on_grid(V, L, 1)[0], 0.0, atol=1e-13)


def test_interpolation_hits_grid_values_and_is_multilinear_between():
    rng = np.random.default_rng(0)
    L, shape = 1.0, (8, 4, 16)
    f = rng.normal(size=shape)
    dz, dy, dx = (L / n for n in shape)
    assert pt.interpolate(f, (3 * dx, 1 * dy, 5 * dz), L) == pytest.approx(f[5, 1, 3])
    # midpoint of a cell: mean of its 8 corners; periodic wrap at the upper edge
    r = (15.5 * dx, 3.5 * dy, 7.5 * dz)
    corners = [f[k, j, i] for k in (7, 0) for j in (3, 0) for i in (15, 0)]
    assert pt.interpolate(f, r, L) == pytest.approx(np.mean(corners))


def test_free_particles_move_uniformly():
    w = ti.small_workload("kgauss", 3, 8, 3, 0, n_tot=1e6)
    cl = w.psi_cl()
    rng = np.random.default_rng(1)
    r0, p0 = rng.random((4, 3)), rng.normal(size=(4, 3))
    _, r, p = pt.run(cl, 0.01, 0.0, 1e-2, 1.0, 3, 1e6, 3, 5, 7, r0, p0)
    assert np.array_equal(p, p0)
    assert np.allclose(r, np.mod(r0 + 7 * 1e-2 * p0, 1.0), atol=1e-13)


def test_leapfrog_is_second_order_in_dt():
    M, hb, C, T = 64, 0.05, 4 * np.pi, 0.4
    x = np.arange(M) / M
    psi = np.sqrt(1 + 0.5 * np.cos(2 * np.pi * x)).astype(np.complex128)
    psi /= np.sqrt(np.mean(np.abs(psi) ** 2))
    r0, p0 = np.array([[0.3]]), np.array([[0.2]])
    out = {}
    for n in (10, 20, 40, 160):
        _, r, p = pt.run(psi, hb, C, T / n, 1.0, 1, 1e9, 0, 0, n, r0, p0, batch=psi[None])
        out[n] = (r[0, 0], p[0, 0])
    e = {n: abs(out[n][0] - out[160][0]) + abs(out[n][1] - out[160][1]) for n in (10, 20, 40)}
    assert 3.0 < e[10] / e[20] < 5.0 and 3.0 < e[20] / e[40] < 5.0
