"""The seeded input generators against the input recipe they implement (the paper's initial-condition
families, Sec. IV): normalization sum |psi|^2 dV = 1 (Sec. III.B.1), each family's density or
spectrum in closed form, the pi/4 time-step rule, layout (x fastest) and seed determinism."""
import math

import numpy as np
import pytest

import twa_inputs as ti


def _norm(psi, g):
    return float(np.sum(np.abs(psi) ** 2) * g.dV)


@pytest.mark.parametrize("w", [ti.workload_1d_bump(), ti.small_workload("kgauss", 3, 16, 2, 1),
                               ti.small_workload("soliton", 3, 16, 2, 1), ti.workload_2d_merger(64, 2),
                               ti.small_workload("cosine", 1, 64, 2, 1), ti.small_workload("kgauss", 2, 32, 2, 1)])
def test_every_family_is_normalized_and_laid_out_x_fastest(w):
    psi = w.psi_cl()
    assert psi.shape == w.grid.shape and psi.dtype == np.complex128
    assert abs(_norm(psi, w.grid) - 1.0) < 1e-12


def test_grid_layout_puts_x_last():
    g = ti.Grid(3, (8, 4, 2), 2.0)
    assert g.shape == (2, 4, 8) and g.cells == 64 and g.dV == pytest.approx((2.0 / 8) * (2.0 / 4) * (2.0 / 2))
    x, y, z = g.coords()
    assert x.shape == (1, 1, 8) and y.shape == (1, 4, 1) and z.shape == (2, 1, 1)
    assert x[0, 0, 3] == pytest.approx(3 * 2.0 / 8)


def test_bump_density_ratio_is_the_closed_form():
    g = ti.Grid.cube(1, 256)
    rho = np.abs(ti.gaussian_bump_1d(g)) ** 2
    x = np.arange(256) / 256.0
    want = 1.0 + 0.5 * np.exp(-((x - 0.5) ** 2) / (2 * 0.05 ** 2))
    assert np.allclose(rho / rho[0], want / want[0], rtol=1e-13)
    assert np.allclose(np.angle(ti.gaussian_bump_1d(g)), 0.0)


def test_cosine_overdensity_has_one_fourier_mode():
    g = ti.Grid.cube(1, 64)
    rho = np.abs(ti.cosine_overdensity(g, 0.1)) ** 2
    r = np.fft.fft(rho)
    assert abs(abs(r[1]) / abs(r[0]) - 0.05) < 1e-13                     # delta / 2
    assert np.all(np.abs(r[2:-1]) < 1e-12 * abs(r[0]))


def test_kspace_gaussian_amplitude_spectrum_and_seeded_phases():
    g = ti.Grid.cube(2, 32)
    k0 = 8.0 * 2.0 * np.pi
    psi = ti.kspace_gaussian(g, k0, 7)
    a = np.abs(np.fft.fftn(psi))
    ky, kx = np.meshgrid(2 * np.pi * np.fft.fftfreq(32, 1 / 32), 2 * np.pi * np.fft.fftfreq(32, 1 / 32),
                         indexing="ij")
    want = np.exp(-(kx ** 2 + ky ** 2) / (2 * k0 ** 2))
    assert np.allclose(a / a[0, 0], want, rtol=1e-10, atol=1e-14)
    assert np.array_equal(psi, ti.kspace_gaussian(g, k0, 7))
    assert not np.allclose(psi, ti.kspace_gaussian(g, k0, 8))


def test_soliton_profile_and_minimum_image():
    g = ti.Grid.cube(3, 32)
    rho = np.abs(ti.soliton(g)) ** 2
    rc = 1.0 / 16.0
    c = rho[16, 16, 16]
    for (iz, iy, ix) in [(16, 16, 20), (16, 10, 16), (3, 16, 16), (0, 0, 0)]:
        r2 = sum(((i / 32.0 - 0.5 + 0.5) % 1.0 - 0.5) ** 2 for i in (ix, iy, iz))
        assert rho[iz, iy, ix] / c == pytest.approx((1 + 0.091 * r2 / rc ** 2) ** -8, rel=1e-12)
    off = ti.soliton(g, center=[0.0, 0.0, 0.0])
    assert np.abs(off[0, 0, 0]) == pytest.approx(np.abs(off).max())
    assert np.abs(off[0, 0, 1]) == pytest.approx(np.abs(off[0, 0, 31]))    # periodic images


def test_two_soliton_merger_boosts_and_separation():
    g = ti.Grid.cube(2, 256)
    psi = ti.two_soliton_2d(g, 99)
    rho = np.abs(psi) ** 2
    row = rho[128]
    left, right = np.argmax(row[:128]), 128 + np.argmax(row[128:])
    assert (right - left) / 256 == pytest.approx(0.3, abs=2 / 256)
    # phase gradient +k on the left soliton, -k on the right, k = 2 pi / (0.1 L), at the peaks
    k = 2 * np.pi / 0.1
    for c, sgn in ((left, 1), (right, -1)):
        dphi = np.angle(psi[128, c + 1] * np.conj(psi[128, c]))
        assert dphi == pytest.approx(sgn * k / 256, rel=0.02)   # the other soliton's tail perturbs it slightly
    assert np.array_equal(psi, ti.two_soliton_2d(g, 99))


@pytest.mark.parametrize("dim,m,hb", [(1, 256, 1.0), (2, 512, 0.0122), (3, 128, 0.0122)])
def test_pi4_rule_puts_the_largest_kinetic_phase_at_pi_over_4(dim, m, hb):
    g = ti.Grid.cube(dim, m)
    dt = ti.dt_pi4_rule(g, hb)
    k2max = dim * (math.pi * m) ** 2
    assert hb * k2max * dt / 2 == pytest.approx(math.pi / 4, rel=1e-14)


def test_bench_workload_matches_its_stated_recipe():
    w = ti.workload_3d_condensation()
    assert w.grid.n == (128, 128, 128) and w.n_real == 256 and w.phys.n_tot == 1e9
    assert w.phys.hbar_m == 0.0122 and w.phys.C == pytest.approx(4 * math.pi)
    assert w.phys.dt == pytest.approx(2.654e-4, rel=1e-3) and w.out_every == 10 and w.psi_cl_seed == 7
