"""Pins for the oracle's Schroedinger-Poisson integrator (Sec. III.B.2, Eq. mft_normed).

Each test checks the oracle against something other than itself: closed forms
(Poisson of a cosine, free Gaussian packet), exact invariants (unitarity), the
Strang splitting's second-order error, and the sign of gravity.
"""
import numpy as np
import pytest

import twa_inputs as ti
from oracle import sp


@pytest.mark.parametrize("dim,modes", [(1, (3,)), (2, (1, 2)), (3, (2, 0, 1))])
def test_poisson_of_a_cosine(dim, modes):
    # rho = 1 + eps cos(k.x)  ->  V = -C eps cos(k.x) / |k|^2  (lap V = C (rho - mean rho)).
    L, m, C, eps = 2.0, 16, 3.7, 0.3
    g = ti.Grid.cube(dim, m, L)
    xs = g.coords()
    kx = 0.0
    k2 = 0.0
    for a in range(dim):
        kx = kx + (2 * np.pi * modes[a] / L) * xs[a]
        k2 += (2 * np.pi * modes[a] / L) ** 2
    rho = np.broadcast_to(1.0 + eps * np.cos(kx), g.shape)
    V = sp.potential(np.sqrt(rho).astype(complex), C, L, dim)
    expect = np.broadcast_to(-C * eps * np.cos(kx) / k2, g.shape)
    assert np.max(np.abs(V - expect)) < 1e-12


def _free_packet(x, t, hbar, x0, s0, k0, L, images=40):
    # Free Gaussian packet (C = 0) summed over periodic images.
    tau = hbar * t / (2 * s0 ** 2)
    out = np.zeros_like(x, dtype=complex)
    for j in range(-images, images + 1):
        xx = x + j * L
        out += ((2 * np.pi * s0 ** 2) ** -0.25 / np.sqrt(1 + 1j * tau)
                * np.exp(-(xx - x0 - hbar * k0 * t) ** 2 / (4 * s0 ** 2 * (1 + 1j * tau)))
                * np.exp(1j * k0 * xx - 1j * 0.5 * hbar * k0 ** 2 * t))
    return out


@pytest.mark.parametrize("order", ["kdk", "dkd"])
def test_free_moving_gaussian_matches_closed_form(order):
    L, m, hbar = 1.0, 256, 0.02
    s0, x0, k0 = L / 30, 0.3, 2 * np.pi * 5 / L
    x = np.arange(m) * (L / m)
    psi0 = _free_packet(x, 0.0, hbar, x0, s0, k0, L)
    dt, n = 0.05, 40
    psi = sp.evolve(psi0, hbar, 0.0, dt, L, 1, n, order)
    expect = _free_packet(x, n * dt, hbar, x0, s0, k0, L)
    assert np.max(np.abs(psi - expect)) < 1e-10
    # the packet moved in +x by hbar k0 t (pins the sign of the kinetic phase)
    # (circular mean of the wrapped density)
    c = np.angle(np.sum(np.exp(2j * np.pi * x / L) * np.abs(psi) ** 2)) * L / (2 * np.pi)
    d = (c - (x0 + hbar * k0 * n * dt)) % L
    assert min(d, L - d) < 1e-6


def test_unitarity_per_step():
    w = ti.small_workload("kgauss", 3, 16, 1, 1)
    psi = w.psi_cl()
    m0 = sp.mass(psi, w.grid.dV, 3)
    for _ in range(5):
        psi = sp.step(psi, w.phys.hbar_m, w.phys.C, w.phys.dt * 20, 1.0, 3)
        assert abs(sp.mass(psi, w.grid.dV, 3) - m0) < 1e-14


def test_gravity_is_attractive():
    # a resting overdensity collapses: its peak density grows at early times
    g = ti.Grid.cube(1, 128)
    psi = ti.gaussian_bump_1d(g)
    p0 = np.abs(psi).max() ** 2
    psi2 = sp.evolve(psi, 0.01, 4 * np.pi, 1e-3, 1.0, 1, 50)
    assert np.abs(psi2).max() ** 2 > p0 * 1.001
    psi3 = sp.evolve(psi, 0.01, -4 * np.pi, 1e-3, 1.0, 1, 50)   # repulsive coupling spreads it
    assert np.abs(psi3).max() ** 2 < p0


def _energy_drift(dt, T, order):
    g = ti.Grid.cube(1, 64)
    psi = ti.cosine_overdensity(g, 0.5)
    hb, C = 0.05, 4 * np.pi
    e0 = sp.energy(psi, hb, C, 1.0, 1)
    worst = 0.0
    for _ in range(int(round(T / dt))):
        psi = sp.step(psi, hb, C, dt, 1.0, 1, order)
        worst = max(worst, abs(sp.energy(psi, hb, C, 1.0, 1) - e0))
    return worst, e0


@pytest.mark.parametrize("order", ["kdk", "dkd"])
def test_energy_error_is_second_order(order):
    e1, e0 = _energy_drift(0.02, 0.6, order)
    e2, _ = _energy_drift(0.01, 0.6, order)
    assert e1 < 5e-2 * abs(e0)
    assert 3.4 < e1 / e2 < 4.6


def test_kdk_and_dkd_converge_to_the_same_flow():
    g = ti.Grid.cube(1, 64)
    psi = ti.cosine_overdensity(g, 0.5)
    hb, C, T = 0.05, 4 * np.pi, 0.4
    ref = sp.evolve(psi, hb, C, T / 800, 1.0, 1, 800, "kdk")
    for order in ("kdk", "dkd"):
        errs = [np.linalg.norm(sp.evolve(psi, hb, C, T / n, 1.0, 1, n, order) - ref) for n in (20, 40)]
        assert 3.5 < errs[0] / errs[1] < 4.5


def test_phase_reduction_is_exact_mod_two_pi():
    rng = np.random.default_rng(0)
    psi = rng.normal(size=32) + 1j * rng.normal(size=32)
    V = rng.normal(size=32)
    hb, tau = 0.3, 0.1
    a = sp.kick(psi, V, tau, hb)
    b = sp.kick(psi, V + 2 * np.pi * hb / tau * 1000, tau, hb)
    assert np.max(np.abs(a - b)) < 1e-9
    assert np.max(np.abs(a - psi * np.exp(-1j * V * tau / hb))) < 1e-14
