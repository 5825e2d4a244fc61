"""Normalized Schroedinger-Poisson system and its split-step integrator (oracle, FP64).

Test infrastructure only (see ``oracle/__init__``).

Equations (Sec. III.C, Eq. mft_normed), with psi normalized to sum |psi|^2 dV = 1:
    d psi / dt = -i ( -hbar/2 lap + V / hbar ) psi,      lap V = C |psi|^2,
where hbar stands for hbar/m and C = 4 pi G M_tot.  On the periodic grid the
Poisson equation is solved spectrally, V_k = -C rho_k / k^2 with V_0 = 0
(this subtracts the mean density; Eq. eqn_Ham's Poisson equation).

Integrator (Sec. III.B.2): Strang splitting with the unitary factors
    U^T(dt) = exp(-i hbar k^2 dt / 2)   (applied in Fourier space),
    U^V(dt) = exp(-i V dt / hbar)       (applied in position space).
The paper prints the kinetic factor with a + sign and the Hamiltonian with
+hbar^2 lap / 2m; both signs are taken from Eq. mft_normed instead, which is
the form the rest of the paper uses.  The default ordering is kick-drift-kick
(KDK); drift-kick-drift (DKD, the order printed in Sec. III.B.2) is an option.
Phase arguments are reduced mod 2 pi in FP64 before the exponential.
"""
from __future__ import annotations

import os

import numpy as np
import scipy.fft as sfft

TWO_PI = 2.0 * np.pi


def _workers() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:  # pragma: no cover
        return os.cpu_count() or 1


WORKERS = _workers()


def axes_of(dim: int):
    return tuple(range(-dim, 0))


def fftn(a, dim):
    return sfft.fftn(a, axes=axes_of(dim), workers=WORKERS)


def ifftn(a, dim):
    return sfft.ifftn(a, axes=axes_of(dim), workers=WORKERS)


def k_squared(shape, L: float) -> np.ndarray:
    """|k|^2 on the FFT grid: k_a = 2 pi n_a / L with n_a in {0..M/2-1, -M/2..-1} (Sec. III.B.1 grid)."""
    dim = len(shape)
    k2 = np.zeros(shape)
    for ax, m in enumerate(shape):
        k = TWO_PI * np.fft.fftfreq(m, d=L / m)
        sh = [1] * dim
        sh[ax] = m
        k2 = k2 + (k ** 2).reshape(sh)
    return k2


def reduce_2pi(theta: np.ndarray) -> np.ndarray:
    """theta mod 2 pi in FP64, result in [0, 2 pi)."""
    return np.remainder(theta, TWO_PI)


def potential(psi: np.ndarray, C: float, L: float, dim: int) -> np.ndarray:
    """V from rho = |psi|^2: V_k = -C rho_k / k^2, V_0 = 0 (Eq. mft_normed Poisson equation)."""
    rho = np.abs(psi) ** 2
    k2 = k_squared(psi.shape[-dim:], L)
    inv = np.zeros_like(k2)
    nz = k2 > 0
    inv[nz] = -C / k2[nz]
    return ifftn(fftn(rho, dim) * inv, dim).real


def kick(psi: np.ndarray, V: np.ndarray, tau: float, hbar: float) -> np.ndarray:
    """U^V(tau): psi * exp(-i V tau / hbar) (Sec. III.B.2)."""
    return psi * np.exp(-1j * reduce_2pi(V * (tau / hbar)))


def drift(psi: np.ndarray, tau: float, hbar: float, L: float, dim: int) -> np.ndarray:
    """U^T(tau) in Fourier space: psi_k * exp(-i hbar k^2 tau / 2) (Sec. III.B.2)."""
    k2 = k_squared(psi.shape[-dim:], L)
    ph = np.exp(-1j * reduce_2pi(hbar * k2 * (tau / 2.0)))
    return ifftn(fftn(psi, dim) * ph, dim)


def step(psi: np.ndarray, hbar: float, C: float, dt: float, L: float, dim: int,
         order: str = "kdk") -> np.ndarray:
    """One split step of Sec. III.B.2 for every field in ``psi`` (leading axes = batch).

    kdk: V(psi) -> U^V(dt/2) -> U^T(dt) -> V(psi) -> U^V(dt/2)
    dkd: U^T(dt/2) -> V(psi) -> U^V(dt) -> U^T(dt/2)
    The potential of each field is a functional of that field alone (Sec. III.A).
    """
    if order == "kdk":
        V = potential(psi, C, L, dim)
        psi = kick(psi, V, 0.5 * dt, hbar)
        psi = drift(psi, dt, hbar, L, dim)
        V = potential(psi, C, L, dim)
        return kick(psi, V, 0.5 * dt, hbar)
    if order == "dkd":
        psi = drift(psi, 0.5 * dt, hbar, L, dim)
        V = potential(psi, C, L, dim)
        psi = kick(psi, V, dt, hbar)
        return drift(psi, 0.5 * dt, hbar, L, dim)
    raise ValueError(order)


def evolve(psi, hbar, C, dt, L, dim, n_steps, order="kdk"):
    for _ in range(n_steps):
        psi = step(psi, hbar, C, dt, L, dim, order)
    return psi


def mass(psi: np.ndarray, dV: float, dim: int) -> np.ndarray:
    """sum_g |psi_g|^2 dV per field (conserved: U^T and U^V are unitary)."""
    return np.sum(np.abs(psi) ** 2, axis=axes_of(dim)) * dV


def energy(psi: np.ndarray, hbar: float, C: float, L: float, dim: int) -> np.ndarray:
    """E = hbar^2/2 int |grad psi|^2 + 1/2 int V |psi|^2 per field.

    hbar times the Hamiltonian functional whose derivative d/dpsi* gives the
    right-hand side of Eq. mft_normed; conserved by the exact flow.
    """
    shape = psi.shape[-dim:]
    M = int(np.prod(shape))
    dV = (L ** dim) / M
    k2 = k_squared(shape, L)
    psik = fftn(psi, dim)
    kin = 0.5 * hbar ** 2 * np.sum(k2 * np.abs(psik) ** 2, axis=axes_of(dim)) * dV / M
    V = potential(psi, C, L, dim)
    pot = 0.5 * np.sum(V * np.abs(psi) ** 2, axis=axes_of(dim)) * dV
    return kin + pot
