"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the CPU oracle.

This module holds only input construction: grid and parameter records, the
classical initial fields psi_cl of the paper's test problems, and the time-step
rule used to pick dt for a workload.  It contains none of the method's
arithmetic (no sampling, no split-step, no Poisson solve, no moments): both the
oracle and the CUDA library implement those independently.

Conventions (normalized units of Sec. III.C, Eq. mft_normed):
  * the box is periodic with side L on every axis; cell g sits at x_g = g * dx,
    dx = L / n_axis (Sec. III.B.1);
  * fields are stored x fastest: numpy shape (nx,), (ny, nx) or (nz, ny, nx);
  * psi_cl is normalized so that sum_g |psi_cl|^2 dV = 1 (Sec. III.B.1).
"""
from __future__ import annotations

import dataclasses
import math
from typing import Sequence, Tuple

import numpy as np

__all__ = [
    "Grid", "Physics", "Workload",
    "normalize", "gaussian_bump_1d", "cosine_overdensity", "kspace_gaussian",
    "soliton", "two_soliton_2d", "dt_pi4_rule",
    "workload_1d_bump", "workload_3d_condensation", "workload_3d_soliton",
    "workload_2d_merger", "small_workload",
]


@dataclasses.dataclass(frozen=True)
class Grid:
    """Periodic box: ``dim`` axes, ``n`` = (nx, ny, nz) cells (unused axes = 1), side ``L``."""
    dim: int
    n: Tuple[int, int, int]
    L: float = 1.0

    @staticmethod
    def cube(dim: int, m: int, L: float = 1.0) -> "Grid":
        n = tuple([m] * dim + [1] * (3 - dim))
        return Grid(dim, n, L)

    @property
    def shape(self) -> Tuple[int, ...]:
        """numpy shape of one field, x fastest."""
        return tuple(reversed(self.n[: self.dim]))

    @property
    def cells(self) -> int:
        return int(np.prod(self.n[: self.dim]))

    @property
    def dx(self) -> Tuple[float, ...]:
        return tuple(self.L / self.n[a] for a in range(self.dim))

    @property
    def dV(self) -> float:
        return float(np.prod(self.dx))

    def coords(self) -> Tuple[np.ndarray, ...]:
        """Cell-position arrays (x, y, z order), broadcastable to ``shape``."""
        out = []
        for a in range(self.dim):
            x = np.arange(self.n[a]) * (self.L / self.n[a])
            sh = [1] * self.dim
            sh[self.dim - 1 - a] = self.n[a]
            out.append(x.reshape(sh))
        return tuple(out)


@dataclasses.dataclass(frozen=True)
class Physics:
    """Parameters of the normalized Schroedinger-Poisson system (Sec. III.C).

    hbar_m : hbar/m (tilde-hbar)
    C      : Poisson coupling in  lap V = C |psi|^2  (C = 4 pi G M_tot)
    dt     : time step
    n_tot  : simulated total particle number (enters only the sampling)
    noise_conv : 0 = complex variance 1/2 per mode (standard coherent-state
                 Wigner function); 1 = variance 1/2 per real component as the
                 paper's Eq. sample is printed.
    """
    hbar_m: float
    C: float
    dt: float
    n_tot: float
    noise_conv: int = 0


@dataclasses.dataclass(frozen=True)
class Workload:
    name: str
    grid: Grid
    phys: Physics
    n_real: int
    n_steps: int
    out_every: int
    psi_cl_seed: int
    noise_seed: int

    def psi_cl(self) -> np.ndarray:
        return _IC_BUILDERS[self.name](self)


def normalize(psi: np.ndarray, dV: float) -> np.ndarray:
    """Scale psi so that sum |psi|^2 dV = 1 (Sec. III.B.1)."""
    return psi / math.sqrt(float(np.sum(np.abs(psi) ** 2)) * dV)


def gaussian_bump_1d(grid: Grid, amp: float = 0.5, x0: float = 0.5, w: float = 0.05) -> np.ndarray:
    """rho proportional to 1 + amp exp(-(x-x0)^2 / (2 w^2)), zero phase (1D workload)."""
    (x,) = grid.coords()
    rho = 1.0 + amp * np.exp(-((x - x0 * grid.L) ** 2) / (2.0 * (w * grid.L) ** 2))
    return normalize(np.sqrt(rho).astype(np.complex128), grid.dV)


def cosine_overdensity(grid: Grid, delta: float = 0.1) -> np.ndarray:
    """Sinusoidal overdensity of Sec. IV.A: psi = sqrt(1 + delta cos(2 pi x / L)) / Norm."""
    x = grid.coords()[0]
    rho = 1.0 + delta * np.cos(2.0 * np.pi * x / grid.L)
    rho = np.broadcast_to(rho, grid.shape)
    return normalize(np.sqrt(rho).astype(np.complex128), grid.dV)


def _kvec(grid: Grid):
    ks = []
    for a in range(grid.dim):
        k = 2.0 * np.pi * np.fft.fftfreq(grid.n[a], d=grid.L / grid.n[a])
        sh = [1] * grid.dim
        sh[grid.dim - 1 - a] = grid.n[a]
        ks.append(k.reshape(sh))
    return ks


def kspace_gaussian(grid: Grid, k0: float, seed: int) -> np.ndarray:
    """Momentum-space Gaussian of Sec. IV.B (Eq. kspaceGauss).

    |psi~(k)| = exp(-k^2 / (2 k0^2)) (so the power spectrum is exp(-k^2/k0^2)),
    phases uniform on [0, 2 pi) from numpy's PCG64 seeded with ``seed``.
    """
    k2 = sum(k ** 2 for k in _kvec(grid))
    rng = np.random.default_rng(seed)
    phi = rng.uniform(0.0, 2.0 * np.pi, size=grid.shape)
    psik = np.exp(-k2 / (2.0 * k0 ** 2) + 1j * phi)
    psi = np.fft.ifftn(psik)
    return normalize(psi, grid.dV)


def _min_image(x: np.ndarray, c: float, L: float) -> np.ndarray:
    d = x - c
    return d - L * np.round(d / L)


def soliton(grid: Grid, rc_frac: float = 1.0 / 16.0, center=None) -> np.ndarray:
    """Soliton profile rho = rho_c [1 + 0.091 (r/r_c)^2]^-8, zero phase, minimum-image r."""
    L = grid.L
    rc = rc_frac * L
    cs = center if center is not None else [0.5 * L] * grid.dim
    r2 = 0.0
    for a, x in enumerate(grid.coords()):
        r2 = r2 + _min_image(x, cs[a], L) ** 2
    rho = (1.0 + 0.091 * r2 / rc ** 2) ** -8
    rho = np.broadcast_to(rho, grid.shape)
    return normalize(np.sqrt(rho).astype(np.complex128), grid.dV)


def two_soliton_2d(grid: Grid, seed: int, rc_frac: float = 1.0 / 20.0, sep: float = 0.3,
                   wavelengths_per: float = 0.1) -> np.ndarray:
    """Two 2D solitons separated by sep*L along x, moving toward each other.

    Each carries one de Broglie wavelength per ``wavelengths_per * L`` (k = 2 pi / (0.1 L));
    the right one gets a uniform random phase from numpy's PCG64 seeded with ``seed``.
    """
    L = grid.L
    kv = 2.0 * np.pi / (wavelengths_per * L)
    x = grid.coords()[0]
    a = soliton(grid, rc_frac, center=[0.5 * L - 0.5 * sep * L, 0.5 * L])
    b = soliton(grid, rc_frac, center=[0.5 * L + 0.5 * sep * L, 0.5 * L])
    phi = np.random.default_rng(seed).uniform(0.0, 2.0 * np.pi)
    psi = a * np.exp(1j * kv * x) + b * np.exp(-1j * kv * x + 1j * phi)
    return normalize(psi, grid.dV)


def dt_pi4_rule(grid: Grid, hbar_m: float) -> float:
    """Largest dt with max_k hbar k^2 dt / 2 <= pi/4 over the full grid (k_max per axis = pi n / L)."""
    k2max = sum((np.pi * grid.n[a] / grid.L) ** 2 for a in range(grid.dim))
    return (np.pi / 4.0) * 2.0 / (hbar_m * k2max)


# ---------------------------------------------------------------------------
# Workloads with the paper's IC families at the sizes used for measurement.
# Unstated constants: C = 4 pi (dynamical time ~ 1 for L = M_tot = 1) and, for
# the 3D/2D systems, hbar/m = 0.0122 (the paper's 0.02 kpc^2/Myr at L = 60 kpc,
# t_c ~ 2.19 Gyr, rescaled to L = 1, t_c = 1).
# ---------------------------------------------------------------------------
HBAR_3D = 0.0122
C_UNIT = 4.0 * np.pi


def workload_1d_bump(m: int = 256, n_real: int = 32, n_steps: int = 1000) -> Workload:
    g = Grid.cube(1, m)
    return Workload("bump1d", g, Physics(1.0, C_UNIT, 1e-3, 1e4), n_real, n_steps, 10, 0, 1234)


def workload_3d_condensation(m: int = 128, n_real: int = 256, n_steps: int = 2000,
                             n_tot: float = 1e9) -> Workload:
    g = Grid.cube(3, m)
    dt = dt_pi4_rule(g, HBAR_3D)
    return Workload("kgauss3d", g, Physics(HBAR_3D, C_UNIT, dt, n_tot), n_real, n_steps, 10, 7, 2024)


def workload_3d_soliton(m: int = 256, n_real: int = 64, n_steps: int = 4000) -> Workload:
    g = Grid.cube(3, m)
    dt = dt_pi4_rule(g, HBAR_3D)
    return Workload("soliton3d", g, Physics(HBAR_3D, C_UNIT, dt, 1e10), n_real, n_steps, 10, 0, 77)


def workload_2d_merger(m: int, n_real: int, n_steps: int = 1000, dt_m: int = 2048) -> Workload:
    g = Grid.cube(2, m)
    dt = dt_pi4_rule(Grid.cube(2, dt_m), HBAR_3D)
    return Workload("merger2d", g, Physics(HBAR_3D, C_UNIT, dt, 1e9), n_real, n_steps, 10, 11, 99)


def small_workload(name: str, dim: int, m: int, n_real: int, n_steps: int, n_tot: float = 1e6,
                   hbar_m: float = None, dt: float = None, out_every: int = 5) -> Workload:
    """Reduced-size workload of one of the IC families (parity cases the oracle runs in seconds)."""
    g = Grid.cube(dim, m)
    hb = hbar_m if hbar_m is not None else (1.0 if name == "bump1d" else HBAR_3D)
    if dt is None:
        dt = 1e-3 if name == "bump1d" else dt_pi4_rule(g, hb)
    return Workload(name, g, Physics(hb, C_UNIT, dt, n_tot), n_real, n_steps, out_every, 5, 4321)


def _ic_bump(w: Workload):
    return gaussian_bump_1d(w.grid)


def _ic_kgauss(w: Workload):
    return kspace_gaussian(w.grid, 8.0 * 2.0 * np.pi / w.grid.L, w.psi_cl_seed)


def _ic_soliton(w: Workload):
    return soliton(w.grid)


def _ic_merger(w: Workload):
    return two_soliton_2d(w.grid, w.psi_cl_seed)


def _ic_cosine(w: Workload):
    return cosine_overdensity(w.grid, 0.1)


_IC_BUILDERS = {
    "bump1d": _ic_bump,
    "kgauss3d": _ic_kgauss,
    "kgauss": _ic_kgauss,
    "soliton3d": _ic_soliton,
    "soliton": _ic_soliton,
    "merger2d": _ic_merger,
    "cosine": _ic_cosine,
}
