"""Test particles of the decoherence experiment (Sec. III.D, the classical equations of motion of
the field-particle system, Eq. cl_int): one particle per stream, moving in that stream's potential,

    dp/dt = -grad V_s(r),   dr/dt = p            (unit mass, normalized units of Eq. mft_normed),

integrated by leapfrog in step with the kick-drift-kick split step: half kick with V of the field
at the step's start, drift of the position, field step, half kick with V of the new field.
grad V at r: the spectral derivative of V on the grid along each axis (the Nyquist component of
an even length set to zero, as for any derivative of a real grid function), interpolated to r
linearly along each axis (trilinear in 3D), periodic.  FP64, test infrastructure only.
"""
from __future__ import annotations

import numpy as np
import scipy.fft as sfft

from . import sp
from .twa import sample


def grad_on_grid(V: np.ndarray, L: float, dim: int):
    """[dV/dx, dV/dy, dV/dz][:dim] on the grid (x is the last array axis)."""
    out = []
    for a in range(dim):
        axis = V.ndim - 1 - a
        m = V.shape[axis]
        k = 2.0 * np.pi * np.fft.fftfreq(m, d=L / m)
        if m % 2 == 0:
            k[m // 2] = 0.0
        sh = [1] * V.ndim
        sh[axis] = m
        out.append(sfft.ifft(1j * k.reshape(sh) * sfft.fft(V, axis=axis), axis=axis).real)
    return out


def interpolate(field: np.ndarray, r, L: float):
    """Periodic multilinear interpolation of a grid field (x last) at position r = (x, y, z)[:dim]."""
    dim = len(r)
    shape = field.shape[-dim:]
    idx0, frac = [], []
    for a in range(dim):
        n = shape[dim - 1 - a]
        s = r[a] / (L / n)
        f = np.floor(s)
        idx0.append(int(f) % n)
        frac.append(s - f)
    val = 0.0
    for corner in range(1 << dim):
        w = 1.0
        ix = [0] * dim
        for a in range(dim):
            n = shape[dim - 1 - a]
            bit = (corner >> a) & 1
            w *= frac[a] if bit else 1.0 - frac[a]
            ix[a] = (idx0[a] + bit) % n
        val += w * field[tuple(reversed(ix))]
    return val


def force(V: np.ndarray, r, L: float, dim: int) -> np.ndarray:
    """-grad V at r."""
    return -np.array([interpolate(g, r, L) for g in grad_on_grid(V, L, dim)])


def run(psi_cl: np.ndarray, hbar: float, C: float, dt: float, L: float, dim: int, n_tot: float,
        n_real: int, seed: int, n_steps: int, r0: np.ndarray, p0: np.ndarray, batch: np.ndarray = None):
    """Sample (or take ``batch``), then n_steps KDK steps of every stream with its particle.
    r0, p0: (n_real + 1, dim) start positions and momenta (slot 0 = the classical field's particle).
    Returns (batch, r, p) with r wrapped into [0, L)."""
    dV = (L ** dim) / psi_cl.size
    if batch is None:
        batch = sample(psi_cl, seed, n_real, n_tot, dV)
    r = np.array(r0, dtype=np.float64).copy()
    p = np.array(p0, dtype=np.float64).copy()
    for _ in range(n_steps):
        for s in range(batch.shape[0]):
            p[s] += 0.5 * dt * force(sp.potential(batch[s], C, L, dim), r[s], L, dim)
            r[s] = np.mod(r[s] + dt * p[s], L)
        batch = sp.step(batch, hbar, C, dt, L, dim)
        for s in range(batch.shape[0]):
            p[s] += 0.5 * dt * force(sp.potential(batch[s], C, L, dim), r[s], L, dim)
    return batch, r, p


def spread(r: np.ndarray, p: np.ndarray, L: float):
    """(Delta x, Delta p) per axis over the streams (slots 1..): standard deviations of the
    minimum-image displacements from the classical field's particle (slot 0) and of the momenta."""
    d = np.mod(r[1:] - r[0] + 0.5 * L, L) - 0.5 * L
    return d.std(axis=0), p[1:].std(axis=0)
