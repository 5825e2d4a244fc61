"""Helpers shared by the GPU parity tests (the oracle is test infrastructure)."""
import math

import numpy as np
import torch

import twa_inputs as ti
from oracle import sp, twa


def field_rel_l2(a, b, dim):
    """Relative L2 error per field (leading axes = fields)."""
    ax = tuple(range(-dim, 0))
    return np.sqrt(np.sum(np.abs(a - b) ** 2, axis=ax) / np.sum(np.abs(b) ** 2, axis=ax))


def oracle_batch(w: ti.Workload, psi_cl, n_steps, instance=0):
    b = twa.sample(psi_cl, w.noise_seed, w.n_real, w.phys.n_tot, w.grid.dV, w.phys.noise_conv, instance)
    for _ in range(n_steps):
        b = sp.step(b, w.phys.hbar_m, w.phys.C, w.phys.dt, w.grid.L, w.grid.dim)
    return b


def make_ensemble(ws, precision=0, want_modes=True):
    from paper_2310_07119_gb300 import Ensemble
    p = ws[0].phys
    return Ensemble([w.grid for w in ws], p.hbar_m, p.C, p.dt, p.n_tot, [w.n_real for w in ws],
                    p.noise_conv, precision, want_modes)
