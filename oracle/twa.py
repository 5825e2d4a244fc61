"""TWA stream ensemble: sampling, run loop and ensemble moments (oracle, FP64).

Test infrastructure only (see ``oracle/__init__``).

Ensemble layout: ``batch[s]`` for stream slot s = 0..N_s; slot 0 holds the
classical field psi_cl (no noise, evolved by the same integrator, Sec. II.C),
slots 1..N_s the sampled streams of Eq. eqn_stream_ensemble with c_i = 1 (the
coherent-state Wigner function is positive, Sec. III.A).

Noise amplitude (Sec. III.B.1, Eq. sample).  In number units b_g = sqrt(n dV) psi_g
a coherent state's Wigner function is a complex Gaussian around z_g.  Two readings:
  noise_conv = 0: complex variance 1/2 per mode, E|delta b|^2 = 1/2, i.e. variance
                  1/(4 n dV) per real component of psi (standard coherent-state
                  Wigner function; the Fock-space test selects this reading);
  noise_conv = 1: variance 1/2 per real component as Eq. sample is printed,
                  i.e. 1/(2 n dV) per component of psi.
The paper writes the variance per grid point without dV; here it is placed on
b_g so that the noise is white and unit-consistent for any dx (by unitarity of
the DFT this is the same noise per Fourier mode).
"""
from __future__ import annotations

import math

import numpy as np

from . import sp
from .philox import wigner_normals


def noise_sigma(n_tot: float, dV: float, noise_conv: int = 0) -> float:
    """Standard deviation of each real component of delta psi (Eq. sample, see module doc)."""
    var_mode = 0.5 if noise_conv == 0 else 1.0
    return math.sqrt(var_mode / (2.0 * n_tot * dV))


def sample(psi_cl: np.ndarray, seed: int, n_real: int, n_tot: float, dV: float,
           noise_conv: int = 0, instance: int = 0) -> np.ndarray:
    """Draw the stream ensemble of Eq. sample: psi_s = psi_cl + sigma (zR + i zI), s = 1..N_s.

    zR, zI are standard normals from Philox4x32-10 (ctr = (cell, s, instance, 0),
    key = seed) through Box-Muller.  Slot 0 is psi_cl itself.
    """
    shape = psi_cl.shape
    n_cells = psi_cl.size
    sig = noise_sigma(n_tot, dV, noise_conv)
    out = np.empty((n_real + 1,) + shape, dtype=np.complex128)
    out[0] = psi_cl
    for s in range(1, n_real + 1):
        zr, zi = wigner_normals(seed, n_cells, s, instance)
        out[s] = psi_cl + sig * (zr + 1j * zi).reshape(shape)
    return out


def moments(batch: np.ndarray, n_tot: float, L: float, dim: int, with_modes: bool = True) -> dict:
    """Ensemble moments of symmetrically ordered operators (Eq. E[op], Sec. III.B.3).

    Averages run over slots 1..N_s; slot 0 supplies the classical density.
      rho_mean = mean |psi|^2 - 1/(2 n dV)          (Weyl symbol of psi^dag psi, normalized units)
      psi_mean = mean psi
      rho_cl   = |psi_cl|^2
      corr     = ||rho_mean - rho_cl||_2 / ||rho_cl||_2
      Q        = sum_g dV (mean|psi|^2 - |mean psi|^2) - M/(2n)      (Eq. Q)
      a_k      = sqrt(n dV / M) DFT(psi)_k     (unitary DFT, number units)
      nk_mean  = mean |a_k|^2 - 1/2
      nk_var   = mean |a_k|^4 - mean |a_k|^2 - (mean |a_k|^2 - 1/2)^2
    The last two are the Weyl symbols of a^dag a and of (a^dag a)^2 = |a|^4 - |a|^2.
    """
    shape = batch.shape[-dim:]
    M = int(np.prod(shape))
    dV = (L ** dim) / M
    ens = batch[1:]
    p2 = np.abs(ens) ** 2
    m2 = p2.mean(axis=0)
    pm = ens.mean(axis=0)
    rho_cl = np.abs(batch[0]) ** 2
    rho_mean = m2 - 1.0 / (2.0 * n_tot * dV)
    out = {
        "rho_mean": rho_mean,
        "psi_mean": pm,
        "rho_cl": rho_cl,
        "corr": float(np.linalg.norm((rho_mean - rho_cl).ravel()) / np.linalg.norm(rho_cl.ravel())),
        "Q": float(np.sum(m2 - np.abs(pm) ** 2) * dV - M / (2.0 * n_tot)),
    }
    if with_modes:
        a = sp.fftn(ens, dim) * math.sqrt(n_tot * dV / M)
        a2 = np.abs(a) ** 2
        ma2 = a2.mean(axis=0)
        ma4 = (a2 ** 2).mean(axis=0)
        out["nk_mean"] = ma2 - 0.5
        out["nk_var"] = ma4 - ma2 - (ma2 - 0.5) ** 2
    return out


def run(psi_cl: np.ndarray, hbar: float, C: float, dt: float, L: float, dim: int,
        n_tot: float, n_real: int, seed: int, n_steps: int, out_every: int,
        noise_conv: int = 0, order: str = "kdk", with_modes: bool = True,
        batch: np.ndarray = None):
    """Sample, then integrate every stream and record moments every ``out_every`` steps.

    Returns (times, list of moment dicts, final batch).  Moments are taken at
    t = 0 and after every ``out_every`` steps (Sec. III.B, the run loop).
    """
    M = psi_cl.size
    dV = (L ** dim) / M
    if batch is None:
        batch = sample(psi_cl, seed, n_real, n_tot, dV, noise_conv)
    times, series = [0.0], [moments(batch, n_tot, L, dim, with_modes)]
    for s in range(1, n_steps + 1):
        batch = sp.step(batch, hbar, C, dt, L, dim, order)
        if s % out_every == 0:
            times.append(s * dt)
            series.append(moments(batch, n_tot, L, dim, with_modes))
    return np.array(times), series, batch


def phase_moments(batch: np.ndarray, n_tot: float, L: float, dim: int) -> dict:
    """Mass-weighted amplitude and phase variances of the ensemble (Eq. varA, Eq. varPhi).

    Per cell, over slots 1..N_s: A_s = |psi_s|, <A> its mean and <dA^2> its (population)
    variance; dphi_s = arg(psi_s conj(mean psi)) in (-pi, pi], the phase of each stream relative
    to the ensemble-mean field (0 reference where the mean field vanishes), and <dphi^2> its mean
    square.  With <rho> the Weyl-corrected mean density of ``moments``:
        Var(A~)   = sum_g dV <rho> <dA^2> / <A>
        Var(phi~) = sum_g dV <rho> <dphi^2> / (pi^2 / 3)
    The printed normalization of the phase variance is pi / sqrt(3), the standard deviation of a
    uniformly distributed phase; it is read as the variance pi^2 / 3, so that a fully random phase
    gives the total mass.
    """
    s = batch[1:]
    dV = (L ** dim) / batch[0].size
    A = np.abs(s)
    a_mean = A.mean(0)
    a_var = (A ** 2).mean(0) - a_mean ** 2
    mean_psi = s.mean(0)
    dphi = np.angle(s * np.conj(mean_psi))
    phi2 = (dphi ** 2).mean(0)
    rho = (np.abs(s) ** 2).mean(0) - 1.0 / (2.0 * n_tot * dV)
    with np.errstate(divide="ignore", invalid="ignore"):
        wa = np.where(a_mean > 0, rho * a_var / a_mean, 0.0)
    return {"var_a_cell": a_var, "a_mean": a_mean, "phi2_cell": phi2,
            "var_a": float(np.sum(wa) * dV), "var_phi": float(np.sum(rho * phi2) * dV / (math.pi ** 2 / 3.0))}


def stream_average(batch: np.ndarray, f, n_tot: float, L: float, dim: int, of_mean: bool = False,
                   modes: bool = False) -> dict:
    """Average of a function of the fields across the streams (Appendix B's synthesizer).

    f(re, im, i, n) takes the real and imaginary parts of the field value, the flat index i of
    the cell or mode (C order of ``batch[s]``, x fastest) and the number of cells n, elementwise
    on arrays, and returns a complex (or real) array.  Over the sampled slots s = 1..N_s:
        per_cell = mean_s f(psi_s)            (of_mean False: f applied to every stream)
        per_cell = f(mean_s psi_s)            (of_mean True: f applied to the averaged field)
        f_cl     = f(psi_0)                   (the classical slot)
        total    = sum over cells of per_cell dV
    With modes, the field is replaced by the number-unit Fourier amplitudes
    a_k = sqrt(n_tot dV / cells) DFT(psi)_k of each slot (as in ``moments``) and the total is the
    plain sum over modes.
    """
    shape = batch.shape[1:]
    cells = batch[0].size
    dV = (L ** dim) / cells
    fields = batch.reshape(batch.shape[0], cells)
    w = dV
    if modes:
        fields = np.sqrt(n_tot * dV / cells) * sp.fftn(batch, dim).reshape(batch.shape[0], cells)
        w = 1.0
    idx = np.arange(cells, dtype=np.int64)

    def g(z):
        return np.asarray(f(z.real, z.imag, idx, cells), dtype=np.complex128) * np.ones(cells)

    if of_mean:
        per_cell = g(fields[1:].mean(0))
    else:
        per_cell = np.zeros(cells, dtype=np.complex128)
        for s in range(1, fields.shape[0]):
            per_cell += g(fields[s])
        per_cell /= fields.shape[0] - 1
    return {"per_cell": per_cell.reshape(shape), "f_cl": g(fields[0]).reshape(shape),
            "total": complex(per_cell.sum() * w)}


def adaptive_dt(batch: np.ndarray, hbar: float, C: float, L: float, dim: int, c_f: float) -> float:
    """Time step of Sec. III.B.2 (the dynamic Delta t rule), read in normalized units:

        Delta t = 2 pi c_f min[ hbar / max|V| ,  L dx / (pi hbar) ]

    The first bound keeps the potential phase V Delta t / hbar of every stream and cell below
    2 pi c_f; the second keeps the gradient of the kinetic phase from aliasing (the footnote's
    dt < 4 pi / (hbar k_max dk) with k_max = pi / dx, dk = 2 pi / L equals it for c_f = 1/pi; the
    printed m L / (M pi hbar) lacks one factor of L, equal to it for L = 1).  dx is the smallest
    cell side; max|V| runs over every stream and cell of the batch.
    """
    shape = batch.shape[-dim:]
    dx = min(L / n for n in shape)
    kin = L * dx / (math.pi * hbar)
    vmax = max(float(np.max(np.abs(sp.potential(b, C, L, dim)))) for b in batch)
    pot = hbar / vmax if vmax > 0 else math.inf
    return 2.0 * math.pi * c_f * min(pot, kin)


def run_adaptive(psi_cl: np.ndarray, hbar: float, C: float, L: float, dim: int, n_tot: float,
                 n_real: int, seed: int, n_out: int, out_every: int, c_f: float,
                 noise_conv: int = 0, with_modes: bool = True, batch: np.ndarray = None):
    """Like ``run`` with the dynamic time step: before each output interval of ``out_every`` KDK
    steps, Delta t is set by ``adaptive_dt`` from the batch at the interval's start and kept for
    the interval.  Returns (times, list of moment dicts, final batch, list of the Delta t used).
    """
    M = psi_cl.size
    dV = (L ** dim) / M
    if batch is None:
        batch = sample(psi_cl, seed, n_real, n_tot, dV, noise_conv)
    t = 0.0
    times, series, dts = [0.0], [moments(batch, n_tot, L, dim, with_modes)], []
    for _ in range(n_out):
        dt = adaptive_dt(batch, hbar, C, L, dim, c_f)
        for _ in range(out_every):
            batch = sp.step(batch, hbar, C, dt, L, dim)
        t += out_every * dt
        dts.append(dt)
        times.append(t)
        series.append(moments(batch, n_tot, L, dim, with_modes))
    return np.array(times), series, batch, dts


def q_physical(Q_sim: float, n_sim: float, n_phys: float) -> float:
    """Q_p = (n_s / n_p) Q_s (Eq. Q_relation), valid while Q << 1."""
    return Q_sim * n_sim / n_phys


def stable_growth_exponent(times: np.ndarray, Q: np.ndarray) -> float:
    """Log-log slope of Q(t) - Q(0) at early times (Sec. V.A: quadratic growth, Q ~ Tr kappa t^2 / 2n).

    Parity partially pinned: the kappa tensor of Eq. DefinitionKappa is garbled in
    the paper, so only the exponent (2) of the early growth is checked.
    """
    dq = np.asarray(Q) - Q[0]
    t = np.asarray(times)
    sel = (t > 0) & (dq > 0)
    return float(np.polyfit(np.log(t[sel]), np.log(dq[sel]), 1)[0])
