"""Thin Python binding of libtwa.so with the C ABI's names (argument marshalling only).

Device memory and streams come from PyTorch; every computation runs in the
library's CUDA kernels.  Buffers are passed as torch tensors (or raw device
addresses); streams as ``torch.cuda.Stream``, raw handles, or None for the
current stream.  There is no CPU path: without CUDA these calls raise.
"""
from __future__ import annotations

import ctypes
from typing import Iterable, Optional, Sequence

import torch

from . import _lib as L

__all__ = [
    "TwaError", "twa_create", "twa_destroy", "twa_batch_elems", "twa_sample", "twa_step_batch",
    "twa_moments", "twa_run", "twa_sync_status", "twa_last_error", "twa_autotune",
    "twa_last_launch_count", "twa_poisson_multiplier", "twa_observable_create", "twa_observable_eval",
    "twa_observable_destroy", "Observable", "twa_advance", "twa_advance_adaptive", "twa_phase_moments", "twa_particles_set", "twa_particles_get", "twa_profile_enable", "twa_profile_read", "Ensemble", "F32",
    "F64_PLAIN", "SCALAR_NAMES", "PASS_NAMES", "twa_set_batch_mode", "twa_get_batch_mode", "twa_set_wait_limit",
    "twa_debug_stall_next_batch", "twa_debug_stall_next_tma", "BATCH_SERIAL", "BATCH_FORK", "BATCH_PERSISTENT",
]

F32, F64_PLAIN = L.TWA_F32, L.TWA_F64_PLAIN
SCALAR_NAMES = L.SCALAR_NAMES
BATCH_SERIAL, BATCH_FORK, BATCH_PERSISTENT = L.TWA_BATCH_SERIAL, L.TWA_BATCH_FORK, L.TWA_BATCH_PERSISTENT
PASS_NAMES = L.PASS_NAMES


class TwaError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"twa error {code}: {msg}")
        self.code = code


def _lib():
    if not torch.cuda.is_available():
        raise TwaError(L.TWA_ECUDA, "no CUDA device: the TWA library has no CPU path")
    return L.load()


def _check(rc: int, h) -> None:
    if rc != 0:
        raise TwaError(rc, L.load().twa_last_error(h).decode())


def _ptr(x) -> Optional[int]:
    if x is None:
        return None
    if isinstance(x, torch.Tensor):
        if not x.is_cuda:
            raise TwaError(L.TWA_EINVAL, "buffers must be CUDA tensors")
        if not x.is_contiguous():
            raise TwaError(L.TWA_EINVAL, "buffers must be contiguous")
        return x.data_ptr()
    return int(x)


def _stream(s) -> int:
    if s is None:
        return torch.cuda.current_stream().cuda_stream
    if isinstance(s, torch.cuda.Stream):
        return s.cuda_stream
    return int(s)


def _grid(g) -> L.Grid:
    if isinstance(g, L.Grid):
        return g
    dim, n, Lb = (g.dim, g.n, g.L) if hasattr(g, "dim") else g
    n = list(n) + [1] * (3 - len(n))
    return L.Grid(int(dim), (ctypes.c_int * 3)(*[int(v) for v in n[:3]]), float(Lb))


def twa_create(grids: Sequence, hbar_m: float, C: float, dt: float, n_tot: float, n_real: Sequence[int],
               noise_conv: int = 0, precision: int = F32, want_modes: bool = True) -> int:
    lib = _lib()
    gs = (L.Grid * len(grids))(*[_grid(g) for g in grids])
    p = L.Params(float(hbar_m), float(C), float(dt), float(n_tot), int(noise_conv), int(precision), int(bool(want_modes)))
    nr = (ctypes.c_int * len(n_real))(*[int(v) for v in n_real])
    h = ctypes.c_void_p()
    rc = lib.twa_create(ctypes.byref(h), gs, ctypes.byref(p), len(grids), nr)
    _check(rc, None)
    return h.value


def twa_destroy(h) -> None:
    _check(_lib().twa_destroy(h), None)


def twa_batch_elems(h) -> int:
    return int(_lib().twa_batch_elems(h))


def twa_sample(h, psi_cl, seed: int, psi, stream=None) -> None:
    _check(_lib().twa_sample(h, _ptr(psi_cl), int(seed), _ptr(psi), _stream(stream)), h)


def twa_step_batch(h, psi, n_steps: int, stream=None) -> None:
    _check(_lib().twa_step_batch(h, _ptr(psi), int(n_steps), _stream(stream)), h)


def twa_moments(h, inst: int, psi, out: dict, stream=None) -> None:
    mo = L.MomentsOut(*[_ptr(out.get(k)) for k in ("rho_mean", "psi_mean", "rho_cl", "nk_mean", "nk_var", "scalars",
                                                    "nk_cl")])
    _check(_lib().twa_moments(h, int(inst), _ptr(psi), ctypes.byref(mo), _stream(stream)), h)


def twa_run(h, psi_cl, seed: int, n_steps: int, out_every: int, psi_work, series, stream=None) -> None:
    _check(_lib().twa_run(h, _ptr(psi_cl), int(seed), int(n_steps), int(out_every), _ptr(psi_work), _ptr(series),
                          _stream(stream)), h)


def twa_advance(h, psi, n_steps: int, out_every: int, series, stream=None) -> None:
    _check(_lib().twa_advance(h, _ptr(psi), int(n_steps), int(out_every), _ptr(series), _stream(stream)), h)


def twa_particles_set(h, inst: int, r, p, stream=None) -> None:
    """Test particles of instance ``inst`` (see include/twa.h): r, p of shape (n_real + 1, dim)."""
    import numpy as np
    r, p = np.asarray(r, dtype=np.float64), np.asarray(p, dtype=np.float64)
    q = np.zeros((r.shape[0], 6))
    q[:, :r.shape[1]] = r
    q[:, 3:3 + p.shape[1]] = p
    buf = (ctypes.c_double * q.size)(*q.ravel())
    _check(_lib().twa_particles_set(h, int(inst), buf, _stream(stream)), h)


def twa_particles_get(h, inst: int, n_slots: int, dim: int, stream=None):
    """(r, p) of instance ``inst``, each (n_slots, dim), synchronized."""
    import numpy as np
    buf = (ctypes.c_double * (6 * n_slots))()
    _check(_lib().twa_particles_get(h, int(inst), buf, _stream(stream)), h)
    q = np.array(buf[:]).reshape(n_slots, 6)
    return q[:, :dim].copy(), q[:, 3:3 + dim].copy()


def twa_phase_moments(h, inst: int, psi, var_a=None, phi2=None, totals=None, stream=None):
    """Amplitude and phase variances (see include/twa.h); returns the device totals [Var A~, Var phi~]."""
    if totals is None:
        totals = torch.empty(2, dtype=torch.float64, device=psi.device)
    _check(_lib().twa_phase_moments(h, int(inst), _ptr(psi), _ptr(var_a), _ptr(phi2), _ptr(totals), _stream(stream)), h)
    return totals


def twa_advance_adaptive(h, psi, n_out: int, out_every: int, c_f: float, series, stream=None):
    """Adaptive-step continuation (see include/twa.h); returns the output times (numpy, n_out + 1)."""
    import numpy as np
    times = (ctypes.c_double * (int(n_out) + 1))()
    _check(_lib().twa_advance_adaptive(h, _ptr(psi), int(n_out), int(out_every), float(c_f), _ptr(series), times,
                                       _stream(stream)), h)
    return np.array(times[:], dtype=np.float64)


def twa_profile_enable(h, on: bool) -> None:
    _check(_lib().twa_profile_enable(h, int(bool(on))), h)


def twa_profile_read(h) -> dict:
    """Per pass kind: launches, total device ms, algorithmic bytes per cell of one launched field,
    fields per launch and cells per field (from the events recorded since the profiler was enabled)."""
    lib = _lib()
    out = {}
    for op, name in enumerate(L.PASS_NAMES):
        n, ms, bpc, fpl, cells = (ctypes.c_longlong(), ctypes.c_double(), ctypes.c_double(), ctypes.c_longlong(),
                                  ctypes.c_longlong())
        _check(lib.twa_profile_read(h, op, ctypes.byref(n), ctypes.byref(ms), ctypes.byref(bpc), ctypes.byref(fpl),
                                    ctypes.byref(cells)), h)
        if n.value:
            out[name] = {"launches": n.value, "total_ms": ms.value, "bytes_per_cell": bpc.value,
                         "fields_per_launch": fpl.value, "cells": cells.value}
    return out


def twa_sync_status(h, stream=None) -> int:
    rc = _lib().twa_sync_status(h, _stream(stream))
    if rc not in (0, L.TWA_ENONFINITE, L.TWA_ETIMEOUT):
        _check(rc, h)
    return rc


def twa_set_batch_mode(h, mode: int) -> None:
    """Run the instances' steps one after another, forked, or as one persistent launch (include/twa.h)."""
    _check(_lib().twa_set_batch_mode(h, int(mode)), h)


def twa_get_batch_mode(h) -> int:
    return int(_lib().twa_get_batch_mode(h))


def twa_set_wait_limit(h, seconds: float) -> None:
    _check(_lib().twa_set_wait_limit(h, float(seconds)), h)


def twa_debug_stall_next_batch(h) -> None:
    _check(_lib().twa_debug_stall_next_batch(h), h)


def twa_debug_stall_next_tma(h) -> None:
    _check(_lib().twa_debug_stall_next_tma(h), h)


def twa_last_error(h) -> str:
    return _lib().twa_last_error(h).decode()


def twa_autotune(h, psi, cache_path: Optional[str] = None, stream=None) -> None:
    cp = cache_path.encode() if cache_path else None
    _check(_lib().twa_autotune(h, _ptr(psi), cp, _stream(stream)), h)


def twa_last_launch_count(h) -> int:
    return int(_lib().twa_last_launch_count(h))


def twa_observable_create(f_re: str, f_im: Optional[str] = None, flags: int = 0):
    """Compile f = f_re + i f_im (C expressions in re, im, i, n, nx, ny, nz) into a stream average."""
    ob = ctypes.c_void_p()
    _check(_lib().twa_observable_create(ctypes.byref(ob), f_re.encode(), f_im.encode() if f_im else None,
                                        int(flags)), None)
    return ob


def twa_observable_eval(ob, h, inst: int, psi, per_cell=None, f_cl=None, total=None, stream=None):
    """Evaluate on one instance; per_cell / f_cl are complex128 device tensors (one value per cell or
    mode) or None; returns the device float64 tensor `total` (real, imaginary)."""
    if total is None:
        total = torch.zeros(2, dtype=torch.float64, device=psi.device)
    _check(_lib().twa_observable_eval(ob, h, int(inst), _ptr(psi), _ptr(per_cell), _ptr(f_cl), _ptr(total),
                                      _stream(stream)), h)
    return total


def twa_observable_destroy(ob) -> None:
    _check(_lib().twa_observable_destroy(ob), None)


class Observable:
    """A compiled stream average of f (Appendix B's synthesizer); see twa_observable_create.

    of_mean: apply f to the streams' mean field instead of averaging f over the streams.
    modes: apply f to the Fourier amplitudes a_k (number units) instead of psi(x).
    fp32: evaluate f in FP32 and sum the streams as float pairs (faster, ~1e-7 per value).
    """

    def __init__(self, f_re: str, f_im: Optional[str] = None, of_mean: bool = False, modes: bool = False,
                 fp32: bool = False):
        flags = ((L.TWA_OBS_OF_MEAN if of_mean else 0) | (L.TWA_OBS_MODES if modes else 0) |
                 (L.TWA_OBS_FP32 if fp32 else 0))
        self.ob = twa_observable_create(f_re, f_im, flags)

    def __call__(self, ens: "Ensemble", inst: int = 0, psi=None, per_cell: bool = True, classical: bool = False,
                 stream=None) -> dict:
        """Evaluate on instance `inst` of an Ensemble's batch (or of `psi`): a dict with the complex
        per-cell (or per-mode) average 'per_cell', f of the classical slot 'f_cl' (if asked) and the
        complex 'total'."""
        psi = ens.psi if psi is None else psi
        cells = ens.cells[inst]
        pc = torch.empty(cells, dtype=torch.complex128, device=psi.device) if per_cell else None
        fc = torch.empty(cells, dtype=torch.complex128, device=psi.device) if classical else None
        tot = twa_observable_eval(self.ob, ens.h, inst, psi, pc, fc, None, stream)
        t = tot.cpu().numpy()
        return {"per_cell": pc, "f_cl": fc, "total": complex(t[0], t[1])}

    def close(self) -> None:
        if self.ob is not None:
            twa_observable_destroy(self.ob)
            self.ob = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def twa_poisson_multiplier(k2, m=None, stream=None):
    """The transform passes' Poisson multiplier 1/k2 (0 where k2 <= 0) of a device float32 tensor."""
    if m is None:
        m = torch.empty_like(k2)
    _check(_lib().twa_poisson_multiplier(_ptr(k2), _ptr(m), int(k2.numel()), _stream(stream)), None)
    return m


class Ensemble:
    """A handle plus torch-owned device buffers for one batch of instances.

    grids: sequence of objects with ``dim``, ``n`` = (nx, ny, nz) and ``L`` (or tuples).
    The batch tensor ``psi`` holds, per instance, slot 0 (classical field) and
    n_real sampled streams, x fastest (see include/twa.h).
    """

    def __init__(self, grids: Sequence, hbar_m: float, C: float, dt: float, n_tot: float,
                 n_real: Sequence[int], noise_conv: int = 0, precision: int = F32, want_modes: bool = True,
                 device="cuda:0"):
        self.device = torch.device(device)
        torch.cuda.set_device(self.device)
        self.grids = [_grid(g) for g in grids]
        self.n_real = list(n_real)
        self.precision = precision
        self.cells = [int(g.n[0] * g.n[1] * g.n[2]) for g in self.grids]
        self.h = twa_create(self.grids, hbar_m, C, dt, n_tot, n_real, noise_conv, precision, want_modes)
        self.ctype = torch.complex64 if precision == F32 else torch.complex128
        self.psi = torch.zeros(twa_batch_elems(self.h), dtype=self.ctype, device=self.device)
        self.offsets = []
        off = 0
        for c, nr in zip(self.cells, self.n_real):
            self.offsets.append(off)
            off += c * (nr + 1)

    def close(self):
        if self.h:
            twa_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def shape(self, inst: int):
        g = self.grids[inst]
        return tuple(reversed([int(g.n[a]) for a in range(g.dim)]))

    def fields(self, inst: int) -> torch.Tensor:
        """View (n_real + 1, *shape) of instance ``inst`` (slot 0 = classical field)."""
        o = self.offsets[inst]
        n = (self.n_real[inst] + 1) * self.cells[inst]
        return self.psi[o:o + n].view((self.n_real[inst] + 1,) + self.shape(inst))

    def psi_cl_tensor(self, psi_cls: Iterable) -> torch.Tensor:
        parts = [torch.as_tensor(p, dtype=torch.complex128).reshape(-1) for p in psi_cls]
        return torch.cat(parts).to(self.device)

    def sample(self, psi_cls: Iterable, seed: int, stream=None):
        cl = self.psi_cl_tensor(psi_cls)
        twa_sample(self.h, cl, seed, self.psi, stream)
        return cl

    def step(self, n_steps: int, stream=None):
        twa_step_batch(self.h, self.psi, n_steps, stream)

    def moments(self, inst: int, modes: bool = True, stream=None) -> dict:
        c = self.cells[inst]
        f64 = dict(dtype=torch.float64, device=self.device)
        out = {"rho_mean": torch.empty(c, **f64), "psi_mean": torch.empty(2 * c, **f64),
               "rho_cl": torch.empty(c, **f64), "scalars": torch.empty(L.TWA_NSCALARS, **f64)}
        if modes:
            out["nk_mean"] = torch.empty(c, **f64)
            out["nk_var"] = torch.empty(c, **f64)
            out["nk_cl"] = torch.empty(c, **f64)
        twa_moments(self.h, inst, self.psi, out, stream)
        return out

    def run(self, psi_cls: Iterable, seed: int, n_steps: int, out_every: int, stream=None) -> torch.Tensor:
        cl = self.psi_cl_tensor(psi_cls)
        n_out = n_steps // out_every + 1
        series = torch.zeros((n_out, len(self.grids), L.TWA_NSCALARS), dtype=torch.float64, device=self.device)
        twa_run(self.h, cl, seed, n_steps, out_every, self.psi, series, stream)
        return series

    def new_series(self, n_steps: int, out_every: int) -> torch.Tensor:
        n_out = n_steps // out_every + 1
        return torch.zeros((n_out, len(self.grids), L.TWA_NSCALARS), dtype=torch.float64, device=self.device)

    def advance(self, n_steps: int, out_every: int, series: Optional[torch.Tensor] = None, stream=None):
        series = self.new_series(n_steps, out_every) if series is None else series
        twa_advance(self.h, self.psi, n_steps, out_every, series, stream)
        return series

    def autotune(self, cache_path: Optional[str] = None, stream=None):
        twa_autotune(self.h, self.psi, cache_path, stream)
