"""Learned correction surrogate: a Fourier neural operator trained on TWA runs of this library.

The network and its training run in libtwa.so (``twa_fno_*``: forward, backward, AdamW, loss and
feature kernels); this module marshals buffers and drives the loop.  Training data come from the
library's own TWA runs: for every run a handle with two instances sharing the classical field — an
input ensemble of a few streams and an independent reference ensemble — evolved with
``twa_step_batch``; per-mode moments from ``twa_moments`` give the classical occupation n_cl, the
few-stream estimate n_est and the reference n_ref.  The target is the correction spectrum
<n_k> - n_k^cl relative to n_cl + n_tot / K (K modes); the surrogate's job is to predict the many-stream value
from the classical spectrum and the few-stream estimate, and the full ensemble stays the fallback and
the reference for its error.
"""
from __future__ import annotations

import ctypes
import dataclasses
import math
from typing import List, Optional, Sequence

import numpy as np
import torch

from . import _lib as L
from .twa import Ensemble, TwaError, _ptr, _stream

C_IN = 4


def _lib():
    if not torch.cuda.is_available():
        raise TwaError(L.TWA_ECUDA, "no CUDA device: the surrogate has no CPU path")
    return L.load()


class FNO:
    """Handle of a twa_fno network (grid^3 mode grid, width, modes per sign per axis, layers)."""

    def __init__(self, grid: int, width: int = 32, modes: int = 6, layers: int = 4, c_in: int = C_IN, c_out: int = 1,
                 seed: int = 0, device="cuda:0"):
        lib = _lib()
        self.device = torch.device(device)
        self.cfg = L.FnoConfig(grid, width, modes, layers, c_in, c_out)
        h = ctypes.c_void_p()
        rc = lib.twa_fno_create(ctypes.byref(h), ctypes.byref(self.cfg), int(seed))
        if rc != 0:
            raise TwaError(rc, lib.twa_last_error(None).decode())
        self.h = h.value
        self.n_params = int(lib.twa_fno_num_params(self.h))
        self.K = grid ** 3
        self._loss = torch.zeros(1, dtype=torch.float32, device=self.device)

    def _check(self, rc):
        if rc != 0:
            raise TwaError(rc, L.load().twa_fno_last_error(self.h).decode())

    def close(self):
        if getattr(self, "h", None):
            L.load().twa_fno_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, theta: torch.Tensor, stream=None):
        theta = theta.to(self.device, torch.float32).contiguous()
        self._check(L.load().twa_fno_set_params(self.h, _ptr(theta), _stream(stream)))

    def get_params(self, which: int = 0, stream=None) -> torch.Tensor:
        out = torch.empty(self.n_params, dtype=torch.float32, device=self.device)
        self._check(L.load().twa_fno_get_params(self.h, _ptr(out), int(which), _stream(stream)))
        return out

    def forward(self, x: torch.Tensor, stream=None) -> torch.Tensor:
        B = x.shape[0]
        y = torch.empty((B, self.cfg.c_out) + tuple(x.shape[2:]), dtype=torch.float32, device=self.device)
        self._x = x.contiguous()
        self._check(L.load().twa_fno_forward(self.h, _ptr(self._x), B, _ptr(y), _stream(stream)))
        return y

    def backward(self, dy: torch.Tensor, want_dx: bool = False, stream=None) -> Optional[torch.Tensor]:
        dx = torch.empty_like(self._x) if want_dx else None
        self._check(L.load().twa_fno_backward(self.h, _ptr(dy.contiguous()), dy.shape[0], _ptr(dx), _stream(stream)))
        return dx

    def zero_grad(self, stream=None):
        self._check(L.load().twa_fno_zero_grad(self.h, _stream(stream)))

    def adamw(self, lr, beta1=0.9, beta2=0.999, eps=1e-8, weight_decay=1e-4, stream=None):
        self._check(L.load().twa_fno_adamw(self.h, lr, beta1, beta2, eps, weight_decay, _stream(stream)))

    def mse(self, y: torch.Tensor, t: torch.Tensor, want_grad: bool = True, stream=None):
        dy = torch.empty_like(y) if want_grad else None
        self._check(L.load().twa_fno_mse(self.h, _ptr(y), _ptr(t.contiguous()), y.numel(), _ptr(self._loss), _ptr(dy),
                                         _stream(stream)))
        return self._loss, dy

    def train_step(self, x: torch.Tensor, t: torch.Tensor, lr: float, weight_decay: float = 1e-4):
        self.zero_grad()
        y = self.forward(x)
        loss, dy = self.mse(y, t)
        self.backward(dy)
        self.adamw(lr, weight_decay=weight_decay)
        return loss


def features(nk_cl: torch.Tensor, nk_est: torch.Tensor, n_tot: float, grid: int,
             nk_ref: Optional[torch.Tensor] = None, stream=None):
    """Kernel-built features x[4][grid^3] (and target t[grid^3] if nk_ref is given)."""
    x = torch.empty((C_IN, grid, grid, grid), dtype=torch.float32, device=nk_cl.device)
    t = torch.empty((1, grid, grid, grid), dtype=torch.float32, device=nk_cl.device) if nk_ref is not None else None
    rc = L.load().twa_fno_features(_ptr(nk_cl), _ptr(nk_est), _ptr(nk_ref), float(n_tot), int(grid), _ptr(x), _ptr(t),
                                   _stream(stream))
    if rc != 0:
        raise TwaError(rc, L.load().twa_last_error(None).decode())
    return x, t


@dataclasses.dataclass
class Sample:
    x: torch.Tensor          # (4, n, n, n) features
    t: torch.Tensor          # (1, n, n, n) target from the reference ensemble
    nk_cl: np.ndarray        # per-mode classical occupation (host, FP64)
    nk_est: np.ndarray       # few-stream estimate of <n_k>
    nk_ref: np.ndarray       # reference-ensemble <n_k>
    n_tot: float
    k0: float
    step: int


def generate(runs: Sequence[dict], grid: int, n_est: int, n_ref: int, snap_steps: Sequence[int],
             hbar_m: float, C: float, dt: float, keep_host: bool = False, device="cuda:0") -> List[Sample]:
    """TWA runs of the condensation family; each run dict has k0 (in units of 2 pi / L), n_tot, seed.

    Every run is one handle of two instances with the same classical field: n_est input streams and
    n_ref reference streams (independent noise: the instance index enters the Philox counter).
    """
    import twa_inputs as ti
    out = []
    g = ti.Grid.cube(3, grid)
    for r in runs:
        psi_cl = ti.kspace_gaussian(g, r["k0"] * 2.0 * np.pi, r["seed"])
        ens = Ensemble([g, g], hbar_m, C, dt, r["n_tot"], [n_est, n_ref], want_modes=True, device=device)
        ens.sample([psi_cl, psi_cl], r["seed"] + 1000003)
        done = 0
        for s in snap_steps:
            ens.step(s - done)
            done = s
            m_est = ens.moments(0)
            m_ref = ens.moments(1)
            x, t = features(m_est["nk_cl"], m_est["nk_mean"], r["n_tot"], grid, nk_ref=m_ref["nk_mean"])
            host = (m_est["nk_cl"].cpu().numpy(), m_est["nk_mean"].cpu().numpy(), m_ref["nk_mean"].cpu().numpy()) \
                if keep_host else (None, None, None)
            out.append(Sample(x, t, *host, n_tot=r["n_tot"], k0=r["k0"], step=s))
        ens.close()
    return out


def run_table(n: int, seed: int, k0_range=(2.0, 5.0), log_ntot_range=(8.0, 10.0)) -> List[dict]:
    """Seeded run parameters: k0 uniform in k0_range (units of 2 pi / L), log10 n_tot uniform."""
    rng = np.random.default_rng(seed)
    return [{"k0": float(rng.uniform(*k0_range)), "n_tot": float(10 ** rng.uniform(*log_ntot_range)),
             "seed": int(rng.integers(1, 2 ** 31))} for _ in range(n)]


def train(model: FNO, data: List[Sample], iters: int, batch: int, lr: float, seed: int = 0, log_every: int = 0):
    """AdamW on the MSE of the target with a cosine learning-rate decay; returns the loss history."""
    rng = np.random.default_rng(seed)
    X = torch.stack([s.x for s in data])
    T = torch.stack([s.t for s in data])
    hist = []
    for it in range(iters):
        idx = torch.as_tensor(rng.choice(len(data), batch, replace=False), device=X.device)
        lr_t = 0.5 * lr * (1.0 + math.cos(math.pi * it / iters))
        loss = model.train_step(X[idx].contiguous(), T[idx].contiguous(), lr_t)
        if log_every and (it % log_every == 0 or it == iters - 1):
            hist.append((it, float(loss.item())))
    return hist


def predict_correction(model: FNO, s: Sample) -> np.ndarray:
    """Predicted <n_k> - n_k^cl (number units) for one sample."""
    y = model.forward(s.x[None].contiguous())[0, 0].double().cpu().numpy().ravel()
    return y * (np.maximum(s.nk_cl, 0.0) + s.n_tot / s.nk_cl.size)


def shell_errors(pred: np.ndarray, ref: np.ndarray, grid: int, nbins: int):
    """Relative L2 error of shell-averaged spectra (shells of integer |m| below nbins)."""
    m = np.fft.fftfreq(grid, d=1.0 / grid)
    r = np.sqrt(m[:, None, None] ** 2 + m[None, :, None] ** 2 + m[None, None, :] ** 2)
    idx = np.rint(r).astype(int).ravel()
    cnt = np.bincount(idx, minlength=nbins)[:nbins]
    sa = lambda f: np.bincount(idx, weights=f, minlength=nbins)[:nbins] / np.maximum(cnt, 1)
    a, b = sa(pred), sa(ref)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def fallback_statistic(pred_corr: np.ndarray, est_corr: np.ndarray, grid: int, nbins: int) -> float:
    """Disagreement of the surrogate with the few-stream estimate it was given: relative L2 distance
    of their shell-averaged correction spectra (number units)."""
    return shell_errors(pred_corr, est_corr, grid, nbins)


def calibrate_fallback(stats: Sequence[float], quantile: float = 0.9) -> float:
    """Threshold on the fallback statistic: its `quantile` over validation samples (runs where the
    surrogate is trusted); above it, a prediction is replaced by a full-ensemble run."""
    v = np.asarray(list(stats), dtype=np.float64)
    if v.size == 0 or not np.all(np.isfinite(v)):
        raise ValueError("calibrate_fallback: need finite validation statistics")
    return float(np.quantile(v, quantile))


def correct_or_fallback(pred_corr: np.ndarray, est_corr: np.ndarray, grid: int, nbins: int, tau: float):
    """(correction, fell_back): the surrogate's correction when it agrees with the few-stream
    estimate within the calibrated threshold tau; otherwise (None, True), and the caller runs the
    full ensemble for that snapshot."""
    stat = fallback_statistic(pred_corr, est_corr, grid, nbins)
    if not np.isfinite(stat) or stat > tau:
        return None, True
    return pred_corr, False


def time_steps(grid: int, modes: int, batch: int, width: int = 32, layers: int = 4, reps: int = 3) -> dict:
    """Device time of one training step (forward, MSE, backward, AdamW) and of one forward, with the
    tensor-core GEMMs on and off, on random inputs (CUDA events on the current stream)."""
    model = FNO(grid, width, modes, layers, seed=1)
    lib = L.load()
    x = torch.randn(batch, C_IN, grid, grid, grid, device=model.device)
    t = torch.randn(batch, 1, grid, grid, grid, device=model.device)
    out = {"grid": grid, "modes": modes, "batch": batch, "width": width, "layers": layers, "params": model.n_params,
           "tensor_core_shapes": int(lib.twa_fno_tensor_core_shapes(model.h))}
    for tc in (1, 0):
        lib.twa_fno_set_tensor_cores(model.h, tc)
        for _ in range(2):
            model.train_step(x, t, 1e-4)
        torch.cuda.synchronize()
        e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        e[0].record()
        for _ in range(reps):
            model.train_step(x, t, 1e-4)
        e[1].record()
        e[2].record()
        model.forward(x)
        e[3].record()
        torch.cuda.synchronize()
        key = "tensor_cores" if tc else "cuda_cores"
        out[key] = {"train_step_ms": e[0].elapsed_time(e[1]) / reps, "forward_ms": e[2].elapsed_time(e[3])}
    model.close()
    return out


def main(argv=None):
    """Train the surrogate on library-generated runs and report held-out errors (JSON lines).

    python -m paper_2310_07119_gb300.fno [--grid 32] [--runs 200] [--iters 3000]
    """
    import argparse
    import json
    import twa_inputs as ti
    ap = argparse.ArgumentParser()
    ap.add_argument("--grid", type=int, default=32)
    ap.add_argument("--runs", type=int, default=200)
    ap.add_argument("--test-runs", type=int, default=12)
    ap.add_argument("--iters", type=int, default=3000)
    ap.add_argument("--lr", type=float, default=5e-4)
    ap.add_argument("--width", type=int, default=32)
    ap.add_argument("--modes", type=int, default=6)
    ap.add_argument("--k0", type=float, nargs=2, default=(2.0, 5.0), help="k0 range in units of 2 pi / L")
    ap.add_argument("--snaps", type=int, nargs="+", default=None,
                    help="snapshot steps (default: 150..400 at 32^3, scaled by (grid / 32)^2 so the times match)")
    ap.add_argument("--batch", type=int, default=8)
    ap.add_argument("--time", action="store_true", help="only time training steps (tensor cores on and off) and exit")
    a = ap.parse_args(argv)
    if a.time:
        print(json.dumps(time_steps(a.grid, a.modes, a.batch, a.width)))
        return None
    grid = a.grid
    dt = ti.dt_pi4_rule(ti.Grid.cube(3, grid), ti.HBAR_3D)
    snaps = a.snaps or [int(round(s * (grid / 32) ** 2)) for s in (150, 200, 250, 300, 350, 400)]
    train_set = generate(run_table(a.runs, 1, k0_range=tuple(a.k0)), grid, 8, 64, snaps, ti.HBAR_3D, ti.C_UNIT, dt)
    # held-out reference: 1024 streams as two independent halves (their difference measures the
    # reference's own sampling noise)
    import twa_inputs as _ti
    g = _ti.Grid.cube(3, grid)
    rows = []
    model = FNO(grid, a.width, a.modes, 4, seed=3)
    import time
    t0 = time.perf_counter()
    hist = train(model, train_set, a.iters, a.batch, a.lr, log_every=max(1, a.iters // 10))
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    nb = grid // 2 - 2
    for r in run_table(a.test_runs, 99, k0_range=tuple(a.k0)):
        psi_cl = _ti.kspace_gaussian(g, r["k0"] * 2.0 * np.pi, r["seed"])
        ens = Ensemble([g, g, g], ti.HBAR_3D, ti.C_UNIT, dt, r["n_tot"], [8, 512, 512], want_modes=True)
        ens.sample([psi_cl] * 3, r["seed"] + 1000003)
        done = 0
        for s in snaps:
            ens.step(s - done)
            done = s
            m = [ens.moments(i) for i in range(3)]
            ncl = m[0]["nk_cl"].cpu().numpy()
            est = m[0]["nk_mean"].cpu().numpy()
            ha, hb = m[1]["nk_mean"].cpu().numpy(), m[2]["nk_mean"].cpu().numpy()
            ref = 0.5 * (ha + hb)
            x, _ = features(m[0]["nk_cl"], m[0]["nk_mean"], r["n_tot"], grid)
            smp = Sample(x, None, ncl, est, ref, r["n_tot"], r["k0"], s)
            pred = predict_correction(model, smp)
            rows.append({"step": s, "n_tot": r["n_tot"], "k0": r["k0"],
                         "fno": shell_errors(pred, ref - ncl, grid, nb),
                         "est8": shell_errors(est - ncl, ref - ncl, grid, nb),
                         "zero": 1.0,
                         "ref_noise": 0.5 * shell_errors(ha - ncl, hb - ncl, grid, nb)})
        ens.close()
    summary = {}
    for s in snaps:
        sel = [r for r in rows if r["step"] == s]
        summary[s] = {k: float(np.median([r[k] for r in sel])) for k in ("fno", "est8", "ref_noise")}
    print(json.dumps({"config": {"grid": grid, "width": a.width, "modes": a.modes, "layers": 4, "train_runs": a.runs,
                                 "snapshots": snaps, "iters": a.iters, "batch": a.batch, "params": model.n_params,
                                 "k0": list(a.k0), "train_seconds": train_s},
                      "loss": hist, "median_shell_rel_err_vs_1024": summary}))
    return summary


if __name__ == "__main__":
    main()
