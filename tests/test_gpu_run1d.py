"""Whole 1D runs in one launch (twa_advance on 1D handles) against the per-interval path and the oracle.

On a handle whose instances are all 1D, twa_advance runs every step and the moment sums of every
output on chip, one launch per instance plus one finishing launch (partial sums of the pairs in pair
order).  Each stream is a line of its own; the two lines of a pair exchange densities and moment
terms by shuffles (2T <= 32 threads) or through shared memory (T >= 32, lengths 512-2048), and both
branches are covered by the lengths below.  With the pass profiler on, the same call runs the per-interval path (one on-chip launch per
output interval and separate moment kernels).  The two do the same arithmetic per field, so the
fields must be bitwise equal; the scalars add the streams in a different order and agree to
rounding.  The series is also checked against the oracle's run (Sec. III.B.3, Eq. E[op], Eq. Q).
"""
import numpy as np
import pytest
import torch

import twa_inputs as ti
from oracle import twa
from paper_2310_07119_gb300 import twa_advance, twa_profile_enable, twa_sync_status
from tests.gpu_common import field_rel_l2, make_ensemble

pytestmark = pytest.mark.gpu

F32_FIELD_TOL = 1e-4
CORR_TOL = 1e-2


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _run(w, n_steps, every, fused, want_modes=True, poison=None):
    ens = make_ensemble([w], 0, want_modes=want_modes)
    ens.sample([w.psi_cl()], w.noise_seed)
    if poison is not None:
        ens.fields(0)[poison] = complex(float("nan"), 0.0)
    twa_profile_enable(ens.h, not fused)
    series = ens.new_series(n_steps, every)
    twa_advance(ens.h, ens.psi, n_steps, every, series)
    rc = twa_sync_status(ens.h)
    out = series.cpu().numpy(), ens.fields(0).cpu().numpy().copy(), rc
    ens.close()
    return out


@pytest.mark.parametrize("n,n_real", [(8, 6), (16, 3), (64, 10), (256, 31), (256, 32), (512, 9), (1024, 4), (2048, 5)])
def test_whole_run_equals_the_per_interval_path(n, n_real):
    w = ti.workload_1d_bump(n, n_real, 0)
    s_f, f_f, rc_f = _run(w, 60, 10, True)
    s_u, f_u, rc_u = _run(w, 60, 10, False)
    assert rc_f == rc_u == 0
    assert np.array_equal(f_f, f_u)
    # Q, corr, mass, mass_cl, non-finite count, n_k sum, |<rho> - rho_cl|, |rho_cl|: the stream sums
    # differ in order (pair partials in FP64 against double-float sums over slots), ~1e-15 relative;
    # <rho> - rho_cl is ~1e-3 of rho, so corr and |<rho> - rho_cl| carry ~1e-12
    assert np.allclose(s_f[:, 0, [2, 3, 7]], s_u[:, 0, [2, 3, 7]], rtol=1e-12, atol=0)
    assert np.allclose(s_f[:, 0, [1, 6]], s_u[:, 0, [1, 6]], rtol=1e-9, atol=0)
    assert np.all(np.abs(s_f[:, 0, 0] - s_u[:, 0, 0]) <= 1e-12 * s_u[:, 0, 2])      # Q: difference of O(1) sums
    assert np.array_equal(s_f[:, 0, 4], s_u[:, 0, 4])
    assert np.allclose(s_f[:, 0, 5], s_u[:, 0, 5], rtol=1e-6)                       # Parseval vs mode sums


def test_whole_run_matches_the_oracle():
    """The 1D workload (256 cells, 32 streams) for 100 steps with an output every 10 steps."""
    w = ti.workload_1d_bump(256, 32, 100)
    series, fields, rc = _run(w, 100, 10, True)
    assert rc == 0
    cl = w.psi_cl()
    _, ref_series, ref_final = twa.run(cl, w.phys.hbar_m, w.phys.C, w.phys.dt, w.grid.L, 1, w.phys.n_tot, w.n_real,
                                       w.noise_seed, 100, 10)
    assert np.all(field_rel_l2(fields.astype(np.complex128), ref_final, 1) < F32_FIELD_TOL)
    for o, mo in enumerate(ref_series):
        assert abs(series[o, 0, 1] - mo["corr"]) <= CORR_TOL * mo["corr"] + 1e-12, o
        assert abs(series[o, 0, 5] - np.sum(mo["nk_mean"])) < 1e-4 * np.sum(np.abs(mo["nk_mean"])), o


def test_chunked_whole_run_at_the_largest_lines():
    """2048 cells x 511 streams: the partial sums of 25 outputs exceed the 256 MB cap, so the run is
    split into launches of whole outputs (each opening and closing with a half kick)."""
    w = ti.workload_1d_bump(2048, 511, 0)
    s_f, f_f, rc_f = _run(w, 50, 2, True, want_modes=False)
    s_u, f_u, rc_u = _run(w, 50, 2, False, want_modes=False)
    assert rc_f == rc_u == 0
    err = field_rel_l2(f_f.astype(np.complex128), f_u.astype(np.complex128), 1)
    assert np.all(err < 1e-5), err.max()
    assert np.allclose(s_f[:, 0, [1, 2, 3]], s_u[:, 0, [1, 2, 3]], rtol=1e-6, atol=0)


def test_nonfinite_value_is_counted_and_flagged():
    w = ti.workload_1d_bump(256, 9, 0)
    series, fields, rc = _run(w, 20, 10, True, poison=(3, 17))
    assert rc == -5                                   # TWA_ENONFINITE
    assert series[-1, 0, 4] > 0
    assert np.all(np.isfinite(fields[[0, 1, 4, 5]]))  # other pairs are untouched by the NaN
