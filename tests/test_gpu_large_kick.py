"""GPU parity of kicks whose phase exceeds 1/4 rad (Sec. III.B.2, the potential factor of the
split step) against the oracle.

The FP32 passes evaluate exp(-i theta) for the kick in two forms: Taylor polynomials when every
|theta| of a thread is at most 1/4, otherwise a reduction of theta mod 2 pi by a two-constant
split of 2 pi followed by sincosf.  The measured workloads kick by less than 0.06 rad, so these
cases are built to kick by 0.6-5 rad: workloads run at several times their usual step (the
3D soliton at the pi/4 rule of its own 32^3 grid; the 2D merger at 3x its step; a 1D cosine
collapse at a coarse step), and the adaptive step of Sec. III.B.2 with c_f = 0.2, whose potential
bound sets max|V| dt / hbar = 2 pi c_f = 1.26 rad for every full kick.  Each case asserts from the
oracle's potential that the general branch is reached.  Steps are few enough that FP32 rounding
cannot grow past the field tolerance (checked on the CPU by perturbing the oracle's run).
"""
import dataclasses

import numpy as np
import pytest
import torch

import twa_inputs as ti
from oracle import sp, twa
from paper_2310_07119_gb300 import twa_advance_adaptive
from tests.gpu_common import field_rel_l2, make_ensemble, oracle_batch

pytestmark = pytest.mark.gpu

F32_FIELD_TOL = 1e-4
RHO_TOL = 1e-5
CORR_TOL = 1e-2


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _fixed_cases():
    mer = ti.small_workload("merger2d", 2, 64, 4, 30, n_tot=1e9)
    mer = dataclasses.replace(mer, phys=dataclasses.replace(mer.phys, dt=0.0048))
    sol_axis = ti.Workload("soliton", ti.Grid(3, (32, 16, 16), 1.0), ti.Physics(ti.HBAR_3D, 4 * np.pi, 0.0042, 1e10),
                           3, 20, 10, 0, 77)
    return {
        "3d_soliton32_plane": ti.small_workload("soliton", 3, 32, 3, 20, n_tot=1e10),
        "3d_soliton_32x16x16_axis": sol_axis,
        "2d_merger64": mer,
        "1d_cosine64": ti.Workload("cosine", ti.Grid.cube(1, 64), ti.Physics(1e-3, 4 * np.pi, 0.02, 1e6), 4, 12, 4, 0, 3),
    }


FIXED = _fixed_cases()


def _max_kick_phase(w, b):
    V = sp.potential(b, w.phys.C, w.grid.L, w.grid.dim)
    return float(np.abs(V).max() * w.phys.dt / w.phys.hbar_m)


@pytest.mark.parametrize("name", list(FIXED))
def test_large_fixed_step_kicks_match_oracle(name):
    w = FIXED[name]
    cl = w.psi_cl()
    b0 = twa.sample(cl, w.noise_seed, w.n_real, w.phys.n_tot, w.grid.dV)
    assert _max_kick_phase(w, b0) > 0.5              # even the half kicks pass the Taylor range
    ens = make_ensemble([w], 0)
    ens.sample([cl], w.noise_seed)
    ens.step(w.n_steps)
    got = ens.fields(0).cpu().numpy().astype(np.complex128)
    ref = oracle_batch(w, cl, w.n_steps)
    err = field_rel_l2(got, ref, w.grid.dim)
    assert np.all(err < F32_FIELD_TOL), err
    m = ens.moments(0)
    mo = twa.moments(ref, w.phys.n_tot, w.grid.L, w.grid.dim, with_modes=False)
    rm = m["rho_mean"].cpu().numpy().reshape(w.grid.shape)
    assert np.linalg.norm(rm - mo["rho_mean"]) / np.linalg.norm(mo["rho_mean"]) < RHO_TOL
    ens.close()


@pytest.mark.parametrize("name", ["3d_soliton32_plane", "2d_merger64"])
def test_large_kicks_through_the_run_series(name):
    """twa_run merges half kicks into full kicks and applies the pending half kick inside the
    moment kernels and the closing kick kernel: all of them take the general branch here."""
    w = FIXED[name]
    every = 5
    n = (w.n_steps // every) * every
    cl = w.psi_cl()
    ens = make_ensemble([w], 0)
    series = ens.run([cl], w.noise_seed, n, every).cpu().numpy()
    t, ref_series, ref_final = twa.run(cl, w.phys.hbar_m, w.phys.C, w.phys.dt, w.grid.L, w.grid.dim, w.phys.n_tot,
                                       w.n_real, w.noise_seed, n, every)
    for o, mo in enumerate(ref_series):
        assert abs(series[o, 0, 1] - mo["corr"]) <= CORR_TOL * mo["corr"] + 1e-12, o
    got = ens.fields(0).cpu().numpy().astype(np.complex128)
    assert np.all(field_rel_l2(got, ref_final, w.grid.dim) < F32_FIELD_TOL)
    ens.close()


def _adaptive_cases():
    return {
        "3d_soliton32_plane": (ti.small_workload("soliton", 3, 32, 3, 0, n_tot=1e10), 3),
        "2d_merger64": (ti.small_workload("merger2d", 2, 64, 4, 0, n_tot=1e9), 3),
        "1d_cosine64": (ti.Workload("cosine", ti.Grid.cube(1, 64), ti.Physics(1e-3, 4 * np.pi, 0.01, 1e6), 4, 0, 5, 0, 3), 2),
    }


ADAPTIVE = _adaptive_cases()


@pytest.mark.parametrize("name", list(ADAPTIVE))
def test_adaptive_step_at_cf_0_2_matches_oracle(name):
    w, n_out = ADAPTIVE[name]
    every, c_f = 5, 0.2
    cl = w.psi_cl()
    ens = make_ensemble([w], 0)
    ens.sample([cl], w.noise_seed)
    series = ens.new_series(n_out * every, every)
    times = twa_advance_adaptive(ens.h, ens.psi, n_out, every, c_f, series)
    got = ens.fields(0).cpu().numpy().astype(np.complex128)
    sc = series.cpu().numpy()
    b0 = twa.sample(cl, w.noise_seed, w.n_real, w.phys.n_tot, w.grid.dV, w.phys.noise_conv)
    t_ref, s_ref, final, dts = twa.run_adaptive(cl, w.phys.hbar_m, w.phys.C, w.grid.L, w.grid.dim, w.phys.n_tot,
                                                w.n_real, w.noise_seed, n_out, every, c_f, batch=b0)
    # the potential bound sets the step: max|V| dt / hbar = 2 pi c_f on the first interval
    V = sp.potential(b0, w.phys.C, w.grid.L, w.grid.dim)
    assert float(np.abs(V).max()) * dts[0] / w.phys.hbar_m == pytest.approx(2 * np.pi * c_f, rel=1e-9)
    assert np.allclose(times, t_ref, rtol=1e-5, atol=0)
    assert np.all(field_rel_l2(got, final, w.grid.dim) < F32_FIELD_TOL), field_rel_l2(got, final, w.grid.dim)
    for o, mo in enumerate(s_ref):
        assert abs(sc[o, 0, 1] - mo["corr"]) <= CORR_TOL * mo["corr"] + 1e-12
    ens.close()
