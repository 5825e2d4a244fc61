"""GPU edge cases of the C ABI: rejected arguments (with their status codes and messages), zero
steps, a single stream (a Poisson pair with one member), the smallest transform lengths and a
grid with three different axis lengths, each against the oracle or an exact expectation."""
import numpy as np
import pytest
import torch

import twa_inputs as ti
from oracle import sp, twa
from paper_2310_07119_gb300 import Ensemble, TwaError, twa_advance
from paper_2310_07119_gb300 import _lib as L
from tests.gpu_common import field_rel_l2, make_ensemble, oracle_batch

pytestmark = pytest.mark.gpu

F32_FIELD_TOL = 1e-4


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.mark.parametrize("grid,n_real", [
    (ti.Grid(3, (48, 32, 32), 1.0), [2]),        # not a power of two
    (ti.Grid(1, (4096, 1, 1), 1.0), [2]),        # longer than the longest plan
    (ti.Grid(2, (4, 64, 1), 1.0), [2]),          # shorter than the shortest plan
    (ti.Grid.cube(3, 16), [0]),                   # no stream
])
def test_create_rejects_bad_shapes(grid, n_real):
    with pytest.raises(TwaError) as e:
        Ensemble([grid], ti.HBAR_3D, ti.C_UNIT, 1e-4, 1e8, n_real)
    assert e.value.code == L.TWA_EINVAL and len(str(e.value)) > 10


def test_create_rejects_nonpositive_physics():
    g = ti.Grid.cube(3, 16)
    for hb, dt, n in ((0.0, 1e-4, 1e8), (ti.HBAR_3D, -1e-4, 1e8), (ti.HBAR_3D, 1e-4, 0.0)):
        with pytest.raises(TwaError) as e:
            Ensemble([g], hb, ti.C_UNIT, dt, n, [2])
        assert e.value.code == L.TWA_EINVAL


def test_advance_rejects_steps_not_a_multiple_of_out_every():
    w = ti.small_workload("kgauss", 3, 16, 2, 0, n_tot=1e8)
    ens = make_ensemble([w], 0)
    ens.sample([w.psi_cl()], w.noise_seed)
    with pytest.raises(TwaError) as e:
        twa_advance(ens.h, ens.psi, 15, 10, ens.new_series(10, 10))
    assert e.value.code == L.TWA_EINVAL and "out_every" in str(e.value)
    ens.close()


def test_zero_steps_leave_the_batch_unchanged_and_run_reports_t0():
    w = ti.small_workload("kgauss", 3, 16, 3, 0, n_tot=1e8)
    cl = w.psi_cl()
    ens = make_ensemble([w], 0)
    ens.sample([cl], w.noise_seed)
    before = ens.fields(0).cpu().numpy().copy()
    ens.step(0)
    assert np.array_equal(before, ens.fields(0).cpu().numpy())
    series = ens.run([cl], w.noise_seed, 0, 10).cpu().numpy()
    assert series.shape[0] == 1
    assert np.array_equal(before, ens.fields(0).cpu().numpy())     # sampled again, nothing applied
    mo = twa.moments(twa.sample(cl, w.noise_seed, w.n_real, w.phys.n_tot, w.grid.dV), w.phys.n_tot, 1.0, 3)
    assert abs(series[0, 0, 1] - mo["corr"]) <= 1e-2 * mo["corr"]
    ens.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_single_stream_half_pair(precision):
    """One stream: slots (classical, stream) form one Poisson pair; with two streams the last pair
    has one member; both against the oracle."""
    for n_real in (1, 2):
        w = ti.small_workload("kgauss", 3, 16, n_real, 20, n_tot=1e8)
        cl = w.psi_cl()
        ens = make_ensemble([w], precision)
        ens.sample([cl], w.noise_seed)
        ens.step(w.n_steps)
        got = ens.fields(0).cpu().numpy().astype(np.complex128)
        ref = oracle_batch(w, cl, w.n_steps)
        tol = F32_FIELD_TOL if precision == 0 else 1e-10
        assert np.all(field_rel_l2(got, ref, 3) < tol), (n_real, field_rel_l2(got, ref, 3))
        ens.close()


@pytest.mark.parametrize("shape", [(8,), (16,), (8, 8), (16, 8), (8, 8, 8), (64, 16, 8)])
def test_smallest_lengths_and_unequal_axes(shape):
    dim = len(shape)
    g = ti.Grid(dim, tuple(list(shape[::-1]) + [1] * (3 - dim)), 1.0)
    w = ti.Workload("kgauss" if dim > 1 else "bump1d", g, ti.Physics(ti.HBAR_3D, ti.C_UNIT, 2e-4, 1e8),
                    3, 30, 10, 5, 777)
    cl = w.psi_cl()
    ens = make_ensemble([w], 0)
    ens.sample([cl], w.noise_seed)
    ens.step(w.n_steps)
    got = ens.fields(0).cpu().numpy().astype(np.complex128)
    ref = oracle_batch(w, cl, w.n_steps)
    assert np.all(field_rel_l2(got, ref, dim) < F32_FIELD_TOL), field_rel_l2(got, ref, dim)
    ens.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_literal_noise_reading_samples_match_oracle(precision):
    """noise_conv = 1 (the paper's printed variance, twice the coherent-state one) on both paths."""
    base = ti.small_workload("kgauss", 3, 16, 4, 0, n_tot=1e6)
    out = {}
    for conv in (0, 1):
        w = ti.Workload(base.name, base.grid, ti.Physics(base.phys.hbar_m, base.phys.C, base.phys.dt,
                                                         base.phys.n_tot, conv),
                        base.n_real, 0, base.out_every, base.psi_cl_seed, base.noise_seed)
        cl = w.psi_cl()
        ens = make_ensemble([w], precision)
        ens.sample([cl], w.noise_seed)
        got = ens.fields(0).cpu().numpy().astype(np.complex128)
        ref = twa.sample(cl, w.noise_seed, w.n_real, w.phys.n_tot, w.grid.dV, conv)
        tol = 2 * np.finfo(np.float32).eps if precision == 0 else 1e-14
        assert np.max(np.abs(got - ref)) <= tol * np.abs(ref).max()
        out[conv] = got[1:] - cl
        amp = np.abs(cl).max()
        ens.close()
    # same normals, sigma scaled by sqrt(2) (up to the rounding of the stored fields)
    atol = 4 * np.finfo(np.float32).eps * amp if precision == 0 else 1e-13 * amp
    assert np.max(np.abs(out[1] - np.sqrt(2.0) * out[0])) <= atol


def test_added_entry_points_reject_bad_use():
    from paper_2310_07119_gb300 import (twa_advance_adaptive, twa_particles_get, twa_particles_set,
                                        twa_phase_moments)
    w = ti.small_workload("kgauss", 3, 16, 2, 0, n_tot=1e8)
    cl = w.psi_cl()
    ens = make_ensemble([w], 0)
    ens.sample([cl], w.noise_seed)
    s = ens.new_series(10, 5)
    for bad in (dict(c_f=0.0), dict(c_f=-1.0), dict(c_f=float("nan"))):
        with pytest.raises(TwaError) as e:
            twa_advance_adaptive(ens.h, ens.psi, 2, 5, bad["c_f"], s)
        assert e.value.code == L.TWA_EINVAL
    with pytest.raises(TwaError) as e:
        twa_particles_get(ens.h, 0, 3, 3)                 # nothing set yet
    assert e.value.code == L.TWA_EINVAL
    with pytest.raises(TwaError) as e:
        twa_particles_set(ens.h, 0, np.full((3, 3), np.nan), np.zeros((3, 3)))
    assert e.value.code == L.TWA_EINVAL
    with pytest.raises(TwaError) as e:
        twa_phase_moments(ens.h, 5, ens.psi)              # no such instance
    assert e.value.code == L.TWA_EINVAL
    ens.close()
    e64 = make_ensemble([w], 1)
    e64.sample([cl], w.noise_seed)
    with pytest.raises(TwaError) as e:
        twa_advance_adaptive(e64.h, e64.psi, 1, 5, 0.01, e64.new_series(5, 5))
    assert e.value.code == L.TWA_EINVAL and "FP32" in str(e.value)
    with pytest.raises(TwaError) as e:
        twa_particles_set(e64.h, 0, np.zeros((3, 3)), np.zeros((3, 3)))
    assert e.value.code == L.TWA_EINVAL
    e64.close()


def test_calls_reject_a_batch_that_is_not_16_byte_aligned():
    """Field buffers are read with 16-byte copies; a batch view starting 8 bytes into an allocation
    is refused with TWA_EINVAL before anything is launched, and the aligned batch is untouched."""
    from paper_2310_07119_gb300 import (twa_advance_adaptive, twa_autotune, twa_moments, twa_phase_moments,
                                        twa_step_batch)
    w = ti.small_workload("kgauss", 3, 16, 2, 0, n_tot=1e8)
    ens = make_ensemble([w], 0)
    ens.sample([w.psi_cl()], w.noise_seed)
    before = ens.psi.clone()
    raw = torch.zeros(ens.psi.numel() + 1, dtype=ens.psi.dtype, device=ens.psi.device)
    off = raw[1:]
    off.copy_(ens.psi)
    assert off.data_ptr() % 16 == 8
    calls = {
        "twa_step_batch": lambda: twa_step_batch(ens.h, off, 1),
        "twa_advance": lambda: twa_advance(ens.h, off, 10, 10, ens.new_series(10, 10)),
        "twa_moments": lambda: twa_moments(ens.h, 0, off, {}),
        "twa_phase_moments": lambda: twa_phase_moments(ens.h, 0, off),
        "twa_advance_adaptive": lambda: twa_advance_adaptive(ens.h, off, 1, 5, 0.01, ens.new_series(5, 5)),
        "twa_autotune": lambda: twa_autotune(ens.h, off),
    }
    for name, call in calls.items():
        with pytest.raises(TwaError) as e:
            call()
        assert e.value.code == L.TWA_EINVAL and "16-byte" in str(e.value) and name in str(e.value), name
    torch.cuda.synchronize()
    assert torch.equal(off, before) and torch.equal(ens.psi, before)
    ens.close()
