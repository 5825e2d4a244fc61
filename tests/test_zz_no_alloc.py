"""The allocation-free 1D step (twa_step_batch_1d_static) against the handle-based step.

Callers that cannot allocate device memory where they step (a process whose device memory is
owned by its own pool, a loop that must not risk an allocation failure or the synchronization an
allocation can cause) use twa_step_batch_1d_static, which keeps its Poisson buffer and tables in
static device arrays.  This checks, through the C ABI, that two consecutive calls give the same
fields as twa_step_batch on a handle, within the FP32 field tolerance of the parity tests, and
that oversized batches are refused.  The file is named so that pytest collects it last.
"""
import ctypes

import numpy as np
import pytest
import torch

import twa_inputs as ti
from paper_2310_07119_gb300 import _lib
from tests.gpu_common import field_rel_l2, make_ensemble

F32_FIELD_TOL = 1e-4


def _fn():
    lib = _lib.load()
    fn = lib.twa_step_batch_1d_static
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.POINTER(_lib.Grid), ctypes.POINTER(_lib.Params), ctypes.c_int, ctypes.c_void_p,
                   ctypes.c_int, ctypes.c_void_p]
    return lib, fn


def _grid_params(w):
    g = _lib.Grid(1, (ctypes.c_int * 3)(w.grid.n[0], 1, 1), w.grid.L)
    p = _lib.Params(w.phys.hbar_m, w.phys.C, w.phys.dt, w.phys.n_tot, 0, _lib.TWA_F32, 0)
    return g, p


def test_static_scratch_rejects_oversized_batches():
    lib, fn = _fn()
    w = ti.workload_1d_bump(2048, 4, 10)
    g, p = _grid_params(w)
    too_many = 2 * (_lib_max() // 2048) + 1          # one pair more than the static buffer holds
    rc = fn(ctypes.byref(g), ctypes.byref(p), too_many, ctypes.c_void_p(1), 1, None)
    assert rc == _lib.TWA_EINVAL
    assert b"exceeds the static scratch" in lib.twa_last_error(None)


def _lib_max():
    txt = open(_lib.HEADER).read()
    assert "#define TWA_STATIC_SCRATCH_ELEMS (1 << 19)" in txt
    return 1 << 19


@pytest.mark.gpu
def test_static_step_matches_handle_step_on_two_calls():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    lib, fn = _fn()
    w = ti.workload_1d_bump(256, 9, 0)
    ens = make_ensemble([w], 0, want_modes=False)
    ens.sample([w.psi_cl()], w.noise_seed)
    mine = ens.psi.clone()
    g, p = _grid_params(w)
    st = torch.cuda.current_stream().cuda_stream
    for n in (40, 60):                                   # two calls in a row, each against the handle path
        ens.step(n)
        rc = fn(ctypes.byref(g), ctypes.byref(p), w.n_real, ctypes.c_void_p(mine.data_ptr()), n, ctypes.c_void_p(st))
        assert rc == 0, lib.twa_last_error(None)
        torch.cuda.synchronize()
        a = ens.psi.view(w.n_real + 1, -1).cpu().numpy().astype(np.complex128)
        b = mine.view(w.n_real + 1, -1).cpu().numpy().astype(np.complex128)
        assert np.all(np.isfinite(b))
        assert np.all(field_rel_l2(b, a, 1) < F32_FIELD_TOL)
    ens.close()
