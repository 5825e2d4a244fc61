"""The allocation-free 1D step (twa_step_batch_1d_static) against the handle step and the oracle.

Callers that cannot allocate device memory where they step (a process whose device memory is
owned by its own pool, a loop that must not risk an allocation failure or the synchronization an
allocation can cause) use twa_step_batch_1d_static, which keeps its Poisson buffer and tables in
static device arrays.  Checked through the C ABI:
  * two consecutive calls give the same fields as twa_step_batch on a handle, within the FP32
    field tolerance of the parity tests, at the smallest, a middle and the largest line length;
  * at the exact size limit ((n_real + 2) / 2 x n = TWA_STATIC_SCRATCH_ELEMS, n = 2048 with 511
    streams) the fields match the FP64 oracle, so the largest accepted batch uses the whole
    static buffer correctly;
  * refused arguments (oversized batches, too many pairs for one launch, a stream count that
    would overflow, a buffer that is not 16-byte aligned) return TWA_EINVAL before any launch,
    so those checks run without a GPU.
The file is named so that pytest collects it last.
"""
import ctypes

import numpy as np
import pytest
import torch

import twa_inputs as ti
from oracle import sp
from paper_2310_07119_gb300 import _lib
from tests.gpu_common import field_rel_l2, make_ensemble

F32_FIELD_TOL = 1e-4
SCRATCH = 1 << 19          # TWA_STATIC_SCRATCH_ELEMS


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


def test_header_states_the_scratch_limit():
    txt = open(_lib.HEADER).read()
    assert "#define TWA_STATIC_SCRATCH_ELEMS (1 << 19)" in txt


@pytest.mark.parametrize("n,n_real,ptr,msg", [
    (2048, 2 * (SCRATCH // 2048) + 1, 256, b"exceeds the static scratch"),     # one pair more than the buffer holds
    (8, 131071, 256, b"65535 stream pairs"),                                   # fits the buffer, not one launch
    (8, 2 ** 31 - 1, 256, b"exceeds the static scratch"),                     # n_real + 1 must not wrap
    (256, 9, 256 + 8, b"16-byte aligned"),                                    # misaligned field buffer
])
def test_refused_arguments_return_einval_before_any_launch(n, n_real, ptr, msg):
    lib, fn = _fn()
    w = ti.workload_1d_bump(n, 4, 10)
    g, p = _grid_params(w)
    # no device memory is behind these addresses: every check must fire before anything launches
    rc = fn(ctypes.byref(g), ctypes.byref(p), n_real, ctypes.c_void_p(ptr), 1, None)
    assert rc == _lib.TWA_EINVAL
    assert msg in lib.twa_last_error(None)


@pytest.mark.gpu
@pytest.mark.parametrize("n,n_real", [(8, 5), (256, 9), (2048, 3)])
def test_static_step_matches_handle_step_on_two_calls(n, n_real):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    lib, fn = _fn()
    w = ti.workload_1d_bump(n, n_real, 0)
    ens = make_ensemble([w], 0, want_modes=False)
    ens.sample([w.psi_cl()], w.noise_seed)
    mine = ens.psi.clone()
    g, p = _grid_params(w)
    st = torch.cuda.current_stream().cuda_stream
    for steps in (40, 60):                              # two calls in a row, each against the handle path
        ens.step(steps)
        rc = fn(ctypes.byref(g), ctypes.byref(p), w.n_real, ctypes.c_void_p(mine.data_ptr()), steps,
                ctypes.c_void_p(st))
        assert rc == 0, lib.twa_last_error(None)
        torch.cuda.synchronize()
        a = ens.psi.view(w.n_real + 1, -1).cpu().numpy().astype(np.complex128)
        b = mine.view(w.n_real + 1, -1).cpu().numpy().astype(np.complex128)
        assert np.all(np.isfinite(b))
        assert np.all(field_rel_l2(b, a, 1) < F32_FIELD_TOL)
    ens.close()


@pytest.mark.gpu
def test_static_step_at_the_size_limit_matches_the_oracle():
    """n = 2048 with 511 streams: 256 pairs x 2048 cells fill the static Poisson buffer exactly."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from oracle import twa
    lib, fn = _fn()
    n, n_real = 2048, 511
    assert (n_real + 2) // 2 * n == SCRATCH
    w = ti.workload_1d_bump(n, n_real, 0)
    cl = w.psi_cl()
    b0 = twa.sample(cl, w.noise_seed, n_real, w.phys.n_tot, w.grid.dV)
    b0 = b0.astype(np.complex64)                      # the FP32 batch both sides start from
    psi = torch.from_numpy(b0.reshape(-1)).cuda()
    g, p = _grid_params(w)
    st = torch.cuda.current_stream().cuda_stream
    ref = b0.astype(np.complex128)
    for steps in (6, 9):                              # two calls in a row
        rc = fn(ctypes.byref(g), ctypes.byref(p), n_real, ctypes.c_void_p(psi.data_ptr()), steps,
                ctypes.c_void_p(st))
        assert rc == 0, lib.twa_last_error(None)
        torch.cuda.synchronize()
        for _ in range(steps):
            ref = sp.step(ref, w.phys.hbar_m, w.phys.C, w.phys.dt, w.grid.L, 1)
        got = psi.view(n_real + 1, n).cpu().numpy().astype(np.complex128)
        err = field_rel_l2(got, ref, 1)
        assert np.all(err < F32_FIELD_TOL), err.max()
