"""Host-side checks of the C ABI (no GPU needed): the library builds, loads and
exports every function include/twa.h declares, and refuses to run without a device."""
import ctypes
import os

import pytest
import torch

from paper_2310_07119_gb300 import _lib


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(_lib.LIB_PATH):
        from paper_2310_07119_gb300.build import build
        build()
    return _lib.load()


def test_every_declared_symbol_is_exported(lib):
    names = _lib.declared_symbols()
    assert {"twa_create", "twa_sample", "twa_step_batch", "twa_moments", "twa_run"} <= set(names)
    for n in names:
        assert hasattr(lib, n), n


def test_header_and_binding_agree_on_constants():
    txt = open(_lib.HEADER).read()
    assert "#define TWA_NSCALARS     8" in txt
    assert len(_lib.SCALAR_NAMES) == _lib.TWA_NSCALARS
    assert ctypes.sizeof(_lib.Params) == 4 * 8 + 3 * 4 + 4  # padded to 8


@pytest.mark.skipif(torch.cuda.is_available(), reason="checks the no-device error path")
def test_create_without_a_device_fails_loudly(lib):
    g = _lib.Grid(1, (ctypes.c_int * 3)(64, 1, 1), 1.0)
    p = _lib.Params(1.0, 1.0, 1e-3, 1e4, 0, 0, 0)
    n = (ctypes.c_int * 1)(4)
    h = ctypes.c_void_p()
    rc = lib.twa_create(ctypes.byref(h), ctypes.byref(g), ctypes.byref(p), 1, n)
    assert rc == _lib.TWA_ECUDA
    assert b"no CUDA device" in lib.twa_last_error(None)


@pytest.mark.skipif(torch.cuda.is_available(), reason="checks the no-device error path")
def test_python_binding_has_no_cpu_path():
    from paper_2310_07119_gb300 import TwaError, twa_create
    with pytest.raises(TwaError):
        twa_create([(1, (64,), 1.0)], 1.0, 1.0, 1e-3, 1e4, [4])


@pytest.mark.parametrize("expr", ["", "re[0]", "re; im", "{re}", "#define x", "\"a\"", "*(double*)0", "p->x",
                                  "__ldg(0)", "asm(\"\")", "re // c"])
def test_observable_refuses_expressions_outside_arithmetic(lib, expr):
    ob = ctypes.c_void_p()
    rc = lib.twa_observable_create(ctypes.byref(ob), expr.encode(), None, 0)
    assert rc == _lib.TWA_EINVAL and not ob.value
    assert b"twa_observable_create" in lib.twa_last_error(None)


def test_observable_rejects_unknown_flags(lib):
    ob = ctypes.c_void_p()
    assert lib.twa_observable_create(ctypes.byref(ob), b"re", None, 8) == _lib.TWA_EINVAL
    assert lib.twa_observable_destroy(None) == _lib.TWA_OK


@pytest.mark.skipif(torch.cuda.is_available(), reason="checks the no-device error path")
def test_observable_without_a_device_fails_loudly(lib):
    ob = ctypes.c_void_p()
    rc = lib.twa_observable_create(ctypes.byref(ob), b"re*re + im*im", None, 0)
    assert rc == _lib.TWA_ECUDA and not ob.value
