"""GPU stream averages of user functions (Appendix B's synthesizer) against the oracle's
stream_average, on the batch the GPU evolved (read back, so both sides see the same stream values):
functions of the field and of the cell index, applied to every stream or to the mean field, in
position space (FP32 and FP64 batches, 1D to 3D) and on the Fourier amplitudes; plus the refused
and non-compiling expressions and the flag combinations that need the FP32 spectral scratch."""
import numpy as np
import pytest
import torch

import twa_inputs as ti
from oracle import twa
from paper_2310_07119_gb300 import Observable, TwaError
from paper_2310_07119_gb300 import _lib as L
from tests.gpu_common import make_ensemble

pytestmark = pytest.mark.gpu

# (C expression re, C expression im, the same function for the oracle)
FUNCS = {
    "density": ("re*re + im*im", None, lambda re, im, i, n: re * re + im * im),
    "field": ("re", "im", lambda re, im, i, n: re + 1j * im),
    "square": ("re*re - im*im", "2*re*im", lambda re, im, i, n: (re + 1j * im) ** 2),
    "angle_abs": ("atan2(im, re)", "sqrt(re*re + im*im) * (double)(i % nx)",
                  None),  # nx filled per grid below
    "quartic": ("pow(re*re + im*im, 2.0) * n", None, lambda re, im, i, n: (re * re + im * im) ** 2 * n),
}


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    try:
        Observable("re").close()
    except TwaError as e:
        if "NVRTC" in str(e):
            pytest.skip("NVRTC is not available: " + str(e))
        raise


def _oracle_f(name, nx):
    if name == "angle_abs":
        return lambda re, im, i, n: np.arctan2(im, re) + 1j * np.sqrt(re * re + im * im) * (i % nx)
    return FUNCS[name][2]


def _evolved(dim, m, n_real, precision=0, steps=5):
    w = ti.small_workload("kgauss", dim, m, n_real, steps, n_tot=1e6)
    ens = make_ensemble([w], precision, want_modes=(precision == 0))
    ens.sample([w.psi_cl()], w.noise_seed)
    ens.step(steps)
    batch = ens.fields(0).cpu().numpy().astype(np.complex128)
    return w, ens, batch


def _check(got, ref, rtol):
    pc = got["per_cell"].cpu().numpy().reshape(ref["per_cell"].shape)
    scale = max(np.abs(ref["per_cell"]).max(), 1e-300)
    assert np.abs(pc - ref["per_cell"]).max() <= rtol * scale
    if got["f_cl"] is not None:
        fc = got["f_cl"].cpu().numpy().reshape(ref["f_cl"].shape)
        assert np.abs(fc - ref["f_cl"]).max() <= rtol * max(np.abs(ref["f_cl"]).max(), 1e-300)
    assert abs(got["total"] - ref["total"]) <= rtol * max(abs(ref["total"]), np.abs(ref["per_cell"]).sum())


@pytest.mark.parametrize("dim,m", [(1, 64), (2, 32), (3, 16)])
@pytest.mark.parametrize("name", list(FUNCS))
@pytest.mark.parametrize("of_mean", [False, True])
def test_position_space_average_matches_the_oracle(dim, m, name, of_mean):
    w, ens, batch = _evolved(dim, m, 6)
    fre, fim, _ = FUNCS[name]
    ob = Observable(fre, fim, of_mean=of_mean)
    got = ob(ens, classical=True)
    ref = twa.stream_average(batch, _oracle_f(name, m), w.phys.n_tot, w.grid.L, dim, of_mean=of_mean)
    _check(got, ref, 1e-12)
    ob.close()
    ens.close()


@pytest.mark.parametrize("dim,m", [(1, 128), (2, 32), (3, 16)])
@pytest.mark.parametrize("name", ["density", "square"])
def test_mode_space_average_matches_the_oracle(dim, m, name):
    """The amplitudes come from the FP32 transform passes: compared with the FP64 DFT of the same
    stream values, to the transforms' rounding."""
    w, ens, batch = _evolved(dim, m, 4)
    fre, fim, f = FUNCS[name]
    ob = Observable(fre, fim, modes=True)
    got = ob(ens, classical=True)
    ref = twa.stream_average(batch, f, w.phys.n_tot, w.grid.L, dim, modes=True)
    _check(got, ref, 2e-5)
    if name == "density":      # Parseval: sum_k <|a_k|^2> = n_tot <sum_x |psi|^2 dV>
        dens = Observable("re*re + im*im")(ens)
        assert abs(got["total"] - w.phys.n_tot * dens["total"]) <= 1e-5 * abs(got["total"])
    ob.close()
    ens.close()


@pytest.mark.parametrize("name", ["density", "field", "angle_abs"])
@pytest.mark.parametrize("of_mean", [False, True])
def test_fp32_evaluation_matches_the_oracle_to_float_rounding(name, of_mean):
    w, ens, batch = _evolved(3, 16, 6)
    fre, fim, _ = FUNCS[name]
    ob = Observable(fre, fim, of_mean=of_mean, fp32=True)
    got = ob(ens, classical=True)
    ref = twa.stream_average(batch, _oracle_f(name, 16), w.phys.n_tot, w.grid.L, 3, of_mean=of_mean)
    _check(got, ref, 2e-6)
    ob.close()
    ens.close()


def test_fp32_evaluation_reports_an_ambiguous_overload():
    with pytest.raises(TwaError) as e:
        Observable("pow(re*re + im*im, 2.0)", fp32=True)
    assert e.value.code == L.TWA_EINVAL and "pow" in str(e.value)
    Observable("pow(re*re + im*im, 2.0f)", fp32=True).close()


def test_fp64_plain_batch():
    w, ens, batch = _evolved(3, 16, 3, precision=1, steps=2)
    ob = Observable("re*re + im*im", "atan2(im, re)")
    got = ob(ens, classical=True)
    ref = twa.stream_average(batch, lambda re, im, i, n: re * re + im * im + 1j * np.arctan2(im, re),
                             w.phys.n_tot, w.grid.L, 3)
    _check(got, ref, 1e-12)
    with pytest.raises(TwaError) as e:
        Observable("re", modes=True)(ens)
    assert e.value.code == L.TWA_EINVAL and "want_modes" in str(e.value)
    ob.close()
    ens.close()


def test_refused_and_broken_expressions_report_why():
    with pytest.raises(TwaError) as e:
        Observable("re +")
    assert e.value.code == L.TWA_EINVAL and "does not compile" in str(e.value) and "error" in str(e.value)
    with pytest.raises(TwaError) as e:
        Observable("re[1]")
    assert e.value.code == L.TWA_EINVAL and "not allowed" in str(e.value)
    with pytest.raises(TwaError) as e:
        Observable("undefined_name * re")
    assert e.value.code == L.TWA_EINVAL


def test_mode_space_needs_the_spectral_scratch():
    w = ti.small_workload("kgauss", 2, 32, 2, 0, n_tot=1e6)
    ens = make_ensemble([w], 0, want_modes=False)
    ens.sample([w.psi_cl()], w.noise_seed)
    with pytest.raises(TwaError) as e:
        Observable("re", modes=True)(ens)
    assert e.value.code == L.TWA_EINVAL
    ens.close()
