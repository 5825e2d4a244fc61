"""The FP32 passes' Poisson multiplier 1/k^2 (Eq. mft_normed: W_k = rho_k / k^2, W_0 = 0) against the
correctly rounded IEEE quotient: a reciprocal approximation refined by one Newton-Raphson step must
stay within 1 ulp everywhere and agree exactly almost everywhere.  Inputs: every distinct k^2 of
the transform grids (float32 sums of the per-axis tables, as the passes form them) and log-uniform
floats in [1e-30, 1e30], where both x and 1/x are normal floats; 0 and negative inputs give 0."""
import numpy as np
import pytest
import torch

from paper_2310_07119_gb300 import TwaError, twa_poisson_multiplier
from paper_2310_07119_gb300 import _lib as L

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _k2_axis(n, L=1.0):
    """k_a^2 = (2 pi m / L)^2 for m in FFT order, rounded to float32 as the tables hold it."""
    m = np.fft.fftfreq(n, d=1.0 / n)
    return ((2.0 * np.pi * m / L) ** 2).astype(np.float32)


def _grid_k2(shape):
    """Distinct float32 values of k2x + k2y (+ k2z) summed in float32, left to right."""
    vals = np.zeros(1, dtype=np.float32)
    for n in shape:
        vals = np.unique((vals[:, None] + np.unique(_k2_axis(n))[None, :]).astype(np.float32).ravel())
    return vals


def _ulp_diff(a, b):
    ia = a.view(np.int32).astype(np.int64)
    ib = b.view(np.int32).astype(np.int64)
    return np.abs(ia - ib)


def test_poisson_multiplier_is_within_one_ulp_of_ieee_division():
    rng = np.random.default_rng(7)
    parts = [_grid_k2((n,)) for n in (8, 64, 2048)]
    parts += [_grid_k2((n, n)) for n in (16, 512)]
    parts += [_grid_k2((128, 128, 128)), _grid_k2((2048, 8, 8))]
    k2 = np.concatenate(parts)
    k2 = k2[k2 > 0]
    rand = np.exp(rng.uniform(np.log(1e-30), np.log(1e30), 1_000_000)).astype(np.float32)
    x = np.concatenate([k2, rand])
    got = twa_poisson_multiplier(torch.from_numpy(x).cuda()).cpu().numpy()
    ref = (np.float32(1.0) / x).astype(np.float32)
    d = _ulp_diff(got, ref)
    assert np.all(np.isfinite(got))
    assert d.max() <= 1, (x[d.argmax()], got[d.argmax()], ref[d.argmax()])
    assert np.mean(d == 0) >= 0.999, np.mean(d == 0)
    dk = _ulp_diff(got[: k2.size], ref[: k2.size])
    assert dk.max() <= 1 and np.mean(dk == 0) >= 0.999


def test_poisson_multiplier_zeroes_the_mean_mode_and_rejects_bad_arguments():
    x = torch.tensor([0.0, -0.0, -4.0, 39.47842], device="cuda")
    got = twa_poisson_multiplier(x).cpu().numpy()
    assert got[0] == 0.0 and got[1] == 0.0 and got[2] == 0.0
    assert _ulp_diff(got[3:], (np.float32(1.0) / np.float32([39.47842])).astype(np.float32)).max() <= 1
    from paper_2310_07119_gb300.twa import _check, _lib
    with pytest.raises(TwaError) as e:
        _check(_lib().twa_poisson_multiplier(None, None, 4, None), None)
    assert e.value.code == L.TWA_EINVAL
