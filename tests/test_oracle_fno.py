"""Pins for the FP64 reference of the FNO surrogate: central finite differences of its gradient."""
import numpy as np
import pytest

from oracle import fno

CFG = dict(W=3, c_in=2, c_out=1, modes=2, layers=2)


def _setup(seed=0, n=8, B=2):
    rng = np.random.default_rng(seed)
    theta = rng.normal(scale=0.3, size=fno.num_params(**CFG))
    x = rng.normal(size=(B, CFG["c_in"], n, n, n))
    t = rng.normal(size=(B, CFG["c_out"], n, n, n))
    return theta, x, t


def _loss(theta, x, t):
    return fno.mse(fno.forward(theta, x, **CFG), t)[0]


def test_backward_matches_central_differences():
    theta, x, t = _setup()
    y, cache = fno.forward(theta, x, **CFG, keep=True)
    _, dy = fno.mse(y, t)
    g, dx = fno.backward(theta, cache, dy, **CFG)
    rng = np.random.default_rng(1)
    idx = rng.choice(theta.size, 40, replace=False)
    eps = 1e-6
    for i in idx:
        tp, tm = theta.copy(), theta.copy()
        tp[i] += eps
        tm[i] -= eps
        fd = (_loss(tp, x, t) - _loss(tm, x, t)) / (2 * eps)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)) + 1e-9, (i, fd, g[i])
    # input gradient too
    for j in rng.choice(x.size, 10, replace=False):
        xp, xm = x.copy().ravel(), x.copy().ravel()
        xp[j] += eps
        xm[j] -= eps
        fd = (_loss(theta, xp.reshape(x.shape), t) - _loss(theta, xm.reshape(x.shape), t)) / (2 * eps)
        assert abs(fd - dx.ravel()[j]) <= 1e-6 * max(1.0, abs(fd)) + 1e-9


def test_truncated_dft_pair_is_adjoint_and_exact_on_kept_modes():
    rng = np.random.default_rng(3)
    n, m = 8, 2
    a = rng.normal(size=(n, n, n))
    s = rng.normal(size=(2 * m,) * 3) + 1j * rng.normal(size=(2 * m,) * 3)
    lhs = np.vdot(fno._dft_trunc(a.astype(complex), n, m), s)
    rhs = np.vdot(a.astype(complex), fno._idft_trunc(s, n, m))
    assert abs(lhs - rhs) < 1e-12
    # a field made only of kept modes is reproduced exactly
    assert np.allclose(fno._dft_trunc(fno._idft_trunc(s, n, m), n, m), s, atol=1e-12)


def test_shell_average_of_radial_function():
    n = 16
    m = np.fft.fftfreq(n, d=1.0 / n)
    r = np.sqrt(m[:, None, None] ** 2 + m[None, :, None] ** 2 + m[None, None, :] ** 2)
    f = np.rint(r) ** 2
    sa = fno.shell_average(f, n)
    assert np.allclose(sa[:8], np.arange(8) ** 2)
