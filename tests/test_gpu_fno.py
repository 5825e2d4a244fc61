"""GPU checks of the surrogate's hand-written kernels against the FP64 oracle network.

The GPU network keeps BF16 weights (biases and the master copy in FP32) and accumulates in FP32;
the oracle runs in FP64 on the same BF16-rounded weights, so forward outputs agree to FP32
accumulation error (~1e-5 relative) and gradients to ~1e-4.
"""
import numpy as np
import pytest
import torch

from oracle import fno as ofno

pytestmark = pytest.mark.gpu

CFG = dict(W=4, c_in=4, c_out=1, modes=2, layers=2)


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _bf16(a: np.ndarray) -> np.ndarray:
    """Round float32 values to bfloat16 (nearest even) and back."""
    u = np.asarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def _weights_as_gpu_sees(theta: np.ndarray) -> np.ndarray:
    out = theta.astype(np.float32).astype(np.float64)
    o = 0
    for name, sh in ofno.param_shapes(**CFG):
        n = int(np.prod(sh))
        if name[0] in "PRWQ":
            out[o:o + n] = _bf16(theta[o:o + n])
        o += n
    return out


def _model_and_data(n=8, B=2, seed=0):
    from paper_2310_07119_gb300.fno import FNO
    rng = np.random.default_rng(seed)
    theta = rng.normal(scale=0.4, size=ofno.num_params(**CFG))
    x = rng.normal(size=(B, CFG["c_in"], n, n, n))
    t = rng.normal(size=(B, CFG["c_out"], n, n, n))
    m = FNO(n, CFG["W"], CFG["modes"], CFG["layers"], CFG["c_in"], CFG["c_out"])
    m.set_params(torch.tensor(theta, dtype=torch.float32))
    return m, theta, x, t


def test_forward_matches_oracle():
    m, theta, x, _ = _model_and_data()
    th = _weights_as_gpu_sees(theta)
    xf = x.astype(np.float32).astype(np.float64)
    y = m.forward(torch.tensor(xf, dtype=torch.float32, device="cuda")).double().cpu().numpy()
    yo = ofno.forward(th, xf, **CFG)
    assert np.max(np.abs(y - yo)) < 1e-4 * np.max(np.abs(yo))


def test_backward_matches_oracle():
    m, theta, x, t = _model_and_data(seed=1)
    th = _weights_as_gpu_sees(theta)
    xf = x.astype(np.float32).astype(np.float64)
    tf = t.astype(np.float32).astype(np.float64)
    xg = torch.tensor(xf, dtype=torch.float32, device="cuda")
    m.zero_grad()
    y = m.forward(xg)
    loss, dy = m.mse(y, torch.tensor(tf, dtype=torch.float32, device="cuda"))
    dx = m.backward(dy, want_dx=True)
    g = m.get_params(which=1).double().cpu().numpy()
    yo, cache = ofno.forward(th, xf, **CFG, keep=True)
    lo, dyo = ofno.mse(yo, tf)
    go, dxo = ofno.backward(th, cache, dyo, **CFG)
    assert abs(loss.item() - lo) < 1e-4 * lo
    assert np.linalg.norm(g - go) < 2e-4 * np.linalg.norm(go)
    o = 0
    for name, sh in ofno.param_shapes(**CFG):      # every parameter block, not just the total
        n_ = int(np.prod(sh))
        assert np.linalg.norm(g[o:o + n_] - go[o:o + n_]) <= 2e-3 * np.linalg.norm(go[o:o + n_]) + 1e-9, name
        o += n_
    assert np.linalg.norm(dx.double().cpu().numpy() - dxo) < 2e-4 * np.linalg.norm(dxo)


def test_adamw_step_matches_definition():
    m, theta, x, t = _model_and_data(seed=2)
    xg = torch.tensor(x, dtype=torch.float32, device="cuda")
    tg = torch.tensor(t, dtype=torch.float32, device="cuda")
    m.zero_grad()
    y = m.forward(xg)
    _, dy = m.mse(y, tg)
    m.backward(dy)
    g = m.get_params(which=1).double().cpu().numpy()
    p0 = m.get_params().double().cpu().numpy()
    lr, b1, b2, eps, wd = 1e-2, 0.9, 0.999, 1e-8, 1e-3
    m.adamw(lr, b1, b2, eps, wd)
    p1 = m.get_params().double().cpu().numpy()
    mh = (1 - b1) * g / (1 - b1)
    vh = (1 - b2) * g * g / (1 - b2)
    expect = p0 - lr * (mh / (np.sqrt(vh) + eps) + wd * p0)
    assert np.max(np.abs(p1 - expect)) < 1e-5


def test_training_is_deterministic():
    out = []
    for _ in range(2):
        m, theta, x, t = _model_and_data(seed=3)
        xg = torch.tensor(x, dtype=torch.float32, device="cuda")
        tg = torch.tensor(t, dtype=torch.float32, device="cuda")
        for _ in range(5):
            m.train_step(xg, tg, 1e-3)
        out.append(m.get_params().cpu().numpy())
        m.close()
    assert np.array_equal(out[0], out[1])


def test_trained_surrogate_gains_over_the_few_stream_estimate():
    """Train on TWA runs of the library (16^3, 8 input streams, 64-stream targets) and compare, on
    held-out runs, the surrogate's prediction and the raw 8-stream estimate against an independent
    256-stream reference (in the normalized units of the target)."""
    import twa_inputs as ti
    from paper_2310_07119_gb300 import fno as F
    grid = 16
    dt = ti.dt_pi4_rule(ti.Grid.cube(3, grid), ti.HBAR_3D)
    snaps = [60, 90, 120]
    train = F.generate(F.run_table(48, 1, k0_range=(1.5, 3.0)), grid, 8, 64, snaps, ti.HBAR_3D, ti.C_UNIT, dt)
    test = F.generate(F.run_table(6, 77, k0_range=(1.5, 3.0)), grid, 8, 256, snaps, ti.HBAR_3D, ti.C_UNIT, dt)
    model = F.FNO(grid, width=16, modes=4, layers=4, seed=5)
    hist = F.train(model, train, iters=400, batch=8, lr=1e-3, log_every=50)
    assert all(np.isfinite(l) for _, l in hist)
    mse_fno, mse_est = 0.0, 0.0
    for s in test:
        y = model.forward(s.x[None].contiguous())[0]
        mse_fno += float(((y - s.t) ** 2).mean())
        mse_est += float(((s.x[1:2] - s.t) ** 2).mean())
    assert mse_fno < 0.85 * mse_est, (mse_fno, mse_est)      # measured: 0.046 vs 0.059 (deterministic)
