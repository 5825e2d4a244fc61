"""GPU parity of the FP32 path's per-mode moments (Sec. III.B.3, Eq. E[op]) against the oracle.

The moments kernel is checked on the batch the GPU itself evolved (copied to the host as
complex128), so the only difference between the two sides is the moment arithmetic: the FP32
transforms to the number-unit amplitudes a_k = sqrt(n dV / M) DFT(psi)_k, and the double-float
stream sums against the oracle's FP64 FFT and sums.

Tolerances, from the arithmetic:
  * n_k of the classical field (nk_cl) and <n_k> (nk_mean): an FP32 transform of a field of
    total occupation n_tot carries an absolute error of about eps_32 sqrt(log2 M) sqrt(n_tot / M)
    per amplitude, which moves |a_k|^2 by about 2 |a_k| times that.  Modes holding at least 1e-5
    of n_tot are held to 1e-4 relative, every mode to 1e-6 n_tot absolute.
  * Var n_k (nk_var) = mean|a|^4 - mean|a|^2 - (mean|a|^2 - 1/2)^2 cancels terms of size <n_k>^2
    down to about <n_k>.  The FP32 amplitude error enters through 2 cov(|a|^2, delta|a|^2); the
    estimator's own sampling error (its influence function x^2 - x - 2(<n_k>) x over the streams,
    x = |a_k|^2) is larger by a factor of order 1 / (sqrt(N_s) eps_32 sqrt(n_tot / M)) or more.
    Each mode's FP32 Var n_k is held to 5 % of that sampling standard error: the arithmetic must
    not add anything a user could see next to the statistical uncertainty of the estimate.
The high-occupation case (the soliton at n_tot = 1e10, 256 streams) is where the cancellation in
Var n_k is hardest: its largest mode holds ~4e8 quanta, so mean|a|^4 ~ 2e17 against a result ~ 4e8.
"""
import math

import numpy as np
import pytest
import torch

import twa_inputs as ti
from oracle import sp, twa
from tests.gpu_common import make_ensemble

pytestmark = pytest.mark.gpu

DT_128 = ti.dt_pi4_rule(ti.Grid.cube(3, 128), ti.HBAR_3D)
DT_2D = ti.dt_pi4_rule(ti.Grid.cube(2, 256), ti.HBAR_3D)
DT_256 = ti.dt_pi4_rule(ti.Grid.cube(3, 256), ti.HBAR_3D)
VAR_FRAC_OF_SE = 0.05


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _cases():
    return {
        "1d_bump256": (ti.workload_1d_bump(256, 31, 0), 30),
        "2d_merger64": (ti.small_workload("merger2d", 2, 64, 15, 0, n_tot=1e9, dt=DT_2D), 30),
        "3d_kgauss16": (ti.small_workload("kgauss", 3, 16, 15, 0, n_tot=1e8, dt=DT_128), 30),
        "3d_kgauss_32x16x16": (ti.Workload("kgauss", ti.Grid(3, (32, 16, 16), 1.0),
                                           ti.Physics(ti.HBAR_3D, 4 * np.pi, DT_128, 1e8), 16, 0, 10, 5, 4321), 30),
        "3d_soliton32_high_occupation": (ti.small_workload("soliton", 3, 32, 256, 0, n_tot=1e10, dt=DT_256), 30),
    }


CASES = _cases()


def _influence_se(b, w):
    """Per-mode standard error of the Var n_k estimator from its influence function (test-side)."""
    M = w.grid.cells
    a = sp.fftn(b[1:], w.grid.dim) * math.sqrt(w.phys.n_tot * w.grid.dV / M)
    x = np.abs(a) ** 2
    m = x.mean(0)
    infl = x ** 2 - x - 2 * (m - 0.5) * x
    return infl.std(0) / math.sqrt(x.shape[0])


@pytest.mark.parametrize("name", list(CASES))
def test_f32_mode_moments_match_oracle_on_the_same_batch(name):
    w, n = CASES[name]
    ens = make_ensemble([w], 0)
    ens.sample([w.psi_cl()], w.noise_seed)
    ens.step(n)
    m = ens.moments(0)
    b = ens.fields(0).cpu().numpy().astype(np.complex128)
    mo = twa.moments(b, w.phys.n_tot, w.grid.L, w.grid.dim)
    sh = w.grid.shape
    n_tot = w.phys.n_tot
    # classical-field occupations (same normalization, FFT order)
    a_cl = sp.fftn(b[0], w.grid.dim) * math.sqrt(n_tot * w.grid.dV / w.grid.cells)
    ref_cl = np.abs(a_cl) ** 2
    got_cl = m["nk_cl"].cpu().numpy().reshape(sh)
    big = ref_cl > 1e-5 * n_tot
    assert big.any()
    assert np.max(np.abs(got_cl[big] - ref_cl[big]) / ref_cl[big]) < 1e-4
    assert np.max(np.abs(got_cl - ref_cl)) < 1e-6 * n_tot
    # <n_k>
    nk = m["nk_mean"].cpu().numpy().reshape(sh)
    big = mo["nk_mean"] > 1e-5 * n_tot
    assert np.max(np.abs(nk[big] - mo["nk_mean"][big]) / mo["nk_mean"][big]) < 1e-4
    assert np.max(np.abs(nk - mo["nk_mean"])) < 1e-6 * n_tot
    # Var n_k against the estimator's own sampling error
    var = m["nk_var"].cpu().numpy().reshape(sh)
    se = _influence_se(b, w)
    ratio = np.abs(var - mo["nk_var"]) / se
    assert np.max(ratio) < VAR_FRAC_OF_SE, (np.max(ratio), np.unravel_index(np.argmax(ratio), sh))
    ens.close()


def test_high_occupation_var_nk_resolves_the_coherent_value_at_t0():
    """At t = 0 the batch is a sampled coherent state: Var n_k = |z_k|^2 within its sampling error.
    The FP32 path must resolve Var n_k ~ 4e8 under mean|a|^4 ~ 2e17 (n_tot = 1e10, 256 streams)."""
    w = CASES["3d_soliton32_high_occupation"][0]
    ens = make_ensemble([w], 0)
    cl = w.psi_cl()
    ens.sample([cl], w.noise_seed)
    m = ens.moments(0)
    b = ens.fields(0).cpu().numpy().astype(np.complex128)
    z2 = np.abs(sp.fftn(cl, 3) * math.sqrt(w.phys.n_tot * w.grid.dV / w.grid.cells)) ** 2
    var = m["nk_var"].cpu().numpy().reshape(w.grid.shape)
    se = _influence_se(b, w)
    big = z2 > 1e-4 * w.phys.n_tot
    assert big.any() and z2.max() > 1e8
    assert np.all(np.abs(var[big] - z2[big]) < 5 * se[big])
    ens.close()


def test_all_moments_at_bench_size_match_oracle_on_the_same_batch():
    """The moments kernels at the bench layout (128^3 x 256 streams + classical field, n_tot = 1e9)
    after 20 KDK steps, every output against oracle.twa.moments of the same batch.

    Beyond the per-mode tolerances above: <rho> is a mean of FP32 |psi|^2 values, each rounded once
    (2^-24 relative, unbiased), summed in double-float, so it is held to 1e-7 of max <rho>; psi_mean
    sums FP32 values exactly (1e-12); rho_cl is formed in FP64 from FP32 values (1e-15); the
    correction norm and Q are sums of those over 2^21 cells, held to 1e-6 and 1e-4 relative."""
    w = ti.workload_3d_condensation(128, 256, 20)
    ens = make_ensemble([w], 0)
    ens.sample([w.psi_cl()], w.noise_seed)
    ens.step(w.n_steps)
    m = {k: v.cpu().numpy() for k, v in ens.moments(0).items()}
    b = ens.fields(0).cpu().numpy().astype(np.complex128)
    ens.close()
    del ens
    torch.cuda.empty_cache()
    mo = twa.moments(b, w.phys.n_tot, w.grid.L, 3)
    sh = w.grid.shape
    rm = m["rho_mean"].reshape(sh)
    assert np.max(np.abs(rm - mo["rho_mean"])) < 1e-7 * np.max(mo["rho_mean"])
    pm = m["psi_mean"].reshape(sh + (2,))
    pm = pm[..., 0] + 1j * pm[..., 1]
    assert np.max(np.abs(pm - mo["psi_mean"])) < 1e-12 * np.max(np.abs(mo["psi_mean"]))
    assert np.max(np.abs(m["rho_cl"].reshape(sh) - mo["rho_cl"])) <= 1e-15 * np.max(mo["rho_cl"])
    sc = m["scalars"]
    assert abs(sc[1] - mo["corr"]) < 1e-6 * mo["corr"]
    assert abs(sc[0] - mo["Q"]) < 1e-4 * abs(mo["Q"]) + 1e-10
    n_tot = w.phys.n_tot
    nk = m["nk_mean"].reshape(sh)
    big = mo["nk_mean"] > 1e-5 * n_tot
    assert big.any()
    assert np.max(np.abs(nk[big] - mo["nk_mean"][big]) / mo["nk_mean"][big]) < 1e-4
    assert np.max(np.abs(nk - mo["nk_mean"])) < 1e-6 * n_tot
    a_cl = sp.fftn(b[0], 3) * math.sqrt(n_tot * w.grid.dV / w.grid.cells)
    ref_cl = np.abs(a_cl) ** 2
    got_cl = m["nk_cl"].reshape(sh)
    big = ref_cl > 1e-5 * n_tot
    assert np.max(np.abs(got_cl[big] - ref_cl[big]) / ref_cl[big]) < 1e-4
    assert np.max(np.abs(got_cl - ref_cl)) < 1e-6 * n_tot
    se = _influence_se(b, w)
    ratio = np.abs(m["nk_var"].reshape(sh) - mo["nk_var"]) / se
    assert np.max(ratio) < VAR_FRAC_OF_SE, np.max(ratio)
