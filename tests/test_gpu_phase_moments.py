"""GPU amplitude and phase variances (Eq. varA, Eq. varPhi) against the oracle: on the very batch
the GPU holds (exact up to FP32 storage and accumulation order), and after evolution against the
oracle's own evolved batch; both paths."""
import numpy as np
import pytest
import torch

import twa_inputs as ti
from oracle import twa
from paper_2310_07119_gb300 import twa_phase_moments
from tests.gpu_common import make_ensemble, oracle_batch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.mark.parametrize("name,precision", [("kgauss3d", 0), ("kgauss3d", 1), ("merger2d", 0), ("bump1d", 0)])
def test_phase_moments_match_oracle(name, precision):
    if name == "kgauss3d":
        w = ti.small_workload("kgauss", 3, 16, 6, 30, n_tot=1e4)
    elif name == "merger2d":
        w = ti.small_workload("merger2d", 2, 64, 6, 30, n_tot=1e4)
    else:
        w = ti.workload_1d_bump(256, 6, 30)
    cl = w.psi_cl()
    ens = make_ensemble([w], precision)
    ens.sample([cl], w.noise_seed)
    ens.step(w.n_steps)
    c = ens.cells[0]
    f64 = dict(dtype=torch.float64, device="cuda")
    va, p2 = torch.empty(c, **f64), torch.empty(c, **f64)
    tot = twa_phase_moments(ens.h, 0, ens.psi, va, p2).cpu().numpy()
    held = ens.fields(0).cpu().numpy().astype(np.complex128)
    mine = twa.phase_moments(held, w.phys.n_tot, w.grid.L, w.grid.dim)
    tol = 1e-5 if precision == 0 else 1e-11
    assert abs(tot[0] - mine["var_a"]) <= tol * abs(mine["var_a"])
    assert abs(tot[1] - mine["var_phi"]) <= tol * abs(mine["var_phi"])
    sh = w.grid.shape
    assert np.allclose(va.cpu().numpy().reshape(sh), mine["var_a_cell"], rtol=1e-3 if precision == 0 else 1e-9,
                       atol=1e-6 * mine["var_a_cell"].max())
    assert np.allclose(p2.cpu().numpy().reshape(sh), mine["phi2_cell"], rtol=1e-3 if precision == 0 else 1e-9,
                       atol=1e-6 * mine["phi2_cell"].max())
    # against the oracle's own evolution of the same sample
    ref = twa.phase_moments(oracle_batch(w, cl, w.n_steps), w.phys.n_tot, w.grid.L, w.grid.dim)
    assert abs(tot[0] - ref["var_a"]) <= 1e-3 * abs(ref["var_a"])
    assert abs(tot[1] - ref["var_phi"]) <= 1e-3 * abs(ref["var_phi"])
    ens.close()
