"""GPU parity of the adaptive time step (Sec. III.B.2, the Delta t rule) against the oracle's
adaptive run: the step sequence, the output times, the moment series and the final fields, for
the 3D plane and axis pipelines, 2D and 1D; and the handle's fixed step afterwards."""
import numpy as np
import pytest
import torch

import twa_inputs as ti
from oracle import twa
from paper_2310_07119_gb300 import twa_advance_adaptive
from tests.gpu_common import field_rel_l2, make_ensemble, oracle_batch

pytestmark = pytest.mark.gpu

F32_FIELD_TOL = 1e-4
CORR_TOL = 1e-2


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _cases():
    phys3 = ti.Physics(ti.HBAR_3D, ti.C_UNIT, 1e-4, 1e8)
    return {
        "3d_kgauss16_plane": ti.small_workload("kgauss", 3, 16, 4, 0, n_tot=1e8),
        "3d_kgauss_32x16x16_axis": ti.Workload("kgauss", ti.Grid(3, (32, 16, 16), 1.0), phys3, 3, 0, 5, 5, 4321),
        "2d_merger64": ti.small_workload("merger2d", 2, 64, 4, 0, n_tot=1e9),
        "1d_bump256": ti.workload_1d_bump(256, 5, 0),
    }


CASES = _cases()


@pytest.mark.parametrize("name", list(CASES))
def test_adaptive_run_matches_oracle(name):
    w = CASES[name]
    n_out, every, c_f = 3, 5, 0.01
    cl = w.psi_cl()
    ens = make_ensemble([w], 0)
    ens.sample([cl], w.noise_seed)
    series = ens.new_series(n_out * every, every)
    times = twa_advance_adaptive(ens.h, ens.psi, n_out, every, c_f, series)
    got = ens.fields(0).cpu().numpy().astype(np.complex128)
    sc = series.cpu().numpy()
    b0 = twa.sample(cl, w.noise_seed, w.n_real, w.phys.n_tot, w.grid.dV, w.phys.noise_conv)
    t_ref, s_ref, final, dts = twa.run_adaptive(cl, w.phys.hbar_m, w.phys.C, w.grid.L, w.grid.dim, w.phys.n_tot,
                                                w.n_real, w.noise_seed, n_out, every, c_f, batch=b0)
    # FP32 potentials set the step to ~1e-7 relative of the FP64 one
    assert np.allclose(times, t_ref, rtol=1e-5, atol=0)
    assert np.all(field_rel_l2(got, final, w.grid.dim) < F32_FIELD_TOL), field_rel_l2(got, final, w.grid.dim)
    for o, mo in enumerate(s_ref):
        assert abs(sc[o, 0, 1] - mo["corr"]) <= CORR_TOL * mo["corr"] + 1e-12
    ens.close()


def test_without_gravity_the_step_is_the_kinetic_bound_and_the_fixed_step_returns():
    g = ti.Grid.cube(3, 16)
    w = ti.Workload("kgauss", g, ti.Physics(ti.HBAR_3D, 0.0, 2e-4, 1e8), 3, 10, 5, 5, 99)
    cl = w.psi_cl()
    ens = make_ensemble([w], 0)
    ens.sample([cl], w.noise_seed)
    c_f = 0.002
    times = twa_advance_adaptive(ens.h, ens.psi, 2, 5, c_f, ens.new_series(10, 5))
    kin = 2 * np.pi * c_f * (1.0 / 16) / (np.pi * ti.HBAR_3D)
    assert np.allclose(times, [0.0, 5 * kin, 10 * kin], rtol=1e-13, atol=0)
    # the handle's own dt (2e-4) is back: ten fixed steps from the same sample match the oracle
    ens.sample([cl], w.noise_seed)
    ens.step(10)
    got = ens.fields(0).cpu().numpy().astype(np.complex128)
    assert np.all(field_rel_l2(got, oracle_batch(w, cl, 10), 3) < F32_FIELD_TOL)
    ens.close()
