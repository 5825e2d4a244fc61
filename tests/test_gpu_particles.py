"""GPU test particles (Sec. III.D) against the oracle integrator on the same sampled streams: the
3D plane and axis pipelines, 2D and 1D, through twa_step_batch; and through twa_advance."""
import numpy as np
import pytest
import torch

import twa_inputs as ti
from oracle import particles as pt
from oracle import twa
from paper_2310_07119_gb300 import twa_particles_get, twa_particles_set
from tests.gpu_common import field_rel_l2, make_ensemble

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _cases():
    phys3 = ti.Physics(ti.HBAR_3D, ti.C_UNIT, 2e-3, 1e8)
    return {
        "3d_kgauss16_plane": ti.Workload("kgauss", ti.Grid.cube(3, 16), phys3, 3, 20, 10, 5, 4321),
        "3d_kgauss_32x16x16_axis": ti.Workload("kgauss", ti.Grid(3, (32, 16, 16), 1.0), phys3, 3, 20, 10, 5, 4321),
        "2d_merger64": ti.Workload("merger2d", ti.Grid.cube(2, 64), phys3, 3, 20, 10, 11, 99),
        "1d_bump256": ti.Workload("bump1d", ti.Grid.cube(1, 256), ti.Physics(0.05, ti.C_UNIT, 2e-3, 1e4), 3, 20, 10, 0, 1234),
    }


CASES = _cases()


def _start(w, seed=7):
    rng = np.random.default_rng(seed)
    return rng.random((w.n_real + 1, w.grid.dim)), 0.3 * rng.normal(size=(w.n_real + 1, w.grid.dim))


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("via", ["step", "advance"])
def test_particles_match_oracle(name, via):
    w = CASES[name]
    cl = w.psi_cl()
    r0, p0 = _start(w)
    ens = make_ensemble([w], 0)
    ens.sample([cl], w.noise_seed)
    twa_particles_set(ens.h, 0, r0, p0)
    if via == "step":
        ens.step(w.n_steps)
    else:
        ens.advance(w.n_steps, w.out_every)
    r, p = twa_particles_get(ens.h, 0, w.n_real + 1, w.grid.dim)
    b0 = twa.sample(cl, w.noise_seed, w.n_real, w.phys.n_tot, w.grid.dV, w.phys.noise_conv)
    batch, r_ref, p_ref = pt.run(cl, w.phys.hbar_m, w.phys.C, w.phys.dt, w.grid.L, w.grid.dim, w.phys.n_tot,
                                 w.n_real, w.noise_seed, w.n_steps, r0, p0, batch=b0)
    got = ens.fields(0).cpu().numpy().astype(np.complex128)
    assert np.all(field_rel_l2(got, batch, w.grid.dim) < 1e-4)
    dr = np.mod(r - r_ref + 0.5, 1.0) - 0.5
    assert np.max(np.abs(dr)) < 1e-6, np.max(np.abs(dr))
    assert np.max(np.abs(p - p_ref)) < 1e-5 * max(1.0, np.max(np.abs(p_ref - p0)) * 10), np.max(np.abs(p - p_ref))
    assert np.max(np.abs(p_ref - p0)) > 1e-4            # the particles did feel the potential
    ens.close()
