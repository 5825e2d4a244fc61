"""Paper-scale cases on the GPU path: the Q relation of Eq. Q_relation (n_s Q_s independent of the
simulated particle number while Q << 1) on the 1D cosine overdensity at hbar/m = 2.5e-4 with 1024
streams, checked against the oracle; and 3D grids whose x lines are 512 to 2048 long."""
import numpy as np
import pytest
import torch

import twa_inputs as ti
from oracle import twa
from tests.gpu_common import field_rel_l2, make_ensemble, oracle_batch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def test_q_relation_on_the_1d_cosine_collapse():
    g = ti.Grid.cube(1, 512)
    hb = 2.5e-4
    dt = ti.dt_pi4_rule(g, hb)
    n_steps, every, ns = 200, 50, 1024
    out = {}
    for n_tot in (1e8, 1e10):
        w = ti.Workload("cosine", g, ti.Physics(hb, ti.C_UNIT, dt, n_tot), ns, n_steps, every, 0, 2023)
        cl = w.psi_cl()
        ens = make_ensemble([w], 0, want_modes=False)
        series = ens.run([cl], w.noise_seed, n_steps, every).cpu().numpy()
        q = series[:, 0, 0]
        out[n_tot] = n_tot * (q - q[0])
        if n_tot == 1e8:
            _, ref, _ = twa.run(cl, hb, ti.C_UNIT, dt, 1.0, 1, n_tot, ns, w.noise_seed, n_steps, every,
                                with_modes=False)
            qr = np.array([s["Q"] for s in ref])
            ref_scaled = n_tot * (qr - qr[0])
            assert np.all(np.abs(out[n_tot][1:] - ref_scaled[1:]) <= 0.02 * np.abs(ref_scaled[1:]) + 1e-6)
        ens.close()
    assert out[1e8][-1] > 0
    assert np.all(np.abs(out[1e10][1:] - out[1e8][1:]) <= 0.05 * np.abs(out[1e10][1:]))


@pytest.mark.parametrize("n", [512, 1024, 2048])
def test_long_x_lines_in_3d(n):
    w = ti.Workload("kgauss", ti.Grid(3, (n, 8, 8), 1.0), ti.Physics(ti.HBAR_3D, ti.C_UNIT, 1e-5, 1e8), 2, 10, 5, 5, 31)
    cl = w.psi_cl()
    ens = make_ensemble([w], 0)
    ens.sample([cl], w.noise_seed)
    ens.step(w.n_steps)
    got = ens.fields(0).cpu().numpy().astype(np.complex128)
    assert np.all(field_rel_l2(got, oracle_batch(w, cl, w.n_steps), 3) < 1e-4)
    ens.close()


def test_soliton_256_cubed_sampled_streams():
    """The stable-object workload at its full layout (256^3 cells x 65 slots, 8.7 GB of FP32 fields), 10 KDK steps:
    the classical field and two sampled streams against the oracle."""
    from oracle import sp
    from oracle.philox import wigner_normals
    w = ti.workload_3d_soliton(256, 64, 10)
    cl = w.psi_cl()
    ens = make_ensemble([w], 0, want_modes=False)
    ens.sample([cl], w.noise_seed)
    ens.step(w.n_steps)
    slots = [0, 1, 64]
    sub = ens.fields(0)[slots].cpu().numpy().astype(np.complex128)
    ens.close()
    torch.cuda.empty_cache()
    sig = twa.noise_sigma(w.phys.n_tot, w.grid.dV, w.phys.noise_conv)
    ref = np.empty((len(slots),) + cl.shape, dtype=np.complex128)
    for j, s_ in enumerate(slots):
        if s_ == 0:
            ref[j] = cl
        else:
            zr, zi = wigner_normals(w.noise_seed, cl.size, s_)
            ref[j] = cl + sig * (zr + 1j * zi).reshape(cl.shape)
    for _ in range(w.n_steps):
        ref = sp.step(ref, w.phys.hbar_m, w.phys.C, w.phys.dt, w.grid.L, 3)
    assert np.all(field_rel_l2(sub, ref, 3) < 1e-4), field_rel_l2(sub, ref, 3)


def test_512_cubed_soliton_sampled_streams():
    """The paper's 3D resolution (512^3, Sec. V) on the stable-object workload: the classical field
    and two sampled streams, 5 KDK steps at the pi/4 step of the 512^3 grid, against the oracle (field
    and per-stream density tolerances of the parity tests)."""
    w = ti.workload_3d_soliton(512, 2, 5)
    cl = w.psi_cl()
    ens = make_ensemble([w], 0, want_modes=False)
    ens.sample([cl], w.noise_seed)
    ens.step(w.n_steps)
    got = ens.fields(0).cpu().numpy().astype(np.complex128)
    ens.close()
    del ens
    torch.cuda.empty_cache()
    ref = oracle_batch(w, cl, w.n_steps)
    assert np.all(field_rel_l2(got, ref, 3) < 1e-4), field_rel_l2(got, ref, 3)
    r_got, r_ref = np.abs(got) ** 2, np.abs(ref) ** 2
    rho_err = np.sqrt(np.sum((r_got - r_ref) ** 2, axis=(1, 2, 3)) / np.sum(r_ref ** 2, axis=(1, 2, 3)))
    assert np.all(rho_err < 1e-5), rho_err
