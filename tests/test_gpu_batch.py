"""The persistent batch launch (TWA_BATCH_PERSISTENT): parity, graph replay and its bounded waits.

One launch runs every KDK step of every instance of a 2D batch as a work list of (step, pass,
instance, pair, tile) items (Sec. III.A: the streams evolve independently).  Each line of a field is
transformed by the same arithmetic as in the one-launch-per-pass modes, so the fields and the moment
series must be bitwise equal to the serial run; they are also checked against the oracle.

The failure path is exercised without a GPU fault: twa_debug_stall_next_batch makes the next launch
wait for a tile that no item produces (a counter the host never releases), the bounded waits run
out after a short limit, twa_sync_status reports TWA_ETIMEOUT, and the handle and the GPU keep
working.
"""
import numpy as np
import pytest
import torch

import twa_inputs as ti
from oracle import sp, twa
from paper_2310_07119_gb300 import (BATCH_PERSISTENT, BATCH_SERIAL, TwaError, twa_debug_stall_next_batch,
                                    twa_get_batch_mode, twa_set_batch_mode, twa_set_wait_limit, twa_sync_status)
from tests.gpu_common import field_rel_l2, make_ensemble

pytestmark = pytest.mark.gpu

F32_FIELD_TOL = 1e-4
DT_2D = ti.dt_pi4_rule(ti.Grid.cube(2, 256), ti.HBAR_3D)


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _mix(n_steps=10):
    base = ti.small_workload("merger2d", 2, 256, 5, n_steps, n_tot=1e9, out_every=5, dt=DT_2D)
    ws = [base]
    for m, nr in ((512, 3), (1024, 2), (2048, 1)):
        ws.append(ti.Workload(base.name, ti.Grid.cube(2, m), base.phys, nr, n_steps, base.out_every,
                              base.psi_cl_seed, base.noise_seed))
    # a non-square instance: rows of 512 cells, columns of 256
    ws.append(ti.Workload(base.name, ti.Grid(2, (512, 256, 1), 1.0), base.phys, 2, n_steps, base.out_every,
                          base.psi_cl_seed, base.noise_seed))
    return ws


def test_persistent_steps_are_bitwise_the_serial_steps_and_match_oracle():
    ws = _mix()
    cls = [w.psi_cl() for w in ws]
    out = {}
    for mode in (BATCH_SERIAL, BATCH_PERSISTENT):
        ens = make_ensemble(ws, 0, want_modes=False)
        twa_set_batch_mode(ens.h, mode)
        assert twa_get_batch_mode(ens.h) == mode
        ens.sample(cls, ws[0].noise_seed)
        ens.step(ws[0].n_steps)
        assert twa_sync_status(ens.h) == 0
        out[mode] = [ens.fields(i).cpu().numpy().copy() for i in range(len(ws))]
        ens.close()
    for a, b in zip(out[BATCH_SERIAL], out[BATCH_PERSISTENT]):
        assert np.array_equal(a, b)
    for i, w in enumerate(ws):
        b = twa.sample(cls[i], w.noise_seed, w.n_real, w.phys.n_tot, w.grid.dV, w.phys.noise_conv, i)
        for _ in range(w.n_steps):
            b = sp.step(b, w.phys.hbar_m, w.phys.C, w.phys.dt, w.grid.L, 2)
        got = out[BATCH_PERSISTENT][i].astype(np.complex128)
        assert np.all(field_rel_l2(got, b, 2) < F32_FIELD_TOL), (i, field_rel_l2(got, b, 2))


def test_persistent_run_replays_its_graph_and_matches_the_serial_series():
    ws = _mix(20)
    cls = [w.psi_cl() for w in ws]
    out = {}
    for mode in (BATCH_SERIAL, BATCH_PERSISTENT):
        ens = make_ensemble(ws, 0)
        twa_set_batch_mode(ens.h, mode)
        s1 = ens.run(cls, ws[0].noise_seed, 20, 5).cpu().numpy()
        s2 = ens.run(cls, ws[0].noise_seed, 20, 5).cpu().numpy()       # second call replays the graph
        assert np.array_equal(s1, s2)
        out[mode] = (s1, [ens.fields(i).cpu().numpy().copy() for i in range(len(ws))])
        ens.close()
    assert np.array_equal(out[BATCH_SERIAL][0], out[BATCH_PERSISTENT][0])
    for a, b in zip(out[BATCH_SERIAL][1], out[BATCH_PERSISTENT][1]):
        assert np.array_equal(a, b)
    # the series against the oracle's run of the smallest instance
    w = ws[0]
    b0 = twa.sample(cls[0], w.noise_seed, w.n_real, w.phys.n_tot, w.grid.dV, w.phys.noise_conv, 0)
    _, ref, _ = twa.run(cls[0], w.phys.hbar_m, w.phys.C, w.phys.dt, w.grid.L, 2, w.phys.n_tot, w.n_real,
                        w.noise_seed, 20, 5, batch=b0)
    for o, mo in enumerate(ref):
        assert abs(out[BATCH_PERSISTENT][0][o, 0, 1] - mo["corr"]) <= 1e-2 * mo["corr"] + 1e-12


def test_a_stalled_dependency_times_out_and_the_handle_keeps_working():
    ws = _mix(6)[:2]
    cls = [w.psi_cl() for w in ws]
    ens = make_ensemble(ws, 0, want_modes=False)
    twa_set_batch_mode(ens.h, BATCH_PERSISTENT)
    twa_set_wait_limit(ens.h, 0.05)
    ens.sample(cls, ws[0].noise_seed)
    twa_debug_stall_next_batch(ens.h)
    ens.step(6)                                      # returns at once; the launch gives up on the device
    assert twa_sync_status(ens.h) == -4              # TWA_ETIMEOUT
    assert twa_sync_status(ens.h) == 0               # the error word was cleared
    x = torch.ones(1 << 20, device="cuda")
    assert float(x.sum()) == float(1 << 20)          # the GPU still answers
    # the next call runs normally: resample and compare with a serial handle
    ens.sample(cls, ws[0].noise_seed)
    ens.step(6)
    assert twa_sync_status(ens.h) == 0
    ref = make_ensemble(ws, 0, want_modes=False)
    twa_set_batch_mode(ref.h, BATCH_SERIAL)
    ref.sample(cls, ws[0].noise_seed)
    ref.step(6)
    for i in range(len(ws)):
        assert np.array_equal(ens.fields(i).cpu().numpy(), ref.fields(i).cpu().numpy())
    ens.close()
    ref.close()


def test_persistent_mode_is_refused_where_it_has_no_kernel():
    w3 = ti.small_workload("kgauss", 3, 16, 2, 0, n_tot=1e8)
    ens = make_ensemble([w3], 0, want_modes=False)
    with pytest.raises(TwaError):
        twa_set_batch_mode(ens.h, BATCH_PERSISTENT)
    with pytest.raises(TwaError):
        twa_debug_stall_next_batch(ens.h)
    with pytest.raises(TwaError):
        twa_set_wait_limit(ens.h, 0.0)
    ens.close()
    w2 = ti.small_workload("merger2d", 2, 128, 2, 0, n_tot=1e9)      # 128-cell lines: no persistent variant
    ens = make_ensemble([w2], 0, want_modes=False)
    with pytest.raises(TwaError):
        twa_set_batch_mode(ens.h, BATCH_PERSISTENT)
    ens.close()


def test_uneven_2d_mix_full_size_persistent():
    """The uneven 2D batch at its full layout (512^2 x 128 + 1024^2 x 64 + 2048^2 x 16 streams) in
    the persistent mode, 10 KDK steps: the classical field and two sampled streams of every instance
    against the oracle."""
    from oracle.philox import wigner_normals
    ws = [ti.workload_2d_merger(m, nr, 10) for m, nr in ((512, 128), (1024, 64), (2048, 16))]
    cls = [w.psi_cl() for w in ws]
    seed = ws[0].noise_seed
    ens = make_ensemble(ws, 0, want_modes=False)
    twa_set_batch_mode(ens.h, BATCH_PERSISTENT)
    ens.sample(cls, seed)
    ens.step(10)
    assert twa_sync_status(ens.h) == 0
    for i, w in enumerate(ws):
        slots = [0, 1, w.n_real]
        sub = ens.fields(i)[slots].cpu().numpy().astype(np.complex128)
        sig = twa.noise_sigma(w.phys.n_tot, w.grid.dV)
        ref = np.empty((len(slots),) + cls[i].shape, dtype=np.complex128)
        for j, sl in enumerate(slots):
            if sl == 0:
                ref[j] = cls[i]
            else:
                zr, zi = wigner_normals(seed, cls[i].size, sl, i)
                ref[j] = cls[i] + sig * (zr + 1j * zi).reshape(cls[i].shape)
        for _ in range(10):
            ref = sp.step(ref, w.phys.hbar_m, w.phys.C, w.phys.dt, 1.0, 2)
        assert np.all(field_rel_l2(sub, ref, 2) < F32_FIELD_TOL), (i, field_rel_l2(sub, ref, 2))
    ens.close()
