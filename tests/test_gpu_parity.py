"""GPU parity of the CUDA path (through the C ABI) against the FP64 oracle.

Tolerances (FP32 batched path): the field relative L2 error per realization
must stay <= 1e-4 after 100 steps; <rho> <= 1e-5 relative; the correction norm
<= 1% relative.  FP32 storage rounds every value to 6e-8 relative and each
transform adds O(log2 N) such roundings, so the per-step field error is a few
1e-7 and 100 steps stay well inside 1e-4 for these non-chaotic intervals.  The
FP64 plain path is held to 1e-10 (rounding of the same arithmetic in FP64).
"""
import math

import numpy as np
import pytest
import torch

import twa_inputs as ti
from oracle import sp, twa
from tests.gpu_common import field_rel_l2, make_ensemble, oracle_batch

pytestmark = pytest.mark.gpu

F32_FIELD_TOL = 1e-4
RHO_TOL = 1e-5
CORR_TOL = 1e-2


# Time steps of the full-size workloads (pi/4 rule of the 128^3 and 256^3 grids, 256^2 for 2D),
# so that per-step phases and the 100-step physical time match the measured configurations.
DT_128 = ti.dt_pi4_rule(ti.Grid.cube(3, 128), ti.HBAR_3D)
DT_256 = ti.dt_pi4_rule(ti.Grid.cube(3, 256), ti.HBAR_3D)
DT_2D = ti.dt_pi4_rule(ti.Grid.cube(2, 256), ti.HBAR_3D)


def _cases():
    return {
        "1d_bump256": ti.workload_1d_bump(256, 7, 100),
        "1d_cosine64": ti.Workload("cosine", ti.Grid.cube(1, 64), ti.Physics(0.01, 4 * np.pi, 1e-3, 1e6), 4, 100, 10, 0, 3),
        "2d_merger64": ti.small_workload("merger2d", 2, 64, 5, 100, n_tot=1e9, dt=DT_2D),
        "3d_kgauss16": ti.small_workload("kgauss", 3, 16, 5, 100, n_tot=1e8, dt=DT_128),
        "3d_kgauss32_pi4": ti.small_workload("kgauss", 3, 32, 3, 100, n_tot=1e8),
        "3d_soliton32": ti.small_workload("soliton", 3, 32, 3, 100, n_tot=1e10, dt=DT_256),
        # nx != ny: runs the per-axis 3D pipeline (square xy planes use the fused plane passes)
        "3d_kgauss_32x16x16": ti.Workload("kgauss", ti.Grid(3, (32, 16, 16), 1.0),
                                          ti.Physics(ti.HBAR_3D, 4 * np.pi, DT_128, 1e8), 4, 100, 10, 5, 4321),
    }


CASES = _cases()


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.mark.parametrize("precision", [0, 1])
def test_sample_matches_oracle(precision):
    w = ti.small_workload("kgauss", 3, 16, 4, 0, n_tot=1e6)
    cl = w.psi_cl()
    ens = make_ensemble([w], precision)
    ens.sample([cl], w.noise_seed)
    got = ens.fields(0).cpu().numpy()
    ref = twa.sample(cl, w.noise_seed, w.n_real, w.phys.n_tot, w.grid.dV)
    if precision == 0:
        # FP64 arithmetic rounded once to FP32
        assert np.max(np.abs(got - ref.astype(np.complex64))) <= 2 * np.finfo(np.float32).eps * np.abs(ref).max()
    else:
        assert np.max(np.abs(got - ref)) < 1e-14 * np.abs(ref).max()
    assert np.array_equal(got[0], ref[0].astype(got.dtype))


@pytest.mark.parametrize("name", list(CASES))
def test_f32_steps_match_oracle(name):
    w = CASES[name]
    cl = w.psi_cl()
    ens = make_ensemble([w], 0)
    ens.sample([cl], w.noise_seed)
    ens.step(w.n_steps)
    got = ens.fields(0).cpu().numpy().astype(np.complex128)
    ref = oracle_batch(w, cl, w.n_steps)
    err = field_rel_l2(got, ref, w.grid.dim)
    assert np.all(err < F32_FIELD_TOL), err
    # moments of the synchronized ensemble
    m = ens.moments(0)
    mo = twa.moments(ref, w.phys.n_tot, w.grid.L, w.grid.dim)
    rm = m["rho_mean"].cpu().numpy().reshape(w.grid.shape)
    assert np.linalg.norm(rm - mo["rho_mean"]) / np.linalg.norm(mo["rho_mean"]) < RHO_TOL
    sc = m["scalars"].cpu().numpy()
    assert abs(sc[1] - mo["corr"]) <= CORR_TOL * mo["corr"]
    mass = sp.mass(ref, w.grid.dV, w.grid.dim)
    assert abs(sc[2] - mass[1:].mean()) < 1e-5 * mass[1:].mean()     # noisy streams carry M/(2n) extra
    assert abs(sc[3] - mass[0]) < 1e-5


@pytest.mark.parametrize("name", ["1d_bump256", "2d_merger64", "3d_kgauss16"])
def test_f64_plain_path_matches_oracle(name):
    w = CASES[name]
    n = 20
    cl = w.psi_cl()
    ens = make_ensemble([w], 1)
    ens.sample([cl], w.noise_seed)
    ens.step(n)
    got = ens.fields(0).cpu().numpy()
    ref = oracle_batch(w, cl, n)
    assert np.all(field_rel_l2(got, ref, w.grid.dim) < 1e-10)
    m = ens.moments(0)
    mo = twa.moments(ref, w.phys.n_tot, w.grid.L, w.grid.dim)
    for k in ("rho_mean", "rho_cl", "nk_mean"):
        g = m[k].cpu().numpy().reshape(w.grid.shape)
        assert np.max(np.abs(g - mo[k])) <= 1e-8 * np.max(np.abs(mo[k])) + 1e-10, k
    # Var n_k = mean|a|^4 - mean|a|^2 - <n_k>^2 cancels terms of size <n_k>^2: FP64 rounding of those
    g = m["nk_var"].cpu().numpy().reshape(w.grid.shape)
    assert np.max(np.abs(g - mo["nk_var"])) <= 1e-13 * np.max(mo["nk_mean"]) ** 2 + 1e-8 * np.max(np.abs(mo["nk_var"]))
    assert abs(m["scalars"][0].item() - mo["Q"]) < 1e-9 * max(1.0, abs(mo["Q"]))


@pytest.mark.parametrize("name", ["2d_merger64", "3d_kgauss16", "1d_bump256", "3d_kgauss_32x16x16"])
def test_f32_moments_match_oracle(name):
    w = CASES[name]
    n = 30
    cl = w.psi_cl()
    ens = make_ensemble([w], 0)
    ens.sample([cl], w.noise_seed)
    ens.step(n)
    m = ens.moments(0)
    ref = oracle_batch(w, cl, n)
    mo = twa.moments(ref, w.phys.n_tot, w.grid.L, w.grid.dim)
    sh = w.grid.shape
    pm = m["psi_mean"].cpu().numpy().reshape(sh + (2,))
    pm = pm[..., 0] + 1j * pm[..., 1]
    assert np.linalg.norm(pm - mo["psi_mean"]) / np.linalg.norm(mo["psi_mean"]) < 1e-5
    assert np.linalg.norm(m["rho_cl"].cpu().numpy().reshape(sh) - mo["rho_cl"]) / np.linalg.norm(mo["rho_cl"]) < 1e-5
    # an FP32 transform resolves |a_k|^2 to ~1e-6 of the total occupation n_tot: check the modes
    # holding at least 1e-5 of it to 1e-3 relative, and all modes to 1e-6 n_tot absolute
    nk = m["nk_mean"].cpu().numpy().reshape(sh)
    tot = np.sum(mo["nk_mean"])
    big = mo["nk_mean"] > 1e-5 * tot
    assert np.max(np.abs(nk[big] - mo["nk_mean"][big]) / mo["nk_mean"][big]) < 1e-3
    assert np.max(np.abs(nk - mo["nk_mean"])) < 1e-6 * tot
    # Q is a small difference of large means: compare against the spread of the ensemble
    sc = m["scalars"].cpu().numpy()
    spread = np.sum(np.abs(ref[1:] - ref[1:].mean(0)) ** 2) / (w.n_real) * w.grid.dV
    assert abs(sc[0] - mo["Q"]) < 2e-3 * spread
    assert abs(sc[5] - np.sum(mo["nk_mean"])) < 1e-4 * np.sum(np.abs(mo["nk_mean"]))


def test_run_series_matches_oracle():
    w = ti.small_workload("kgauss", 3, 16, 6, 40, n_tot=1e8, out_every=10, dt=DT_128)
    cl = w.psi_cl()
    ens = make_ensemble([w], 0)
    series = ens.run([cl], w.noise_seed, w.n_steps, w.out_every).cpu().numpy()
    t, ref_series, ref_final = twa.run(cl, w.phys.hbar_m, w.phys.C, w.phys.dt, w.grid.L, 3, w.phys.n_tot,
                                       w.n_real, w.noise_seed, w.n_steps, w.out_every)
    assert series.shape[0] == len(ref_series)
    for o, mo in enumerate(ref_series):
        assert abs(series[o, 0, 1] - mo["corr"]) <= CORR_TOL * mo["corr"] + 1e-12
        assert abs(series[o, 0, 5] - np.sum(mo["nk_mean"])) < 1e-4 * np.sum(np.abs(mo["nk_mean"]))
    got = ens.fields(0).cpu().numpy().astype(np.complex128)
    assert np.all(field_rel_l2(got, ref_final, 3) < F32_FIELD_TOL)


def test_run_is_bitwise_deterministic_and_replays_graph():
    w = ti.small_workload("merger2d", 2, 64, 4, 30, n_tot=1e9, out_every=10, dt=DT_2D)
    cl = w.psi_cl()
    ens = make_ensemble([w], 0)
    s1 = ens.run([cl], w.noise_seed, w.n_steps, w.out_every).cpu().numpy()
    f1 = ens.fields(0).cpu().numpy().copy()
    s2 = ens.run([cl], w.noise_seed, w.n_steps, w.out_every).cpu().numpy()
    f2 = ens.fields(0).cpu().numpy()
    assert np.array_equal(s1, s2) and np.array_equal(f1, f2)


def test_uneven_multi_instance_batch():
    w1 = ti.small_workload("merger2d", 2, 64, 5, 20, n_tot=1e9, dt=DT_2D)
    w2 = ti.small_workload("merger2d", 2, 32, 3, 20, n_tot=1e9, dt=DT_2D)
    w2 = ti.Workload(w2.name, w2.grid, w1.phys, w2.n_real, w2.n_steps, w2.out_every, w2.psi_cl_seed, w1.noise_seed)
    ens = make_ensemble([w1, w2], 0)
    ens.sample([w1.psi_cl(), w2.psi_cl()], w1.noise_seed)
    ens.step(20)
    for i, w in enumerate((w1, w2)):
        ref = oracle_batch(w, w.psi_cl(), 20, instance=i)
        got = ens.fields(i).cpu().numpy().astype(np.complex128)
        assert np.all(field_rel_l2(got, ref, 2) < F32_FIELD_TOL)


def test_forked_instances_match_serial_run_and_oracle():
    """A three-instance uneven batch runs each instance on its own graph branch; the result is
    bitwise the same as the serial run (the pass profiler keeps one stream) and matches the oracle."""
    from paper_2310_07119_gb300 import twa_profile_enable
    base = ti.small_workload("merger2d", 2, 64, 4, 30, n_tot=1e9, out_every=10, dt=DT_2D)
    ws = [base]
    for m, nr in ((32, 3), (128, 2)):
        g = ti.Grid.cube(2, m)
        ws.append(ti.Workload(base.name, g, base.phys, nr, base.n_steps, base.out_every, base.psi_cl_seed, base.noise_seed))
    cls = [w.psi_cl() for w in ws]
    out = []
    for serial in (True, False):
        ens = make_ensemble(ws, 0)
        twa_profile_enable(ens.h, serial)
        series = ens.run(cls, base.noise_seed, base.n_steps, base.out_every).cpu().numpy()
        out.append((series, [ens.fields(i).cpu().numpy().copy() for i in range(len(ws))]))
        ens.close()
    assert np.array_equal(out[0][0], out[1][0])
    for a, b in zip(out[0][1], out[1][1]):
        assert np.array_equal(a, b)
    for i, w in enumerate(ws):
        b0 = twa.sample(cls[i], w.noise_seed, w.n_real, w.phys.n_tot, w.grid.dV, w.phys.noise_conv, i)
        _, ref_series, ref_final = twa.run(cls[i], w.phys.hbar_m, w.phys.C, w.phys.dt, w.grid.L, 2, w.phys.n_tot,
                                           w.n_real, w.noise_seed, w.n_steps, w.out_every, batch=b0)
        assert np.all(field_rel_l2(out[1][1][i].astype(np.complex128), ref_final, 2) < F32_FIELD_TOL)
        for o, mo in enumerate(ref_series):
            assert abs(out[1][0][o, i, 1] - mo["corr"]) <= CORR_TOL * mo["corr"] + 1e-12


def test_streams_are_independent_of_batch_size():
    # slots keep their Poisson partner (2p, 2p+1) when the batch grows, so results are bitwise equal
    base = ti.small_workload("kgauss", 3, 16, 3, 10, n_tot=1e8)
    big = ti.Workload(base.name, base.grid, base.phys, 7, 10, 5, base.psi_cl_seed, base.noise_seed)
    cl = base.psi_cl()
    out = []
    for w in (base, big):
        ens = make_ensemble([w], 0)
        ens.sample([cl], w.noise_seed)
        ens.step(10)
        out.append(ens.fields(0).cpu().numpy())
    assert np.array_equal(out[0], out[1][:4])


def test_nonfinite_input_is_flagged_and_contained_to_its_pair():
    from paper_2310_07119_gb300 import twa_sync_status
    w = ti.small_workload("merger2d", 2, 32, 5, 5, n_tot=1e9)
    cl = w.psi_cl()
    clean = make_ensemble([w], 0)
    clean.sample([cl], w.noise_seed)
    clean.step(5)
    ens = make_ensemble([w], 0)
    ens.sample([cl], w.noise_seed)
    f = ens.fields(0)
    f[3, 5, 7] = complex(float("nan"), 0.0)          # slot 3 (pair 1 = slots 2, 3)
    ens.step(5)
    m = ens.moments(0)
    assert m["scalars"][4].item() > 0
    assert twa_sync_status(ens.h) == -5
    a, b = ens.fields(0).cpu().numpy(), clean.fields(0).cpu().numpy()
    for s in (0, 1, 4, 5):
        assert np.array_equal(a[s], b[s]), s
    assert not np.all(np.isfinite(a[3]))


def test_autotune_keeps_parity(tmp_path):
    w = ti.small_workload("kgauss", 3, 32, 4, 20, n_tot=1e8, dt=DT_128)
    cl = w.psi_cl()
    ens = make_ensemble([w], 0)
    cache = str(tmp_path / "tune.json")
    ens.autotune(cache)
    assert open(cache).read().count("op") >= 6
    ens.sample([cl], w.noise_seed)
    ens.step(20)
    got = ens.fields(0).cpu().numpy().astype(np.complex128)
    assert np.all(field_rel_l2(got, oracle_batch(w, cl, 20), 3) < F32_FIELD_TOL)


def test_bench_size_sampled_realizations():
    """128^3 x 256 streams (the bench layout), 100 KDK steps: sampled streams vs the oracle.

    The oracle evolves the classical field and two sampled streams (same Philox counters) for
    the same 100 steps; field and per-stream density must meet the field (1e-4) and <rho>
    (1e-5) tolerances, and every stream must conserve its mass.
    """
    w = ti.workload_3d_condensation(128, 256, 100)
    cl = w.psi_cl()
    ens = make_ensemble([w], 0, want_modes=False)
    ens.sample([cl], w.noise_seed)
    f = ens.fields(0)
    mass0 = (f.abs() ** 2).sum(dim=(1, 2, 3)).double().cpu().numpy() * w.grid.dV
    ens.step(w.n_steps)
    mass = (f.abs() ** 2).sum(dim=(1, 2, 3)).double().cpu().numpy() * w.grid.dV
    assert np.all(np.abs(mass - mass0) < 1e-5 * mass0)          # unitarity of every stream
    slots = [0, 137, 256]
    sub = f[slots].cpu().numpy().astype(np.complex128)
    del f, ens
    torch.cuda.empty_cache()
    sig = twa.noise_sigma(w.phys.n_tot, w.grid.dV)
    from oracle.philox import wigner_normals
    ref = np.empty((len(slots),) + cl.shape, dtype=np.complex128)
    for i, s in enumerate(slots):
        if s == 0:
            ref[i] = cl
        else:
            zr, zi = wigner_normals(w.noise_seed, cl.size, s)
            ref[i] = cl + sig * (zr + 1j * zi).reshape(cl.shape)
    for _ in range(w.n_steps):
        ref = sp.step(ref, w.phys.hbar_m, w.phys.C, w.phys.dt, 1.0, 3)
    assert np.all(field_rel_l2(sub, ref, 3) < F32_FIELD_TOL)
    r_got, r_ref = np.abs(sub) ** 2, np.abs(ref) ** 2
    rho_err = np.sqrt(np.sum((r_got - r_ref) ** 2, axis=(1, 2, 3)) / np.sum(r_ref ** 2, axis=(1, 2, 3)))
    assert np.all(rho_err < RHO_TOL), rho_err




def test_uneven_2d_mix_full_size_sampled():
    """The uneven 2D batch at its full layout (two-soliton merger, 512^2 x 128 + 1024^2 x 64 +
    2048^2 x 16 streams in one handle, forked per instance), 10 KDK steps: the classical field and
    two sampled streams of every instance against the oracle."""
    from oracle.philox import wigner_normals
    ws = [ti.workload_2d_merger(m, nr, 10) for m, nr in ((512, 128), (1024, 64), (2048, 16))]
    cls = [w.psi_cl() for w in ws]
    seed = ws[0].noise_seed
    ens = make_ensemble(ws, 0, want_modes=False)
    ens.sample(cls, seed)
    ens.step(10)
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

PIPE = 1 << 16     # flag on a pass's "lines" value selecting its cp.async-pipelined variant
PIPE_OPS = (0, 1, 2, 3, 5, 6, 7)     # drift, kick_drift, kick_drift_vinv, drift_rho, fwd, fwd_mul_inv, inv
THREADS_PER_LINE = {32: 2, 64: 8, 128: 8, 256: 16, 512: 32, 1024: 64, 2048: 128}    # N / registers-per-thread of the line FFT


def _force_pipelined(w, path, axis_pipeline):
    """Autotune cache that selects the pipelined variant of every line pass that has one."""
    import json
    n = list(w.grid.shape[::-1]) + [1] * (3 - w.grid.dim)          # fastest axis first
    key = f"{n[0]}x{n[1]}x{n[2]}:slots{w.n_real + 1}"
    cache = {f"{key}:axis9:op0": 0 if axis_pipeline else 1}
    for ax in range(w.grid.dim):
        T = THREADS_PER_LINE[n[ax]]
        lines = max(4 if ax > 0 else 1, 128 // T)
        for op in PIPE_OPS:
            cache[f"{key}:axis{ax}:op{op}"] = PIPE | lines
    json.dump(cache, open(path, "w"))


# line passes each pipeline runs per step: (axis, op)
RUN_PASSES = {"3d_axis": [(0, 2), (1, 0), (2, 3), (0, 5), (1, 6), (2, 7)], "3d_plane": [(2, 3), (2, 7)],
              "2d": [(0, 1), (1, 3), (0, 6), (1, 7)]}


@pytest.mark.parametrize("name,axis_pipeline", [("3d_kgauss64", True), ("3d_kgauss64", False), ("2d_merger64", True),
                                                ("2d_merger2048", True)])
def test_pipelined_passes_match_oracle(name, axis_pipeline, tmp_path):
    """The pipelined line passes, forced through the autotune cache, against the oracle (the cache
    the tuner writes back shows that it kept the pipelined variant of every pass the step runs)."""
    import json
    if name == "3d_kgauss64":
        w = ti.small_workload("kgauss", 3, 64, 3, 40, n_tot=1e8, dt=DT_128)
        runs = RUN_PASSES["3d_axis" if axis_pipeline else "3d_plane"]
    elif name == "2d_merger64":
        w = ti.small_workload("merger2d", 2, 64, 5, 40, n_tot=1e9, dt=DT_2D)
        runs = RUN_PASSES["2d"]
    else:
        w = ti.small_workload("merger2d", 2, 2048, 1, 8, n_tot=1e9, dt=DT_2D)
        runs = RUN_PASSES["2d"]
    path = str(tmp_path / "force_pipe.json")
    _force_pipelined(w, path, axis_pipeline)
    cl = w.psi_cl()
    ens = make_ensemble([w], 0)
    ens.autotune(path)
    chosen = json.load(open(path))
    n = list(w.grid.shape[::-1]) + [1] * (3 - w.grid.dim)
    key = f"{n[0]}x{n[1]}x{n[2]}:slots{w.n_real + 1}"
    for ax, op in runs:
        assert chosen[f"{key}:axis{ax}:op{op}"] & PIPE, (ax, op)
    if w.grid.dim == 3:
        assert chosen[f"{key}:axis9:op0"] == (0 if axis_pipeline else 1)
    ens.sample([cl], w.noise_seed)
    ens.step(w.n_steps)
    got = ens.fields(0).cpu().numpy().astype(np.complex128)
    ref = oracle_batch(w, cl, w.n_steps)
    assert np.all(field_rel_l2(got, ref, w.grid.dim) < F32_FIELD_TOL)


DUAL = 1 << 17     # flag on a pass's "lines" value selecting its two-field variant (both slots of a pair per thread)
DUAL_OPS = (0, 1, 2, 3)     # drift, kick_drift, kick_drift_vinv, drift_rho


def _force_dual(w, path, axis_pipeline, dual=True):
    """Autotune cache that selects the 3D pipeline and, for every pass that has one, the two-field
    variant (dual) or the single-field variant with the same lines per CTA."""
    import json
    n = list(w.grid.shape[::-1]) + [1] * (3 - w.grid.dim)
    key = f"{n[0]}x{n[1]}x{n[2]}:slots{w.n_real + 1}"
    cache = {f"{key}:axis9:op0": 0 if axis_pipeline else 1}
    for ax in range(w.grid.dim):
        T = THREADS_PER_LINE.get(n[ax], 1)
        lines = max(4 if ax > 0 else 2, 128 // T)
        for op in DUAL_OPS:
            cache[f"{key}:axis{ax}:op{op}"] = (DUAL if dual else 0) | lines
    json.dump(cache, open(path, "w"))


@pytest.mark.parametrize("name,axis_pipeline", [("3d_kgauss64", True), ("3d_kgauss64_odd", True),
                                                ("3d_kgauss64", False), ("2d_merger64", True), ("2d_merger2048", True)])
def test_dual_passes_match_oracle_and_the_single_field_passes(name, axis_pipeline, tmp_path):
    """The two-field variants (both slots of a pair transformed by the same threads), forced through
    the autotune cache: bitwise the single-field passes (the same arithmetic per line) and the oracle."""
    import json
    if name == "3d_kgauss64":
        w = ti.small_workload("kgauss", 3, 64, 3, 30, n_tot=1e8, dt=DT_128)
    elif name == "3d_kgauss64_odd":
        w = ti.small_workload("kgauss", 3, 64, 4, 30, n_tot=1e8, dt=DT_128)      # 5 slots: a lone last slot
    elif name == "2d_merger64":
        w = ti.small_workload("merger2d", 2, 64, 5, 30, n_tot=1e9, dt=DT_2D)
    else:
        w = ti.small_workload("merger2d", 2, 2048, 2, 8, n_tot=1e9, dt=DT_2D)
    cl = w.psi_cl()
    out = []
    for forced in (True, False):
        path = str(tmp_path / f"force_dual{int(forced)}.json")
        _force_dual(w, path, axis_pipeline, dual=forced)
        ens = make_ensemble([w], 0)
        ens.autotune(path)
        if forced:
            chosen = json.load(open(path))
            n = list(w.grid.shape[::-1]) + [1] * (3 - w.grid.dim)
            key = f"{n[0]}x{n[1]}x{n[2]}:slots{w.n_real + 1}"
            assert any(v & DUAL for k, v in chosen.items() if k.startswith(key) and ":op" in k)
        ens.sample([cl], w.noise_seed)
        ens.step(w.n_steps)
        out.append(ens.fields(0).cpu().numpy().copy())
        ens.close()
    assert np.array_equal(out[0], out[1])
    ref = oracle_batch(w, cl, w.n_steps)
    assert np.all(field_rel_l2(out[0].astype(np.complex128), ref, w.grid.dim) < F32_FIELD_TOL)


TMA = 1 << 18      # with PIPE: the column pass whose tiles the Tensor Memory Accelerator copies
COLUMN_OPS = (0, 3, 5, 6, 7)     # drift, drift_rho, fwd, fwd_mul_inv, inv


def _force_columns(w, path, axis_pipeline, tma, narrow=False):
    """Autotune cache that selects the pipelined variant of every column pass (y and z axes), with
    TMA tile copies or with the threads' cp.async copies (narrow: the TMA variant with two lines per
    CTA, for lines of 64 or more threads); the x passes get one fixed shape."""
    import json
    n = list(w.grid.shape[::-1]) + [1] * (3 - w.grid.dim)
    key = f"{n[0]}x{n[1]}x{n[2]}:slots{w.n_real + 1}"
    cache = {f"{key}:axis9:op0": 0 if axis_pipeline else 1}
    for ax in range(1, w.grid.dim):
        lines = max(4, 128 // THREADS_PER_LINE[n[ax]])
        if narrow and tma and THREADS_PER_LINE[n[ax]] >= 64:
            lines = 2
        for op in COLUMN_OPS:
            cache[f"{key}:axis{ax}:op{op}"] = PIPE | (TMA if tma else 0) | lines
    for op in (1, 2, 6):     # one fixed shape for the x passes, so both runs do the same arithmetic
        cache[f"{key}:axis0:op{op}"] = max(1, 128 // THREADS_PER_LINE.get(n[0], 128))
    json.dump(cache, open(path, "w"))


@pytest.mark.parametrize("name,axis_pipeline", [("3d_kgauss64", True), ("3d_kgauss64_odd", True),
                                                ("3d_kgauss64", False), ("2d_merger64", True), ("2d_merger512", True),
                                                ("2d_merger2048", True), ("2d_merger2048_narrow", True),
                                                ("2d_merger1024_narrow", True)])
def test_tma_column_passes_match_cp_async_and_oracle(name, axis_pipeline, tmp_path):
    """The column passes with TMA tile copies (4D tensor maps over the batch, boxes of LINES x 256
    elements, mbarrier completion) against the same passes fed by cp.async: the same values reach
    the same shared-memory layout, so the fields are bitwise equal; and against the oracle.  The odd
    case has a lone last slot (a stage with nothing to copy)."""
    import json
    from paper_2310_07119_gb300 import twa_sync_status
    if name == "3d_kgauss64":
        w = ti.small_workload("kgauss", 3, 64, 3, 20, n_tot=1e8, dt=DT_128)
    elif name == "3d_kgauss64_odd":
        w = ti.small_workload("kgauss", 3, 64, 4, 20, n_tot=1e8, dt=DT_128)
    elif name == "2d_merger64":
        w = ti.small_workload("merger2d", 2, 64, 5, 20, n_tot=1e9, dt=DT_2D)
    elif name == "2d_merger512":
        w = ti.small_workload("merger2d", 2, 512, 3, 10, n_tot=1e9, dt=DT_2D)
    elif name == "2d_merger1024_narrow":
        w = ti.small_workload("merger2d", 2, 1024, 4, 8, n_tot=1e9, dt=DT_2D)
    else:
        w = ti.small_workload("merger2d", 2, 2048, 2, 6, n_tot=1e9, dt=DT_2D)
    narrow = name.endswith("_narrow")
    cl = w.psi_cl()
    out = []
    for tma in (True, False):
        path = str(tmp_path / f"force_cols{int(tma)}.json")
        _force_columns(w, path, axis_pipeline, tma, narrow)
        ens = make_ensemble([w], 0)
        ens.autotune(path)
        chosen = json.load(open(path))
        n = list(w.grid.shape[::-1]) + [1] * (3 - w.grid.dim)
        key = f"{n[0]}x{n[1]}x{n[2]}:slots{w.n_real + 1}"
        for ax in range(1, w.grid.dim):
            for op in COLUMN_OPS:
                k = f"{key}:axis{ax}:op{op}"
                assert chosen[k] & PIPE and bool(chosen[k] & TMA) == tma, (k, chosen[k])
        ens.sample([cl], w.noise_seed)
        ens.step(w.n_steps)
        assert twa_sync_status(ens.h) == 0
        out.append(ens.fields(0).cpu().numpy().copy())
        ens.close()
    assert np.array_equal(out[0], out[1])
    ref = oracle_batch(w, cl, w.n_steps)
    assert np.all(field_rel_l2(out[0].astype(np.complex128), ref, w.grid.dim) < F32_FIELD_TOL)


ROW_OPS = (1, 2, 5, 6, 7)     # kick_drift, kick_drift_vinv, fwd, fwd_mul_inv, inv


def _force_rows(w, path, axis_pipeline, tma):
    """Autotune cache that selects the pipelined variant of every row pass (x axis), its tiles copied
    by one bulk copy per row (TMA) or by the threads' cp.async copies; other passes get fixed shapes."""
    import json
    n = list(w.grid.shape[::-1]) + [1] * (3 - w.grid.dim)
    key = f"{n[0]}x{n[1]}x{n[2]}:slots{w.n_real + 1}"
    cache = {f"{key}:axis9:op0": 0 if axis_pipeline else 1}
    lines = max(1, 128 // THREADS_PER_LINE[n[0]])
    for op in ROW_OPS:
        cache[f"{key}:axis0:op{op}"] = PIPE | (TMA if tma else 0) | lines
    for ax in range(1, w.grid.dim):
        for op in COLUMN_OPS:
            cache[f"{key}:axis{ax}:op{op}"] = max(4, 128 // THREADS_PER_LINE[n[ax]])
    json.dump(cache, open(path, "w"))


@pytest.mark.parametrize("name,axis_pipeline", [("3d_kgauss64", True), ("3d_kgauss64_odd", True),
                                                ("2d_merger64", True), ("2d_merger512", True),
                                                ("2d_merger2048", True)])
def test_tma_row_passes_match_cp_async_and_oracle(name, axis_pipeline, tmp_path):
    """The row passes with their tiles moved by bulk copies (cp.async.bulk, one per row, completion
    on the stage's mbarrier) against the same passes fed by cp.async (bitwise) and the oracle."""
    import json
    from paper_2310_07119_gb300 import twa_sync_status
    if name == "3d_kgauss64":
        w = ti.small_workload("kgauss", 3, 64, 3, 20, n_tot=1e8, dt=DT_128)
    elif name == "3d_kgauss64_odd":
        w = ti.small_workload("kgauss", 3, 64, 4, 20, n_tot=1e8, dt=DT_128)
    elif name == "2d_merger64":
        w = ti.small_workload("merger2d", 2, 64, 5, 20, n_tot=1e9, dt=DT_2D)
    elif name == "2d_merger512":
        w = ti.small_workload("merger2d", 2, 512, 3, 10, n_tot=1e9, dt=DT_2D)
    else:
        w = ti.small_workload("merger2d", 2, 2048, 2, 6, n_tot=1e9, dt=DT_2D)
    cl = w.psi_cl()
    out = []
    for tma in (True, False):
        path = str(tmp_path / f"force_rows{int(tma)}.json")
        _force_rows(w, path, axis_pipeline, tma)
        ens = make_ensemble([w], 0)
        ens.autotune(path)
        chosen = json.load(open(path))
        n = list(w.grid.shape[::-1]) + [1] * (3 - w.grid.dim)
        key = f"{n[0]}x{n[1]}x{n[2]}:slots{w.n_real + 1}"
        used = [k for k in chosen if k.startswith(f"{key}:axis0:") and int(k.rsplit("op", 1)[1]) in ROW_OPS]
        assert used and all(bool(chosen[k] & TMA) == tma and chosen[k] & PIPE for k in used), chosen
        ens.sample([cl], w.noise_seed)
        ens.step(w.n_steps)
        assert twa_sync_status(ens.h) == 0
        out.append(ens.fields(0).cpu().numpy().copy())
        ens.close()
    assert np.array_equal(out[0], out[1])
    ref = oracle_batch(w, cl, w.n_steps)
    assert np.all(field_rel_l2(out[0].astype(np.complex128), ref, w.grid.dim) < F32_FIELD_TOL)


def test_a_stalled_tma_tile_times_out_and_the_handle_keeps_working(tmp_path):
    """Fault injection on the host side of the TMA tile pipeline: the next TMA pass expects 16 bytes
    per tile that no copy delivers, so every CTA's bounded wait runs out (wait limit 0.05 s), the
    pass stops and twa_sync_status reports TWA_ETIMEOUT; the GPU keeps answering and the next call
    (after resampling) matches a handle that never stalled, bitwise."""
    from paper_2310_07119_gb300 import twa_debug_stall_next_tma, twa_set_wait_limit, twa_sync_status
    w = ti.small_workload("merger2d", 2, 512, 3, 4, n_tot=1e9, dt=DT_2D)
    cl = w.psi_cl()
    path = str(tmp_path / "force_cols.json")
    _force_columns(w, path, True, True)
    ens = make_ensemble([w], 0)
    ens.autotune(path)
    twa_set_wait_limit(ens.h, 0.05)
    ens.sample([cl], w.noise_seed)
    twa_debug_stall_next_tma(ens.h)
    ens.step(2)
    assert twa_sync_status(ens.h) == -4                  # TWA_ETIMEOUT
    assert twa_sync_status(ens.h) == 0                   # the error word was cleared
    x = torch.ones(1 << 20, device="cuda")
    assert float(x.sum()) == float(1 << 20)              # the GPU still answers
    ens.sample([cl], w.noise_seed)
    ens.step(w.n_steps)
    assert twa_sync_status(ens.h) == 0
    got = ens.fields(0).cpu().numpy().copy()
    ens.close()
    ref = make_ensemble([w], 0)
    ref.autotune(path)
    ref.sample([cl], w.noise_seed)
    ref.step(w.n_steps)
    assert np.array_equal(got, ref.fields(0).cpu().numpy())
    ref.close()


@pytest.mark.parametrize("n_real", [3, 4])
def test_sixteen_line_512_columns_match_eight_lines_and_oracle(n_real, tmp_path):
    """512-point column passes with 16 lines per CTA (512 threads; a warp reads two whole 128-byte
    rows per access) against the 8-line passes (the same arithmetic per line: bitwise) and the
    oracle; n_real = 4 leaves a lone last slot."""
    import json
    w = ti.small_workload("merger2d", 2, 512, n_real, 10, n_tot=1e9, dt=DT_2D)
    cl = w.psi_cl()
    key = f"512x512x1:slots{w.n_real + 1}"
    out = []
    for lines in (16, 8):
        path = str(tmp_path / f"cols{lines}.json")
        cache = {f"{key}:axis1:op{op}": lines for op in (3, 4, 5, 7)}
        cache.update({f"{key}:axis0:op{op}": 4 for op in (1, 6, 9)})
        json.dump(cache, open(path, "w"))
        ens = make_ensemble([w], 0)
        ens.autotune(path)
        chosen = json.load(open(path))
        assert all(chosen[f"{key}:axis1:op{op}"] == lines for op in (3, 4, 5, 7))
        ens.sample([cl], w.noise_seed)
        ens.step(w.n_steps)
        out.append(ens.fields(0).cpu().numpy().copy())
        ens.close()
    assert np.array_equal(out[0], out[1])
    ref = oracle_batch(w, cl, w.n_steps)
    assert np.all(field_rel_l2(out[0].astype(np.complex128), ref, w.grid.dim) < F32_FIELD_TOL)


@pytest.mark.parametrize("n_real", [3, 4])
def test_hybrid_3d_pipeline_matches_plane_pipeline_and_oracle(n_real, tmp_path):
    """The hybrid 3D pipeline (axis passes for the fields, the xy-plane pass for the Poisson field,
    autotune cache value 2) against the plane pipeline (value 1): the same per-line arithmetic, so
    fields and the moment series of twa_advance are bitwise equal; and the fields against the oracle."""
    import json
    from paper_2310_07119_gb300 import twa_advance, twa_sync_status
    w = ti.small_workload("kgauss", 3, 64, n_real, 20, n_tot=1e8, dt=DT_128)
    cl = w.psi_cl()
    key = f"64x64x64:slots{w.n_real + 1}"
    out = []
    for pipeline in (2, 1):
        path = str(tmp_path / f"pipe{pipeline}.json")
        json.dump({f"{key}:axis9:op0": pipeline}, open(path, "w"))
        ens = make_ensemble([w], 0)
        ens.autotune(path)
        assert json.load(open(path))[f"{key}:axis9:op0"] == pipeline
        ens.sample([cl], w.noise_seed)
        series = ens.new_series(w.n_steps, 10)
        twa_advance(ens.h, ens.psi, w.n_steps, 10, series)
        assert twa_sync_status(ens.h) == 0
        out.append((ens.fields(0).cpu().numpy().copy(), series.cpu().numpy().copy()))
        ens.close()
    assert np.array_equal(out[0][0], out[1][0])
    assert np.array_equal(out[0][1], out[1][1])
    ref = oracle_batch(w, cl, w.n_steps)
    assert np.all(field_rel_l2(out[0][0].astype(np.complex128), ref, w.grid.dim) < F32_FIELD_TOL)
