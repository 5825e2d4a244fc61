"""Pins for the oracle's TWA sampling and ensemble moments (Sec. III.A-III.C).

Checked against: the coherent-state Wigner function's exact moments, the
exactness of the TWA for a quadratic Hamiltonian (free field), the paper's
n_s Q_s invariance (Eq. Q_relation), brute-force Fock-space evolution of a
3-site lattice (the exact quantum answer), and the single-mode Kerr oscillator
of Fig. 2 in closed form.
"""
import math

import numpy as np
import pytest

import twa_inputs as ti
from oracle import fock, kerr, sp, twa


def _bump(m=64):
    g = ti.Grid.cube(1, m)
    return g, ti.cosine_overdensity(g, 0.5)


def test_sample_slot0_is_classical_and_noise_variance():
    g, psi = _bump()
    n, Ns = 1e4, 400
    b = twa.sample(psi, 3, Ns, n, g.dV)
    assert np.array_equal(b[0], psi)
    d = (b[1:] - psi[None]).ravel()
    sig2 = 1.0 / (4.0 * n * g.dV)                    # complex variance 1/2 per mode
    for comp in (d.real, d.imag):
        assert abs(comp.var() / sig2 - 1.0) < 5 * math.sqrt(2.0 / comp.size)
    lit = twa.sample(psi, 3, Ns, n, g.dV, noise_conv=1)
    assert np.allclose((lit[1:] - psi).var(), 2.0 * (b[1:] - psi).var(), rtol=1e-12)


def test_noise_is_white_with_half_quantum_per_mode():
    g, psi = _bump(32)
    n, Ns = 1e6, 2000
    b = twa.sample(psi, 11, Ns, n, g.dV)
    da = np.fft.fft(b[1:] - psi, axis=-1) * math.sqrt(n * g.dV / g.cells)
    e = (np.abs(da) ** 2).mean(axis=0)                 # E |delta a_k|^2 per mode
    assert np.all(np.abs(e - 0.5) < 5 * 0.5 / math.sqrt(Ns))


def test_moments_of_the_initial_coherent_state():
    g, psi = _bump(32)
    n, Ns = 50.0, 20000
    b = twa.sample(psi, 5, Ns, n, g.dV)
    m = twa.moments(b, n, 1.0, 1)
    z2 = np.abs(np.fft.fft(psi) * math.sqrt(n * g.dV / g.cells)) ** 2
    # a coherent state has <n_k> = |z_k|^2 and Var n_k = |z_k|^2 (Poisson)
    se = np.sqrt((z2 + 0.25) / Ns)
    assert np.all(np.abs(m["nk_mean"] - z2) < 5 * se)
    se_var = np.sqrt((2 * z2 ** 2 + 4 * z2 + 1) / Ns) + 1e-3
    assert np.all(np.abs(m["nk_var"] - z2) < 6 * se_var)
    # Q(0): a coherent state has Q = 0; the sample estimator's bias is -M/(2 n N_s)
    M = g.cells
    assert abs(m["Q"] + M / (2 * n * Ns)) < 6 * (M / (2 * n)) / math.sqrt(M * Ns)
    assert np.allclose(m["rho_cl"], np.abs(psi) ** 2)
    assert abs(np.sum(m["rho_mean"]) * g.dV - 1.0) < 5e-3


def test_free_field_twa_is_exact():
    # quadratic H: every |a_k|^2 is conserved stream by stream, and so are Q and Var n_k
    g, psi = _bump(64)
    n = 1e3
    t, series, _ = twa.run(psi, 0.05, 0.0, 0.01, 1.0, 1, n, 16, 9, 30, 10)
    for s in series[1:]:
        assert np.max(np.abs(s["nk_mean"] - series[0]["nk_mean"])) < 1e-9
        assert np.max(np.abs(s["nk_var"] - series[0]["nk_var"])) < 1e-9 * (1 + np.max(series[0]["nk_var"]))
        assert abs(s["Q"] - series[0]["Q"]) < 1e-12


def test_free_field_keeps_the_coherent_state_moments_at_late_times():
    # the TWA is exact for the free field: <n_k> = Var n_k = |z_k|^2 at every t (here after 200
    # steps, long after every mode has rotated many times), within the sampling error
    g, psi = _bump(32)
    n, Ns = 50.0, 20000
    t, series, _ = twa.run(psi, 0.2, 0.0, 0.01, 1.0, 1, n, Ns, 5, 200, 200)
    m = series[-1]
    z2 = np.abs(np.fft.fft(psi) * math.sqrt(n * g.dV / g.cells)) ** 2
    assert np.all(np.abs(m["nk_mean"] - z2) < 5 * np.sqrt((z2 + 0.25) / Ns))
    assert np.all(np.abs(m["nk_var"] - z2) < 6 * (np.sqrt((2 * z2 ** 2 + 4 * z2 + 1) / Ns) + 1e-3))


def test_correction_norm_of_constructed_batches():
    # streams psi0 e^{i theta_s}: every |psi_s|^2 = rho_cl, so <rho> - rho_cl = -1/(2 n dV) in every
    # cell and corr = sqrt(M) / (2 n dV ||rho_cl||); streams c_s psi0 (real c_s) give
    # <rho> - rho_cl = (mean c^2 - 1) rho_cl - 1/(2 n dV)
    M, n_tot, L = 32, 1e3, 2.0
    dV = L / M
    rng = np.random.default_rng(9)
    psi0 = (1.0 + rng.random(M)) * np.exp(1j * rng.uniform(0, 2 * np.pi, M))
    w = 1.0 / (2.0 * n_tot * dV)
    rho = np.abs(psi0) ** 2
    theta = np.array([0.3, -1.2, 2.0])
    rot = np.concatenate([psi0[None], psi0[None] * np.exp(1j * theta)[:, None]])
    m = twa.moments(rot, n_tot, L, 1, with_modes=False)
    assert m["corr"] == pytest.approx(math.sqrt(M) * w / np.linalg.norm(rho), rel=1e-12)
    c = np.array([0.9, 1.05, 1.2, 0.7])
    sc = np.concatenate([psi0[None], c[:, None] * psi0[None]])
    m = twa.moments(sc, n_tot, L, 1, with_modes=False)
    expect = np.linalg.norm((np.mean(c ** 2) - 1.0) * rho - w) / np.linalg.norm(rho)
    assert m["corr"] == pytest.approx(expect, rel=1e-12)


def test_correction_norm_of_the_initial_coherent_state():
    # At t = 0, psi_s = psi_cl + d_s with complex Gaussian d_s of variance 2 sigma^2 = 1/(2 n dV):
    # X_s = |psi_cl + d_s|^2 - rho_cl - 1/(2 n dV) has mean 0 and variance 4 sigma^2 rho_cl + 4 sigma^4
    # per cell, so E ||<rho> - rho_cl||^2 = sum_g (4 sigma^2 rho_g + 4 sigma^4) / N_s.  A missing Weyl
    # offset adds M / (2 n dV)^2 (five times the expectation here); a wrong noise variance doubles it.
    g, psi = _bump(64)
    n, Ns, R = 50.0, 16, 400
    sig2 = 1.0 / (4.0 * n * g.dV)
    rho = np.abs(psi) ** 2
    expect = np.sum(4 * sig2 * rho + 4 * sig2 ** 2) / Ns
    vals = []
    for r in range(R):
        m = twa.moments(twa.sample(psi, 1000 + r, Ns, n, g.dV), n, 1.0, 1, with_modes=False)
        vals.append((m["corr"] * np.linalg.norm(rho)) ** 2)
    vals = np.array(vals)
    assert abs(vals.mean() - expect) < 5 * vals.std() / math.sqrt(R)
    assert abs(vals.mean() - expect) < 0.05 * expect


def test_nsQs_is_independent_of_the_sampling_n():
    # Eq. Q_relation: with the same normals, n_s Q_s agrees across n_s while Q << 1
    g, psi = _bump(64)
    out = []
    for n in (1e8, 1e10):
        t, series, _ = twa.run(psi, 0.01, 4 * np.pi, 2e-3, 1.0, 1, n, 32, 21, 150, 50,
                               with_modes=False)
        q = np.array([s["Q"] for s in series])
        out.append(n * (q - q[0]))
    assert np.all(np.abs(out[0][1:] - out[1][1:]) < 0.02 * np.abs(out[1][1:]) + 1e-9)
    assert out[1][-1] > 0


def _fock_case(M, C=200.0, amp=0.9, n=10.0, times=(0.0, 0.02, 0.05)):
    x = np.arange(M) / M
    psi = np.sqrt(1 + amp * np.cos(2 * np.pi * x)).astype(complex)
    psi /= np.sqrt(np.sum(np.abs(psi) ** 2) / M)
    return psi, C, n, np.array(times)


def _twa_nk(psi, C, n, times, Ns, noise_conv=0, dt=1e-3):
    """<n_k> and Var n_k of the TWA ensemble from oracle.twa.moments, with standard errors.

    The standard errors are the test's own: the spread of |a_k|^2 over the streams for <n_k>, and
    the delta-method influence function of the Var n_k estimator for Var n_k."""
    M = psi.size
    cur = twa.sample(psi, 7, Ns, n, 1.0 / M, noise_conv)
    res = []
    s = 0
    for t in times:
        while s < int(round(t / dt)):
            cur = sp.step(cur, 1.0, C, dt, 1.0, 1)
            s += 1
        mo = twa.moments(cur, n, 1.0, 1)
        a = np.fft.fft(cur, axis=-1) * math.sqrt(n * (1.0 / M) / M)
        a2 = np.abs(a[1:]) ** 2
        m2 = a2.mean(0)
        infl = a2 ** 2 - a2 - 2 * (m2 - 0.5) * a2            # delta-method influence function
        res.append((mo["nk_mean"], a2.std(0) / math.sqrt(Ns), mo["nk_var"], infl.std(0) / math.sqrt(Ns),
                    np.abs(a[0]) ** 2))
    return res


@pytest.mark.parametrize("M", [2, 3, 4])
def test_twa_matches_brute_force_fock_evolution(M):
    psi, C, n, times = _fock_case(M)
    nk, var, prob = fock.mode_occupations(psi, 1.0, 1.0, C, n, times, n_max=40)
    assert np.all(prob > 1 - 1e-9)
    worst_cl = 0.0
    for ti_, (m, se, v, sev, cl) in enumerate(_twa_nk(psi, C, n, times, 20000)):
        assert np.all(np.abs(m - nk[ti_]) < 3.5 * se), (ti_, m, nk[ti_], se)
        assert np.all(np.abs(v - var[ti_]) < 4.0 * sev), (ti_, v, var[ti_], sev)
        worst_cl = max(worst_cl, float(np.max(np.abs(cl - nk[ti_]) / se)))
    if M == 3:
        # the classical (mean-field) trajectory misses the quantum correction by many sigma
        assert worst_cl > 6.0


def test_paper_literal_noise_reading_disagrees_with_fock():
    psi, C, n, times = _fock_case(3, times=(0.0,))
    nk, _, _ = fock.mode_occupations(psi, 1.0, 1.0, C, n, times, n_max=40)
    m, se, _, _, _ = _twa_nk(psi, C, n, times, 20000, noise_conv=1)[0]
    assert np.all(np.abs(m - nk[0]) > 8 * se)       # off by +1/2 per mode


def test_kerr_ensemble_matches_closed_forms():
    z, lam, Ns = math.sqrt(20.0), 1.0, 200000
    # one "cell" with n dV = 1: psi is the mode amplitude itself
    alpha0 = twa.sample(np.array([z + 0j]), 13, Ns, 1.0, 1.0)[1:, 0]
    for th in (0.02, 0.05, 0.1):
        mc = kerr.twa_trajectory(alpha0, lam, th).mean()
        cf = kerr.twa_mean_closed_form(z, lam, th)
        se = math.sqrt(0.5 / Ns) * 3
        assert abs(mc - cf) < 4 * se
        ex = kerr.exact_mean(z, lam, th)
        mf = z * np.exp(-1j * lam * (abs(z) ** 2 - 1) * th)        # mean-field, no spread
        assert abs(cf - ex) < 0.25 * abs(mf - ex)


def test_q_physical_scaling():
    assert twa.q_physical(1e-3, 1e8, 1e98) == pytest.approx(1e-93)


@pytest.mark.parametrize("seed", [1, 2])
def test_early_growth_of_Q_is_quadratic(seed):
    # Sec. V.A: Q - Q(0) grows as t^2 at early times (Eq. DefinitionKappa's prefactor is garbled,
    # so only the exponent is pinned)
    g = ti.Grid.cube(1, 64)
    psi = ti.cosine_overdensity(g, 0.5)
    t, series, _ = twa.run(psi, 0.05, 4 * np.pi, 2e-3, 1.0, 1, 1e8, 400, seed, 60, 6, with_modes=False)
    q = np.array([s["Q"] for s in series])
    assert 1.7 < twa.stable_growth_exponent(t, q) < 2.3


def _cosine_field(M, n, eps, L=1.0):
    x = np.arange(M) * L / M
    return np.sqrt(1.0 + eps * np.cos(2 * np.pi * n * x / L)).astype(np.complex128)


def test_adaptive_dt_potential_bound_matches_the_cosine_closed_form():
    # rho = 1 + eps cos(k x)  ->  V = -C eps cos(k x) / k^2,  max|V| = C eps / k^2
    M, n, eps, C, hb, c_f = 64, 2, 0.3, 4 * np.pi, 1e-3, 0.1
    psi = _cosine_field(M, n, eps)
    k = 2 * np.pi * n
    expect_pot = 2 * np.pi * c_f * hb * k * k / (C * eps)
    kin = 2 * np.pi * c_f * (1.0 / M) / (np.pi * hb)
    assert expect_pot < kin
    got = twa.adaptive_dt(psi[None], hb, C, 1.0, 1, c_f)
    assert got == pytest.approx(expect_pot, rel=1e-12)


def test_adaptive_dt_kinetic_bound_is_the_gradient_aliasing_rule():
    # C = 0: only the kinetic bound; for c_f = 1/pi it is the footnote's 4 pi / (hbar k_max dk)
    hb, L = 0.0122, 2.0
    for shape in ((64,), (32, 64), (16, 32, 128)):
        psi = np.ones(shape, dtype=np.complex128)
        dx = min(L / m for m in shape)
        kmax, dk = np.pi / dx, 2 * np.pi / L
        got = twa.adaptive_dt(psi[None], hb, 0.0, L, len(shape), 1.0 / np.pi)
        assert got == pytest.approx(4 * np.pi / (hb * kmax * dk), rel=1e-12)


def test_adaptive_run_without_gravity_is_the_fixed_step_run():
    M, hb = 64, 1e-2
    psi = _cosine_field(M, 3, 0.2)
    psi /= np.sqrt(np.sum(np.abs(psi) ** 2) / M)
    dt = twa.adaptive_dt(psi[None], hb, 0.0, 1.0, 1, 0.05)
    ta, sa, ba, dts = twa.run_adaptive(psi, hb, 0.0, 1.0, 1, 1e4, 3, 11, 4, 5, 0.05)
    tf, sf, bf = twa.run(psi, hb, 0.0, dt, 1.0, 1, 1e4, 3, 11, 20, 5)
    assert dts == [dt] * 4
    assert np.allclose(ta, tf, rtol=0, atol=1e-15) and np.array_equal(ba, bf)


def test_adaptive_dt_shrinks_while_an_overdensity_collapses():
    M, hb, C = 128, 2e-3, 4 * np.pi
    x = np.arange(M) / M
    psi = np.sqrt(1 + 2.0 * np.exp(-(x - 0.5) ** 2 / (2 * 0.05 ** 2))).astype(np.complex128)
    psi /= np.sqrt(np.sum(np.abs(psi) ** 2) / M)
    _, _, _, dts = twa.run_adaptive(psi, hb, C, 1.0, 1, 1e6, 2, 5, 6, 20, 0.02)
    assert all(b <= a * (1 + 1e-12) for a, b in zip(dts, dts[1:])) and dts[-1] < 0.9 * dts[0]


def _weyl(n_tot, dV):
    return 1.0 / (2.0 * n_tot * dV)


def test_phase_variance_of_rotated_copies_is_the_variance_of_the_angles():
    # streams psi0 e^{i theta_s}: amplitudes equal (Var A = 0), dphi_s = theta_s - mean angle
    M, n_tot = 32, 1e6
    rng = np.random.default_rng(3)
    psi0 = (1.0 + 0.5 * rng.random(M)) * np.exp(1j * rng.uniform(0, 2 * np.pi, M))
    theta = np.array([-0.3, -0.1, 0.05, 0.15, 0.2])
    theta -= theta.mean()
    batch = np.concatenate([psi0[None], psi0[None] * np.exp(1j * theta)[:, None]])
    pm = twa.phase_moments(batch, n_tot, 1.0, 1)
    dV = 1.0 / M
    rho = np.abs(psi0) ** 2 - _weyl(n_tot, dV)
    assert pm["var_a"] == pytest.approx(0.0, abs=1e-12)
    # the mean field psi0 mean(e^{i theta}) sits at the phase of psi0 plus arg mean(e^{i theta})
    ref_phase = np.angle(np.mean(np.exp(1j * theta)))
    expect = np.sum(rho * np.mean((theta - ref_phase) ** 2)) * dV / (np.pi ** 2 / 3)
    assert pm["var_phi"] == pytest.approx(expect, rel=1e-12)


def test_amplitude_variance_of_scaled_copies():
    # streams c_s psi0 with real c_s > 0: phases equal, Var A = Var(c) |psi0|^2, <A> = mean(c) |psi0|
    M, n_tot = 16, 1e5
    psi0 = np.exp(1j * np.linspace(0, 1, M)) * (1 + np.arange(M) / M)
    c = np.array([0.8, 1.0, 1.1, 1.3])
    batch = np.concatenate([psi0[None], c[:, None] * psi0[None]])
    pm = twa.phase_moments(batch, n_tot, 2.0, 1)
    dV = 2.0 / M
    a2 = np.abs(psi0) ** 2
    rho = np.mean(c ** 2) * a2 - _weyl(n_tot, dV)
    expect = np.sum(rho * np.var(c) * a2 / (np.mean(c) * np.abs(psi0))) * dV
    assert pm["var_a"] == pytest.approx(expect, rel=1e-12)
    assert pm["var_phi"] == pytest.approx(0.0, abs=1e-20)


def test_fully_random_phase_gives_about_the_mass():
    # equally spaced phases about a vanishing mean field: <dphi^2> -> pi^2/3 (1 + 2/N^2)
    N, M, n_tot = 64, 8, 1e9
    phases = 2 * np.pi * (np.arange(N) + 0.5) / N - np.pi
    batch = np.concatenate([np.ones((1, M)), np.exp(1j * phases)[:, None] * np.ones((1, M))]).astype(np.complex128)
    pm = twa.phase_moments(batch, n_tot, 1.0, 1)
    mass = np.sum(np.mean(np.abs(batch[1:]) ** 2, 0) - _weyl(n_tot, 1.0 / M)) / M
    assert pm["var_phi"] == pytest.approx(mass, rel=2e-3)
