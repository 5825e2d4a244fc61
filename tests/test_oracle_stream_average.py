"""Pins of the oracle's stream average (Appendix B's synthesizer: averages of arbitrary functions of
the streams' fields, per cell or mode and in total, applied to every stream or to the mean field):
brute-force loops with an explicit DFT on a tiny batch, the antithetic-streams closed form, and
Parseval's relation between the position-space and mode-space totals."""
import cmath
import math

import numpy as np
import pytest

from oracle import twa


def _tiny_batch(shape, n_slots, seed):
    rng = np.random.default_rng(seed)
    return rng.normal(size=(n_slots,) + shape) + 1j * rng.normal(size=(n_slots,) + shape)


def _brute(batch, fz, L, n_tot, of_mean, modes):
    """Pure-Python loops: the DFT as an explicit sum, then the average over slots 1.."""
    n_slots = batch.shape[0]
    shape = batch.shape[1:]
    dim = len(shape)
    cells = int(np.prod(shape))
    dV = L ** dim / cells
    flat = [list(batch[s].reshape(-1)) for s in range(n_slots)]
    if modes:
        idx = list(np.ndindex(*shape))
        amp = math.sqrt(n_tot * dV / cells)
        tr = []
        for s in range(n_slots):
            out = []
            for k in idx:
                acc = 0j
                for xi, x in enumerate(idx):
                    ph = sum(k[a] * x[a] / shape[a] for a in range(dim))
                    acc += flat[s][xi] * cmath.exp(-2j * math.pi * ph)
                out.append(amp * acc)
            tr.append(out)
        flat = tr
    per = []
    for c in range(cells):
        if of_mean:
            m = sum(flat[s][c] for s in range(1, n_slots)) / (n_slots - 1)
            per.append(fz(m, c, cells))
        else:
            per.append(sum(fz(flat[s][c], c, cells) for s in range(1, n_slots)) / (n_slots - 1))
    cl = [fz(flat[0][c], c, cells) for c in range(cells)]
    total = sum(per) * (1.0 if modes else dV)
    return np.array(per).reshape(shape), np.array(cl).reshape(shape), total


FUNCS = [
    (lambda re, im, i, n: re * re + im * im, lambda z, c, n: abs(z) ** 2),
    (lambda re, im, i, n: np.arctan2(im, re) + 1j * np.sqrt(re * re + im * im) * (i % 3),
     lambda z, c, n: math.atan2(z.imag, z.real) + 1j * abs(z) * (c % 3)),
    (lambda re, im, i, n: (re + 1j * im) ** 2 * n, lambda z, c, n: z * z * n),
]


@pytest.mark.parametrize("shape", [(6,), (4, 3), (2, 3, 2)])
@pytest.mark.parametrize("of_mean", [False, True])
@pytest.mark.parametrize("modes", [False, True])
@pytest.mark.parametrize("fi", range(len(FUNCS)))
def test_stream_average_matches_brute_force_loops(shape, of_mean, modes, fi):
    f, fz = FUNCS[fi]
    batch = _tiny_batch(shape, 4, 11 + fi)
    L, n_tot = 1.7, 3.0e4
    got = twa.stream_average(batch, f, n_tot, L, len(shape), of_mean=of_mean, modes=modes)
    per, cl, total = _brute(batch, fz, L, n_tot, of_mean, modes)
    scale = max(1.0, np.abs(per).max(), np.abs(cl).max())
    assert np.allclose(got["per_cell"], per, rtol=0, atol=1e-12 * scale)
    assert np.allclose(got["f_cl"], cl, rtol=0, atol=1e-12 * scale)
    assert abs(got["total"] - total) <= 1e-12 * max(1.0, abs(total))


def test_antithetic_streams_give_the_classical_mean_and_its_density_plus_the_noise():
    rng = np.random.default_rng(5)
    cl = rng.normal(size=(8, 8)) + 1j * rng.normal(size=(8, 8))
    d = 0.1 * (rng.normal(size=(3, 8, 8)) + 1j * rng.normal(size=(3, 8, 8)))
    batch = np.concatenate([cl[None], cl + d, cl - d])     # streams psi_cl +- d_j
    mean = twa.stream_average(batch, lambda re, im, i, n: re + 1j * im, 1e6, 1.0, 2, of_mean=True)
    assert np.allclose(mean["per_cell"], cl, atol=1e-14)
    rho = twa.stream_average(batch, lambda re, im, i, n: re * re + im * im, 1e6, 1.0, 2)
    assert np.allclose(rho["per_cell"], np.abs(cl) ** 2 + (np.abs(d) ** 2).mean(0), rtol=1e-13)
    assert np.allclose(rho["f_cl"], np.abs(cl) ** 2, rtol=1e-14)


def test_mode_total_of_the_occupation_is_the_particle_number():
    """Parseval: sum_k |a_k|^2 = n_tot dV sum_x |psi|^2, per stream and hence on average."""
    batch = _tiny_batch((16, 8), 5, 3)
    n_tot, L = 2.5e5, 2.0
    occ = twa.stream_average(batch, lambda re, im, i, n: re * re + im * im, n_tot, L, 2, modes=True)
    dens = twa.stream_average(batch, lambda re, im, i, n: re * re + im * im, n_tot, L, 2)
    assert abs(occ["total"] - n_tot * dens["total"]) <= 1e-12 * abs(occ["total"])
