"""Host logic of the surrogate's fallback rule (no GPU): the disagreement statistic between the
surrogate's correction and the few-stream estimate, the threshold calibrated on validation samples,
and the decision."""
import numpy as np
import pytest

from paper_2310_07119_gb300 import fno

G, NB = 8, 6


def _spectrum(rng, scale=1.0):
    return scale * (1.0 + rng.random(G ** 3))


def test_statistic_is_zero_for_agreement_and_scale_free():
    rng = np.random.default_rng(0)
    est = _spectrum(rng)
    assert fno.fallback_statistic(est, est, G, NB) == 0.0
    pred = est * 1.1
    s1 = fno.fallback_statistic(pred, est, G, NB)
    s2 = fno.fallback_statistic(1e3 * pred, 1e3 * est, G, NB)
    assert s1 == pytest.approx(0.1, rel=1e-12) and s2 == pytest.approx(s1, rel=1e-12)


def test_calibrated_threshold_flags_outliers_only():
    rng = np.random.default_rng(1)
    val = []
    for _ in range(200):
        est = _spectrum(rng)
        val.append(fno.fallback_statistic(est * (1 + 0.05 * rng.standard_normal(est.size)), est, G, NB))
    tau = fno.calibrate_fallback(val, 0.9)
    assert np.mean(np.asarray(val) > tau) == pytest.approx(0.1, abs=0.01)
    est = _spectrum(rng)
    good = est * (1 + 0.01 * rng.standard_normal(est.size))
    corr, fell = fno.correct_or_fallback(good, est, G, NB, tau)
    assert not fell and corr is good
    corr, fell = fno.correct_or_fallback(2.0 * est, est, G, NB, tau)
    assert fell and corr is None
    corr, fell = fno.correct_or_fallback(np.full_like(est, np.nan), est, G, NB, tau)
    assert fell


def test_calibration_rejects_empty_or_nonfinite():
    with pytest.raises(ValueError):
        fno.calibrate_fallback([], 0.9)
    with pytest.raises(ValueError):
        fno.calibrate_fallback([0.1, float("nan")], 0.9)
