"""Pins of the oracle's noise statistics (Sec. 4.5, calculation of mean and standard
deviation): level statistics without rejection are the textbook mean and deviation
of the decimated series; with iterated 2-sigma rejection on Gaussian noise they
converge to the closed-form fixed point of the truncated normal; outliers are
removed; the per-width table reproduces Eq. whitenoise for white noise and the
level values at powers of two."""
import math

import numpy as np
import pytest
from scipy import optimize, stats

import oracle
import spd_synth


def _decimate(x, k):
    B = 1 << k
    n = x.shape[1] // B
    return x[:, : n * B].reshape(x.shape[0], n, B).sum(axis=2)


def test_no_rejection_is_plain_mean_and_deviation():
    x = spd_synth.gaussian_noise(3, 10007, 11, mu=0.7, sigma=2.5, dtype=np.float64)
    mu, sg, n = oracle.msd_levels(x, 8, thr=0.0)
    for k in range(8):
        d = _decimate(x, k)
        assert np.array_equal(n[:, k], np.full(3, d.shape[1]))
        assert np.allclose(mu[:, k], d.mean(axis=1), rtol=1e-12, atol=1e-12)
        assert np.allclose(sg[:, k], d.std(axis=1), rtol=1e-12)


def _fixed_point(thr):
    # s = sd of N(0,1) truncated to |v| <= thr * s  (the iteration's limit)
    def g(s):
        c = thr * s
        var = 1.0 - 2.0 * c * stats.norm.pdf(c) / (2.0 * stats.norm.cdf(c) - 1.0)
        return math.sqrt(var) - s
    return optimize.brentq(g, 0.1, 1.0)


def test_rejection_converges_to_truncated_normal_fixed_point():
    x = spd_synth.gaussian_noise(2, 1 << 22, 12, dtype=np.float64)
    mu, sg, n = oracle.msd_levels(x, 5, thr=2.0, max_passes=50)
    s_star = _fixed_point(2.0)  # ~0.77 for a 2-sigma cut
    for k in range(5):
        sd_true = math.sqrt(1 << k)
        nv = (1 << 22) >> k
        assert np.all(np.abs(sg[:, k] / sd_true - s_star) < 6.0 / math.sqrt(nv)), (k, sg[:, k] / sd_true, s_star)
        assert np.all(np.abs(mu[:, k] / sd_true) < 6.0 / math.sqrt(nv))
        # kept fraction = P(|v| <= thr * s*)
        frac = n[:, k] / nv
        assert np.all(np.abs(frac - (2 * stats.norm.cdf(2 * s_star) - 1)) < 6.0 / math.sqrt(nv))


def test_outliers_are_rejected():
    x = spd_synth.gaussian_noise(1, 1 << 20, 13, dtype=np.float64)
    spikes = np.random.default_rng(13).choice(1 << 20, 5000, replace=False)
    x[0, spikes] += 50.0
    mu0, sg0, _ = oracle.msd_levels(x, 1, thr=0.0)
    mu, sg, n = oracle.msd_levels(x, 1, thr=3.0, max_passes=50)
    assert sg0[0, 0] > 3.0  # the spikes inflate the plain deviation
    assert abs(sg[0, 0] - _fixed_point(3.0)) < 0.01 and abs(mu[0, 0]) < 0.01
    assert n[0, 0] <= (1 << 20) - 5000


def test_constant_series_and_short_rows():
    x = np.full((2, 100), 3.0)
    mu, sg, n = oracle.msd_levels(x, 8, thr=2.0)
    for k in range(8):
        nv = 100 >> k
        assert np.all(n[:, k] == nv)
        if nv:
            assert np.all(mu[:, k] == 3.0 * (1 << k)) and np.all(sg[:, k] == 0.0)
        else:
            assert np.all(mu[:, k] == 0.0) and np.all(sg[:, k] == 0.0)


def test_table_white_law_and_levels_at_powers_of_two():
    x = spd_synth.gaussian_noise(2, 1 << 18, 14, mu=0.3, sigma=1.7, dtype=np.float64)
    mu, sg, n = oracle.msd_levels(x, 10, thr=0.0)
    widths = np.array([1, 2, 3, 5, 8, 12, 100, 512, 700, 4000], np.int32)
    tm, ts = oracle.msd_table(mu, sg, n, widths)
    for w_i, L in enumerate(widths):
        if L & (L - 1) == 0:
            k = int(L).bit_length() - 1
            assert np.allclose(tm[:, w_i], mu[:, k], rtol=1e-12)
            assert np.allclose(ts[:, w_i], sg[:, k], rtol=1e-12)
    # white noise: mu_L = L mu, sigma_L = sqrt(L) sigma (Eq. whitenoise), within sampling error
    assert np.allclose(tm / widths, 0.3, atol=0.05)
    assert np.allclose(ts / np.sqrt(widths), 1.7, rtol=0.05)
    # exactly white level statistics give the white law at every width, beyond the last level too
    lm = 0.3 * (1 << np.arange(10))[None, :].repeat(2, 0)
    ls = 1.7 * np.sqrt(1 << np.arange(10))[None, :].repeat(2, 0)
    tm, ts = oracle.msd_table(lm, ls, np.full((2, 10), 100), widths)
    assert np.allclose(tm, 0.3 * widths, rtol=1e-12) and np.allclose(ts, 1.7 * np.sqrt(widths), rtol=1e-12)
