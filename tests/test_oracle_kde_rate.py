"""Pins of the oracle's KDE rate estimate (Sec. 3.3: Silverman-rule kernel density of a
channel's quantised symbols, PMF(y) = CDF(y + 1/2) - CDF(y - 1/2), rate = -mean log2 PMF).

* the PMF equals scipy.stats.gaussian_kde with the 'silverman' bandwidth integrated over
  [k - 1/2, k + 1/2] (the library's own kernel density);
* the PMF sums to one over the integers;
* a constant channel (sigma = 0, h = 1) has the closed form -log2(Phi(1/2) - Phi(-1/2));
* the rate is a cross-entropy: never below the empirical entropy of the symbols, and for a
  wide discretised normal within a few hundredths of a bit of it and of the differential
  entropy 1/2 log2(2 pi e sigma^2).
"""
import math

import numpy as np
import scipy.stats

from oracle import kde_rate as kr


def test_pmf_equals_scipy_gaussian_kde():
    rng = np.random.default_rng(0)
    for sigma, n in ((0.7, 400), (6.0, 1000), (25.0, 700)):
        y = rng.normal(3.0, sigma, n) + rng.uniform(-0.5, 0.5, n)
        s = kr.symbols(y)
        kde = scipy.stats.gaussian_kde(s.astype(np.float64), bw_method="silverman")
        ks = np.arange(s.min() - 3, s.max() + 4)
        want = np.array([kde.integrate_box_1d(k - 0.5, k + 0.5) for k in ks])
        got = kr.pmf(s, ks)
        assert np.allclose(got, want, rtol=1e-10, atol=1e-14), sigma


def test_pmf_sums_to_one():
    rng = np.random.default_rng(1)
    s = kr.symbols(rng.gamma(2.0, 5.0, 3000))
    h = kr.bandwidth(s)
    ks = np.arange(s.min() - int(12 * h) - 2, s.max() + int(12 * h) + 3)
    assert abs(kr.pmf(s, ks).sum() - 1.0) < 1e-12


def test_constant_channel_closed_form():
    y = np.full(500, 7.2)
    want = -math.log2(scipy.stats.norm.cdf(0.5) - scipy.stats.norm.cdf(-0.5))
    assert abs(kr.rate(y) - want) < 1e-12
    assert kr.bandwidth(kr.symbols(y)) == 1.0


def test_rate_is_a_cross_entropy():
    rng = np.random.default_rng(2)
    for sigma in (0.8, 3.0, 20.0):
        s = kr.symbols(rng.normal(0.0, sigma, 20000))
        _, c = np.unique(s, return_counts=True)
        p = c / c.sum()
        h_emp = float(-(p * np.log2(p)).sum())
        r = kr.rate(s)
        assert r >= h_emp - 1e-9, sigma
        if sigma >= 20.0:
            assert r - h_emp < 0.02
            assert abs(r - 0.5 * math.log2(2 * math.pi * math.e * sigma ** 2)) < 0.03
