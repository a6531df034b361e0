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


# ---- training form: noise-injected values, density of their symbols held fixed

def test_training_rate_equals_symbol_rate_on_integers():
    rng = np.random.default_rng(3)
    for sigma in (0.6, 5.0, 30.0):
        y = np.rint(rng.normal(-2.0, sigma, 800))
        assert abs(kr.rate_continuous(y) - kr.rate(y)) < 1e-12


def test_training_gradient_matches_central_differences():
    """Moving one value by +-1e-5 (away from a rounding boundary) keeps every symbol and h,
    so only that value's own term -log2 P(y_i) / N changes: its difference quotient is the
    fixed-density derivative.  A full-rate difference quotient agrees too, to its rounding."""
    rng = np.random.default_rng(4)
    for sigma, n in ((0.7, 400), (6.0, 600), (25.0, 500)):
        y = rng.normal(1.0, sigma, n) + rng.uniform(-0.5, 0.5, n)
        s = kr.symbols(y)
        g = kr.rate_continuous_grad(y)
        frac = np.abs(y - np.floor(y) - 0.5)
        for i in np.flatnonzero(frac > 0.01)[:12]:
            e = 1e-5
            pp, pm = kr.pmf_at(s, [y[i] + e, y[i] - e])
            fd = -(np.log2(pp) - np.log2(pm)) / (2 * e * n)
            assert abs(fd - g[i]) <= 1e-6 * abs(g[i]) + 1e-13, (sigma, i, fd, g[i])
            yp, ym = y.copy(), y.copy()
            yp[i] += e
            ym[i] -= e
            fd_all = (kr.rate_continuous(yp) - kr.rate_continuous(ym)) / (2 * e)
            assert abs(fd_all - g[i]) <= 1e-4 * abs(g[i]) + 1e-10, (sigma, i, fd_all, g[i])


def test_training_constant_channel_closed_form():
    """All values round to 7: sigma = 0, h = 1, P(x) = Phi(x - 6.5) - Phi(x - 7.5)."""
    rng = np.random.default_rng(5)
    y = 7.0 + rng.uniform(-0.45, 0.45, 300)
    n = y.shape[0]
    norm = scipy.stats.norm
    p = norm.cdf(y - 6.5) - norm.cdf(y - 7.5)
    want_r = float(-np.log2(p).mean())
    want_g = -(norm.pdf(y - 6.5) - norm.pdf(y - 7.5)) / (p * n * math.log(2.0))
    assert abs(kr.rate_continuous(y) - want_r) < 1e-12
    assert np.allclose(kr.rate_continuous_grad(y), want_g, rtol=1e-10, atol=1e-15)


def test_training_gradient_points_away_from_the_mode():
    """For a unimodal channel the rate rises as a value moves into the tail: the gradient has
    the sign of (value - mode) for values clearly off the mode."""
    rng = np.random.default_rng(6)
    y = rng.normal(0.0, 8.0, 4000) + rng.uniform(-0.5, 0.5, 4000)
    g = kr.rate_continuous_grad(y)
    far = np.abs(y) > 6.0
    assert np.all(np.sign(g[far]) == np.sign(y[far]))
