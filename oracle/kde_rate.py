"""Oracle of the KDE rate estimate of the keyframe RD loss (Sec. 3.3, Eq. of P_PMF): the
bits an entropy coder spends on the quantised symbols of one attribute channel, estimated
from a Gaussian kernel density of the channel's own symbols.  TEST INFRASTRUCTURE ONLY.

Readings (the paper names the ingredients - Silverman-rule bandwidth, the CDF of the kernel
density, PMF(y) = CDF(y + 1/2) - CDF(y - 1/2), rate = -mean log2 PMF - and computes the CDF
by FFT convolution on a grid):

* symbols s_i = round(y_i) (round half to even), i = 1..N, of one channel;
* bandwidth h = sigma (3 N / 4)^(-1/5), sigma the sample standard deviation of the symbols
  (ddof 1) - the normal-reference (Silverman) rule; h = 1 when sigma = 0;
* CDF(x) = (1/N) sum_i Phi((x - s_i) / h), Phi the standard normal CDF;
* PMF(k) = CDF(k + 1/2) - CDF(k - 1/2) for every integer k (exactly a convolution of the
  symbol histogram with the kernel w(d) = Phi((d + 1/2) / h) - Phi((d - 1/2) / h), which the
  paper evaluates with an FFT);
* rate = -(1/N) sum_i log2 max(PMF(s_i), 2^-40) bits per symbol.

Here everything is evaluated from that definition in FP64 (sums over the samples).
The training form (rate of noise-injected values and its gradient) follows below.
"""
import numpy as np
from scipy.special import ndtr

PMF_FLOOR = 2.0 ** -40


def symbols(y) -> np.ndarray:
    return np.rint(np.asarray(y, np.float64)).astype(np.int64)


def bandwidth(s) -> float:
    s = np.asarray(s, np.float64)
    n = s.shape[0]
    sd = float(np.std(s, ddof=1)) if n > 1 else 0.0
    return sd * (0.75 * n) ** (-0.2) if sd > 0 else 1.0


def pmf(s, k, h=None) -> np.ndarray:
    """PMF at the integers k from the symbols s (sums over every sample)."""
    s = np.asarray(s, np.float64)
    h = bandwidth(s) if h is None else h
    k = np.asarray(k, np.float64)
    out = np.zeros(k.shape)
    for j, kj in enumerate(k.reshape(-1)):
        out.reshape(-1)[j] = np.mean(ndtr((kj + 0.5 - s) / h) - ndtr((kj - 0.5 - s) / h))
    return out


def rate(y) -> float:
    """Bits per symbol of one channel."""
    s = symbols(y)
    vals, counts = np.unique(s, return_counts=True)
    p = pmf(s, vals)
    return float(-(counts * np.log2(np.maximum(p, PMF_FLOOR))).sum() / s.shape[0])


# --------------------------------------------------------------------------- training form
#
# Reading (Sec. 3.3, differentiable quantisation): during training the attribute values carry
# the injected uniform noise, y~_i = y_i + u_i (in units of the quantisation step; the caller
# draws u).  The density model is the kernel density of the symbols s_j = round(y~_j) above
# (the histogram the paper's FFT convolves), held fixed; the rate is evaluated at the
# continuous values:  R = -(1/N) sum_i log2 max(P(y~_i), 2^-40),  P(x) = CDF(x + 1/2) -
# CDF(x - 1/2).  The gradient flows through the evaluation points only:
#   dR/dy~_i = -(1/(N ln 2)) (pdf(y~_i + 1/2) - pdf(y~_i - 1/2)) / P(y~_i)   (0 at the floor),
#   pdf(x) = (1/(N h)) sum_j phi((x - s_j) / h).
# For integer inputs R equals rate() above.


def pmf_at(s, x, h=None) -> np.ndarray:
    """P(x) = CDF(x + 1/2) - CDF(x - 1/2) at real points x (sums over every sample)."""
    s = np.asarray(s, np.float64)
    h = bandwidth(s) if h is None else h
    vals, counts = np.unique(s, return_counts=True)
    x = np.asarray(x, np.float64).reshape(-1)
    out = np.empty(x.shape)
    for i, xi in enumerate(x):
        out[i] = np.sum(counts * (ndtr((xi + 0.5 - vals) / h) - ndtr((xi - 0.5 - vals) / h))) / s.shape[0]
    return out


def pdf_at(s, x, h=None) -> np.ndarray:
    """pdf(x) = (1/(N h)) sum_j phi((x - s_j) / h) at real points x."""
    s = np.asarray(s, np.float64)
    h = bandwidth(s) if h is None else h
    vals, counts = np.unique(s, return_counts=True)
    x = np.asarray(x, np.float64).reshape(-1)
    out = np.empty(x.shape)
    for i, xi in enumerate(x):
        z = (xi - vals) / h
        out[i] = np.sum(counts * np.exp(-0.5 * z * z)) / (np.sqrt(2.0 * np.pi) * h * s.shape[0])
    return out


def rate_continuous(y) -> float:
    """R of the training form: the symbols' density evaluated at the continuous values."""
    y = np.asarray(y, np.float64)
    s = symbols(y)
    p = pmf_at(s, y)
    return float(-np.log2(np.maximum(p, PMF_FLOOR)).sum() / y.shape[0])


def rate_continuous_grad(y) -> np.ndarray:
    """dR/dy~_i of the training form, density held fixed."""
    y = np.asarray(y, np.float64)
    s = symbols(y)
    n = y.shape[0]
    p = pmf_at(s, y)
    dp = pdf_at(s, y + 0.5) - pdf_at(s, y - 0.5)
    g = -dp / (np.maximum(p, PMF_FLOOR) * n * np.log(2.0))
    return np.where(p > PMF_FLOOR, g, 0.0)
