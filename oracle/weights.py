"""Robust weighting of the source update, Sect. 5.1.2."""
import numpy as np


def w_agis(z):
    """Downweighting factor w(z), Eq. dw: 1 for |z| <= 2, cubic join for 2 <= |z| < 3,
    exp(-|z|/3) beyond (t = |z| - 2)."""
    a = np.abs(np.asarray(z, dtype=np.float64))
    t = a - 2.0
    return np.where(a <= 2.0, 1.0,
                    np.where(a < 3.0, 1.0 - 1.773735 * t * t + 1.141615 * t * t * t, np.exp(-a / 3.0)))


def w_huber(z, c=2.0):
    """Huber weight, Eq. dwH."""
    a = np.abs(np.asarray(z, dtype=np.float64))
    with np.errstate(divide="ignore", invalid="ignore"):
        return np.where(a <= c, 1.0, c * (2.0 * a - c) / (a * a))


def intersextile_half_range(x):
    """Robust standard deviation: half the range between the 1/6 and 5/6 quantiles (Sect. 5.1.2).

    Quantile definition (a reading; the paper does not fix it): linear interpolation between
    order statistics at position p*(n-1) (Hyndman-Fan type 7).
    """
    x = np.sort(np.asarray(x, dtype=np.float64))
    n = x.size
    if n == 0:
        return 0.0

    def q(p):
        h = p * (n - 1)
        lo = int(np.floor(h))
        hi = min(lo + 1, n - 1)
        return x[lo] + (h - lo) * (x[hi] - x[lo])
    return 0.5 * (q(5.0 / 6.0) - q(1.0 / 6.0))
