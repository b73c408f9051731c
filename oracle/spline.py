"""B-splines, App. B of the paper.

Knots are int64 nanoseconds; differences are formed in integers before being
converted to float64, so that long missions keep nanosecond resolution.
"""
import numpy as np


def uniform_knots(knot0_ns, dt_ns, n_coef, M=4):
    """Regular knot sequence with M-fold end knots (App. B.3): tau_0..tau_{M-1} = t_beg,
    tau_{N}..tau_{N+M-1} = t_end, and N-M+1 regular intervals in between."""
    K = n_coef - M + 1
    k = np.arange(n_coef + M, dtype=np.int64) - (M - 1)
    k = np.clip(k, 0, K)
    return np.int64(knot0_ns) + k * np.int64(dt_ns)


def left_index(knots, t_ns, n_coef, M=4):
    """Left index l with tau_l <= t < tau_{l+1}, restricted to M-1 <= l <= N-1 (Sect. 3.3;
    t = tau_N belongs to the last interval)."""
    t_ns = np.asarray(t_ns, dtype=np.int64)
    l = np.searchsorted(knots, t_ns, side="right") - 1
    return np.clip(l, M - 1, n_coef - 1)


def deboor(knots, t_ns, l, M=4):
    """Algorithm B.1: the M non-zero B-splines b_j = B_{l-M+1+j}(t), j = 0..M-1.

    Vectorised over t (and l).  R_i = tau_{l+i+1} - t and L_i = t - tau_{l-i}.
    """
    t_ns = np.asarray(t_ns, dtype=np.int64)
    l = np.asarray(l, dtype=np.int64)
    shape = t_ns.shape
    b = np.zeros(shape + (M,))
    b[..., 0] = 1.0
    R = np.zeros(shape + (M - 1,))
    L = np.zeros(shape + (M - 1,))
    for i in range(M - 1):
        R[..., i] = (knots[l + i + 1] - t_ns).astype(np.float64)
        L[..., i] = (t_ns - knots[l - i]).astype(np.float64)
        s = np.zeros(shape)
        for j in range(i + 1):
            u = b[..., j] / (R[..., j] + L[..., i - j])
            b[..., j] = s + R[..., j] * u
            s = L[..., i - j] * u
        b[..., i + 1] = s
    return b


def cox_deboor(knots, t_ns, n, M=4):
    """B_n(t) of order M by the Cox-de Boor recursion (textbook definition, used as a pin
    for Algorithm B.1); 0/0 is taken as 0."""
    t = np.asarray(t_ns, dtype=np.int64)

    def rec(j, k):
        if k == 1:
            return ((knots[j] <= t) & (t < knots[j + 1])).astype(np.float64)
        d1 = float(knots[j + k - 1] - knots[j])
        d2 = float(knots[j + k] - knots[j + 1])
        out = np.zeros(t.shape)
        if d1 > 0:
            out = out + (t - knots[j]).astype(np.float64) / d1 * rec(j, k - 1)
        if d2 > 0:
            out = out + (knots[j + k] - t).astype(np.float64) / d2 * rec(j + 1, k - 1)
        return out
    return rec(n, M)


def uniform_cubic(u):
    """Closed form of the four cubic B-splines on a regular knot interval, u in [0, 1)
    (used as a pin for Algorithm B.1)."""
    u = np.asarray(u, dtype=np.float64)
    v = 1.0 - u
    return np.stack([v ** 3 / 6, (3 * u ** 3 - 6 * u ** 2 + 4) / 6, (-3 * u ** 3 + 3 * u ** 2 + 3 * u + 1) / 6,
                     u ** 3 / 6], axis=-1)
