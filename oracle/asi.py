"""Accelerated simple iteration (ASI, Sect. 4.7), FP64 (TEST INFRASTRUCTURE ONLY).

Once the simple iteration has run for a while its updates keep their direction and shrink by
a nearly constant ratio, d^(k+1) ~ lambda d^(k): the slowest eigenvector of the iteration
matrix dominates and lambda is its eigenvalue.  The updates still to come then sum to the
geometric series d^(k+1) (1 + lambda + lambda^2 + ...) = d^(k+1) / (1 - lambda), and ASI
applies that factor in iteration k+1.  The paper estimates lambda statistically from the
parallax updates of a small fraction of the sources (a change of the frame orientation
between iterations leaves the parallaxes alone).

Readings where the paper leaves the details open:
  sample     the sources i = 0, m, 2m, ... (m = stride)
  estimate   the lower median of the ratios d_varpi,i^(k+1) / d_varpi,i^(k) of the plain
             S-block updates of the last two iterations, sources with a zero previous update
             or a non-finite ratio skipped; clamped to [0, lambda_max]
  factor     applied to the source update of the S block only; the A and C blocks then solve
             against the extrapolated sources, reading the residuals corrected to first
             order (R - A c for a source correction c).  For two blocks iterated in
             Gauss-Seidel order this removes the slowest error component exactly, while
             extrapolating both blocks overshoots (tests/test_oracle_asi.py shows both).

Pins: tests/test_oracle_asi.py (the estimator on hand-worked samples; the two-block linear
system solved exactly by one accelerated step; the first-order residual correction against
residuals re-evaluated at the corrected sources).
"""
import numpy as np

from . import agis as G


def lambda_estimate(d_prev, d_cur, stride, lam_max):
    """(median, lambda, factor 1/(1 - lambda), number of ratios) from two [n_src, 5] updates."""
    idx = np.arange(0, np.asarray(d_cur).shape[0], stride)
    d0 = np.asarray(d_prev, dtype=np.float64)[idx, 2]
    d1 = np.asarray(d_cur, dtype=np.float64)[idx, 2]
    with np.errstate(divide="ignore", invalid="ignore"):
        r = np.where(d0 != 0.0, d1 / np.where(d0 != 0.0, d0, 1.0), np.nan)
    r = np.sort(r[(d0 != 0.0) & np.isfinite(r)])
    if r.size == 0:
        return 0.0, 0.0, 1.0, 0
    med = float(r[(r.size - 1) // 2])
    lam = min(max(med, 0.0), lam_max)
    return med, lam, 1.0 / (1.0 - lam), int(r.size)


def correction(d, factor):
    """The part of the extrapolated update f d that the S block has not applied: (f - 1) d."""
    return (factor - 1.0) * np.asarray(d, dtype=np.float64)


def apply_to_sources(src, c):
    """src + c in tangent units (alpha* turned into alpha with cos(delta) of src), as the S
    block applies its own update (footnote to Eq. ubardiff)."""
    out = np.array(src, dtype=np.float64, copy=True)
    out[:, 0] += c[:, 0] / np.cos(out[:, 1])
    out[:, 1:] += c[:, 1:]
    return out


def corrected_residuals(P, R, A, c):
    """R_l - A_l c_i for every observation l of source i; A = design rows -dR/ds'."""
    return np.asarray(R) - np.einsum("lk,lk->l", A, np.asarray(c)[P.src])


def iterate(P, state, st, n_iter, stride, lam_max, ref=None, d_prev=None):
    """n_iter accelerated iterations.  d_prev: the plain S-block update of the iteration
    before the first (None: the first iteration is a plain one).  Returns (state, per-iteration
    list of (IterStats, (median, lambda, factor, count) or None, plain S-block update d),
    the last plain update)."""
    out = []
    for _ in range(n_iter):
        est = [None]

        def after_s(src1, sres, ev, d_prev=d_prev):
            if d_prev is None:
                return src1, sres.R
            e = lambda_estimate(d_prev, sres.d, stride, lam_max)
            est[0] = e
            c = correction(sres.d, e[2])
            return apply_to_sources(src1, c), corrected_residuals(P, sres.R, ev["A"], c)

        state, stats, sres = G.iterate_once(P, state, st, ref=ref, after_s=after_s)
        d_prev = sres.d
        out.append((stats, est[0], sres.d))
    return state, out, d_prev
