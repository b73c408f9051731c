"""Tolerances of the source-update statistics (Q_i, eps_i^2, W_l) derived from the residuals.

Q_i, eps_i^2 and W_l are functions of the residuals R_l of a source (Sect. 5.1.2, Eqs. Qi, dw,
epsi).  Two implementations that evaluate the FP64 model with different arithmetic give
residuals that differ by delta_l (the residual parity floor, ~1e-16 rad, relative to sigma ~5e-10
rad: ~2e-7 per observation).  These bounds propagate the measured delta_l to first order,
with s_l^2 = sigma_l^2 + eps_i^2 and z_l = R_l / s_l:

  * a weight w(z) changes by |dw| <= 1.6 w |dz|: |d ln w / dz| is at most 1.54 on the cubic join of
    Eq. dw (largest near |z| = 2.7), 1/3 on its exponential tail and below 0.2 for Eq. dwH;
  * Q = sum w R^2 / s^2 changes through the residuals and the weights by at most
    S1 = sum_l w_l (2 |z_l| + 1.6 z_l^2) delta_l / s_l;
  * eps^2 = y solves Q(y) = nu (the rational steps of Eq. epsi); the implicit change is
    |dy| <= S1 / S2 with S2 = -Q'(y) = sum_l w_l z_l^2 / s_l^2; with y = 0 (no excess noise)
    only Q moves;
  * W_l = w_l / s_l^2 changes by |dW / W| <= 1.6 (delta_l / s_l + |z_l| |dy| / (2 s_l^2)) + |dy| / s_l^2.

Each bound is taken three times over (the weights of a round come from the residuals of the
previous round, whose differences are of the same size), plus 1e-12 relative for the rounding of
the sums and of the rational steps themselves.
"""
import numpy as np

D_LN_W = 1.6
SAFETY = 3.0
FLOOR = 1e-12


def stat_tolerances(src, n_src, sigma, R_ref, R_test, W_ref, eps2_ref, Q_ref):
    """Per-source tolerances of Q and eps^2 (absolute) and per-observation tolerance of W
    (absolute), from the reference statistics and the measured residual differences."""
    src = np.asarray(src)
    s2 = np.asarray(sigma, dtype=np.float64) ** 2 + np.asarray(eps2_ref)[src]
    s = np.sqrt(s2)
    w = np.asarray(W_ref) * s2                     # the downweighting factor w_l
    z = np.asarray(R_ref) / s
    dl = np.abs(np.asarray(R_test) - np.asarray(R_ref)) / s
    S1 = np.bincount(src, w * (2 * np.abs(z) + D_LN_W * z * z) * dl, minlength=n_src)
    S2 = np.bincount(src, w * z * z / s2, minlength=n_src)
    dy = np.where(S2 > 0, S1 / np.where(S2 > 0, S2, 1.0), 0.0)
    dy = np.where(np.asarray(eps2_ref) > 0, dy, 0.0)
    tol_Q = SAFETY * S1 * (1.0 + (np.asarray(eps2_ref) > 0)) + FLOOR * np.abs(Q_ref)
    s2min = np.full(n_src, np.inf)
    np.minimum.at(s2min, src, s2)
    s2min = np.where(np.isfinite(s2min), s2min, 0.0)
    tol_eps2 = SAFETY * dy + FLOOR * s2min
    dyl = dy[src]
    rel_W = SAFETY * (D_LN_W * (dl + np.abs(z) * dyl / (2 * s2)) + dyl / s2) + FLOOR
    tol_W = rel_W * np.abs(np.asarray(W_ref))
    return tol_Q, tol_eps2, tol_W


def assert_stats_close(src, n_src, sigma, R_ref, R_test, W_ref, W_test, eps2_ref, eps2_test, Q_ref, Q_test,
                       what=""):
    tol_Q, tol_eps2, tol_W = stat_tolerances(src, n_src, sigma, R_ref, R_test, W_ref, eps2_ref, Q_ref)
    for name, ref, test, tol in (("W", W_ref, W_test, tol_W), ("Q", Q_ref, Q_test, tol_Q),
                                 ("eps2", eps2_ref, eps2_test, tol_eps2)):
        d = np.abs(np.asarray(test) - np.asarray(ref))
        ok = d <= tol
        if not ok.all():
            i = int(np.argmax(d - tol))
            raise AssertionError(f"{what}{name}: {int((~ok).sum())} off; worst at {i}: |diff| {d[i]:.3e} "
                                 f"> tol {tol[i]:.3e} (value {np.asarray(ref)[i]:.6e})")
    # how tight the bounds are, for the record
    return {"W": float(np.max(np.abs(np.asarray(W_test) - W_ref) / np.maximum(tol_W, 1e-300))),
            "Q": float(np.max(np.abs(np.asarray(Q_test) - Q_ref) / np.maximum(tol_Q, 1e-300))),
            "eps2": float(np.max(np.abs(np.asarray(eps2_test) - eps2_ref) / np.maximum(tol_eps2, 1e-300)))}


def chi2_tolerance(R_ref, R_test, W_ref, tol_W):
    """Bound on |chi2_test - chi2_ref| for chi2 = sum W R^2 from the measured residual differences
    and the weight tolerances above."""
    R = np.abs(np.asarray(R_ref))
    dR = np.abs(np.asarray(R_test) - np.asarray(R_ref))
    W = np.abs(np.asarray(W_ref))
    return float(np.sum(tol_W * R * R + W * (2 * R * dR + dR * dR)) + FLOOR * np.sum(W * R * R))
