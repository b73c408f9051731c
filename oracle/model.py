"""Observation model, residuals and partial derivatives (FP64).

Follows Sects. 3.2 (astrometric model), 3.3 (attitude model), 3.4 (geometric
instrument model), 3.6 (synthesis model) and the partial derivatives of
Sects. 5.1.3 and 5.2.3-5.2.4.  Readings where the paper is silent:
  * the proper direction is the standard model (Eq. astro-standard) with the
    Roemer delay (Eq. roemer) followed by classical aberration (Eq. classAberr);
    no light deflection and no global parameters;
  * only five source parameters are unknowns, mu_r = 0 (Sect. 3.2);
  * the barycentric ephemeris is a circular 1-AU orbit in the ecliptic turned to
    ICRS by the obliquity (auxiliary data h);
  * the field index f of an observation is the one recorded with it; the
    computed sign(phi) of Eq. srspropeta agrees for every valid observation;
  * calibration: one AL offset per (field, AF CCD, day) and one AC offset per
    (field, AC row, day) -- the r = 0 terms of Eq. etazeta with g = 0;
  * the attitude partials include the factor 1/||s|| of the normalisation in
    Eq. qspline: dR/da_n = dR/dq B_n / ||s||, which is exact because dR/dq is
    orthogonal to q (it equals Eq. dfadq when ||s|| = 1).
"""
from dataclasses import dataclass

import numpy as np

from . import calgeneric as CG
from . import quat as Q
from . import spline

YEAR_S = 365.25 * 86400.0


@dataclass
class Problem:
    """Geometry, auxiliary data and observations (sorted by source)."""
    # instrument (Eq. etazeta0)
    gamma_c: float
    focal_length: float
    p_ac: float
    mu_c: float
    eta0: np.ndarray        # [62]
    x_fpa: np.ndarray       # [62]
    x_centre: np.ndarray    # [2]: fov 0 (f = +1), fov 1 (f = -1)
    ccd_row: np.ndarray     # [62]
    # ephemeris
    orb_L0: float
    obliquity: float
    au_light_s: float
    # epochs and knots
    t_ep_ns: int
    t_fr_ns: int
    knot0_ns: int
    knot_dt_ns: int
    n_coef: int
    # calibration intervals
    cal_t0_ns: int
    cal_dt_ns: int
    n_cal_days: int
    # observations
    t_ns: np.ndarray
    src: np.ndarray
    ccd: np.ndarray
    fov: np.ndarray
    kind: np.ndarray
    sigma: np.ndarray
    mu: np.ndarray
    n_src: int
    # full geometric calibration (Eq. etazeta): its layout and the gate of each observation;
    # None: the per-day offsets
    calg: object = None
    gate: np.ndarray = None

    @property
    def n_obs(self):
        return int(self.t_ns.shape[0])

    @property
    def n_cal(self):
        if self.calg is not None:
            return int(self.calg.n_params)
        return int(self.n_cal_days * 2 * (62 + 7))

    def knots(self):
        return spline.uniform_knots(self.knot0_ns, self.knot_dt_ns, self.n_coef)

    def src_offsets(self):
        return np.searchsorted(self.src, np.arange(self.n_src + 1)).astype(np.int64)

    def f_sign(self, idx=slice(None)):
        return np.where(self.fov[idx] == 0, 1.0, -1.0)


def problem_from_dataset(ds):
    g = ds.geometry
    return Problem(
        gamma_c=g["gamma_c"], focal_length=g["focal_length"], p_ac=g["p_ac"], mu_c=g["mu_c"],
        eta0=np.asarray(g["eta0"]), x_fpa=np.asarray(g["x_fpa"]), x_centre=np.asarray(g["x_centre"]),
        ccd_row=np.asarray(g["ccd_row"]), orb_L0=g["orb_L0"], obliquity=g["obliquity"],
        au_light_s=g["au_light_s"], t_ep_ns=int(g["t_ep_ns"]), t_fr_ns=int(g["t_fr_ns"]),
        knot0_ns=int(g["knot0_ns"]), knot_dt_ns=int(g["knot_dt_ns"]), n_coef=int(g["n_coef"]),
        cal_t0_ns=int(g["cal_t0_ns"]), cal_dt_ns=int(g["cal_dt_ns"]), n_cal_days=int(g["n_cal_days"]),
        t_ns=ds.t_ns, src=ds.src, ccd=ds.ccd, fov=ds.fov, kind=ds.kind, sigma=ds.sigma, mu=ds.mu,
        n_src=ds.n_src,
        calg=(CG.Layout(n_ccd=62, n_gate=int(g["n_gate"]), n_j=int(g["n_cal_days"]), j_per_k=int(g["cal_j_per_k"]),
                        n_col=int(g["n_col"]), col_bin=int(g["cal_col_bin"])) if g.get("cal_generic") else None),
        gate=ds.gate)


# ---------------------------------------------------------------------------
# auxiliary data and source geometry
# ---------------------------------------------------------------------------

def ephemeris(P, t_ns):
    """Barycentric position b_G (AU) and velocity v_G (AU/s) of Gaia, ICRS components."""
    t_s = np.asarray(t_ns, dtype=np.int64).astype(np.float64) * 1e-9
    L = P.orb_L0 + 2.0 * np.pi * (t_s / YEAR_S)
    n = 2.0 * np.pi / YEAR_S
    ce, se = np.cos(P.obliquity), np.sin(P.obliquity)
    cL, sL = np.cos(L), np.sin(L)
    b = np.stack([cL, ce * sL, se * sL], axis=-1)
    v = np.stack([-n * sL, ce * n * cL, se * n * cL], axis=-1)
    return b, v


def normal_triad(alpha, delta):
    """[p q r] of a source, Eq. normal-triad (columns returned as three [...,3] arrays)."""
    sa, ca = np.sin(alpha), np.cos(alpha)
    sd, cd = np.sin(delta), np.cos(delta)
    z = np.zeros_like(sa)
    p = np.stack([-sa, ca, z], axis=-1)
    q = np.stack([-sd * ca, -sd * sa, cd], axis=-1)
    r = np.stack([cd * ca, cd * sa, sd], axis=-1)
    return p, q, r


def unit(v):
    return v / np.linalg.norm(v, axis=-1, keepdims=True)


def proper_direction(P, s5, t_ns):
    """Coordinate direction (Eq. astro-standard with Eq. roemer) and proper direction
    u = <u_bar + v_G/c> (Eq. classAberr).  s5 rows: (alpha, delta, parallax, mu_a*, mu_d)
    in rad and rad/yr, broadcast against t_ns.

    Returns u, u_bar, p, q, r, b_G, v_G/c, tau (years)."""
    s5 = np.asarray(s5, dtype=np.float64)
    p, q, r = normal_triad(s5[..., 0], s5[..., 1])
    b, v = ephemeris(P, t_ns)
    dt_s = (np.asarray(t_ns, dtype=np.int64) - np.int64(P.t_ep_ns)).astype(np.float64) * 1e-9
    tB_rel = dt_s + np.sum(r * b, axis=-1) * P.au_light_s            # t_B - t_ep, Eq. roemer
    tau = tB_rel / YEAR_S
    ubar = unit(r + tau[..., None] * (p * s5[..., 3:4] + q * s5[..., 4:5]) - s5[..., 2:3] * b)
    vc = v * P.au_light_s                                             # v_G / c
    u = unit(ubar + vc)
    return u, ubar, p, q, r, b, vc, tau


# ---------------------------------------------------------------------------
# attitude
# ---------------------------------------------------------------------------

def attitude(P, att, t_ns, knots=None):
    """Spline attitude q(t) = <sum a_n B_n(t)>, Eq. qspline.

    Returns q (unit), s (unnormalised sum), l (left index), B (the 4 non-zero B-splines)."""
    if knots is None:
        knots = P.knots()
    l = spline.left_index(knots, t_ns, P.n_coef)
    B = spline.deboor(knots, t_ns, l)
    idx = l[..., None] + np.arange(-3, 1)
    s = np.sum(att[idx] * B[..., None], axis=-2)
    return Q.qunit(s), s, l, B


# ---------------------------------------------------------------------------
# field angles, calibrated observation lines, residuals
# ---------------------------------------------------------------------------

def cal_day(P, t_ns):
    d = (np.asarray(t_ns, dtype=np.int64) - np.int64(P.cal_t0_ns)) // np.int64(P.cal_dt_ns)
    return np.clip(d, 0, P.n_cal_days - 1)


def cal_index(P, t_ns, fov, ccd, kind):
    """Index of the calibration parameter of an observation (input data convention):
    AL: (day*2 + fov)*62 + ccd;  AC: n_days*124 + (day*2 + fov)*7 + row(ccd)."""
    day = cal_day(P, t_ns)
    fov = np.asarray(fov, dtype=np.int64)
    ccd = np.asarray(ccd, dtype=np.int64)
    al = (day * 2 + fov) * 62 + ccd
    ac = P.n_cal_days * 124 + (day * 2 + fov) * 7 + P.ccd_row[ccd]
    return np.where(np.asarray(kind) == 0, al, ac)


def field_angles(u_srs):
    """Instrument angles phi, zeta, Eq. srsprop1."""
    phi = np.arctan2(u_srs[..., 1], u_srs[..., 0])
    zeta = np.arctan2(u_srs[..., 2], np.sqrt(u_srs[..., 0] ** 2 + u_srs[..., 1] ** 2))
    return phi, zeta


def observation_lines(P, cal, idx=slice(None)):
    """Calibrated observation lines eta_fng and zeta_fng of the observations, Eqs. etazeta0 and
    etazeta: the r = 0 offsets, or with P.calg the full model (oracle/calgeneric.py; the nominal
    lines the same for every gate).  Returns (lines, k): k the parameter index of each
    observation, or with P.calg the (cols, vals) of its calibration terms."""
    t_ns, fov, ccd, kind, mu = P.t_ns[idx], P.fov[idx], P.ccd[idx], P.kind[idx], P.mu[idx]
    if P.calg is not None:
        k = CG.design(P.calg, kind, fov, ccd, P.gate[idx], cal_day(P, t_ns), mu)
        term = CG.line_term(cal, *k)
    else:
        k = cal_index(P, t_ns, fov, ccd, kind)
        term = np.asarray(cal)[k]
    eta_line = P.eta0[ccd] + term
    f = np.where(fov == 0, 0, 1)
    zeta0 = -(P.x_fpa[ccd] - (mu - P.mu_c) * P.p_ac - P.x_centre[f]) / P.focal_length
    zeta_line = zeta0 + term
    return np.where(kind == 0, eta_line, zeta_line), k


def evaluate(P, src, att, cal, idx=slice(None), knots=None, partials=True):
    """Residuals R_l (Eqs. resAL, resAC) and, optionally, the partial derivatives of the
    observations selected by idx.

    Returns a dict with
      R      residual (rad)
      A      design rows -dR/ds' (5 per observation), Eqs. dfads, srsprop1diffsol, ubardiff, duds
      gq     dR/dq (4 per observation, quaternion), Eq. dfadq
      s      unnormalised spline sum (4), B (4 B-splines), l (left index)
      cal_k  calibration parameter index (dR/dc_k = +1, Eq. pdC); with the full calibration
             model cal_cols, cal_vals instead (dR/dc = the factor, Eq. pdC)
    """
    t_ns = P.t_ns[idx]
    s5 = np.asarray(src)[P.src[idx]]
    kind = P.kind[idx]
    f = P.f_sign(idx)
    u, ubar, p, q, r, b, vc, tau = proper_direction(P, s5, t_ns)
    qa, s, l, B = attitude(P, att, t_ns, knots)
    us = Q.frame_rotate(qa, u)                                        # Eq. srsprop
    phi, zeta = field_angles(us)
    eta = phi - f * P.gamma_c / 2.0                                   # Eq. srspropeta
    line, k = observation_lines(P, cal, idx)
    R = np.where(kind == 0, line - eta, line - zeta)
    out = dict(R=R, s=s, B=B, l=l, phi=phi, zeta=zeta, u=u, q=qa)
    if P.calg is not None:
        out.update(cal_k=None, cal_cols=k[0], cal_vals=k[1])
    else:
        out.update(cal_k=k)
    if not partials:
        return out
    # source partials
    pb = np.zeros(b.shape)
    rb = np.sum(r * b, axis=-1, keepdims=True)
    dpar = -(b - r * rb)                                              # -(I - r r') b_G / A_u
    dubar = np.stack([p, q, dpar, p * tau[..., None], q * tau[..., None]], axis=-1)   # [...,3,5]
    del pb
    ubv = np.sum(ubar * vc, axis=-1)
    # Eq. duds: du/ds' = [(1 - ubar'v/c) I - ubar v'/c] dubar/ds'
    vdu = np.einsum("...i,...ij->...j", vc, dubar)
    du = (1.0 - ubv)[..., None, None] * dubar - ubar[..., :, None] * vdu[..., None, :]
    # to the SRS, Eq. srspropdiff (column by column)
    du_s = np.stack([Q.frame_rotate(qa, du[..., :, j]) for j in range(5)], axis=-1)
    sp, cp = np.sin(phi), np.cos(phi)
    sz, cz = np.sin(zeta), np.cos(zeta)
    z0 = np.zeros_like(sp)
    m = np.stack([-sp, cp, z0], axis=-1)                              # Eq. srspqr
    n = np.stack([-sz * cp, -sz * sp, cz], axis=-1)
    A_al = np.einsum("...i,...ij->...j", m, du_s) / cz[..., None]     # -dR_AL/ds'
    A_ac = np.einsum("...i,...ij->...j", n, du_s)                     # -dR_AC/ds'
    A = np.where((kind == 0)[..., None], A_al, A_ac)
    # attitude partials, Eq. dfadq: -dR_AL/dq = -2 sec(zeta) q {n,0};  -dR_AC/dq = 2 q {m,0}
    g_al = 2.0 / cz[..., None] * Q.qmul(qa, Q.vq(n))
    g_ac = -2.0 * Q.qmul(qa, Q.vq(m))
    gq = np.where((kind == 0)[..., None], g_al, g_ac)
    out.update(A=A, gq=gq)
    return out


def attitude_design(ev):
    """dR/da_n for the 4 coefficients n = l-3..l: (dR/dq) B_n / ||s|| (Eq. dfadq with the
    normalisation of Eq. qspline).  Returns [..., 4 (n), 4 (component)]."""
    ns = Q.qnorm(ev["s"])
    return ev["B"][..., :, None] * (ev["gq"] / ns[..., None])[..., None, :]


def norm_deviation(ev):
    """D_l = 1 - ||s||^2 (Eq. Dl) and dD_l/da_n = -2 s B_n (Eq. dDldan, exact form)."""
    s = ev["s"]
    D = 1.0 - np.sum(s * s, axis=-1)
    dD = -2.0 * ev["B"][..., :, None] * s[..., None, :]
    return D, dD
