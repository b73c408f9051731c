"""The S, A and C update blocks (Sect. 5) and the frame rotator (Sect. 6.1), FP64.

Readings where the paper is silent or leaves a choice:
  * inner iteration (Sect. 5.1.2): the robust sigma is half the intersextile
    range of h_l / sigma_l (AL and AC pooled after dividing by their own
    sigma), initial w_l = w(h_l / (sigma_l varsigma)); then exactly
    ``n_rounds`` (4) rounds of [excess-noise solve; w_l <- w(R_l / sqrt(sigma_l^2 + eps^2))]
    followed by a final excess-noise solve with the last w_l;
  * excess-noise solve: at most ``n_eps`` (3) rational steps
    dy = (1 - Q/nu) Q / Q', y <- max(0, y + dy) (a variance cannot be negative),
    stopping early when |dy| <= 1e-12 min(sigma_l^2);
    Q'(y) = -sum w_l R_l^2 / (sigma_l^2 + y)^2 (envelope theorem: the update d
    minimises Q at fixed y);
  * nu = n_i - n_out - 5 counts AL and AC components; n_out = #(w_l < 0.2);
    eps = 0 when nu <= 0;
  * residuals and weights passed to A and C are the final ones of the source
    update: R_l = h_l - A_l d (the first line of Eq. precond2) and
    W_l = w_l / (sigma_l^2 + eps_i^2); the excess attitude noise is zero;
  * attitude regularisation: the lambda^2 dD dD' W term of Eq. normAmod enters
    the matrix; its right-hand-side term is included only when
    ``rhs_norm_term`` is set (the paper-literal form);
  * attitude segmentation (Sect. 5.2.2): segments of ``seg_len`` knot
    intervals with 2L overlapping intervals; segment K updates a_n up to and
    including n = x - floor(M/2) where tau_x is its cross-over knot;
  * calibration constraints: Eq. cc1 (per day, over both fields and all 62 AF
    CCDs) and Eq. cc3 (per field and day over the 7 AC parameters), enforced by
    the projection of Eq. calCon;
  * frame rotator: unit weights, all sources in S_PM with the reference values
    given, comparison epoch t = t_ep = t_fr (Eq. cond-mu3).
"""
from dataclasses import dataclass, field

import numpy as np

from . import calgeneric as CG
from . import cholesky as CH
from . import model as M
from . import quat as Q
from . import weights as WF

MAS = np.pi / 648000.0 * 1e-3


@dataclass
class Settings:
    robust: bool = True          # inner iteration with downweighting and excess noise
    n_rounds: int = 4            # weight rounds
    n_eps: int = 3               # excess-noise steps per round
    weight_fn: str = "agis"      # "agis" (Eq. dw) or "huber" (Eq. dwH)
    lam: float = 1e-3            # attitude regularisation lambda, Eq. JfuncMod
    rhs_norm_term: bool = False  # include lambda^2 dD D W on the right-hand side
    seg_len: int = 720           # attitude segment length in knot intervals
    seg_overlap: int = 12        # L
    block_mask: str = "SAC"      # blocks run by an iteration
    frame_each_iter: bool = True
    # order of the blocks within an iteration (Sect. 4.6): "S[AC]" A and C from the residuals
    # after the source update (Eq. precondS(CAG)); "SAC" C also after the attitude update
    # (Gauss-Seidel, Eq. precond); "[SAC]" A and C from the residuals before the source
    # update (Jacobi, Eq. precond(SCAG))
    block_order: str = "S[AC]"
    # excess attitude noise (Sect. 5.2.5): bucket length in ns, 0 = not estimated
    att_noise_bucket_ns: int = 0


def _wfun(st):
    return WF.w_agis if st.weight_fn == "agis" else WF.w_huber


# ---------------------------------------------------------------------------
# S block, Sect. 5.1
# ---------------------------------------------------------------------------

@dataclass
class SourceResult:
    d: np.ndarray          # [n_src, 5] updates (alpha*, delta, parallax, mu_a*, mu_d)
    eps2: np.ndarray       # excess source variance
    Qi: np.ndarray         # Eq. Qi with the final weights
    nu: np.ndarray
    n_out: np.ndarray
    D: np.ndarray          # significance, Eq. D
    cov: np.ndarray        # [n_src, 5, 5] inverse normal matrix
    rank_def: np.ndarray
    R: np.ndarray          # [n_obs] final residuals h - A d
    W: np.ndarray          # [n_obs] final statistical weights


def _solve_weighted(A, h, Wt):
    """Normal equations A'WA d = A'Wh (Eq. normSmat) by C.1-C.3."""
    N = A.T @ (A * Wt[:, None])
    b = A.T @ (h * Wt)
    d, U, rd = CH.solve(N, b)
    return d, U, rd


def _eps_solve(A, h, sig2, w, nu, st):
    """Excess-noise solve for fixed downweighting factors (Eq. epsi).

    Returns y = eps_i^2, d, R, Q(y), Q(0), U, rank defect."""
    y = 0.0
    d, U, rd = _solve_weighted(A, h, w / sig2)
    R = h - A @ d
    Qy = float(np.sum(w * R * R / sig2))
    Q0 = Qy
    if nu <= 0 or Q0 <= nu:
        return y, d, R, Qy, Q0, U, rd
    tol = 1e-12 * float(np.min(sig2))
    for _ in range(st.n_eps):
        dQ = -float(np.sum(w * R * R / (sig2 + y) ** 2))
        dy = (1.0 - Qy / nu) * Qy / dQ
        y = max(0.0, y + dy)
        d, U, rd = _solve_weighted(A, h, w / (sig2 + y))
        R = h - A @ d
        Qy = float(np.sum(w * R * R / (sig2 + y)))
        if abs(dy) <= tol:
            break
    return y, d, R, Qy, Q0, U, rd


def source_update_one(A, h, sig2, st):
    """Inner iteration of one source (Sect. 5.1.2).  A: [n, 5] design rows -dR/ds',
    h: [n] residuals at the current parameters, sig2: [n] sigma_l^2."""
    n = h.size
    wf = _wfun(st)
    if not st.robust:
        w = np.ones(n)
        d, U, rd = _solve_weighted(A, h, w / sig2)
        R = h - A @ d
        nu = n - 5
        Qi = float(np.sum(R * R / sig2))
        return dict(d=d, eps2=0.0, R=R, W=w / sig2, Qi=Qi, nu=nu, n_out=0,
                    D=(Qi - nu) / np.sqrt(2 * nu) if nu > 0 else 0.0, U=U, rd=rd)
    sig = np.sqrt(sig2)
    x = h / sig
    vs = WF.intersextile_half_range(x)
    w = wf(x / vs) if vs > 0 else np.ones(n)
    res = None
    for rnd in range(st.n_rounds + 1):
        n_out = int(np.sum(w < 0.2))
        nu = n - n_out - 5
        y, d, R, Qy, Q0, U, rd = _eps_solve(A, h, sig2, w, nu, st)
        res = (y, d, R, Qy, Q0, U, rd, nu, n_out, w)
        if rnd < st.n_rounds:
            w = wf(R / np.sqrt(sig2 + y))
    y, d, R, Qy, Q0, U, rd, nu, n_out, w = res
    D = (Q0 - nu) / np.sqrt(2.0 * nu) if nu > 0 else 0.0
    return dict(d=d, eps2=y, R=R, W=w / (sig2 + y), Qi=Qy, nu=nu, n_out=n_out, D=D, U=U, rd=rd)


def source_update(P, src, att, cal, st, ev=None, sig2=None):
    """S block: per-source 5x5 solves (Eq. normS) and the parameter update (footnote to
    Eq. ubardiff: alpha += d0 / cos(delta)).  sig2: the observation variances to use (default
    sigma_l^2; sigma~_l^2 with the excess attitude noise, Eq. W).  Returns (new sources,
    SourceResult, ev)."""
    if ev is None:
        ev = M.evaluate(P, src, att, cal)
    off = P.src_offsets()
    ns = P.n_src
    res = SourceResult(d=np.zeros((ns, 5)), eps2=np.zeros(ns), Qi=np.zeros(ns), nu=np.zeros(ns, np.int64),
                       n_out=np.zeros(ns, np.int64), D=np.zeros(ns), cov=np.zeros((ns, 5, 5)),
                       rank_def=np.zeros(ns, np.int64), R=np.zeros(P.n_obs), W=np.zeros(P.n_obs))
    if sig2 is None:
        sig2 = P.sigma.astype(np.float64) ** 2
    for i in range(ns):
        a, b = off[i], off[i + 1]
        if b == a:
            continue
        r = source_update_one(ev["A"][a:b], ev["R"][a:b], sig2[a:b], st)
        res.d[i] = r["d"]
        res.eps2[i] = r["eps2"]
        res.Qi[i] = r["Qi"]
        res.nu[i] = r["nu"]
        res.n_out[i] = r["n_out"]
        res.D[i] = r["D"]
        res.cov[i] = CH.inverse(r["U"])
        res.rank_def[i] = r["rd"]
        res.R[a:b] = r["R"]
        res.W[a:b] = r["W"]
    new = np.array(src, dtype=np.float64, copy=True)
    new[:, 0] += res.d[:, 0] / np.cos(src[:, 1])
    new[:, 1] += res.d[:, 1]
    new[:, 2:5] += res.d[:, 2:5]
    return new, res, ev


# ---------------------------------------------------------------------------
# A block, Sect. 5.2
# ---------------------------------------------------------------------------

def segments(P, st):
    """Overlapping segments (Sect. 5.2.2).  Returns a list of
    (l_lo, l_hi, n_lo, n_hi, upd_lo, upd_hi): interval range [l_lo, l_hi], unknowns
    [n_lo, n_hi] = [l_lo-3, l_hi] and the coefficients it updates [upd_lo, upd_hi]."""
    Mo = 4
    N = P.n_coef
    K = N - Mo + 1
    S, L = st.seg_len, st.seg_overlap
    nseg = max(1, -(-K // S))
    out = []
    for k in range(nseg):
        x0 = (Mo - 1) + k * S          # cross-over knot with the previous segment
        x1 = (Mo - 1) + (k + 1) * S    # with the next
        l_lo = max(Mo - 1, x0 - L)
        l_hi = min(N - 1, x1 + L - 1)
        upd_lo = 0 if k == 0 else x0 - Mo // 2 + 1
        upd_hi = N - 1 if k == nseg - 1 else x1 - Mo // 2
        out.append((l_lo, l_hi, l_lo - (Mo - 1), l_hi, upd_lo, upd_hi))
    return out


def attitude_normals(P, ev, R, W, st, l_lo, l_hi):
    """Banded normal equations of one segment, Eq. normAmod: band storage of width 16
    over the 4(n_hi - n_lo + 1) unknowns (4 per coefficient)."""
    l = ev["l"]
    sel = np.nonzero((l >= l_lo) & (l <= l_hi))[0]
    n_lo, n_hi = l_lo - 3, l_hi
    nu = 4 * (n_hi - n_lo + 1)
    w = 16
    Nb = np.zeros((nu, w))
    b = np.zeros(nu)
    if sel.size:
        G = M.attitude_design({k: v[sel] for k, v in ev.items() if k in ("B", "gq", "s")})  # [m,4,4]
        D, dD = M.norm_deviation({k: v[sel] for k, v in ev.items() if k in ("B", "s")})
        Gf = G.reshape(sel.size, 16)
        dDf = dD.reshape(sel.size, 16)
        Wl = W[sel]
        base = 4 * (l[sel] - 3 - n_lo)                 # first unknown of each observation
        lam2 = st.lam ** 2
        for i in range(16):
            for j in range(i, 16):
                v = (Gf[:, i] * Gf[:, j] + lam2 * dDf[:, i] * dDf[:, j]) * Wl
                np.add.at(Nb, (base + i, j - i), v)
            rhs = -Gf[:, i] * R[sel] * Wl
            if st.rhs_norm_term:
                rhs = rhs - lam2 * dDf[:, i] * D * Wl
            np.add.at(b, base + i, rhs)
    return Nb, b


def attitude_update(P, att, ev, R, W, st):
    """A block: segmented banded solves with the robust Cholesky (App. C) and the update of
    the spline coefficients.  Returns (new attitude, total rank defect)."""
    new = np.array(att, dtype=np.float64, copy=True)
    rd_total = 0
    for (l_lo, l_hi, n_lo, n_hi, u_lo, u_hi) in segments(P, st):
        Nb, b = attitude_normals(P, ev, R, W, st, l_lo, l_hi)
        x, Ub, rd = CH.band_solve(Nb, b)
        rd_total += rd
        dx = x.reshape(-1, 4)
        new[u_lo:u_hi + 1] += dx[u_lo - n_lo:u_hi - n_lo + 1]
    return new, rd_total


# ---------------------------------------------------------------------------
# C block, Sect. 5.3
# ---------------------------------------------------------------------------

def calibration_constraint_groups(P):
    """Columns of the constraint matrix C (Eq. genericConstraint) for Eqs. cc1 and cc3, as
    lists of parameter indices with unit coefficients."""
    nd = P.n_cal_days
    groups = []
    for d in range(nd):
        groups.append(np.arange((d * 2) * 62, (d * 2 + 2) * 62))                      # cc1
    for d in range(nd):
        for f in range(2):
            a = nd * 124 + (d * 2 + f) * 7
            groups.append(np.arange(a, a + 7))                                         # cc3
    return groups


def calibration_update(P, cal, ev, R, W):
    """C block: block-diagonal normals (Eq. normC with dR/dc = 1, Eq. pdC), the 1x1 robust
    solves (Algorithms C.1-C.3: x = (b / sqrt(N)) / sqrt(N), or 0 with a rank defect when
    N = 0) and the constraint projection d = d~ - C (C'C)^-1 C' d~ (Eq. calCon).  The
    constraint columns of Eqs. cc1 and cc3 have disjoint supports, so C'C is diagonal and
    the projection subtracts, within each column's support, C'd~ / C'C.
    With the full calibration model (P.calg) the update of oracle/calgeneric.py instead.
    Returns (new calibration, rank defect)."""
    if P.calg is not None:
        d, rd = CG.update(P.calg, ev["cal_cols"], ev["cal_vals"], R, W)
        return np.asarray(cal) + d, rd
    k = ev["cal_k"]
    Ncc = np.bincount(k, weights=W, minlength=P.n_cal)
    bc = np.bincount(k, weights=-R * W, minlength=P.n_cal)
    pos = Ncc > 0
    U = np.where(pos, np.sqrt(np.where(pos, Ncc, 1.0)), 0.0)
    dt = np.zeros(P.n_cal)
    dt[pos] = (bc[pos] / U[pos]) / U[pos]
    rd = int(np.sum(~pos))
    d = dt.copy()
    for g in calibration_constraint_groups(P):
        ctd = float(np.sum(dt[g]))
        ctc = float(g.size)
        d[g] -= ctd / ctc
    return np.asarray(cal) + d, rd


# ---------------------------------------------------------------------------
# frame rotator, Sect. 6.1
# ---------------------------------------------------------------------------

def frame_f(P, eps, omega, t_ns):
    """Frame rotator quaternion f(t) = Q[(t - t_fr) omega] Q(eps), Eq. fr1 (t in years for omega)."""
    dt = (np.asarray(t_ns, dtype=np.int64) - np.int64(P.t_fr_ns)).astype(np.float64) * 1e-9 / M.YEAR_S
    return Q.qmul(Q.Q(dt[..., None] * np.asarray(omega)), Q.Q(np.broadcast_to(eps, np.shape(dt) + (3,))))


def frame_fit(P, src, ref):
    """Least-squares (eps, omega) from Eq. cond-mu3 with t = t_ep = t_fr and unit weights.
    src: AGIS parameters; ref: reference (alpha, delta, mu_a*, mu_d) in the ICRS, epoch t_ep."""
    p, q, r = M.normal_triad(src[:, 0], src[:, 1])
    _, _, rh = M.normal_triad(ref[:, 0], ref[:, 1])
    dr = r - rh
    da = np.sum(p * dr, axis=-1)          # Eq. fr-Delta1 with t = t_ep = t_PM
    dd = np.sum(q * dr, axis=-1)
    dpa = src[:, 3] - ref[:, 2]
    dpd = src[:, 4] - ref[:, 3]
    tt = (P.t_ep_ns - P.t_fr_ns) * 1e-9 / M.YEAR_S
    n = src.shape[0]
    z3 = np.zeros((n, 3))
    # unknowns x = (eps_X, eps_Y, eps_Z, omega_X, omega_Y, omega_Z)
    rows = np.concatenate([
        np.concatenate([z3, q], axis=1),                 # q'omega = dmu_a*
        np.concatenate([z3, -p], axis=1),                # -p'omega = dmu_d
        np.concatenate([q, tt * q], axis=1),             # q'(eps + (t - t_fr) omega) = Delta alpha*
        np.concatenate([-p, -tt * p], axis=1),           # -p'(eps + (t - t_fr) omega) = Delta delta
    ], axis=0)
    rhs = np.concatenate([dpa, dpd, da, dd])
    N = rows.T @ rows
    b = rows.T @ rhs
    x, U, rd = CH.solve(N, b)
    return x[:3], x[3:]


def frame_apply_sources(P, src, eps, omega):
    """Rigorous transformation of the astrometric parameters (Sect. 6.1.2, steps 1-5)."""
    f = frame_f(P, eps, omega, np.full(src.shape[0], P.t_ep_ns, dtype=np.int64))          # step 1
    pt, qt, r_t = M.normal_triad(src[:, 0], src[:, 1])                                     # step 2
    w = np.asarray(omega)
    mu_t = pt * src[:, 3:4] + qt * src[:, 4:5] - np.cross(np.broadcast_to(w, r_t.shape), r_t)  # Eq. mu-agis
    r_c = Q.frame_rotate(f, r_t)                                                           # step 3, Eq. fr-r
    mu_c = Q.frame_rotate(f, mu_t)                                                         # Eq. fr-mu
    alpha = np.arctan2(r_c[:, 1], r_c[:, 0])                                               # step 4, Eq. fr-ad
    delta = np.arctan2(r_c[:, 2], np.sqrt(r_c[:, 0] ** 2 + r_c[:, 1] ** 2))
    p, q, _ = M.normal_triad(alpha, delta)
    out = np.array(src, dtype=np.float64, copy=True)
    out[:, 0] = np.mod(alpha, 2 * np.pi)
    out[:, 1] = delta
    out[:, 3] = np.sum(p * mu_c, axis=-1)                                                  # step 5
    out[:, 4] = np.sum(q * mu_c, axis=-1)
    return out


def frame_apply_attitude(P, att, eps, omega):
    """a_n = f(t_n)^-1 a~_n with t_n the mid-time of the support of B_n (Eqs. fr-q4, RF4)."""
    kn = P.knots()
    n = np.arange(P.n_coef)
    tbar = (kn[n] + kn[n + 4]) // 2
    f = frame_f(P, eps, omega, tbar)
    return Q.qmul(Q.qinv(f), att)
