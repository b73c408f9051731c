"""Pins for the S, A, C blocks, the frame rotator and the S[ACG] step (Sects. 4.5-6.1)."""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spl

import synth
from oracle import agis as G
from oracle import blocks as B
from oracle import model as M
from oracle import quat as Q
from oracle import weights as WF

UAS = synth.UAS


# ---------------------------------------------------------------------------
# inner iteration
# ---------------------------------------------------------------------------

def test_excess_noise_one_rational_step_is_exact_for_equal_sigma():
    # Q(y) = Q(0) s^2 / (s^2 + y) when all sigma are equal and w = 1: the rational model of the
    # footnote to Eq. epsi is exact and one step gives y* = s^2 (Q(0)/nu - 1)
    rng = np.random.default_rng(0)
    n = 200
    A = rng.normal(size=(n, 5))
    s2 = 1e-18
    h = A @ rng.normal(size=5) * 1e-9 + rng.normal(size=n) * 3e-9
    st = B.Settings(n_eps=1)
    nu = n - 5
    y, d, R, Qy, Q0, U, rd = B._eps_solve(A, h, np.full(n, s2), np.ones(n), nu, st)
    assert Q0 > nu
    assert abs(y / (s2 * (Q0 / nu - 1)) - 1) < 1e-12
    assert abs(Qy / nu - 1) < 1e-10


def test_source_update_recovers_exact_linear_data():
    rng = np.random.default_rng(1)
    n = 300
    A = rng.normal(size=(n, 5))
    d_true = rng.normal(size=5) * 1e-8
    h = A @ d_true
    r = B.source_update_one(A, h, np.full(n, 1e-18), B.Settings())
    assert np.allclose(r["d"], d_true, rtol=1e-10, atol=1e-22)
    assert r["eps2"] == 0.0 and r["n_out"] == 0


def test_outlier_is_downweighted():
    rng = np.random.default_rng(2)
    n = 300
    A = rng.normal(size=(n, 5))
    sig = 1e-9
    h = A @ (rng.normal(size=5) * 1e-8) + rng.normal(size=n) * sig
    h[17] += 30 * sig
    r = B.source_update_one(A, h, np.full(n, sig * sig), B.Settings())
    assert r["W"][17] < 1e-3 * np.median(r["W"])
    assert r["n_out"] >= 1


# ---------------------------------------------------------------------------
# truth is a fixed point (noise-free data from the independent simulator)
# ---------------------------------------------------------------------------

def test_truth_is_a_fixed_point(small_noisefree):
    ds = small_noisefree
    P = M.problem_from_dataset(ds)
    st = B.Settings(seg_len=720)
    state = G.State(ds.src_true.copy(), ds.att_true.copy(), ds.cal_true.copy())
    new, stats, sres = G.iterate_once(P, state, st, ref=ds.src_true[:, [0, 1, 3, 4]])
    # the only residuals at truth come from rounding the observation times to integer ns
    # (0.016 uas RMS per observation): updates stay at that floor
    e = G.source_errors(new.src, ds.src_true)
    assert np.all(np.sqrt(np.mean(e ** 2, axis=0)) < 0.1 * UAS)
    assert np.max(np.abs(e)) < 1.0 * UAS
    dc = new.cal - ds.cal_true
    assert np.sqrt(np.mean(dc ** 2)) < 0.01 * UAS
    # the attitude is fixed by the data at the observation times (not coefficient by coefficient)
    R0 = M.evaluate(P, ds.src_true, ds.att_true, ds.cal_true, partials=False)["R"]
    R1 = M.evaluate(P, ds.src_true, new.att, ds.cal_true, partials=False)["R"]
    assert np.sqrt(np.mean((R1 - R0) ** 2)) < 0.01 * UAS
    assert np.max(np.abs(stats.frame)) < 0.01 * UAS


# ---------------------------------------------------------------------------
# one S[ACG] iteration equals d = K^-1 b (Eqs. precond1, precond2, precondS(CAG))
# ---------------------------------------------------------------------------

def _jacobian(P, ev, lam):
    n = P.n_obs
    ns, nc = P.n_src, P.n_coef
    rows = np.arange(n)
    Js = sp.csr_matrix((-ev["A"].ravel(), (np.repeat(rows, 5), (P.src[:, None] * 5 + np.arange(5)).ravel())),
                       shape=(n, 5 * ns))
    Ga = M.attitude_design(ev).reshape(n, 16)
    col_a = (4 * (ev["l"][:, None] - 3) + np.arange(16)).ravel()
    Ja = sp.csr_matrix((Ga.ravel(), (np.repeat(rows, 16), col_a)), shape=(n, 4 * nc))
    D, dD = M.norm_deviation(ev)
    Jd = sp.csr_matrix((dD.reshape(n, 16).ravel(), (np.repeat(rows, 16), col_a)), shape=(n, 4 * nc))
    Jc = sp.csr_matrix((np.ones(n), (rows, ev["cal_k"])), shape=(n, P.n_cal))
    return Js, Ja, Jd, Jc


def _reduced_solve(Nm, b):
    keep = np.asarray(abs(Nm).sum(axis=1)).ravel() > 0
    x = np.zeros(b.size)
    if keep.any():
        x[keep] = spl.spsolve(sp.csc_matrix(Nm[keep][:, keep]), b[keep])
    return x


@pytest.mark.parametrize("order", ["S[AC]", "SAC", "[SAC]"])
def test_one_iteration_equals_preconditioner_solve(order):
    # the three block orders of Sect. 4.6: S[AC] (Eq. precondS(CAG), N_as and N_cs below the
    # diagonal), SAC (Gauss-Seidel, Eq. precond: also N_ca) and [SAC] (Jacobi, Eq.
    # precond(SCAG): block diagonal)
    ds = synth.simulate(synth.config("small1yr", n_src=6000, span_days=180, min_transits=6, seed=11))
    P = M.problem_from_dataset(ds)
    K = P.n_coef - 3
    st = B.Settings(robust=False, seg_len=K + 10, lam=1e-3, frame_each_iter=False, block_order=order)
    state = G.State(ds.src0.copy(), ds.att0.copy(), ds.cal0.copy())
    new, stats, sres = G.iterate_once(P, state, st)
    ev = M.evaluate(P, state.src, state.att, state.cal)
    Js, Ja, Jd, Jc = _jacobian(P, ev, st.lam)
    Wm = sp.diags(1.0 / P.sigma.astype(np.float64) ** 2)
    R0 = ev["R"]
    Nss = (Js.T @ Wm @ Js).tocsc()
    bs = -(Js.T @ (Wm @ R0))
    ds_ = _reduced_solve(Nss, bs)
    assert np.allclose(ds_.reshape(-1, 5), sres.d, rtol=1e-7, atol=1e-6 * np.abs(sres.d).max())
    Naa = (Ja.T @ Wm @ Ja + st.lam ** 2 * (Jd.T @ Wm @ Jd)).tocsc()
    ba = -(Ja.T @ (Wm @ R0))
    if order != "[SAC]":
        ba = ba - (Ja.T @ Wm @ Js) @ ds_
    da = _reduced_solve(Naa, ba)
    # compare where the data determine the update: its effect on the residuals, J_a d_a
    # (directions with J_a v ~ 0, e.g. the spline scale regularised only by lambda^2, are
    # solver-dependent and invisible to the observations)
    ya = Ja @ (new.att - state.att).ravel()
    yr = Ja @ da
    assert np.linalg.norm(ya - yr) < 1e-6 * np.linalg.norm(yr)
    Ncc = (Jc.T @ Wm @ Jc).diagonal()
    bc = -(Jc.T @ (Wm @ R0))
    if order != "[SAC]":
        bc = bc - (Jc.T @ Wm @ Js) @ ds_
    if order == "SAC":
        bc = bc - (Jc.T @ Wm @ Ja) @ da
    dc = np.where(Ncc > 0, bc / np.where(Ncc > 0, Ncc, 1), 0.0)
    for g in B.calibration_constraint_groups(P):
        dc[g] -= dc[g].mean()
    assert np.allclose(new.cal - state.cal, dc, rtol=1e-6, atol=1e-6 * np.abs(dc).max())


def test_null_space_vectors(small_noisefree):
    # Sect. 6.1.5: N V = 0 up to the absolute frame information carried by aberration and
    # parallax through the ICRS ephemeris (Sect. 4.4), of relative size ~ v/c = 1e-4.
    # Reading: with the frame conventions of Eqs. fr1, fr-q4 and cond-mu3 the printed V_s and
    # V_a describe rotations of opposite sense; (V_s, -V_a) is the null-space pair (with the
    # printed signs the source and attitude terms add instead of cancelling).
    ds = small_noisefree
    P = M.problem_from_dataset(ds)
    ev = M.evaluate(P, ds.src_true, ds.att_true, ds.cal_true)
    Js, Ja, Jd, Jc = _jacobian(P, ev, 0.0)
    p, q, r = M.normal_triad(ds.src_true[:, 0], ds.src_true[:, 1])
    tau = (P.t_ep_ns - P.t_fr_ns) * 1e-9 / M.YEAR_S
    ns = P.n_src
    Vs = np.zeros((ns, 5, 6))
    Vs[:, 0, :3], Vs[:, 0, 3:] = q, tau * q
    Vs[:, 1, :3], Vs[:, 1, 3:] = -p, -tau * p
    Vs[:, 3, 3:] = q
    Vs[:, 4, 3:] = -p
    kn = P.knots()
    n = np.arange(P.n_coef)
    tn = ((kn[n] + kn[n + 4]) // 2 - P.t_fr_ns) * 1e-9 / M.YEAR_S
    a = ds.att_true
    ax, ay, az, aw = a[:, 0], a[:, 1], a[:, 2], a[:, 3]
    Va = np.zeros((P.n_coef, 4, 6))
    base = np.stack([np.stack([-aw, -az, ay], -1), np.stack([az, -aw, -ax], -1),
                     np.stack([-ay, ax, -aw], -1), np.stack([ax, ay, az], -1)], axis=1)
    Va[:, :, :3] = 0.5 * base
    Va[:, :, 3:] = 0.5 * base * tn[:, None, None]
    for k in range(6):
        js = Js @ Vs[:, :, k].ravel()
        ja = Ja @ (-Va[:, :, k]).ravel()
        # residual changes from the source part and the attitude part cancel
        assert np.linalg.norm(js + ja) < 3e-4 * np.linalg.norm(js)
        assert np.linalg.norm(js) > 0


# ---------------------------------------------------------------------------
# C block constraints, A-block segmentation and rank defects
# ---------------------------------------------------------------------------

def test_calibration_constraints_hold(small_noisy):
    ds = small_noisy
    P = M.problem_from_dataset(ds)
    ev = M.evaluate(P, ds.src_true, ds.att_true, ds.cal0)
    cal1, rd = B.calibration_update(P, ds.cal0, ev, ev["R"], 1.0 / ds.sigma.astype(float) ** 2)
    for g in B.calibration_constraint_groups(P):
        assert abs(cal1[g].sum()) < 1e-12 * max(1e-12, np.abs(cal1[g]).sum())
    assert rd > 0  # CCD-days without data are reported, not an error


def test_segmented_attitude_matches_single_segment(small_noisefree):
    ds = small_noisefree
    P = M.problem_from_dataset(ds)
    ev = M.evaluate(P, ds.src_true, ds.att0, ds.cal_true)
    W = 1.0 / ds.sigma.astype(float) ** 2
    a_seg, _ = B.attitude_update(P, ds.att0, ev, ev["R"], W, B.Settings(seg_len=240))
    a_one, _ = B.attitude_update(P, ds.att0, ev, ev["R"], W, B.Settings(seg_len=P.n_coef))
    ev_seg = M.evaluate(P, ds.src_true, a_seg, ds.cal_true, partials=False)["R"]
    ev_one = M.evaluate(P, ds.src_true, a_one, ds.cal_true, partials=False)["R"]
    # 2L = 24 overlapping knot intervals make the seams practically invisible (Sect. 5.2.2)
    assert np.sqrt(np.mean((ev_seg - ev_one) ** 2)) < 0.05 * np.sqrt(np.mean(ev["R"] ** 2))


def test_segment_assignment_covers_every_coefficient_once():
    class PP:
        n_coef = 1000
    st = B.Settings(seg_len=97, seg_overlap=12)
    segs = B.segments(PP, st)
    hit = np.zeros(1000, int)
    for (l_lo, l_hi, n_lo, n_hi, u_lo, u_hi) in segs:
        assert n_lo <= u_lo and u_hi <= n_hi
        hit[u_lo:u_hi + 1] += 1
    assert np.all(hit == 1)


# ---------------------------------------------------------------------------
# frame rotator
# ---------------------------------------------------------------------------

def _to_agis_frame(P, src, eps, om):
    """Inverse of the rigorous transformation: ICRS parameters -> AGIS frame (Eqs. fr-r, mu)."""
    f = B.frame_f(P, eps, om, np.full(src.shape[0], P.t_ep_ns, dtype=np.int64))
    p, q, r = M.normal_triad(src[:, 0], src[:, 1])
    mu = p * src[:, 3:4] + q * src[:, 4:5]
    rt = Q.vector_rotate(f, r)
    mut = Q.vector_rotate(f, mu)
    a = np.mod(np.arctan2(rt[:, 1], rt[:, 0]), 2 * np.pi)
    d = np.arctan2(rt[:, 2], np.hypot(rt[:, 0], rt[:, 1]))
    pt, qt, _ = M.normal_triad(a, d)
    m = mut + np.cross(np.broadcast_to(om, rt.shape), rt)
    out = src.copy()
    out[:, 0], out[:, 1] = a, d
    out[:, 3], out[:, 4] = np.sum(pt * m, 1), np.sum(qt * m, 1)
    return out


def test_frame_rotator_recovers_injected_rotation(small_noisefree):
    ds = small_noisefree
    P = M.problem_from_dataset(ds)
    mas = synth.MAS
    eps = np.array([12.0, -7.0, 15.0]) * mas
    om = np.array([-3.0, 9.0, 4.0]) * mas            # per year
    agis_src = _to_agis_frame(P, ds.src_true, eps, om)
    e_fit, o_fit = B.frame_fit(P, agis_src, ds.src_true[:, [0, 1, 3, 4]])
    assert np.allclose(e_fit, eps, atol=1e-5 * UAS)
    assert np.allclose(o_fit, om, atol=1e-5 * UAS)
    back = B.frame_apply_sources(P, agis_src, eps, om)
    err = G.source_errors(back, ds.src_true)
    assert np.max(np.abs(err)) < 1e-3 * UAS


def test_frame_rotation_leaves_residuals_invariant(small_noisefree):
    # rotating sources and attitude together (Eqs. fr1, fr-q4) changes the residuals only
    # through aberration/parallax (ICRS ephemeris) and the coefficient-level transform
    ds = small_noisefree
    P = M.problem_from_dataset(ds)
    mas = synth.MAS
    eps, om = np.array([20.0, -10.0, 5.0]) * mas, np.array([2.0, 1.0, -3.0]) * mas
    agis_src = _to_agis_frame(P, ds.src_true, eps, om)
    kn = P.knots()
    n = np.arange(P.n_coef)
    f = B.frame_f(P, eps, om, (kn[n] + kn[n + 4]) // 2)
    agis_att = Q.qmul(f, ds.att_true)
    assert np.allclose(B.frame_apply_attitude(P, agis_att, eps, om), ds.att_true, atol=1e-15)
    idx = np.arange(0, P.n_obs, 7)
    R0 = M.evaluate(P, ds.src_true, ds.att_true, ds.cal_true, idx=idx, partials=False)["R"]
    R1 = M.evaluate(P, agis_src, agis_att, ds.cal_true, idx=idx, partials=False)["R"]
    assert np.max(np.abs(R1 - R0)) < 1e-3 * 20 * mas


def test_rigorous_transform_agrees_with_linear_form(small_noisefree):
    # Eq. fr3: for 20 mas rotations second-order terms are below 0.002 uas
    ds = small_noisefree
    P = M.problem_from_dataset(ds)
    mas = synth.MAS
    eps, om = np.array([20.0, 0.0, 0.0]) * mas, np.zeros(3)
    src = ds.src_true[:50]
    out = B.frame_apply_sources(P, src, eps, om)
    _, _, r = M.normal_triad(src[:, 0], src[:, 1])
    _, _, r1 = M.normal_triad(out[:, 0], out[:, 1])
    lin = r + np.cross(r, np.broadcast_to(eps, r.shape))   # Eq. fr3 with t = t_fr
    assert np.max(np.linalg.norm(r1 - lin, axis=1)) < 0.002 * UAS


def test_source_statistics_against_the_noise():
    # Gaussian noise without outliers, sources updated from the truth (attitude and calibration
    # at the truth): (1) the formal covariances describe the errors, the robust scale estimate
    # of the normalised errors (0.390152 x the 10-90% range, the RSE of the paper's tables) is
    # 1 within its sampling error; (2) Q0 = sum w R^2 / sigma^2 with the weights of Eq. dw, which
    # already fall below 1 beyond |z| = 2, has the expectation nu E[w(z) z^2] for standard
    # normal z (about 0.93 nu, not nu): the mean of Q0 / nu over the sources, from
    # D = (Q0 - nu) / sqrt(2 nu), against that expectation by quadrature
    from scipy import integrate
    from scipy.stats import norm
    ds = synth.simulate(synth.config("small1yr", n_src=2000, seed=31, outlier_frac=0.0, min_transits=8))
    P = M.problem_from_dataset(ds)
    src1, sres, _ = B.source_update(P, ds.src_true, ds.att_true, ds.cal_true, B.Settings(seg_len=720))
    z = G.source_errors(src1, ds.src_true) / np.sqrt(np.einsum("ikk->ik", sres.cov))
    rse = 0.390152 * (np.quantile(z, 0.9, axis=0) - np.quantile(z, 0.1, axis=0))
    assert np.all(np.abs(rse - 1.0) < 0.08), rse          # sampling error of the RSE ~0.025 here
    ok = sres.nu > 20
    q0nu = 1.0 + sres.D[ok] * np.sqrt(2.0 / sres.nu[ok])
    wz2 = lambda t: WF.w_agis(t) * t * t * norm.pdf(t)  # noqa: E731
    expect = 2.0 * sum(integrate.quad(wz2, lo, hi, epsabs=1e-13)[0] for lo, hi in ((0, 2), (2, 3), (3, 40)))
    se = q0nu.std() / np.sqrt(ok.sum())
    assert 0.92 < expect < 0.94
    assert abs(q0nu.mean() - expect) < 4 * se, (q0nu.mean(), expect, se)


def test_attitude_normals_without_the_norm_term_are_singular_along_the_coefficients():
    # Sect. 5.2.3: the observations see only q = s / |s|, so scaling every coefficient of a
    # segment changes no residual and the normals from the observations alone have exactly one
    # null direction, the coefficient vector itself; the lambda^2 term of Eq. JfuncMod lifts it
    from oracle import cholesky as CH
    ds = synth.simulate(synth.config("small1yr", n_src=3000, seed=21))
    P = M.problem_from_dataset(ds)
    l_lo, l_hi = 500, 547                                  # 48 knot intervals, 51 coefficients
    kn = P.knots()
    sel = np.nonzero((ds.t_ns >= kn[l_lo]) & (ds.t_ns < kn[l_hi + 1]))[0]
    ev = M.evaluate(P, ds.src_true, ds.att_true, ds.cal_true, idx=sel)
    W = 1.0 / P.sigma[sel].astype(np.float64) ** 2
    a = ds.att_true[l_lo - 3:l_hi + 1].ravel()
    for lam in (0.0, 1e-3):
        Nb, _ = B.attitude_normals(P, ev, ev["R"], W, B.Settings(seg_len=720, lam=lam), l_lo, l_hi)
        N = CH.band_to_dense(Nb)
        e = np.linalg.eigvalsh(N) / np.linalg.eigvalsh(N)[-1]
        if lam == 0.0:
            assert e[0] < 1e-15 and e[1] > 1e-13
            assert np.linalg.norm(N @ a) < 1e-14 * np.linalg.norm(N, 2) * np.linalg.norm(a)
        else:
            assert e[0] > 1e-11


def test_first_source_update_hardly_depends_on_the_starting_sources():
    # The source update is independent of the current source values (Sect. 4.5, the footnote
    # on the zero columns of the iteration matrix) up to what a Gauss-Newton step keeps of its
    # starting point: second order in
    # the offset through the model's curvature (positions: halving the offset quarters the
    # difference) and first order through the aberration-level approximation of the partials
    # (Eq. duds; parallax and proper motions: halving halves it).  From the demonstration's
    # starting values (50 mas, zero parallax and proper motion) the update lands within 1 uas
    # of the one started at the truth; noise-free data, attitude and calibration at the truth.
    ds = synth.simulate(synth.config("small1yr", n_src=500, seed=41, min_transits=8, noise_free=True))
    P = M.problem_from_dataset(ds)
    st = B.Settings(seg_len=720, robust=False)
    rng = np.random.default_rng(0)
    off = np.column_stack([rng.normal(size=(ds.n_src, 2)) * 50 * synth.MAS, -ds.src_true[:, 2:]])
    out = {}
    for scale in (0.0, 0.5, 1.0):
        s0 = ds.src_true.copy()
        s0[:, 0] += scale * off[:, 0] / np.cos(s0[:, 1])
        s0[:, 1] += scale * off[:, 1]
        s0[:, 2:] += scale * off[:, 2:]
        out[scale], _, _ = B.source_update(P, s0, ds.att_true, ds.cal_true, st)
    full = np.abs(G.source_errors(out[1.0], out[0.0])).max(axis=0)
    half = np.abs(G.source_errors(out[0.5], out[0.0])).max(axis=0)
    assert np.all(full < 1.0 * UAS), full / UAS
    assert np.all(half < 0.6 * full), half / full
