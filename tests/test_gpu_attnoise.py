"""The excess attitude noise (Sect. 5.2.5) on the GPU, in the FP64 and the mixed form, against
the oracle's iteration with the same buckets (oracle/attnoise.py, oracle/agis.py), on the
one-year 3000-source set of the parity tests with a stretch of bad attitude injected as in
the oracle's pin: eps_a^2 per component and bucket after each iteration, and the sources,
attitude (weighed with the attitude weights of Eqs. W, wl) and calibration.  8-hour buckets
(runs of a few hundred observations, staged in shared memory) and 30-day buckets (runs of tens
of thousands, selected from global memory).  The pin's own 120-day set is not used here: a few
of its sources are so poorly determined by 120 days of data that their 5x5 solutions, and the
frame fit they dominate, change with the rounding of the platform (the oracle's own on two
hosts).

Tolerance of eps_a^2.  The estimate is an order statistic (or a linear interpolation between
two adjacent ones) of x_l = R_l^2 - sigma_l^2 - eps_i^2, and an order statistic moves by no
more than the largest change of its inputs.  With the measured residual differences dR_l
after the source update and the eps_i^2 tolerance propagated from them (tests/parity_tol.py),
each x_l moves by at most 2 |R| dR + dR^2 + tol(eps_i^2): the bound is the largest of these
over the observations.  The chi^2 of the source update is compared within the bound that the
same residual differences and weight tolerances give."""
import dataclasses

import numpy as np
import pytest

import synth
from oracle import agis as OG
from oracle import attnoise as OAN
from oracle import blocks as OB
from oracle import model as OM
from oracle import quat as OQ
from parity_tol import chi2_tolerance, stat_tolerances

pytestmark = pytest.mark.gpu

UAS = synth.UAS
TOL_SRC = 0.5 * UAS
HOUR_NS = 3600 * 10**9


@pytest.fixture(scope="module")
def lib():
    import paper_1112_4139_gb300 as pkg
    pkg.build()
    from paper_1112_4139_gb300 import agis
    agis.load()
    return agis


def _with_bad_attitude(ds):
    # AL observation times of the 8-hour buckets 100..139 shifted by N(0, 5 us): ~3 sigma_AL
    # of extra AL residual there, as in the oracle's pin
    P0 = OM.problem_from_dataset(ds)
    b = OAN.bucket_of(ds.t_ns, P0.knot0_ns, 8 * HOUR_NS)
    sel = (ds.kind == 0) & (b >= 100) & (b < 140)
    dt = np.zeros(ds.n_obs, dtype=np.int64)
    dt[sel] = np.round(np.random.default_rng(7).normal(0, 5000, sel.sum())).astype(np.int64)
    return dataclasses.replace(ds, t_ns=ds.t_ns + dt)


@pytest.fixture(scope="module")
def data():
    return _with_bad_attitude(synth.simulate(synth.config("small1yr", n_src=3000, seed=21)))


@pytest.fixture(scope="module")
def data_determined():
    # for the mixed form: every source with at least 8 transits.  Its pivot tolerance (the
    # reach of FP32 normals, 64 / 2^24 of the diagonal) zeroes the weak directions of one
    # source of the set above, whose FP64 solution moves tens of mas along them.
    return _with_bad_attitude(synth.simulate(synth.config("small1yr", n_src=3000, seed=21, min_transits=8)))


def _attitude_angle_diff(P, a1, a2, t_ns):
    q1 = OM.attitude(P, a1, t_ns)[0]
    q2 = OM.attitude(P, a2, t_ns)[0]
    return np.max(np.abs(OQ.diffrot(q1, q2)))


def _deviation(P, g, state, t_ns):
    """The GPU state against the oracle's: the residuals it predicts (RMS, 99.9% quantile, the
    largest difference more than two days from the ends of the mission) and the RMS source
    difference."""
    R_or = OM.evaluate(P, state.src, state.att, state.cal, partials=False)["R"]
    dR = np.abs(g.evaluate() - R_or)
    day = 86400 * 10**9
    inner = (t_ns > t_ns.min() + 2 * day) & (t_ns < t_ns.max() - 2 * day)
    e = np.sqrt(np.mean(OG.source_errors(g.sources(), state.src) ** 2))
    return np.array([np.sqrt(np.mean(dR ** 2)), np.quantile(dR, 0.999), dR[inner].max(), e])


def _bounds(P, sres, sig2_used, g):
    """Bounds of eps_a^2 and of chi^2 from the measured differences of the residuals after the
    source update (sig2_used: the variances sigma~^2 the source update used)."""
    Rg, _ = g.residuals()
    tol_Q, tol_eps2, tol_W = stat_tolerances(P.src, P.n_src, np.sqrt(sig2_used), sres.R, Rg, sres.W, sres.eps2,
                                             sres.Qi)
    dR = np.abs(Rg - sres.R)
    eps_b = float(np.max(2 * np.abs(sres.R) * dR + dR ** 2 + tol_eps2[P.src]))
    return eps_b, chi2_tolerance(sres.R, Rg, sres.W, tol_W)


@pytest.mark.parametrize("bucket_h,n_iter,precision", [(8, 2, 0), (720, 1, 0), (8, 2, 1)])
def test_iterations_match_oracle(lib, data, data_determined, bucket_h, n_iter, precision):
    # precision 1: the mixed form (FP32 normals around float-pair residuals), whose estimate
    # is compared within the same bounds, derived from its own measured residual differences
    if precision == 1:
        data = data_determined
    plain_dev = []
    if precision == 1:
        # The mixed form's attitude update rounds its normals to FP32; on these sparse noisy
        # data (about 55 observations per knot interval) that moves its weakly determined
        # directions by tens of uas (the multiple knots at the ends of the mission by tens of
        # mas), which the observations see at the 0.1-1 uas level, and the next source update
        # inherits it.  After one iteration its attitude (through the residuals it predicts)
        # is compared against the plain mixed iteration's own deviation from the plain oracle
        # iteration on the same data: the excess attitude noise may not add to it.
        P_ = OM.problem_from_dataset(data)
        ref_ = data.src_true[:, [0, 1, 3, 4]]
        sp = OG.State(data.src_true.copy(), data.att_true.copy(), data.cal_true.copy())
        gp = lib.from_dataset(data, seg_len=720, seg_overlap=12, precision=1)
        gp.set_state(src=data.src_true, att=data.att_true, cal=data.cal_true)
        for _ in range(n_iter):
            sp, _, _ = OG.iterate_once(P_, sp, OB.Settings(seg_len=720, seg_overlap=12), ref_)
            gp.iterate(1)
            plain_dev.append(_deviation(P_, gp, sp, data.t_ns))
        gp.close()
    bucket_ns = bucket_h * HOUR_NS
    st = OB.Settings(seg_len=720, seg_overlap=12, att_noise_bucket_ns=bucket_ns)
    P = OM.problem_from_dataset(data)
    ref = data.src_true[:, [0, 1, 3, 4]]
    state = OG.State(data.src_true.copy(), data.att_true.copy(), data.cal_true.copy())
    g = lib.from_dataset(data, seg_len=720, seg_overlap=12, precision=precision)
    g.set_state(src=data.src_true, att=data.att_true, cal=data.cal_true)
    g.set_attnoise(bucket_ns)
    assert np.array_equal(g.attnoise(), np.zeros((3, int(OAN.bucket_of(data.t_ns, P.knot0_ns, bucket_ns).max()) + 1)))
    sig2 = P.sigma.astype(np.float64) ** 2
    comp = OAN.component(P.kind, P.fov)
    bucket = OAN.bucket_of(P.t_ns, P.knot0_ns, bucket_ns)
    for k in range(n_iter):
        eps2_prev = state.eps2_a if state.eps2_a is not None else np.zeros((OAN.N_COMP, int(bucket.max()) + 1))
        sig2_used = OAN.adjusted_variance(sig2, eps2_prev, comp, bucket)
        state, stats, sres = OG.iterate_once(P, state, st, ref)
        it = g.iterate(1)[0]
        e_g, e_o = g.attnoise(), state.eps2_a
        assert e_g.shape == e_o.shape
        bound, chi2_tol = _bounds(P, sres, sig2_used, g)
        d = np.abs(e_g - e_o)
        print(f"precision {precision}, bucket {bucket_h} h, iteration {k}: eps_a^2 max diff {d.max():.3e} rad^2, bound {bound:.3e}, "
              f"max eps_a^2 {e_o.max():.3e}, non-zero {np.count_nonzero(e_o)} / {e_o.size}")
        assert np.all(d <= bound), (np.argmax(d), d.max(), bound)
        if k == 0 and bucket_h == 8:
            # the injected stretch is where the estimate puts it (the oracle's pin: the
            # stretch above 0.25 and the rest below 0.05 of the injected variance)
            lo = e_g[0, 100:140].min()
            assert lo > 0.0 and np.max(np.r_[e_g[0, :95], e_g[0, 145:]]) < 0.25 * lo
        assert abs(it["s"]["chi2"] - stats.chi2) <= chi2_tol, (it["s"]["chi2"], stats.chi2, chi2_tol)
        e = OG.source_errors(g.sources(), state.src)
        if precision == 0 or k == 0:
            assert np.max(np.abs(e)) < TOL_SRC, f"max source diff {np.max(np.abs(e)) / UAS:.3e} uas"
        if precision == 0:
            assert _attitude_angle_diff(P, g.attitude(), state.att, data.t_ns) < TOL_SRC
        else:
            dev = _deviation(P, g, state, data.t_ns)
            print(f"mixed form, iteration {k}: deviation from the oracle (residuals RMS, 99.9%, max away from "
                  f"the ends; sources RMS) {np.round(dev / UAS, 4)} uas; plain mixed form "
                  f"{np.round(plain_dev[k] / UAS, 4)} uas")
            # After the first iteration the state carries that deviation through attitude
            # normals that the noise weakens by up to 1 + eps_a^2 / sigma^2 (about 60 in the
            # injected stretch), so it is not compared element-wise there; the source update of
            # that iteration is held by eps_a^2 and chi^2 within their derived bounds above (and
            # the calibration, which reads its residuals, is compared after the first only).
            if k == 0:
                assert np.all(dev <= 2.0 * plain_dev[k] + 0.01 * UAS), (dev / UAS, plain_dev[k] / UAS)
        if precision == 0 or k == 0:
            assert np.max(np.abs(g.calibration() - state.cal)) < 1e-3 * UAS
    g.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_attitude_weights_change_the_attitude_only(lib, data, precision):
    # one iteration from the truth with and without the noise: the sources (S sees eps_a^2 = 0
    # in the first iteration) and the calibration (S weights) are the same bit for bit, the
    # attitude is not; switching the noise off again restores the plain iteration
    out = {}
    for name in ("plain", "noise", "off"):
        g = lib.from_dataset(data, seg_len=720, seg_overlap=12, frame_each_iter=0, precision=precision)
        g.set_state(src=data.src_true, att=data.att_true, cal=data.cal_true)
        if name != "plain":
            g.set_attnoise(8 * HOUR_NS)
        if name == "off":
            g.set_attnoise(0)
            assert g.attnoise() is None
        g.iterate(1)
        out[name] = (g.sources(), g.attitude(), g.calibration())
        g.close()
    assert np.array_equal(out["plain"][0], out["noise"][0])
    assert np.array_equal(out["plain"][2], out["noise"][2])
    assert not np.array_equal(out["plain"][1], out["noise"][1])
    for a, b in zip(out["plain"], out["off"]):
        assert np.array_equal(a, b)


def test_rejections(lib, data):
    with pytest.raises(lib.AgisError):
        g = lib.from_dataset(data, seg_len=720, seg_overlap=12)
        try:
            g.set_attnoise(-1)
        finally:
            g.close()
    for kw in (dict(block_order=2), dict(block_order=2, precision=1)):
        g = lib.from_dataset(data, seg_len=720, seg_overlap=12, **kw)
        with pytest.raises(lib.AgisError):
            g.set_attnoise(8 * HOUR_NS)
        g.close()
    g = lib.from_dataset(data, seg_len=720, seg_overlap=12)
    g.set_asi(16, 0.9)
    with pytest.raises(lib.AgisError):
        g.set_attnoise(8 * HOUR_NS)
    g.set_asi(0)
    g.set_attnoise(8 * HOUR_NS)
    with pytest.raises(lib.AgisError):
        g.set_asi(16, 0.9)
    with pytest.raises(lib.AgisError):
        g.set_proposal(np.zeros(lib.MLP_N_PARAMS, dtype=np.float32), 5)
    g.close()
    # observations before the first bucket
    geo = dict(data.geometry)
    geo["knot0_ns"] = int(data.t_ns.min()) + 1
    d2 = dataclasses.replace(data, geometry=geo)
    g = lib.from_dataset(d2, seg_len=720, seg_overlap=12)
    with pytest.raises(lib.AgisError, match="precedes"):
        g.set_attnoise(8 * HOUR_NS)
    g.close()
