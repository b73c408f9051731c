"""Parity of the GPU library (through the C ABI) with the FP64 oracle, block by block.

Tolerances: residuals |R_gpu - R_cpu| <= 1e-9 |R_cpu| + 1e-15 rad (the FP64 floor reading of
"1e-9 relative on residuals"); source parameters, calibration and attitude within 0.5 uas
(uas/yr for proper motions), the stated parity bound for the source parameters.
"""
import numpy as np
import pytest

import synth
from oracle import agis as OG
from oracle import blocks as OB
from oracle import model as OM
from oracle import quat as OQ
from parity_tol import assert_stats_close

pytestmark = pytest.mark.gpu

UAS = synth.UAS
TOL_SRC = 0.5 * UAS


def _r_ok(Rg, Rc, floor=1e-15):
    return np.abs(Rg - Rc) <= 1e-9 * np.abs(Rc) + floor


# residuals after a source update, R = h - A d, inherit the rounding of the solved d: their
# floor is the source-parameter tolerance times |A| ~ 1 instead of the fixed-parameter 1e-15
R_AFTER_S_FLOOR = 1e-3 * UAS


@pytest.fixture(scope="module")
def lib():
    import paper_1112_4139_gb300 as pkg
    pkg.build()
    from paper_1112_4139_gb300 import agis
    agis.load()
    return agis


@pytest.fixture(scope="module")
def data():
    # 3000 sources, 1 yr, 1-h knots: ~5e5 observations, 8769 coefficients, 13 segments of
    # 720 intervals with a ragged last one
    return synth.simulate(synth.config("small1yr", n_src=3000, seed=21))


def _settings(**kw):
    base = dict(seg_len=720, seg_overlap=12)
    base.update(kw)
    return OB.Settings(**base)


def _gpu(lib, ds, **kw):
    base = dict(seg_len=720, seg_overlap=12)
    base.update(kw)
    return lib.from_dataset(ds, **base)


def test_residuals_at_start(lib, data):
    P = OM.problem_from_dataset(data)
    Rc = OM.evaluate(P, data.src0, data.att0, data.cal0, partials=False)["R"]
    g = _gpu(lib, data)
    Rg = g.evaluate()
    ok = _r_ok(Rg, Rc)
    assert ok.all(), f"{(~ok).sum()} residuals off, max diff {np.abs(Rg - Rc).max():.3e}"
    # and at the truth, where the residuals are the injected noise
    g.set_state(src=data.src_true, att=data.att_true, cal=data.cal_true)
    Rt = g.evaluate()
    assert np.all(np.abs(Rt - data.noise) <= 1e-9 * np.abs(data.noise) + 2e-15)
    g.close()


def _compare_source_block(lib, ds, st, **cfg):
    P = OM.problem_from_dataset(ds)
    src1, sres, ev = OB.source_update(P, ds.src0, ds.att0, ds.cal0, st)
    g = _gpu(lib, ds, **cfg)
    stats = g.source_update()
    sg = g.sources()
    e = OG.source_errors(sg, src1)
    assert np.max(np.abs(e)) < TOL_SRC, f"max source diff {np.max(np.abs(e)) / UAS:.3e} uas"
    Rg, Wg = g.residuals()
    assert _r_ok(Rg, sres.R, R_AFTER_S_FLOOR).all(), f"R after S: max diff {np.abs(Rg - sres.R).max():.3e}"
    ss = g.source_stats()
    assert np.array_equal(ss["nu"].astype(int), sres.nu)
    assert np.array_equal(ss["n_out"].astype(int), sres.n_out)
    # W = w / (sigma^2 + eps^2), Q_i and eps_i^2 within the first-order propagation of the
    # measured residual differences (tests/parity_tol.py)
    assert_stats_close(P.src, ds.n_src, P.sigma, sres.R, Rg, sres.W, Wg, sres.eps2, ss["eps2"], sres.Qi, ss["Q"])
    assert np.allclose(ss["cov"], sres.cov, rtol=1e-7, atol=1e-12 * np.abs(sres.cov).max())
    assert abs(stats["chi2"] / np.sum(sres.W * sres.R ** 2) - 1) < 1e-10
    return g, P, src1, sres, ev


def test_source_update(lib, data):
    g, *_ = _compare_source_block(lib, data, _settings())
    g.close()


def test_source_update_plain_weights(lib, data):
    g, *_ = _compare_source_block(lib, data, _settings(robust=False), robust=0)
    g.close()


def test_source_update_huber(lib, data):
    g, *_ = _compare_source_block(lib, data, _settings(weight_fn="huber"), weight_fn=1)
    g.close()


def _attitude_angle_diff(P, a1, a2, t_ns):
    q1 = OM.attitude(P, a1, t_ns)[0]
    q2 = OM.attitude(P, a2, t_ns)[0]
    return np.max(np.abs(OQ.diffrot(q1, q2)))


def test_attitude_and_calibration_update(lib, data):
    # the paper-literal right-hand side (rhs_norm_term) is compared at 30-s knots, where its
    # lambda^2 D term is at the rounding level (tests/test_gpu_benchshape.py); at these 1-h
    # knots it asks for a spline-scale change that the matrix stiffens only at the 4 lambda^2
    # level, so its solution is not unique to the parity bound
    rhs_norm = 0
    st = _settings(rhs_norm_term=bool(rhs_norm))
    P = OM.problem_from_dataset(data)
    src1, sres, ev = OB.source_update(P, data.src0, data.att0, data.cal0, st)
    att1, rda = OB.attitude_update(P, data.att0, ev, sres.R, sres.W, st)
    cal1, rdc = OB.calibration_update(P, data.cal0, ev, sres.R, sres.W)
    g = _gpu(lib, data, rhs_norm_term=rhs_norm)
    g.source_update()
    sa = g.attitude_update()
    sc = g.calibration_update()
    ag = g.attitude()
    cg = g.calibration()
    # attitude compared as rotation angles at the observation times
    assert _attitude_angle_diff(P, ag, att1, data.t_ns) < TOL_SRC
    assert np.max(np.abs(cg - cal1)) < 1e-3 * UAS
    assert sa["rank_defect"] == rda
    assert sc["rank_defect"] == rdc
    g.close()


def test_frame_rotator(lib, data):
    st = _settings()
    P = OM.problem_from_dataset(data)
    src1, sres, ev = OB.source_update(P, data.src0, data.att0, data.cal0, st)
    ref = data.src_true[:, [0, 1, 3, 4]]
    e_c, o_c = OB.frame_fit(P, src1, ref)
    g = _gpu(lib, data)
    g.source_update()
    eo = g.frame_rotate()
    assert np.allclose(eo[:3], e_c, atol=1e-4 * UAS) and np.allclose(eo[3:], o_c, atol=1e-4 * UAS)
    s_c = OB.frame_apply_sources(P, src1, e_c, o_c)
    a_c = OB.frame_apply_attitude(P, data.att0, e_c, o_c)
    assert np.max(np.abs(OG.source_errors(g.sources(), s_c))) < TOL_SRC
    assert np.max(np.abs(g.attitude() - a_c)) < 1e-14
    # subset fit
    sub = np.arange(0, data.n_src, 3)
    g2 = _gpu(lib, data)
    g2.source_update()
    eo2 = g2.frame_rotate(sub)
    e2, o2 = OB.frame_fit(P, src1[sub], ref[sub])
    assert np.allclose(eo2, np.concatenate([e2, o2]), atol=1e-4 * UAS)
    g.close()
    g2.close()


@pytest.mark.parametrize("use_graph", [0, 1])
def test_two_iterations(lib, data, use_graph):
    st = _settings()
    P = OM.problem_from_dataset(data)
    ref = data.src_true[:, [0, 1, 3, 4]]
    state = OG.State(data.src0.copy(), data.att0.copy(), data.cal0.copy())
    hist = []
    for _ in range(2):
        state, stats, _ = OG.iterate_once(P, state, st, ref)
        hist.append(stats)
    g = _gpu(lib, data, use_graph=use_graph)
    it = g.iterate(2)
    assert len(it) == 2
    for k in range(2):
        assert abs(it[k]["s"]["chi2"] / hist[k].chi2 - 1) < 1e-8
        assert np.allclose(it[k]["frame"], hist[k].frame, atol=1e-3 * UAS)
    e = OG.source_errors(g.sources(), state.src)
    q1 = OM.attitude(P, g.attitude(), data.t_ns)[0]
    q2 = OM.attitude(P, state.att, data.t_ns)[0]
    ang = np.abs(OQ.diffrot(q1, q2))
    print(f"two iterations: sources max {np.max(np.abs(e)) / UAS:.3g} uas, attitude max {ang.max() / UAS:.3g} uas, "
          f"RMS {np.sqrt(np.mean(ang ** 2)) / UAS:.3g} uas")
    assert np.max(np.abs(e)) < TOL_SRC, f"max source diff {np.max(np.abs(e)) / UAS:.3e} uas"
    # A one-ulp random change of every starting source parameter and attitude coefficient moves
    # the oracle's own attitude after these two iterations by up to 0.36 uas (RMS 0.0012 uas,
    # at a few weakly determined knots): the attitude is compared at three times that.
    assert ang.max() < 1.1 * UAS
    assert np.sqrt(np.mean(ang ** 2)) < 0.004 * UAS
    assert np.max(np.abs(g.calibration() - state.cal)) < 1e-3 * UAS
    g.close()


def test_edge_cases_empty_and_short_sources(lib):
    # sources without observations and with fewer than 5 observations (singular 5x5)
    ds = synth.simulate(synth.config("small1yr", n_src=600, seed=5, min_transits=10))
    keep = np.ones(ds.n_obs, bool)
    first = ds.src_offsets()
    keep[first[7] + 3:first[8]] = False       # source 7: 3 observations
    keep[first[11]:first[12]] = False          # source 11: none
    keep[first[12]:first[13]] = False          # source 12: none
    import dataclasses
    sel = lambda a: np.ascontiguousarray(a[keep])  # noqa: E731
    d2 = dataclasses.replace(ds, t_ns=sel(ds.t_ns), src=sel(ds.src), ccd=sel(ds.ccd), fov=sel(ds.fov),
                             kind=sel(ds.kind), sigma=sel(ds.sigma), mu=sel(ds.mu), noise=sel(ds.noise))
    st = _settings()
    P = OM.problem_from_dataset(d2)
    src1, sres, ev = OB.source_update(P, d2.src0, d2.att0, d2.cal0, st)
    g = _gpu(lib, d2)
    g.source_update()
    sg = g.sources()
    # the 3-observation source has a rank-deficient 5x5 system: its parameters are not unique
    # (App. C), its fitted residuals are
    err = np.abs(OG.source_errors(sg, src1))
    err[7] = 0.0
    assert np.max(err) < TOL_SRC, f"source {np.argmax(err.max(axis=1))}: {err.max() / UAS:.3e} uas"
    Rg, _ = g.residuals()
    o7 = slice(P.src_offsets()[7], P.src_offsets()[8])
    assert np.all(np.abs(Rg[o7] - sres.R[o7]) < 1e-3 * UAS)
    assert np.array_equal(sg[11], d2.src0[11]) and np.array_equal(sg[12], d2.src0[12])
    ss = g.source_stats()
    assert ss["nu"][7] < 0 and np.isfinite(sg[7]).all()
    g.attitude_update()
    g.calibration_update()
    assert np.isfinite(g.attitude()).all() and np.isfinite(g.calibration()).all()
    g.close()


def test_invalid_inputs_are_rejected(lib, data):
    from paper_1112_4139_gb300.agis import AgisError
    obs = lib.obs_from_dataset(data)
    bad = dict(obs)
    bad["src"] = obs["src"][::-1].copy()
    with pytest.raises(AgisError, match="sorted"):
        lib.Agis(data.geometry, lib.default_config(), bad, data.src0, data.att0, data.cal0)
    bad = dict(obs)
    s = obs["sigma"].copy()
    s[5] = 0.0
    bad["sigma"] = s
    with pytest.raises(AgisError, match="sigma"):
        lib.Agis(data.geometry, lib.default_config(), bad, data.src0, data.att0, data.cal0)
    with pytest.raises(AgisError, match="n_cal"):
        lib.Agis(data.geometry, lib.default_config(), obs, data.src0, data.att0, data.cal0[:-1])
    # non-finite starting values and observations
    for name, arr, idx in (("src0", data.src0, (4, 2)), ("att0", data.att0, (100, 1)), ("cal0", data.cal0, (7,))):
        for v in (np.nan, np.inf, -np.inf):
            a = arr.copy()
            a[idx] = v
            args = dict(src0=data.src0, att0=data.att0, cal0=data.cal0)
            args[name] = a
            with pytest.raises(AgisError, match="non-finite starting value"):
                lib.Agis(data.geometry, lib.default_config(), obs, args["src0"], args["att0"], args["cal0"])
    bad = dict(obs)
    m = obs["mu"].copy()
    m[np.flatnonzero(data.kind == 1)[3]] = np.nan
    bad["mu"] = m
    with pytest.raises(AgisError, match="mu of an AC observation"):
        lib.Agis(data.geometry, lib.default_config(), bad, data.src0, data.att0, data.cal0)
    bad = dict(obs)
    s = obs["sigma"].copy()
    s[9] = np.inf
    bad["sigma"] = s
    with pytest.raises(AgisError, match="sigma not positive and finite"):
        lib.Agis(data.geometry, lib.default_config(), bad, data.src0, data.att0, data.cal0)
    g = _gpu(lib, data)
    with pytest.raises(AgisError, match="source update first"):
        g.attitude_update()
    g.close()


def test_attitude_data_gap(lib):
    # a 12-hour gap in the data (twelve 1-h knot intervals, more than M = 4): the coefficients
    # that no observation reaches give zero rows of the banded normals, which the robust
    # Cholesky zeroes and counts as rank defects (App. C.3) instead of failing; the attitude
    # elsewhere matches the oracle's and nothing becomes non-finite
    ds = synth.simulate(synth.config("small1yr", n_src=3000, seed=23))
    t0 = ds.geometry["knot0_ns"] + 2000 * 3600 * 10**9
    keep = (ds.t_ns < t0) | (ds.t_ns >= t0 + 12 * 3600 * 10**9)
    assert (~keep).sum() > 100
    import dataclasses
    sel = lambda a: np.ascontiguousarray(a[keep])  # noqa: E731
    d2 = dataclasses.replace(ds, t_ns=sel(ds.t_ns), src=sel(ds.src), ccd=sel(ds.ccd), fov=sel(ds.fov),
                             kind=sel(ds.kind), sigma=sel(ds.sigma), mu=sel(ds.mu), noise=sel(ds.noise))
    st = _settings()
    P = OM.problem_from_dataset(d2)
    src1, sres, ev = OB.source_update(P, d2.src0, d2.att0, d2.cal0, st)
    att1, rda = OB.attitude_update(P, d2.att0, ev, sres.R, sres.W, st)
    g = _gpu(lib, d2)
    g.source_update()
    sa = g.attitude_update()
    ag = g.attitude()
    assert rda >= 4 * 8, rda          # at least the eight coefficients inside the gap
    assert sa["rank_defect"] == rda
    assert np.isfinite(ag).all()
    assert _attitude_angle_diff(P, ag, att1, d2.t_ns) < TOL_SRC
    # the coefficients the data do not reach keep their values on both sides
    untouched = np.all(att1 == d2.att0, axis=1)
    assert untouched.sum() >= 8 and np.array_equal(ag[untouched], d2.att0[untouched])
    it = g.iterate(2)
    assert all(np.isfinite(x["s"]["chi2"]) for x in it) and np.isfinite(g.attitude()).all()
    g.close()
