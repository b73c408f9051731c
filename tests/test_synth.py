"""The seeded input generator: determinism, layout and the statistics it promises."""
import numpy as np

import synth


def test_deterministic_and_sorted():
    a = synth.simulate(synth.config("small1yr", n_src=200))
    b = synth.simulate(synth.config("small1yr", n_src=200))
    assert a.n_obs == b.n_obs and np.array_equal(a.t_ns, b.t_ns) and np.array_equal(a.mu, b.mu)
    assert np.all(np.diff(a.src) >= 0)
    c = synth.simulate(synth.config("small1yr", n_src=200, seed=99))
    assert not np.array_equal(a.src_true, c.src_true)


def test_layout_and_ranges():
    ds = synth.simulate(synth.config("small1yr", n_src=500))
    assert ds.ccd.max() < 62 and set(np.unique(ds.fov)) <= {0, 1} and set(np.unique(ds.kind)) <= {0, 1}
    ac = ds.kind == 1
    assert np.all((ds.mu[ac] > 14) & (ds.mu[ac] < 1979))
    assert np.all(ds.t_ns >= 0) and np.all(ds.t_ns < ds.geometry["span_ns"])
    # nine AL observations per transit (eight on the row without its ninth strip) and one AC
    n_al, n_ac = np.sum(~ac), np.sum(ac)
    assert 8.5 < n_al / n_ac < 9.0
    assert ds.att_true.shape == (ds.geometry["n_coef"], 4)
    # the calibration truth satisfies the constraints
    nd = ds.geometry["n_cal_days"]
    al = ds.cal_true[:nd * 124].reshape(nd, 124)
    acp = ds.cal_true[nd * 124:].reshape(nd, 2, 7)
    assert np.allclose(al.sum(axis=1), 0, atol=1e-18) and np.allclose(acp.sum(axis=2), 0, atol=1e-17)


def test_noise_statistics():
    ds = synth.simulate(synth.config("small1yr", n_src=2000))
    z = ds.noise / ds.sigma.astype(float)
    out = np.abs(z) > 6
    assert 0.005 < out.mean() < 0.015                      # 1% outliers at 10 sigma
    assert abs(np.std(z[~out]) - 1.0) < 0.02


def test_magnitude_dependent_sigma():
    ds = synth.simulate(synth.config("uneven5yr", n_src=300, span_days=365.25, knot_dt_s=3600, min_transits=0,
                                     max_transits=0))
    s_al = ds.sigma[ds.kind == 0].astype(float) / synth.UAS
    assert 45 < s_al.min() and s_al.max() < 520


def test_independent_of_the_thread_count_in_both_calibration_modes():
    # every source draws from its own counter-based stream (and the gates from a stream of
    # their own), so the data do not depend on how the sources are split among threads
    fields = ("t_ns", "src", "ccd", "fov", "kind", "sigma", "mu", "noise", "gate", "cal_true", "att_true", "src0")
    for extra in ({}, dict(cal_generic=True, n_gate=3, cal_j_per_k=5, cal_col_bin=131)):
        a = synth.simulate(synth.config("small1yr", n_src=1500, span_days=20, seed=3, n_threads=1, **extra))
        b = synth.simulate(synth.config("small1yr", n_src=1500, span_days=20, seed=3, n_threads=4, **extra))
        assert a.n_obs > 1000
        for f in fields:
            assert np.array_equal(getattr(a, f), getattr(b, f)), (extra, f)
