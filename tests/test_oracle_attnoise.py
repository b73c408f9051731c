"""Pins of the excess attitude noise (Sect. 5.2.5, oracle/attnoise.py): the component and
bucket mapping, the 68% quantile on values where it is obvious, the estimator's expectation
for Gaussian residuals in closed form, and the attitude weights reducing to those of the
source update when there is no excess attitude noise."""
import numpy as np
from scipy.stats import norm

from oracle import attnoise as AN
from oracle import weights as WF


def test_components_and_buckets():
    kind = np.array([0, 0, 1, 1])
    fov = np.array([0, 1, 0, 1])
    assert AN.component(kind, fov).tolist() == [0, 0, 1, 2]
    t0, dt = 1_000, 600
    t = np.array([1_000, 1_599, 1_600, 1_000 + 10 * 600 + 5])
    assert AN.bucket_of(t, t0, dt).tolist() == [0, 0, 1, 10]


def test_quantile_on_values_where_it_is_obvious():
    # 101 values 0..100 in one bucket: the 68% quantile is 68 exactly; shifted below zero the
    # estimate is clamped to 0; an empty bucket gives 0; components do not mix
    x = np.arange(101.0)
    sig2 = np.zeros(101)
    R = np.sqrt(x)
    comp = np.zeros(101, dtype=int)
    bucket = np.zeros(101, dtype=int)
    e = AN.estimate(R, sig2, np.zeros(101), comp, bucket, n_buckets=2)
    assert e.shape == (3, 2)
    assert e[0, 0] == 68.0 and e[0, 1] == 0.0 and np.all(e[1:] == 0.0)
    e = AN.estimate(R, sig2 + 200.0, np.zeros(101), comp, bucket, n_buckets=1)
    assert e[0, 0] == 0.0
    # the source's excess variance is removed like the formal one
    e = AN.estimate(R, sig2, np.full(101, 10.0), comp, bucket, n_buckets=1)
    assert e[0, 0] == 58.0
    # values of another component in the same bucket change nothing
    R2 = np.r_[R, np.full(50, 1e3)]
    e = AN.estimate(R2, np.zeros(151), np.zeros(151), np.r_[comp, np.full(50, 2)], np.zeros(151, dtype=int), 1)
    assert e[0, 0] == 68.0 and e[2, 0] == 1e6


def test_estimator_expectation_for_gaussian_residuals():
    # R ~ N(0, s^2), s^2 = sigma^2 + eps_i^2 + eps_a^2: R^2 = s^2 chi^2_1, whose 68% quantile
    # is s^2 Phi^-1(0.84)^2 = 0.9889 s^2; the estimator expects 0.9889 s^2 - sigma^2 - eps_i^2
    # (slightly below eps_a^2), and clamps a negative value to 0 when eps_a = 0
    rng = np.random.default_rng(0)
    n = 400_000
    sig2, eps_i2 = 1.0, 0.3
    k = norm.ppf(0.84) ** 2
    for eps_a2, bucket_n in ((2.0, 0), (0.5, 1), (0.0, 2)):
        s2 = sig2 + eps_i2 + eps_a2
        R = rng.normal(0.0, np.sqrt(s2), n)
        e = AN.estimate(R, np.full(n, sig2), np.full(n, eps_i2), np.zeros(n, dtype=int), np.full(n, bucket_n), 3)
        expect = max(0.0, k * s2 - sig2 - eps_i2)
        # sampling error of the quantile: sqrt(p (1-p) / n) / density of R^2 there, ~0.3% of s^2
        assert abs(e[0, bucket_n] - expect) < 0.01 * s2, (eps_a2, e[0, bucket_n], expect)


def test_attitude_weights_reduce_to_the_source_update_weights():
    rng = np.random.default_rng(1)
    n = 1000
    sig2 = rng.uniform(0.5, 2.0, n)
    R = rng.normal(0, 1, n) * np.sqrt(sig2) * 3
    comp = rng.integers(0, 3, n)
    bucket = rng.integers(0, 4, n)
    W = AN.attitude_weights(R, sig2, np.zeros(n), np.zeros((3, 4)), comp, bucket, WF.w_agis)
    assert np.array_equal(W, WF.w_agis(R / np.sqrt(sig2)) / sig2)
    # excess attitude noise widens the variance: an observation flagged by the source update
    # (|z| = 5) is no longer downweighted when eps_a^2 = 24 sigma^2 (|z| = 1)
    W1 = AN.attitude_weights(np.array([5.0]), np.array([1.0]), np.zeros(1), np.full((3, 1), 24.0),
                             np.zeros(1, dtype=int), np.zeros(1, dtype=int), WF.w_agis)
    assert W1[0] == 1.0 / 25.0 and WF.w_agis(np.array([5.0]))[0] < 1.0


def test_iteration_finds_an_injected_stretch_of_bad_attitude():
    # AL observation times of buckets 100..139 (8-h buckets) shifted by N(0, 5 us): about
    # 300 uas of extra AL residual there (3 sigma_AL).  One iteration from the truth with the
    # excess attitude noise estimated: those buckets get eps_AL^2 well above zero (the source
    # update's excess noise absorbs part of it for the sources observed then, and Eq. e09
    # subtracts it), the other AL buckets stay near zero, and the attitude weights downweight
    # far fewer of the affected observations than the source update did.
    import dataclasses
    import synth
    from oracle import agis as G
    from oracle import blocks as B
    from oracle import model as M
    ds = synth.simulate(synth.config("small1yr", n_src=2000, span_days=120, seed=5))
    P0 = M.problem_from_dataset(ds)
    bucket_ns = 8 * int(ds.geometry["knot_dt_ns"])
    b = AN.bucket_of(ds.t_ns, P0.knot0_ns, bucket_ns)
    al = ds.kind == 0
    sel = al & (b >= 100) & (b < 140)
    dt = np.zeros(ds.n_obs, dtype=np.int64)
    dt[sel] = np.round(np.random.default_rng(7).normal(0, 5000, sel.sum())).astype(np.int64)
    ds2 = dataclasses.replace(ds, t_ns=ds.t_ns + dt)
    P = M.problem_from_dataset(ds2)
    inj = (M.evaluate(P, ds.src_true, ds.att_true, ds.cal_true, partials=False)["R"]
           - M.evaluate(P0, ds.src_true, ds.att_true, ds.cal_true, partials=False)["R"])
    v = np.mean(inj[sel] ** 2)
    st = B.Settings(seg_len=720, att_noise_bucket_ns=bucket_ns)
    state, _, sres = G.iterate_once(P, G.State(ds.src_true.copy(), ds.att_true.copy(), ds.cal_true.copy()), st,
                                    ref=ds.src_true[:, [0, 1, 3, 4]])
    e = state.eps2_a
    assert e.shape == (3, int(b.max()) + 1)
    assert np.all(e[0, 100:140] > 0.25 * v) and np.all(e[0, 100:140] < 1.1 * v)
    quiet = np.r_[e[0, :95], e[0, 145:]]
    assert np.max(quiet) < 0.05 * v
    # downweighting (w < 0.2) among the affected AL observations: source update vs attitude
    sig2 = P.sigma.astype(np.float64) ** 2
    comp = AN.component(P.kind, P.fov)
    eps_i = sres.eps2[P.src]
    w_s = sres.W * (AN.adjusted_variance(sig2, np.zeros_like(e), comp, b) + eps_i)
    W_a = AN.attitude_weights(sres.R, sig2, eps_i, e, comp, b, B._wfun(st))
    w_a = W_a * (AN.adjusted_variance(sig2, e, comp, b) + eps_i)
    n_s, n_a = np.sum(w_s[sel] < 0.2), np.sum(w_a[sel] < 0.2)
    assert n_s > 0 and n_a < 0.5 * n_s, (n_s, n_a)
