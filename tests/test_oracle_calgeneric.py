"""Pins of the full geometric calibration (Sect. 3.4 Eq. etazeta, Sect. 5.3; oracle/calgeneric.py):
the shifted Legendre polynomials in closed form, the reduction to the offsets-only model, the
null space of a group's AL normals (exactly three transfer vectors per long interval when the
observations sit at column centres), the constrained solution against the paper's own two
forms where the degeneracy is exact and against brute-force solves where it is not,
recovery of a constrained truth from noise-free data, the constraints after an update, the
basic angle of Eq. DeltaGamma, parameters without observations, and the column rounding."""
import numpy as np

from oracle import calgeneric as G
from oracle import cholesky as CH
from oracle import model as OM


def _obs(L, n, rng, centres=False, ac_frac=0.2, cols=None):
    kind = (rng.random(n) < ac_frac).astype(np.int64)
    fov = rng.integers(0, 2, n)
    ccd = rng.integers(0, L.n_ccd, n)
    gate = rng.integers(0, L.n_gate, n)
    j = rng.integers(0, L.n_j, n)
    c = rng.integers(0, L.n_col, n) if cols is None else rng.choice(cols, n)
    mu = 14.0 + c + (0.0 if centres else rng.uniform(-0.5, 0.5, n))
    mu = np.clip(mu, 13.5, 13.5 + L.n_col - 1e-9)
    return kind, fov, ccd, gate, j, mu


def test_legendre_star_closed_form():
    x = np.array([0.0, 0.5, 1.0])
    assert np.array_equal(G.legendre_star(0, x), [1.0, 1.0, 1.0])
    assert np.array_equal(G.legendre_star(1, x), [-1.0, 0.0, 1.0])
    assert np.array_equal(G.legendre_star(2, x), [1.0, -0.5, 1.0])
    # orthogonal on [0, 1] with norm 1 / (2r + 1): 5-point Gauss-Legendre is exact to degree 9
    t, w = np.polynomial.legendre.leggauss(5)
    xq, wq = 0.5 * (t + 1.0), 0.5 * w
    for r in range(3):
        for s in range(3):
            v = np.sum(wq * G.legendre_star(r, xq) * G.legendre_star(s, xq))
            assert abs(v - (1.0 / (2 * r + 1) if r == s else 0.0)) < 1e-15


def test_column_rounding():
    L = G.Layout(n_col=1966)
    mu = np.array([13.6, 14.0, 14.49, 14.5, 15.49, 1979.0, 1979.4])
    assert L.column(mu).tolist() == [0, 0, 0, 1, 1, 1965, 1965]
    assert abs(L.x(13.5)) == 0.0 and L.x(13.5 + 1966) == 1.0


def test_reduces_to_the_offsets_model(small_noisefree):
    # the r = 0 terms of one gate, one short interval per day and no small-scale terms give
    # the offsets model of oracle.model exactly (same parameter values, same lines)
    ds = small_noisefree
    P = OM.problem_from_dataset(ds)
    nd = P.n_cal_days
    L = G.Layout(n_ccd=62, n_gate=1, n_j=nd, j_per_k=1)
    rng = np.random.default_rng(0)
    cal = rng.normal(size=P.n_cal) * 1e-8
    gen = np.zeros(L.n_params)
    day = OM.cal_day(P, P.t_ns)
    for d in range(nd):
        for f in (0, 1):
            n = np.arange(62)
            gen[L.deta_large(n, 0, d, f, 0)] = cal[(d * 2 + f) * 62 + n]
            gen[L.dzeta_large(n, 0, d, f, 0)] = cal[nd * 124 + (d * 2 + f) * 7 + P.ccd_row[n]]
    cols, vals = G.design(L, P.kind, P.fov, P.ccd, np.zeros(P.n_obs, int), day, P.mu)
    k = OM.cal_index(P, P.t_ns, P.fov, P.ccd, P.kind)
    assert np.array_equal(G.line_term(gen, cols, vals), cal[k])


def _degenerate_group(seed, n=3000):
    # one CCD, one gate, one long interval of two short ones, 12 columns; AL observations at
    # column centres covering every (f, j, column)
    L = G.Layout(n_ccd=1, n_gate=1, n_j=2, j_per_k=2, n_col=12)
    rng = np.random.default_rng(seed)
    kind, fov, ccd, gate, j, mu = _obs(L, n, rng, centres=True, ac_frac=0.0)
    cols, vals = G.design(L, kind, fov, ccd, gate, j, mu)
    R = rng.normal(size=n) * 1e-9
    W = rng.uniform(0.5, 2.0, n) * 1e16
    Nal, bal, _, _ = G.group_normals(L, cols, vals, R, W)
    return L, Nal[0], bal[0]


def _transfer_vectors(L):
    # a quadratic moved from the large-scale terms of every j in k (both fields) into the
    # small-scale terms
    Z = np.zeros((L.al_size, 3))
    xm = (np.arange(L.n_col) + 0.5) / L.n_col
    for r in range(3):
        for jj in range(L.j_per_k):
            for f in (0, 1):
                Z[jj * 6 + f * 3 + r, r] = -1.0
        Z[6 * L.j_per_k:, r] = G.legendre_star(r, xm)
    return Z


def test_null_space_of_the_al_normals():
    L, N, _ = _degenerate_group(1)
    ev = np.linalg.eigvalsh(N)
    assert np.sum(ev < 1e-13 * ev.max()) == 3 and ev[3] > 1e-6 * ev.max()
    Z = _transfer_vectors(L)
    assert np.linalg.norm(N @ Z) < 1e-13 * np.linalg.norm(N) * np.linalg.norm(Z)
    # cc2 fixes exactly those directions
    C2 = G.cc2_matrix(L)
    assert np.linalg.cond(C2.T @ Z) < 1e3


def test_constrained_solution_equals_the_papers_forms_where_degenerate():
    L, N, b = _degenerate_group(2)
    C2 = G.cc2_matrix(L)
    x, rd = G.constrained_solve(N, b, C2)
    assert rd == 0
    scale = np.abs(x).max()
    # feasible (the normal equations hold: the constraint only picks among their solutions)
    assert np.linalg.norm(N @ x - b) < 1e-9 * np.linalg.norm(b)
    assert np.abs(C2.T @ x).max() < 1e-12 * scale * L.n_col
    # (N + lambda^2 C C') x = b for any lambda (the paper's positive-definite form)
    m = np.trace(N) / N.shape[0]
    for lam2 in (1e-3 * m, m, 1e3 * m):
        xl, _, _ = CH.solve(N + lam2 * (C2 @ C2.T), b)
        assert np.abs(xl - x).max() < 1e-8 * scale
    # and the oblique form of Eq. calCon: any feasible solution minus the null-space component
    # that violates the constraint, d~ - Z (C'Z)^-1 C' d~
    Z = _transfer_vectors(L)
    dt = np.linalg.lstsq(N, b, rcond=1e-13)[0] + Z @ np.array([3e-9, -1e-9, 2e-9])
    xo = dt - Z @ np.linalg.solve(C2.T @ Z, C2.T @ dt)
    assert np.abs(xo - x).max() < 1e-8 * scale


def test_constrained_solution_matches_brute_force_where_not_degenerate():
    # continuous mu: the r = 0 transfer stays an exact null direction (L*_0 = 1), the r = 1, 2
    # ones are near-null, and the unconstrained least squares break cc2.  Two brute-force
    # solves of the constrained problem: the KKT system with its blocks balanced (N ~ 1e16
    # beside C ~ 1 would leave it at cond ~ 1e35), and the projected system on an SVD basis of
    # the constraint's null space solved by least squares
    import scipy.linalg as sl
    L = G.Layout(n_ccd=1, n_gate=1, n_j=2, j_per_k=2, n_col=12)
    rng = np.random.default_rng(3)
    kind, fov, ccd, gate, j, mu = _obs(L, 3000, rng, ac_frac=0.0)
    cols, vals = G.design(L, kind, fov, ccd, gate, j, mu)
    R = rng.normal(size=3000) * 1e-9
    W = np.full(3000, 1e16)
    Nal, bal, _, _ = G.group_normals(L, cols, vals, R, W)
    N, b = Nal[0], bal[0]
    C2 = G.cc2_matrix(L)
    x, rd = G.constrained_solve(N, b, C2)
    s = L.al_size
    sc = np.sqrt(np.trace(N) / s)
    K = np.block([[N, sc * C2], [sc * C2.T, np.zeros((3, 3))]])
    xk = np.linalg.solve(K, np.concatenate([b, np.zeros(3)]))[:s]
    assert rd == 0 and np.abs(x - xk).max() < 1e-8 * np.abs(xk).max()
    Z = sl.null_space(C2.T)
    xs = Z @ np.linalg.lstsq(Z.T @ N @ Z, Z.T @ b, rcond=None)[0]
    assert np.abs(x - xs).max() < 1e-10 * np.abs(xs).max()
    x_free = np.linalg.lstsq(N, b, rcond=None)[0]
    assert np.abs(C2.T @ x_free).max() > 1e3 * np.abs(C2.T @ x).max()


def _constrained_truth(L, rng):
    c = rng.normal(size=L.n_params) * 1e-8
    C2 = G.cc2_matrix(L)
    for g in range(L.n_groups):
        v = c[g * L.al_size:(g + 1) * L.al_size]
        v -= C2 @ np.linalg.solve(C2.T @ C2, C2.T @ v)
    for idx in G.zero_point_groups(L):
        c[idx] -= np.mean(c[idx])
    return c


def _constraint_sums(L, c):
    C2 = G.cc2_matrix(L)
    s2 = max(np.abs(C2.T @ c[g * L.al_size:(g + 1) * L.al_size]).max() for g in range(L.n_groups))
    s13 = max(abs(np.sum(c[idx])) for idx in G.zero_point_groups(L))
    return s2, s13


def test_update_recovers_a_constrained_truth_from_noise_free_data():
    L = G.Layout(n_ccd=3, n_gate=2, n_j=4, j_per_k=2, n_col=24, col_bin=2)
    rng = np.random.default_rng(4)
    n = 20_000
    kind, fov, ccd, gate, j, mu = _obs(L, n, rng)
    cols, vals = G.design(L, kind, fov, ccd, gate, j, mu)
    c_true = _constrained_truth(L, rng)
    # residuals at c = 0 of data whose residuals vanish at the truth: R = line(0) - line(c_true)
    R = -G.line_term(c_true, cols, vals)
    W = rng.uniform(0.5, 2.0, n) * 1e16
    d, rd = G.update(L, cols, vals, R, W)
    assert rd == 0
    assert np.abs(d - c_true).max() < 1e-9 * np.abs(c_true).max()


def test_constraints_hold_after_an_update():
    L = G.Layout(n_ccd=3, n_gate=2, n_j=4, j_per_k=2, n_col=24)
    rng = np.random.default_rng(5)
    n = 20_000
    kind, fov, ccd, gate, j, mu = _obs(L, n, rng)
    cols, vals = G.design(L, kind, fov, ccd, gate, j, mu)
    R = rng.normal(size=n) * 1e-9
    W = rng.uniform(0.5, 2.0, n) * 1e16
    d, _ = G.update(L, cols, vals, R, W)
    s2, s13 = _constraint_sums(L, d)
    assert s2 < 1e-12 * np.abs(d).max() * L.n_col and s13 < 1e-13 * np.abs(d).max() * L.n_ccd


def test_basic_angle():
    # a basic-angle change delta shows up as +delta/2 in the preceding and -delta/2 in the
    # following field (Sect. 3.4); Eq. DeltaGamma returns it, and a common offset cancels
    L = G.Layout(n_ccd=62, n_gate=1, n_j=3, j_per_k=3, n_col=12)
    c = np.zeros(L.n_params)
    n = np.arange(62)
    rng = np.random.default_rng(6)
    delta = np.array([1e-9, -2e-9, 0.0])
    for jj in range(3):
        common = rng.normal(size=62) * 1e-8
        c[L.deta_large(n, 0, jj, 0, 0)] = common + delta[jj] / 2
        c[L.deta_large(n, 0, jj, 1, 0)] = common - delta[jj] / 2
    assert np.allclose(G.delta_gamma(L, c), delta, rtol=0, atol=1e-22)
    # recovered by an update from noise-free data (the change satisfies cc1)
    kind, fov, ccd, gate, j, mu = _obs(L, 30_000, rng, ac_frac=0.0)
    cols, vals = G.design(L, kind, fov, ccd, gate, j, mu)
    c_true = np.zeros(L.n_params)
    for jj in range(3):
        c_true[L.deta_large(n, 0, jj, 0, 0)] = delta[jj] / 2
        c_true[L.deta_large(n, 0, jj, 1, 0)] = -delta[jj] / 2
    d, _ = G.update(L, cols, vals, -G.line_term(c_true, cols, vals), np.full(30_000, 1e16))
    assert np.allclose(G.delta_gamma(L, d), delta, rtol=0, atol=1e-18)


def test_parameters_without_observations():
    # AL observations on half of the columns only, no AC: the other small-scale parameters
    # and every AC parameter are 0 and count in the rank defect; the observed ones equal the
    # KKT solution of the observed part with cc2 summed over the observed columns
    L = G.Layout(n_ccd=1, n_gate=1, n_j=2, j_per_k=2, n_col=12)
    rng = np.random.default_rng(7)
    seen = np.arange(0, 12, 2)
    kind, fov, ccd, gate, j, mu = _obs(L, 3000, rng, ac_frac=0.0, cols=seen)
    cols, vals = G.design(L, kind, fov, ccd, gate, j, mu)
    R = rng.normal(size=3000) * 1e-9
    W = np.full(3000, 1e16)
    d, rd = G.update(L, cols, vals, R, W)
    small = d[12:24]
    unseen = np.setdiff1d(np.arange(12), seen)
    assert np.all(small[unseen] == 0.0) and np.all(d[L.n_al:] == 0.0)
    assert rd == unseen.size + 6
    Nal, bal, _, _ = G.group_normals(L, cols, vals, R, W)
    F = np.r_[np.arange(12), 12 + seen]
    C = G.cc2_matrix(L)[F]
    NF = Nal[0][np.ix_(F, F)]
    sc = np.sqrt(np.trace(NF) / F.size)   # balanced blocks, as in the brute-force test above
    K = np.block([[NF, sc * C], [sc * C.T, np.zeros((3, 3))]])
    xk = np.linalg.solve(K, np.concatenate([bal[0][F], np.zeros(3)]))[:F.size]
    # cc1 then subtracts the mean of the two fields' r = 0 terms of each j (one CCD here)
    for jj in range(2):
        i0, i1 = jj * 6 + 0, jj * 6 + 3
        m = 0.5 * (xk[i0] + xk[i1])
        xk[i0] -= m
        xk[i1] -= m
    assert np.abs(d[F] - xk).max() < 1e-8 * np.abs(xk).max()


def test_cc2_weights_are_the_column_centre_legendre_values():
    # Eq. cc2 weighs column m with L*_r((m - 13.5) / n_col), m = 14 for the first column, i.e.
    # x at the column centres (c + 1/2) / n_col; a bin sums its columns
    L = G.Layout(n_col=10, col_bin=1)
    xc = (np.arange(10) + 0.5) / 10
    expect = np.array([np.ones(10), 2 * xc - 1, 6 * xc ** 2 - 6 * xc + 1])
    assert np.allclose(G.cc2_weights(L), expect, rtol=0, atol=1e-15)
    Lb = G.Layout(n_col=10, col_bin=3)
    got = G.cc2_weights(Lb)
    assert got.shape == (3, 4)
    assert np.allclose(got[:, 0], expect[:, 0:3].sum(axis=1)) and np.allclose(got[:, 3], expect[:, 9])


def test_zero_point_constraints_cover_the_nongated_offsets():
    # Eq. cc1: the r = 0, g = 0 AL terms of every CCD and both fields, one sum per short
    # interval; Eq. cc3: the r = 0, g = 0 AC terms of every CCD, one sum per field and long
    # interval; nothing else
    L = G.Layout(n_ccd=4, n_gate=3, n_j=6, j_per_k=3, n_col=8)
    groups = G.zero_point_groups(L)
    assert len(groups) == L.n_j + 2 * L.n_k
    for j in range(L.n_j):
        expect = {int(L.deta_large(n, 0, j, f, 0)) for n in range(4) for f in (0, 1)}
        assert set(groups[j].tolist()) == expect
    for k in range(L.n_k):
        for f in (0, 1):
            expect = {int(L.dzeta_large(n, 0, k, f, 0)) for n in range(4)}
            assert set(groups[L.n_j + 2 * k + f].tolist()) == expect
    # and the layout gives every parameter one index
    idx = [L.deta_large(n, g, j, f, r) for n in range(4) for g in range(3) for j in range(6) for f in (0, 1)
           for r in range(3)]
    idx += [L.deta_small(n, g, k, b) for n in range(4) for g in range(3) for k in range(2) for b in range(8)]
    idx += [L.dzeta_large(n, g, k, f, r) for n in range(4) for g in range(3) for k in range(2) for f in (0, 1)
            for r in range(3)]
    assert sorted(int(i) for i in idx) == list(range(L.n_params))


# --- the generic model through the oracle's observation model and C block, on generated data

import pytest  # noqa: E402

import synth  # noqa: E402
from oracle import blocks as OB  # noqa: E402


@pytest.fixture(scope="module")
def generic_ds():
    # noise-free, 40k sources over 30 days: 2 gates (G + N(0, 0.15) below 13 gated), one
    # 30-day long interval, 10 column bins; ~5.4e5 observations, every (CCD, gate) group
    # determined
    return synth.simulate(synth.config("small1yr", n_src=40_000, span_days=30, seed=11, noise_free=True,
                                       cal_generic=True, n_gate=2, cal_j_per_k=30, cal_col_bin=197))


def test_generated_data_follow_the_generic_model(generic_ds):
    # the residuals of the oracle's model at the truth are the generator's realised noise (here
    # the rounding of the times to ns), so the two implementations of Eq. etazeta agree; the
    # data carry gated observations, sources seen with both gates, AL pixel coordinates
    ds = generic_ds
    P = OM.problem_from_dataset(ds)
    assert P.calg is not None and P.n_cal == ds.n_cal
    R = OM.evaluate(P, ds.src_true, ds.att_true, ds.cal_true, partials=False)["R"]
    assert np.all(np.abs(R - ds.noise) <= 1e-9 * np.abs(ds.noise) + 1e-15)
    assert 0.05 < np.mean(ds.gate > 0) < 0.5
    lo = np.full(ds.n_src, 9)
    hi = np.zeros(ds.n_src, int)
    np.minimum.at(lo, ds.src, ds.gate)
    np.maximum.at(hi, ds.src, ds.gate)
    assert np.sum(lo != hi) > 500
    al = ds.kind == 0
    assert ds.mu[al].min() > 14.0 and ds.mu[al].max() < 1979.0


def test_one_calibration_update_recovers_the_truth(generic_ds):
    # sources and attitude at the truth, calibration from zero: one C update (Sect. 5.3) gives
    # back the truth to the noise of the data (|noise| <= 0.05 uas from the ns rounding): every
    # observed parameter, the residuals, and the basic angle of every day
    ds = generic_ds
    P = OM.problem_from_dataset(ds)
    ev = OM.evaluate(P, ds.src_true, ds.att_true, np.zeros(ds.n_cal))
    W = 1.0 / ds.sigma.astype(np.float64) ** 2
    cal1, rd = OB.calibration_update(P, np.zeros(ds.n_cal), ev, ev["R"], W)
    noise = np.abs(ds.noise).max()
    Nal, _, Nac, _ = G.group_normals(P.calg, ev["cal_cols"], ev["cal_vals"], ev["R"], W)
    obs = np.r_[np.concatenate([np.diagonal(N) for N in Nal]), np.concatenate([np.diagonal(N) for N in Nac])] > 0
    assert rd == np.sum(~obs)                       # the only rank defects: unobserved parameters
    assert np.abs(cal1 - ds.cal_true)[obs].max() < 2 * noise
    R1 = OM.evaluate(P, ds.src_true, ds.att_true, cal1, partials=False)["R"]
    assert np.abs(R1).max() < 2 * noise
    assert np.abs(G.delta_gamma(P.calg, cal1) - G.delta_gamma(P.calg, ds.cal_true)).max() < noise


def test_constrained_solve_over_random_layouts():
    # random group shapes (short intervals per long one, columns, bin width) and random data:
    # the null-space solution equals the balanced KKT solve and satisfies cc2
    for seed in range(12):
        rng = np.random.default_rng(100 + seed)
        nj = int(rng.integers(1, 4))
        L = G.Layout(n_ccd=1, n_gate=1, n_j=nj, j_per_k=nj, n_col=int(rng.integers(6, 21)),
                     col_bin=int(rng.integers(1, 4)))
        n = 200 * L.al_size
        kind, fov, ccd, gate, j, mu = _obs(L, n, rng, ac_frac=0.0)
        cols, vals = G.design(L, kind, fov, ccd, gate, j, mu)
        R = rng.normal(size=n) * 1e-9
        W = rng.uniform(0.2, 5.0, n) * 1e16
        Nal, bal, _, _ = G.group_normals(L, cols, vals, R, W)
        N, b = Nal[0], bal[0]
        C2 = G.cc2_matrix(L)
        x, rd = G.constrained_solve(N, b, C2)
        sc = np.sqrt(np.trace(N) / L.al_size)
        K = np.block([[N, sc * C2], [sc * C2.T, np.zeros((3, 3))]])
        xk = np.linalg.solve(K, np.concatenate([b, np.zeros(3)]))[:L.al_size]
        assert rd == 0, (seed, rd)
        assert np.abs(x - xk).max() < 1e-8 * np.abs(xk).max(), seed
        assert np.abs(C2.T @ x).max() < 1e-12 * np.abs(x).max() * L.n_col, seed


def test_truth_is_a_fixed_point_of_the_whole_iteration():
    # one S[AC] iteration with the frame rotator (oracle/agis.py) from the truth of noise-free
    # one-year data of the full model (one gate, 3-day long intervals, 2 column bins): every
    # block sees residuals at the nanosecond-rounding floor (0.016 uas RMS, 0.044 max per
    # observation) and stays there.  The lines seen by the observations (attitude and
    # calibration together) move by < 0.03 uas RMS; the sources by < 0.2 uas RMS per parameter
    # (the offsets-only model, with a quarter of the calibration unknowns, stays below 0.1).
    from oracle import agis as OG
    ds = synth.simulate(synth.config("small1yr", n_src=3000, seed=21, noise_free=True, cal_generic=True,
                                     n_gate=1, cal_j_per_k=3, cal_col_bin=983))
    P = OM.problem_from_dataset(ds)
    new, stats, _ = OG.iterate_once(P, OG.State(ds.src_true.copy(), ds.att_true.copy(), ds.cal_true.copy()),
                                    OB.Settings(seg_len=720), ref=ds.src_true[:, [0, 1, 3, 4]])
    UAS = synth.UAS
    e = OG.source_errors(new.src, ds.src_true)
    assert np.all(np.sqrt(np.mean(e ** 2, axis=0)) < 0.2 * UAS)
    R0 = OM.evaluate(P, ds.src_true, ds.att_true, ds.cal_true, partials=False)["R"]
    R1 = OM.evaluate(P, ds.src_true, new.att, new.cal, partials=False)["R"]
    assert np.sqrt(np.mean((R1 - R0) ** 2)) < 0.03 * UAS and np.abs(R1 - R0).max() < 0.5 * UAS
    assert np.abs(stats.frame).max() < 0.01 * UAS
    s2 = max(np.abs(G.cc2_matrix(P.calg).T @ new.cal[g * P.calg.al_size:(g + 1) * P.calg.al_size]).max()
             for g in range(P.calg.n_groups))
    assert s2 < 1e-12 * np.abs(new.cal).max() * P.calg.n_col


def test_block_elimination_gives_the_same_constrained_solution():
    # An independent route to a group's constrained least-squares solution: eliminate each
    # short interval's 6x6 block of large-scale terms (the Schur complement onto the
    # small-scale terms), impose cc2 on the reduced system (it acts on the small-scale terms
    # alone), back-substitute.  Equal to the oracle's dense null-space solve.
    import scipy.linalg as sl
    L = G.Layout(n_ccd=1, n_gate=1, n_j=4, j_per_k=4, n_col=30, col_bin=2)
    rng = np.random.default_rng(11)
    kind, fov, ccd, gate, j, mu = _obs(L, 6000, rng, ac_frac=0.0)
    cols, vals = G.design(L, kind, fov, ccd, gate, j, mu)
    Nal, bal, _, _ = G.group_normals(L, cols, vals, rng.normal(size=6000) * 1e-9, rng.uniform(0.5, 2, 6000) * 1e16)
    N, b = Nal[0], bal[0]
    C2 = G.cc2_matrix(L)
    x, rd = G.constrained_solve(N, b, C2)
    big = [np.arange(6 * k, 6 * k + 6) for k in range(L.j_per_k)]
    sm = np.arange(6 * L.j_per_k, L.al_size)
    S = N[np.ix_(sm, sm)].copy()
    bs = b[sm].copy()
    for J in big:
        Bj, Cj = N[np.ix_(J, J)], N[np.ix_(J, sm)]
        S -= Cj.T @ np.linalg.solve(Bj, Cj)
        bs -= Cj.T @ np.linalg.solve(Bj, b[J])
    Z = sl.null_space(C2[sm].T)
    v = Z @ np.linalg.solve(Z.T @ S @ Z, Z.T @ bs)
    u = [np.linalg.solve(N[np.ix_(J, J)], b[J] - N[np.ix_(J, sm)] @ v) for J in big]
    xe = np.concatenate(u + [v])
    assert rd == 0 and np.abs(x - xe).max() < 1e-9 * np.abs(xe).max()
