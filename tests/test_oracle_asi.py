"""Pins of the accelerated simple iteration (Sect. 4.7, oracle/asi.py): the lambda estimator
on hand-worked samples, the extrapolation on a linear two-block system where one accelerated
step must land on the exact solution (and where extrapolating both blocks must not), and the
first-order residual correction against residuals re-evaluated at the corrected sources."""
import numpy as np
import scipy.linalg as sl

from oracle import asi as ASI
from oracle import model as M


def _upd(plx):
    d = np.zeros((len(plx), 5))
    d[:, 2] = plx
    return d


def test_lambda_estimate_hand_worked():
    d0 = _upd([2.0, 1.0, 0.0, 4.0, 1.0, 2.0, 1.0, 3.0])
    d1 = _upd([1.0, 0.3, 5.0, 2.0, 0.9, -0.2, 0.8, 2.7])
    # ratios 0.5, 0.3, (d0 = 0: skipped), 0.5, 0.9, -0.1, 0.8, 0.9; sorted
    # -0.1 0.3 0.5 0.5 0.8 0.9 0.9: 7 values, lower median the 4th = 0.5
    med, lam, f, n = ASI.lambda_estimate(d0, d1, 1, 0.95)
    assert (med, lam, n) == (0.5, 0.5, 7) and f == 2.0
    # stride 2: sources 0, 2, 4, 6 -> ratios 0.5, (skipped), 0.9, 0.8 -> lower median 0.8
    med, lam, f, n = ASI.lambda_estimate(d0, d1, 2, 0.95)
    assert (med, n) == (0.8, 3) and abs(f - 5.0) < 1e-15
    # an even count takes the lower of the two middle values: 0.3 0.5 | 0.8 0.9 -> 0.5
    med, _, _, n = ASI.lambda_estimate(d0[[1, 3, 4, 6]], d1[[1, 3, 4, 6]], 1, 0.95)
    assert n == 4 and med == 0.5


def test_lambda_estimate_clamps_and_empty_sample():
    d0 = _upd([1.0, 2.0, 3.0])
    assert ASI.lambda_estimate(d0, -0.5 * d0, 1, 0.9) == (-0.5, 0.0, 1.0, 3)      # oscillation: no step
    med, lam, f, n = ASI.lambda_estimate(d0, 0.99 * d0, 1, 0.9)                  # clamp
    assert abs(med - 0.99) < 1e-15 and lam == 0.9 and abs(f - 10.0) < 1e-12
    assert ASI.lambda_estimate(_upd([0.0, 0.0]), _upd([1.0, 2.0]), 1, 0.9) == (0.0, 0.0, 1.0, 0)
    inf = ASI.lambda_estimate(_upd([1.0, 1.0, 1.0]), _upd([np.inf, 0.7, np.nan]), 1, 0.9)
    assert inf[0] == 0.7 and inf[3] == 1


def test_lambda_estimate_is_robust_to_a_minority_of_wild_ratios():
    rng = np.random.default_rng(0)
    n = 1001
    d0 = _upd(rng.normal(size=n))
    d1 = 0.7 * d0
    wild = rng.choice(n, 450, replace=False)
    d1[wild[:225], 2] = 50.0 * np.abs(d0[wild[:225], 2])
    d1[wild[225:], 2] = -50.0 * np.abs(d0[wild[225:], 2])
    med, lam, f, cnt = ASI.lambda_estimate(d0, d1, 1, 0.95)
    assert cnt == n and abs(med - 0.7) < 1e-15


def _two_block_system(seed, n_src=6, n_a=7, lam=0.8):
    """SPD normal matrix [[N_ss, N_sa], [N_sa', N_aa]] with N_ss block-diagonal (5x5 per
    source, as in the S block) and a rank-one coupling N_sa = k u w', so that the
    Gauss-Seidel iteration matrix has the single non-zero eigenvalue
    lam = k^2 (u' N_ss^-1 u)(w' N_aa^-1 w)."""
    rng = np.random.default_rng(seed)
    blocks = []
    for _ in range(n_src):
        m = rng.normal(size=(5, 5))
        blocks.append(m @ m.T + 5 * np.eye(5))
    Nss = sl.block_diag(*blocks)
    m = rng.normal(size=(n_a, n_a))
    Naa = m @ m.T + n_a * np.eye(n_a)
    u, w = rng.normal(size=5 * n_src), rng.normal(size=n_a)
    k = np.sqrt(lam / ((u @ np.linalg.solve(Nss, u)) * (w @ np.linalg.solve(Naa, w))))
    Nsa = k * np.outer(u, w)
    b_s, b_a = rng.normal(size=5 * n_src), rng.normal(size=n_a)
    full = np.block([[Nss, Nsa], [Nsa.T, Naa]])
    x = np.linalg.solve(full, np.concatenate([b_s, b_a]))
    return Nss, Nsa, Naa, b_s, b_a, x[:5 * n_src], x[5 * n_src:]


def test_one_accelerated_step_solves_a_two_block_system_with_rank_one_coupling():
    # S then A in Gauss-Seidel order, as in S[ACG].  With a rank-one coupling the error after
    # the first iteration lies along the only eigenvector of the iteration matrix, the source
    # updates of iterations 3 and 4 are exactly proportional, and extrapolating the source
    # update of iteration 4 by 1/(1 - lambda) (A then solving against the extrapolated
    # sources) leaves no error at all.
    n_src = 6
    Nss, Nsa, Naa, b_s, b_a, s_star, a_star = _two_block_system(1, n_src=n_src)
    s_update = lambda s, a: np.linalg.solve(Nss, b_s - Nss @ s - Nsa @ a)
    a_update = lambda s, a: np.linalg.solve(Naa, b_a - Nsa.T @ s - Naa @ a)
    s, a = np.zeros_like(s_star), np.zeros_like(a_star)
    hist = []
    for _ in range(3):
        d = s_update(s, a)
        s = s + d
        a = a + a_update(s, a)
        hist.append(d)
    d4 = s_update(s, a)
    med, lam, f, cnt = ASI.lambda_estimate(hist[-1].reshape(n_src, 5), d4.reshape(n_src, 5), 1, 0.99)
    assert cnt == n_src and abs(lam - 0.8) < 1e-9
    scale = np.linalg.norm(np.concatenate([s_star, a_star]))
    # plain step: the error shrinks by lambda only
    s_p = s + d4
    a_p = a + a_update(s_p, a)
    err_plain = np.linalg.norm(np.concatenate([s_p - s_star, a_p - a_star])) / scale
    # accelerated step (source update only)
    s_x = s + d4 + ASI.correction(d4.reshape(n_src, 5), f).ravel()
    a_x = a + a_update(s_x, a)
    err_asi = np.linalg.norm(np.concatenate([s_x - s_star, a_x - a_star])) / scale
    # both blocks extrapolated: overshoots the attitude-like block by lambda / (1 - lambda)
    a_b = a + f * a_update(s_x, a)
    err_both = np.linalg.norm(np.concatenate([s_x - s_star, a_b - a_star])) / scale
    assert err_plain > 1e-2
    assert err_asi < 1e-10
    assert err_both > err_plain


def test_residual_correction_is_first_order(small_noisefree):
    ds = small_noisefree
    P = M.problem_from_dataset(ds)
    src = ds.src_true
    ev = M.evaluate(P, src, ds.att_true, ds.cal_true)
    rng = np.random.default_rng(3)
    c = rng.normal(size=(P.n_src, 5)) * 1e-6          # rad and rad/yr, tangent units
    diffs = []
    for s in (1.0, 0.5):
        cs = s * c
        lin = ASI.corrected_residuals(P, ev["R"], ev["A"], cs)
        true = M.evaluate(P, ASI.apply_to_sources(src, cs), ds.att_true, ds.cal_true, partials=False)["R"]
        first = np.abs(np.einsum("lk,lk->l", ev["A"], cs[P.src])).max()
        diffs.append(np.abs(true - lin).max())
        assert diffs[-1] < 1e-4 * first
    # the remainder is quadratic in the correction: halving c quarters it
    assert 3.0 < diffs[0] / diffs[1] < 5.0
