"""Pins for the B-spline evaluation (App. B)."""
import numpy as np

from oracle import spline as S

DT = 3_600_000_000_000


def _knots(N=40):
    return S.uniform_knots(0, DT, N)


def test_end_knots_multiplicity():
    kn = _knots(40)
    assert kn.shape == (44,)
    assert np.all(kn[:4] == 0) and np.all(kn[-4:] == kn[40])
    assert np.all(np.diff(kn) >= 0)


def test_partition_of_unity_and_positivity():
    kn = _knots(40)
    rng = np.random.default_rng(0)
    t = rng.integers(0, kn[-1], size=2000)
    l = S.left_index(kn, t, 40)
    b = S.deboor(kn, t, l)
    assert np.allclose(b.sum(axis=1), 1.0, atol=1e-15)
    assert np.all(b >= -1e-18)


def test_deboor_equals_cox_deboor_including_end_knots():
    kn = _knots(12)
    t = np.linspace(0, kn[-1] - 1, 997).astype(np.int64)
    l = S.left_index(kn, t, 12)
    b = S.deboor(kn, t, l)
    for j in range(4):
        ref = np.array([S.cox_deboor(kn, np.array([tt]), int(ll) - 3 + j)[0] for tt, ll in zip(t, l)])
        assert np.allclose(b[:, j], ref, atol=1e-14)


def test_deboor_equals_uniform_closed_form_inside():
    kn = _knots(60)
    rng = np.random.default_rng(1)
    t = rng.integers(kn[8], kn[52], size=3000)
    l = S.left_index(kn, t, 60)
    u = (t - kn[l]).astype(np.float64) / DT
    assert np.allclose(S.deboor(kn, t, l), S.uniform_cubic(u), atol=1e-15)


def test_c2_continuity_at_interior_knots():
    # Two adjacent cubic pieces differ only by c (t - tau_k)^3: value, first and second
    # derivatives are continuous at the knot (App. B, maximally smooth spline).
    kn = _knots(30)
    rng = np.random.default_rng(2)
    c = rng.normal(size=30)

    def piece(l, t):
        t = np.asarray(t, dtype=np.int64)
        b = S.deboor(kn, t, np.full(t.shape, l))
        return b @ c[l - 3:l + 1]
    h = 600 * 1_000_000_000
    for k in range(6, 26):
        d = np.array([-2 * h, -h, 0, h, 2 * h])
        diff = piece(k - 1, kn[k] + d) - piece(k, kn[k] + d)
        assert abs(diff[2]) < 1e-14
        assert np.allclose(diff[[0, 1, 3, 4]] / np.array([-8.0, -1.0, 1.0, 8.0]), diff[3], rtol=1e-6, atol=1e-15)


def test_left_index_clamps():
    kn = _knots(20)
    l = S.left_index(kn, np.array([0, kn[-1], kn[-1] - 1]), 20)
    assert l[0] == 3 and l[1] == 19 and l[2] == 19
