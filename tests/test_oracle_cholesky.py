"""Pins for the robust Cholesky (App. C) against LAPACK and the paper's accuracy experiment."""
import json
import os

import numpy as np

from oracle import cholesky as CH

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "cholesky_accuracy.json")))


def test_spd_matches_lapack():
    rng = np.random.default_rng(0)
    for n in (1, 2, 5, 17):
        A = rng.normal(size=(3 * n, n))
        N = A.T @ A
        b = rng.normal(size=n)
        x, U, d = CH.solve(N, b)
        assert d == 0
        assert np.allclose(U.T @ U, N, rtol=1e-12, atol=1e-12 * np.abs(N).max())
        assert np.allclose(x, np.linalg.solve(N, b), rtol=1e-10)
        assert np.allclose(CH.inverse(U), np.linalg.inv(N), rtol=1e-9, atol=1e-12)


def _psd(rng, n, r):
    # Higham-style random PSD matrix of rank r
    X = rng.normal(size=(n, r)) * np.logspace(0, -3, r)
    return X @ X.T


def test_semidefinite_accuracy_like_paper():
    rng = np.random.default_rng(1)
    u = 2.0 ** -52
    rho_N, rho_b = [], []
    for _ in range(300):
        n = int(rng.integers(5, 13))
        r = int(rng.integers(1, n))
        N = _psd(rng, n, r)
        x = rng.normal(size=n)
        b = N @ x
        xt, U, d = CH.solve(N, b)
        rho_N.append(np.linalg.norm(N - U.T @ U) / (u * np.linalg.norm(N)))
        rho_b.append(np.linalg.norm(b - N @ xt) / (u * np.linalg.norm(b)))
        assert np.all(np.isfinite(xt))
    assert np.percentile(rho_N, 99) < GOLD["rho_N_p99_max"]
    assert np.percentile(rho_b, 99) < GOLD["rho_b_p99_max"]


def test_rank_defect_counted_on_exact_zero_pivots():
    N = np.diag([4.0, 0.0, 9.0, 0.0])
    x, U, d = CH.solve(N, np.array([4.0, 0.0, 9.0, 0.0]))
    assert d == 2
    assert np.allclose(x, [1, 0, 1, 0])


def test_band_equals_dense():
    rng = np.random.default_rng(2)
    n, w = 60, 16
    A = np.zeros((3 * n, n))
    for i in range(3 * n):
        j = int(rng.integers(0, n - w + 1))
        A[i, j:j + w] = rng.normal(size=w)
    N = A.T @ A
    Nb = np.zeros((n, w))
    for k in range(w):
        Nb[:n - k, k] = np.diagonal(N, k)
    assert np.allclose(CH.band_to_dense(Nb), N)
    b = rng.normal(size=n)
    xb, Ub, db = CH.band_solve(Nb, b)
    xd, Ud, dd = CH.solve(N, b)
    assert db == dd
    assert np.allclose(xb, xd, rtol=1e-9, atol=1e-12)
