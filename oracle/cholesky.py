"""Robust Cholesky for positive semidefinite matrices without pivoting, App. C.

Algorithms C.1 (factor, with rank-defect estimate), C.2 (forward) and C.3
(back substitution) written as stated, on dense matrices and on matrices
stored by their upper band (the envelope is preserved, App. C.2).

Reading: C.1 tests a pivot N_jj - s against zero.  In floating point an exactly
singular direction leaves a positive pivot of rounding size (~1e-15 N_jj) and
the division by it amplifies rounding without bound (the paper notes that the
rank estimate of C.1 is unreliable).  A pivot N_jj - s <= PIVOT_TOL * N_jj
(original diagonal) is therefore treated as zero; PIVOT_TOL = 1e-12 keeps
every genuinely determined direction, including the attitude scale that
Eq. JfuncMod regularises at the lambda^2 ~ 1e-6 level.
"""
import numpy as np

PIVOT_TOL = 1e-12


def chol_c1(N):
    """Algorithm C.1: upper-triangular U with U'U = N and the rank-defect estimate d."""
    N = np.asarray(N, dtype=np.float64)
    n = N.shape[0]
    U = N.copy()
    diag = np.diagonal(N).copy()
    d = 0
    for j in range(n):
        for i in range(j + 1):
            s = float(np.dot(U[:i, i], U[:i, j])) if i > 0 else 0.0
            if i < j:
                U[i, j] = (U[i, j] - s) / U[i, i] if U[i, i] > 0 else 0.0
            else:
                if U[j, j] - s > PIVOT_TOL * diag[j]:
                    U[j, j] = np.sqrt(U[j, j] - s)
                else:
                    U[j, j] = 0.0
                    d += 1
        U[j + 1:, j] = 0.0
    return U, d


def chol_c2(U, b):
    """Algorithm C.2: y with U'y = b (zero where U_ii = 0)."""
    y = np.array(b, dtype=np.float64, copy=True)
    n = U.shape[0]
    for i in range(n):
        if U[i, i] > 0:
            y[i] = (y[i] - np.dot(U[:i, i], y[:i])) / U[i, i]
        else:
            y[i] = 0.0
    return y


def chol_c3(U, y):
    """Algorithm C.3: x with Ux = y (zero where U_ii = 0)."""
    x = np.array(y, dtype=np.float64, copy=True)
    n = U.shape[0]
    for i in range(n - 1, -1, -1):
        if U[i, i] > 0:
            x[i] = (x[i] - np.dot(U[i, i + 1:], x[i + 1:])) / U[i, i]
        else:
            x[i] = 0.0
    return x


def solve(N, b):
    """N x = b by C.1-C.3; returns (x, U, rank defect)."""
    U, d = chol_c1(N)
    return chol_c3(U, chol_c2(U, b)), U, d


def inverse(U):
    """Full inverse N^-1 = U^-1 U'^-1 from the factor, by C.2-C.3 on the unit vectors (App. C.2)."""
    n = U.shape[0]
    out = np.zeros((n, n))
    for i in range(n):
        e = np.zeros(n)
        e[i] = 1.0
        out[:, i] = chol_c3(U, chol_c2(U, e))
    return out


# --------------------------------------------------------------------------
# banded storage: Nb[i, k] = N[i, i+k] for 0 <= k < w (upper band, half-width w-1)
# --------------------------------------------------------------------------

def band_c1(Nb):
    """Algorithm C.1 restricted to a band of width w (no fill-in outside the envelope)."""
    Nb = np.asarray(Nb, dtype=np.float64)
    n, w = Nb.shape
    Ub = Nb.copy()
    diag = Nb[:, 0].copy()
    d = 0
    # U[i, j] is stored at Ub[i, j - i]
    for j in range(n):
        i0 = max(0, j - w + 1)
        for i in range(i0, j + 1):
            # s = sum_{k=i0..i-1} U[k,i] U[k,j]
            k = np.arange(max(i0, j - w + 1), i)
            s = float(np.dot(Ub[k, i - k], Ub[k, j - k])) if k.size else 0.0
            if i < j:
                Uii = Ub[i, 0]
                Ub[i, j - i] = (Ub[i, j - i] - s) / Uii if Uii > 0 else 0.0
            else:
                if Ub[j, 0] - s > PIVOT_TOL * diag[j]:
                    Ub[j, 0] = np.sqrt(Ub[j, 0] - s)
                else:
                    Ub[j, 0] = 0.0
                    d += 1
    return Ub, d


def band_c2(Ub, b):
    """Algorithm C.2 on the band factor."""
    n, w = Ub.shape
    y = np.array(b, dtype=np.float64, copy=True)
    for i in range(n):
        if Ub[i, 0] > 0:
            k = np.arange(max(0, i - w + 1), i)
            y[i] = (y[i] - np.dot(Ub[k, i - k], y[k])) / Ub[i, 0]
        else:
            y[i] = 0.0
    return y


def band_c3(Ub, y):
    """Algorithm C.3 on the band factor."""
    n, w = Ub.shape
    x = np.array(y, dtype=np.float64, copy=True)
    for i in range(n - 1, -1, -1):
        if Ub[i, 0] > 0:
            m = min(w, n - i)
            x[i] = (x[i] - np.dot(Ub[i, 1:m], x[i + 1:i + m])) / Ub[i, 0]
        else:
            x[i] = 0.0
    return x


def band_solve(Nb, b):
    Ub, d = band_c1(Nb)
    return band_c3(Ub, band_c2(Ub, b)), Ub, d


def band_to_dense(Nb):
    n, w = Nb.shape
    N = np.zeros((n, n))
    for k in range(w):
        idx = np.arange(n - k)
        N[idx, idx + k] = Nb[idx, k]
        N[idx + k, idx] = Nb[idx, k]
    return N
