"""Full geometric calibration: observation lines and calibration update, FP64 (TEST
INFRASTRUCTURE ONLY).

Observation lines (Eq. etazeta), for field f, CCD n, gate g, AC pixel coordinate mu and time t
in short interval j and long interval k:

    eta_fng(mu, t)  = eta0_ng  + sum_r Deta_rfngj L*_r(x) + deta_ngkm
    zeta_fng(mu, t) = zeta0_fng(mu) + sum_r Dzeta_rfngk L*_r(x)

with r = 0, 1, 2, x = (mu - 13.5) / n_col, L*_r the shifted Legendre polynomials
(L*_0 = 1, L*_1 = 2x - 1, L*_2 = 6x^2 - 6x + 1) and m = floor(mu + 1/2) the nearest pixel
column (mu = 14 at the first of the n_col columns).  The calibration model is linear, so the
partial of a residual R = line - (eta or zeta) with respect to a parameter is the factor it
multiplies (Eq. pdC).  Nominal lines are the caller's; this module supplies the calibration
terms and the update.

Calibration update (Sect. 5.3, Eqs. normC, calCon).  The normals are block-diagonal: an
observation touches the parameters of one CCD/gate, and within it those of one long interval
k (Deta of the short intervals j inside k, deta of k; Dzeta of k).  Each (n, g, k) group is an
independent system.  Constraints (Eqs. cc1-cc3):
  cc1  sum over f and n of Deta_0fn0j = 0, for each j
  cc2  sum over m of deta_ngkm L*_r((m - 13.5) / n_col) = 0, for each r, n, g, k
  cc3  sum over n of Dzeta_0fn0k = 0, for each f, k

Readings where the paper is silent or at odds with itself:
  cc2 and the   The AL normals of a group are singular: a quadratic in x moved from the
  projection    large-scale terms of every j in k (both fields) into the small-scale terms
                leaves every residual unchanged (three null vectors per group: the constant
                one always, the linear and quadratic ones exactly when every observation sits
                at a column centre and nearly otherwise).  Eq. calCon's
                projection d~ - C (C'C)^-1 C' d~ keeps a least-squares solution only if C spans
                that null space, which the paper states as the condition; the cc2 vectors act
                on deta alone and the null vectors do not.  Each AL group's update is therefore
                the constrained least-squares solution, minimum of the weighted residual sum
                subject to cc2, by the null-space method: d = Z y with Z an orthonormal basis
                of {C2' d = 0} (from the QR factors of C2) and (Z' N Z) y = Z' b solved by the
                robust Cholesky of App. C.  Where the degeneracy is exact this equals the
                solution of (N + lambda^2 C2 C2') d = b for every lambda != 0, the paper's
                statement of the equivalence (pinned); where it is not, the normals alone
                determine the split only through the variation of x within a column, and the
                constraint decides it.
  cc2 gates     Eq. cc2 is stated for g = 0 only; without it the AL normals of every gated
                group stay singular, against the paper's condition that the constraints span
                the null space.  cc2 is applied to every gate.
  cc1, cc3      They fix the zero points of the field angles, which the attitude shares; they
                are not null directions of the calibration normals.  As for the offsets-only
                model, they are applied by the projection of Eq. calCon after the group
                solves (disjoint supports: subtract the mean of the constrained parameters).
  binned        Columns may be binned (col_bin columns share one deta); cc2 then weighs a bin
  columns       with the sum of L*_r over its columns (the constraint on per-column values
                that are constant within the bin).
  rounding      m = floor(mu + 1/2): a half rounds up.
  empty         A parameter without observations is 0 and counts in the rank defect (the
                constraints are then sums over the observed ones); further rank defects of a
                group come from the robust Cholesky's pivot test.

Basic angle (Eq. DeltaGamma): Delta Gamma_j = (1/n_ccd) sum_n sum_f f Deta_0fn0j, f = +1 for
the preceding field (fov 0) and -1 for the following one.

Pins: tests/test_oracle_calgeneric.py.
"""
from dataclasses import dataclass

import numpy as np

from . import cholesky as CH


def legendre_star(r, x):
    """Shifted Legendre polynomial L*_r(x), r = 0, 1, 2 (orthogonal on [0, 1])."""
    x = np.asarray(x, dtype=np.float64)
    if r == 0:
        return np.ones_like(x)
    if r == 1:
        return 2.0 * x - 1.0
    if r == 2:
        return 6.0 * x * x - 6.0 * x + 1.0
    raise ValueError("r in 0..2")


@dataclass
class Layout:
    """Parameter layout of the generic calibration.

    Groups (n, g, k) in the order n, g, k; within an AL group: Deta[j_in_k, f, r] (6 per short
    interval) then deta[bin]; the AC groups follow all AL groups, Dzeta[f, r] (6 each)."""
    n_ccd: int = 62
    n_gate: int = 1
    n_j: int = 1            # short intervals (large-scale AL)
    j_per_k: int = 1        # short intervals per long interval
    n_col: int = 1966       # AC pixel columns
    col_bin: int = 1        # columns per small-scale parameter

    @property
    def n_k(self):
        return -(-self.n_j // self.j_per_k)

    @property
    def n_bin(self):
        return -(-self.n_col // self.col_bin)

    @property
    def al_size(self):
        return 6 * self.j_per_k + self.n_bin

    @property
    def n_groups(self):
        return self.n_ccd * self.n_gate * self.n_k

    @property
    def n_al(self):
        return self.n_groups * self.al_size

    @property
    def n_params(self):
        return self.n_al + 6 * self.n_groups

    def group(self, ccd, gate, k):
        return (np.asarray(ccd, dtype=np.int64) * self.n_gate + np.asarray(gate, dtype=np.int64)) * self.n_k \
            + np.asarray(k, dtype=np.int64)

    def deta_large(self, ccd, gate, j, fov, r):
        """Index of Deta_{r f n g j}."""
        j = np.asarray(j, dtype=np.int64)
        k, jj = j // self.j_per_k, j % self.j_per_k
        return self.group(ccd, gate, k) * self.al_size + jj * 6 + np.asarray(fov, dtype=np.int64) * 3 + r

    def deta_small(self, ccd, gate, k, b):
        """Index of deta_{n g k m} for the bin b of column m."""
        return self.group(ccd, gate, k) * self.al_size + 6 * self.j_per_k + np.asarray(b, dtype=np.int64)

    def dzeta_large(self, ccd, gate, k, fov, r):
        """Index of Dzeta_{r f n g k}."""
        return self.n_al + self.group(ccd, gate, k) * 6 + np.asarray(fov, dtype=np.int64) * 3 + r

    def column(self, mu):
        """Pixel column index 0..n_col-1 of the nearest column, m = floor(mu + 1/2) - 14."""
        m = np.floor(np.asarray(mu, dtype=np.float64) + 0.5).astype(np.int64) - 14
        return np.clip(m, 0, self.n_col - 1)

    def x(self, mu):
        return (np.asarray(mu, dtype=np.float64) - 13.5) / self.n_col


def design(L, kind, fov, ccd, gate, j, mu):
    """Parameters and factors of each observation's calibration term (Eqs. etazeta, pdC):
    cols, vals [n_obs, 4]; AL: Deta_r (r = 0..2) and deta; AC: Dzeta_r and an unused slot
    (col -1, factor 0)."""
    kind = np.asarray(kind)
    j = np.asarray(j, dtype=np.int64)
    k = j // L.j_per_k
    x = L.x(mu)
    lr = np.stack([legendre_star(r, x) for r in range(3)], axis=-1)
    n = kind.shape[0]
    cols = np.full((n, 4), -1, dtype=np.int64)
    vals = np.zeros((n, 4))
    al = kind == 0
    for r in range(3):
        cols[:, r] = np.where(al, L.deta_large(ccd, gate, j, fov, r), L.dzeta_large(ccd, gate, k, fov, r))
        vals[:, r] = lr[:, r]
    b = L.column(mu) // L.col_bin
    cols[:, 3] = np.where(al, L.deta_small(ccd, gate, k, b), -1)
    vals[:, 3] = np.where(al, 1.0, 0.0)
    return cols, vals


def line_term(cal, cols, vals):
    """The calibration part of each observation line, sum of factor x parameter."""
    cal = np.asarray(cal, dtype=np.float64)
    return np.sum(np.where(cols >= 0, vals * cal[np.maximum(cols, 0)], 0.0), axis=1)


def cc2_weights(L):
    """[3, n_bin]: weight of each bin in the three cc2 sums, sum of L*_r over its columns."""
    m = np.arange(L.n_col)
    xm = (m + 14 - 13.5) / L.n_col
    w = np.zeros((3, L.n_bin))
    for r in range(3):
        np.add.at(w[r], m // L.col_bin, legendre_star(r, xm))
    return w


def group_normals(L, cols, vals, R, W):
    """Dense normals N, b = -sum Phi R W (Eq. normC) of every AL group [n_groups, s, s] and AC
    group [n_groups, 6, 6], s = al_size: the sums over observations of W Phi Phi' and
    -W Phi R, scattered into the group of each observation."""
    s = L.al_size
    R = np.asarray(R, dtype=np.float64)
    W = np.asarray(W, dtype=np.float64)
    al = cols[:, 0] < L.n_al
    out = []
    for sel, base, size, nslot in ((al, 0, s, 4), (~al, L.n_al, 6, 3)):
        c = cols[sel][:, :nslot] - base
        v = vals[sel][:, :nslot]
        g = c[:, 0] // size
        loc = c - g[:, None] * size
        N = np.zeros(L.n_groups * size * size)
        b = np.zeros(L.n_groups * size)
        w, r = W[sel], R[sel]
        for a in range(nslot):
            for e in range(nslot):
                np.add.at(N, (g * size + loc[:, a]) * size + loc[:, e], w * v[:, a] * v[:, e])
            np.add.at(b, g * size + loc[:, a], -v[:, a] * r * w)
        out += [N.reshape(L.n_groups, size, size), b.reshape(L.n_groups, size)]
    return out[0], out[1], out[2], out[3]


def cc2_matrix(L):
    """C2 [al_size, 3]: the cc2 vectors of one AL group (zero on its large-scale part)."""
    C = np.zeros((L.al_size, 3))
    C[6 * L.j_per_k:, :] = cc2_weights(L).T
    return C


def zero_point_groups(L):
    """Index sets of the constraints cc1 (per j: Deta_0fn0j over f, n) and cc3 (per f, k:
    Dzeta_0fn0k over n), each a constraint with unit weights."""
    out = []
    n = np.arange(L.n_ccd)
    for j in range(L.n_j):
        out.append(np.concatenate([L.deta_large(n, 0, j, f, 0) for f in (0, 1)]))
    for k in range(L.n_k):
        for f in (0, 1):
            out.append(L.dzeta_large(n, 0, k, f, 0))
    return out


def constrained_solve(N, b, C):
    """Minimum of x'Nx - 2 b'x subject to C'x = 0 (the weighted least squares of normals N, b
    under the constraints C), by the null-space method; parameters with a zero diagonal are
    held at 0.  Returns (x, rank defect)."""
    n = N.shape[0]
    obs = np.diagonal(N) > 0.0
    x = np.zeros(n)
    if not obs.any():
        return x, n
    F = np.flatnonzero(obs)
    NF, bF = N[np.ix_(F, F)], b[F]
    CF = C[F, :]
    Qc, Rc = np.linalg.qr(CF, mode="complete")
    rdiag = np.abs(np.diagonal(Rc)) if Rc.shape[0] else np.zeros(0)
    rank = int(np.sum(rdiag > 1e-12 * max(1.0, float(rdiag.max()) if rdiag.size else 1.0)))
    Z = Qc[:, rank:]
    y, _, rd = CH.solve(Z.T @ NF @ Z, Z.T @ bF)
    x[F] = Z @ y
    return x, (n - F.size) + rd


def update(L, cols, vals, R, W):
    """Calibration update d (Sect. 5.3): each AL group's constrained least-squares solution
    under cc2, each AC group from N d = b (robust Cholesky, App. C), then the projection of
    Eq. calCon onto cc1 and cc3.  Returns (d, rank defect)."""
    Nal, bal, Nac, bac = group_normals(L, cols, vals, R, W)
    C2 = cc2_matrix(L)
    d = np.zeros(L.n_params)
    rd = 0
    for g in range(L.n_groups):
        x, r = constrained_solve(Nal[g], bal[g], C2)
        d[g * L.al_size:(g + 1) * L.al_size] = x
        rd += r
        x, r = constrained_solve(Nac[g], bac[g], np.zeros((6, 0)))
        d[L.n_al + 6 * g:L.n_al + 6 * (g + 1)] = x
        rd += r
    for idx in zero_point_groups(L):
        d[idx] -= np.sum(d[idx]) / idx.size
    return d, rd


def delta_gamma(L, cal):
    """Basic-angle offset of each short interval, Eq. DeltaGamma (f = +1 for fov 0)."""
    cal = np.asarray(cal, dtype=np.float64)
    n = np.arange(L.n_ccd)
    out = np.zeros(L.n_j)
    for j in range(L.n_j):
        out[j] = (np.sum(cal[L.deta_large(n, 0, j, 0, 0)]) - np.sum(cal[L.deta_large(n, 0, j, 1, 0)])) / L.n_ccd
    return out
