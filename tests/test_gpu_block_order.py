"""The block orders of Sect. 4.6 on the GPU: block Gauss-Seidel SAC (C reads the residuals
with the attitude update added, Eq. precond) and block Jacobi [SAC] (A and C read the
residuals before the source update, Eq. precond(SCAG)) against the oracle's iteration with
the same order, the mixed form following the FP64 form of the same order, and the
rejections (out-of-range order; ASI and the proposal under the Jacobi order)."""
import numpy as np
import pytest

import synth
from oracle import agis as OG
from oracle import blocks as OB
from oracle import model as OM
from oracle import quat as OQ

pytestmark = pytest.mark.gpu

UAS = synth.UAS
TOL_SRC = 0.5 * UAS
ORDERS = {1: "SAC", 2: "[SAC]"}
# Attitude difference allowed after two iterations, per order: three times the oracle's own
# sensitivity to rounding, measured on this set as the change of its attitude after two
# iterations when every starting source parameter and attitude coefficient moves by one ulp
# in a random direction: 0.20 uas at most (RMS 0.0007 uas) under SAC, 0.52 uas (RMS 0.0019
# uas) under Jacobi, where A reads the residuals from before the source update.  A handful of
# weakly determined knots carry these maxima.
TOL_ATT = {1: 0.6 * UAS, 2: 1.6 * UAS}
TOL_ATT_RMS = {1: 0.0025 * UAS, 2: 0.006 * UAS}


@pytest.fixture(scope="module")
def lib():
    import paper_1112_4139_gb300 as pkg
    pkg.build()
    from paper_1112_4139_gb300 import agis
    agis.load()
    return agis


@pytest.fixture(scope="module")
def data():
    return synth.simulate(synth.config("small1yr", n_src=3000, seed=21))


def _attitude_angles(P, a1, a2, t_ns):
    q1 = OM.attitude(P, a1, t_ns)[0]
    q2 = OM.attitude(P, a2, t_ns)[0]
    return np.abs(OQ.diffrot(q1, q2))


@pytest.mark.parametrize("order", [1, 2])
def test_two_iterations_match_oracle(lib, data, order):
    st = OB.Settings(seg_len=720, seg_overlap=12, block_order=ORDERS[order])
    P = OM.problem_from_dataset(data)
    ref = data.src_true[:, [0, 1, 3, 4]]
    state = OG.State(data.src0.copy(), data.att0.copy(), data.cal0.copy())
    hist = []
    for _ in range(2):
        state, stats, _ = OG.iterate_once(P, state, st, ref)
        hist.append(stats)
    g = lib.from_dataset(data, seg_len=720, seg_overlap=12, block_order=order)
    it = g.iterate(2)
    for k in range(2):
        assert abs(it[k]["s"]["chi2"] / hist[k].chi2 - 1) < 1e-8
        assert np.allclose(it[k]["frame"], hist[k].frame, atol=1e-3 * UAS)
    e = OG.source_errors(g.sources(), state.src)
    assert np.max(np.abs(e)) < TOL_SRC, f"max source diff {np.max(np.abs(e)) / UAS:.3e} uas"
    ang = _attitude_angles(P, g.attitude(), state.att, data.t_ns)
    print("attitude difference: max %.3g uas, RMS %.3g uas" % (ang.max() / UAS, np.sqrt(np.mean(ang ** 2)) / UAS))
    assert ang.max() < TOL_ATT[order]
    assert np.sqrt(np.mean(ang ** 2)) < TOL_ATT_RMS[order]
    assert np.max(np.abs(g.calibration() - state.cal)) < 1e-3 * UAS
    g.close()


def test_orders_differ_where_the_paper_says(lib, data):
    # one iteration: the sources (S first in every order) are the same; the calibration
    # differs between S[AC] and SAC only by the attitude term, and Jacobi changes both A and C
    out = {}
    for order in (0, 1, 2):
        g = lib.from_dataset(data, seg_len=720, seg_overlap=12, block_order=order, frame_each_iter=0)
        g.iterate(1)
        out[order] = (g.sources(), g.attitude(), g.calibration())
        g.close()
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][0], out[2][0])
    assert np.array_equal(out[0][1], out[1][1])          # A is the same in S[AC] and SAC
    assert not np.array_equal(out[0][2], out[1][2])      # C sees the attitude update in SAC
    assert not np.array_equal(out[0][1], out[2][1])      # A reads h in Jacobi


@pytest.mark.parametrize("order", [1, 2])
def test_mixed_follows_fp64_of_the_same_order(lib, order):
    ds = synth.simulate(synth.config("scale5yr", n_src=20_000, knot_dt_s=3600, seed=77))
    K = 20
    runs = {}
    for prec in (0, 1):
        g = lib.from_dataset(ds, seg_len=720, seg_overlap=12, precision=prec, refresh_every=8, block_order=order)
        its = g.iterate(K)
        runs[prec] = (g.sources(), its[-1]["s"]["chi2"])
        g.close()
    e = OG.source_errors(runs[1][0], runs[0][0]) / UAS
    print("order", order, "mixed vs FP64 after", K, "iterations, max uas:", np.max(np.abs(e), axis=0))
    assert np.all(np.max(np.abs(e), axis=0) < 0.5)
    assert abs(runs[1][1] / runs[0][1] - 1) < 1e-4


def test_rejections(lib, data):
    with pytest.raises(lib.AgisError):
        lib.from_dataset(data, seg_len=720, seg_overlap=12, block_order=3)
    g = lib.from_dataset(data, seg_len=720, seg_overlap=12, block_order=2)
    with pytest.raises(lib.AgisError):
        g.set_asi(16, 0.9)
    with pytest.raises(lib.AgisError):
        g.set_proposal(np.zeros(lib.MLP_N_PARAMS, dtype=np.float32), 5)
    g.close()
