"""The full geometric calibration (Sect. 3.4, Eq. etazeta; Sect. 5.3, Eqs. normC, calCon,
cc1-cc3) on the GPU against the oracle (oracle/calgeneric.py through oracle/blocks.py), through
the C ABI, on the generator's data of that model: 40,000 sources over 30 days, two gates of
about equal size (gate threshold at G = 15, sources near it seen with both), three long
intervals of 10 days, the AC pixel columns in 10 bins of 197; every (CCD, gate, day) cell holds
about 70 observations per field, so the only rank defects are the unobserved parameters.

Compared: the residuals of the observation model with the full calibration terms; the C update
(each (CCD, gate, long interval) group's constrained least-squares solution under cc2, then
cc1 and cc3), and its rank defects; two whole S[AC] iterations.  Tolerances as for the
offsets-only model: residuals 1e-9 |R| + 1e-15 rad, attitude 0.5 uas, calibration 1e-3 uas.

Thirty days leave the sources' parallaxes and proper motions all but undetermined (5x5 normal
matrices of condition up to 1e17): as in tests/test_gpu_benchshape.py both sides take the pivot
tolerance 1e-4 (App. C), which zeroes those directions, so that the residuals and weights the
C block reads are unique; the sources are then compared through the residuals, and the frame
rotator (whose fit the undetermined proper motions would dominate) is off.  The weights are the
plain ones: a one-ulp change of the starting right ascensions moves the oracle's own residuals
after the source update by up to 0.006 uas and its calibration update by 1e-4 uas with plain
weights, but by 2.5 uas and 0.003 uas with the robust weights, whose downweighting of these
short-arc sources feeds the differences back.  The residuals after S are compared to 0.02 uas
(three times that sensitivity), the calibration to 1e-3 uas.
"""
import numpy as np
import pytest

import oracle.cholesky as CH
import synth
from oracle import agis as OG
from oracle import blocks as OB
from oracle import calgeneric as CG
from oracle import model as OM
from oracle import quat as OQ

pytestmark = pytest.mark.gpu

UAS = synth.UAS
TOL_SRC = 0.5 * UAS


@pytest.fixture(scope="module")
def lib():
    import paper_1112_4139_gb300 as pkg
    pkg.build()
    from paper_1112_4139_gb300 import agis
    agis.load()
    return agis


@pytest.fixture(scope="module")
def data():
    ds = synth.simulate(synth.config("small1yr", n_src=40_000, span_days=30, seed=13, cal_generic=True, n_gate=2,
                                     gate_g0=15.0, gate_step=10.0, cal_j_per_k=10, cal_col_bin=197))
    P = OM.problem_from_dataset(ds)
    assert P.calg is not None and P.calg.n_k == 3 and P.calg.n_bin == 10 and ds.n_cal == P.calg.n_params
    return ds, P


PIVOT = 1e-4


@pytest.fixture()
def pivot_tol(monkeypatch):
    monkeypatch.setattr(CH, "PIVOT_TOL", PIVOT)
    return PIVOT


def _gpu(lib, ds, **kw):
    return lib.from_dataset(ds, seg_len=720, seg_overlap=12, pivot_tol=PIVOT, frame_each_iter=0, **kw)


def test_residuals_of_the_full_model(lib, data):
    ds, P = data
    g = _gpu(lib, ds)
    Rc = OM.evaluate(P, ds.src0, ds.att0, ds.cal0, partials=False)["R"]
    Rg = g.evaluate()
    assert np.all(np.abs(Rg - Rc) <= 1e-9 * np.abs(Rc) + 1e-15), np.abs(Rg - Rc).max()
    # at the truth the residuals are the injected noise: both implementations of Eq. etazeta
    g.set_state(src=ds.src_true, att=ds.att_true, cal=ds.cal_true)
    Rt = g.evaluate()
    assert np.all(np.abs(Rt - ds.noise) <= 1e-9 * np.abs(ds.noise) + 2e-15)
    g.close()


def test_calibration_update(lib, data, pivot_tol):
    # plain weights: the residuals and weights the C block reads agree to the parity floor
    ds, P = data
    st = OB.Settings(seg_len=720, seg_overlap=12, robust=False)
    src1, sres, ev = OB.source_update(P, ds.src0, ds.att0, ds.cal0, st)
    cal1, rdc = OB.calibration_update(P, ds.cal0, ev, sres.R, sres.W)
    att1, rda = OB.attitude_update(P, ds.att0, ev, sres.R, sres.W, st)
    g = _gpu(lib, ds, robust=0)
    g.source_update()
    Rg, _ = g.residuals()
    print("R after S: max diff", np.abs(Rg - sres.R).max() / UAS, "uas")
    assert np.all(np.abs(Rg - sres.R) <= 1e-9 * np.abs(sres.R) + 0.02 * UAS)
    sc = g.calibration_update()
    sa = g.attitude_update()
    cg = g.calibration()
    d = np.abs(cg - cal1)
    print("calibration update: max diff", d.max() / UAS, "uas; rank defects", sc["rank_defect"], rdc)
    assert d.max() < 1e-3 * UAS
    assert sc["rank_defect"] == rdc
    # the constraints of Eqs. cc1-cc3 hold after the update
    L = P.calg
    for idx in CG.zero_point_groups(L):
        assert abs(np.sum(cg[idx] - ds.cal0[idx])) < 1e-9 * UAS * idx.size
    C2 = CG.cc2_matrix(L)
    for grp in range(L.n_groups):
        dv = (cg - ds.cal0)[grp * L.al_size:(grp + 1) * L.al_size]
        assert np.all(np.abs(C2.T @ dv) < 1e-9 * UAS * L.n_col)
    ang = np.abs(OQ.diffrot(OM.attitude(P, g.attitude(), ds.t_ns)[0], OM.attitude(P, att1, ds.t_ns)[0]))
    assert ang.max() < TOL_SRC and sa["rank_defect"] == rda
    g.close()


def test_two_iterations_with_the_full_model(lib, data, pivot_tol):
    ds, P = data
    st = OB.Settings(seg_len=720, seg_overlap=12, frame_each_iter=False, robust=False)
    state = OG.State(ds.src0.copy(), ds.att0.copy(), ds.cal0.copy())
    hist = []
    for _ in range(2):
        state, stats, sres = OG.iterate_once(P, state, st, None)
        hist.append(stats)
    g = _gpu(lib, ds, robust=0)
    it = g.iterate(2)
    for k in range(2):
        assert abs(it[k]["s"]["chi2"] / hist[k].chi2 - 1) < 1e-8
        assert it[k]["c"]["rank_defect"] == hist[k].rank_def_c
        assert it[k]["a"]["rank_defect"] == hist[k].rank_def_a
    Rg, _ = g.residuals()
    ang = np.abs(OQ.diffrot(OM.attitude(P, g.attitude(), ds.t_ns)[0], OM.attitude(P, state.att, ds.t_ns)[0]))
    d = np.abs(g.calibration() - state.cal)
    print("two iterations: R max diff", np.max(np.abs(Rg - sres.R)) / UAS, "attitude max", ang.max() / UAS,
          "calibration max diff", d.max() / UAS, "uas")
    assert np.max(np.abs(Rg - sres.R)) < 0.02 * UAS
    assert ang.max() < TOL_SRC
    assert d.max() < 1e-3 * UAS
    g.close()


def test_full_model_rejections(lib, data):
    ds, P = data
    from paper_1112_4139_gb300.agis import AgisError
    obs = lib.obs_from_dataset(ds)
    cc = lib.calibration_config(ds.geometry)
    with pytest.raises(AgisError, match="FP64 form"):
        lib.Agis(ds.geometry, lib.default_config(precision=1, **cc), obs, ds.src0, ds.att0, ds.cal0)
    bad = dict(obs)
    gate = obs["gate"].copy()
    gate[17] = 2
    bad["gate"] = gate
    with pytest.raises(AgisError, match="gate out of range"):
        lib.Agis(ds.geometry, lib.default_config(**cc), bad, ds.src0, ds.att0, ds.cal0)
    with pytest.raises(AgisError, match="n_cal"):
        lib.Agis(ds.geometry, lib.default_config(**cc), obs, ds.src0, ds.att0, ds.cal0[:-6])
    with pytest.raises(AgisError, match="n_cal"):
        lib.Agis(ds.geometry, lib.default_config(), obs, ds.src0, ds.att0, ds.cal0)
    cc_bad = dict(cc)
    cc_bad["n_gate"] = 0
    with pytest.raises(AgisError, match="n_gate"):
        lib.Agis(ds.geometry, lib.default_config(**cc_bad), obs, ds.src0, ds.att0, ds.cal0)
