"""Parity at the full size of the benchmark workload: 1M sources, 5 years, 30-s knots (8.2e8
observations, 5.26e6 attitude coefficients), in the configuration the bench times (FP64
form, graph-captured iteration, one-day attitude segments).  The oracle cannot run this
workload whole, so the test compares what it can compute one by one, and checks properties
that hold at any size:
* residuals at the start values of 20,000 sampled observations (|dR| <= 1e-9 |R| + 1e-15 rad);
* the source update of 100 sampled sources, which depends only on the attitude and
  calibration it starts from (Sect. 5.1): parameters within 0.5 uas, their residuals after
  the update, nu and n_out exactly;
* after the attitude and calibration updates, and after one more graph-captured iteration,
  the calibration constraints (Eqs. cc1, cc3: zero sum of the AL offsets per day, of the AC
  offsets per field and day) to rounding, and finite states."""
import numpy as np
import pytest

import synth
from oracle import agis as OG
from oracle import blocks as OB
from oracle import model as OM

pytestmark = pytest.mark.gpu

UAS = synth.UAS
TOL_SRC = 0.5 * UAS
R_AFTER_S_FLOOR = 1e-3 * UAS


@pytest.fixture(scope="module")
def lib():
    import paper_1112_4139_gb300 as pkg
    pkg.build()
    from paper_1112_4139_gb300 import agis
    agis.load()
    return agis


@pytest.fixture(scope="module")
def ds():
    return synth.simulate(synth.config("scale5yr"))


def _constraints_hold(cal, n_days):
    al = cal[:n_days * 124].reshape(n_days, 124)
    ac = cal[n_days * 124:].reshape(n_days, 2, 7)
    scale = max(np.abs(cal).max(), 1e-30)
    return np.abs(al.sum(axis=1)).max() <= 1e-12 * scale and np.abs(ac.sum(axis=2)).max() <= 1e-12 * scale


def test_full_size_sampled_parity(lib, ds):
    assert ds.n_src == 1_000_000 and ds.n_obs > 8e8
    rng = np.random.default_rng(1112)
    cfg = lib.default_config(seg_len=2880, use_graph=1, frame_each_iter=1, precision=0)
    g = lib.Agis(ds.geometry, cfg, lib.obs_from_dataset(ds), np.ascontiguousarray(ds.src0),
                 np.ascontiguousarray(ds.att0), np.ascontiguousarray(ds.cal0),
                 src_ref=np.ascontiguousarray(ds.src_true[:, [0, 1, 3, 4]]))
    P = OM.problem_from_dataset(ds)
    # residuals at the start values
    sample = np.sort(rng.choice(ds.n_obs, 20_000, replace=False))
    Rc = OM.evaluate(P, ds.src0, ds.att0, ds.cal0, idx=sample, partials=False)["R"]
    Rg = g.evaluate()[sample]
    ok = np.abs(Rg - Rc) <= 1e-9 * np.abs(Rc) + 1e-15
    assert ok.all(), f"{(~ok).sum()} sampled residuals off, max diff {np.abs(Rg - Rc).max():.3e}"
    # one source update: the sampled sources against the oracle's update of those sources
    g.source_update()
    idx = np.sort(rng.choice(ds.n_src, 100, replace=False))
    sub = ds.subset_sources(idx)
    st = OB.Settings(seg_len=2880, seg_overlap=12)
    src1, sres, _ = OB.source_update(OM.problem_from_dataset(sub), sub.src0, sub.att0, sub.cal0, st)
    e = OG.source_errors(g.sources()[idx], src1)
    assert np.max(np.abs(e)) < TOL_SRC, f"max source diff {np.max(np.abs(e)) / UAS:.3e} uas"
    Rg_all, _ = g.residuals()
    off = ds.src_offsets()
    Rg_sub = np.concatenate([Rg_all[off[i]:off[i + 1]] for i in idx])
    assert np.all(np.abs(Rg_sub - sres.R) <= 1e-9 * np.abs(sres.R) + R_AFTER_S_FLOOR)
    del Rg_all
    ss = g.source_stats()
    assert np.array_equal(ss["nu"][idx].astype(int), sres.nu)
    assert np.array_equal(ss["n_out"][idx].astype(int), sres.n_out)
    # the rest of the iteration, then one graph-captured iteration: properties at any size
    n_days = int(ds.geometry["n_cal_days"])
    g.attitude_update()
    g.calibration_update()
    assert _constraints_hold(g.calibration(), n_days)
    it = g.iterate(1)[0]
    assert np.isfinite(it["s"]["chi2"]) and it["s"]["chi2"] > 0
    assert _constraints_hold(g.calibration(), n_days)
    assert np.isfinite(g.sources()).all() and np.isfinite(g.attitude()).all()
    g.close()
