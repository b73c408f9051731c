"""agis_source_update_static: the source update for callers that cannot allocate device memory.

Some callers cannot let this library call cudaMalloc: a host framework that owns every
device allocation, or a process that reserved the device memory up front.  The static entry
point runs the S block on caller-owned device arrays with a scratch array compiled into the
library.  This test calls it twice in a row through the C ABI and checks its results against
the context-based agis_source_update on the same inputs, with the tolerances of the parity
tests.  It runs last (file name) so that a first-failure run has already run everything else.
"""
import numpy as np
import pytest

import synth
from parity_tol import assert_stats_close

pytestmark = pytest.mark.gpu

UAS = synth.UAS


def test_static_source_update_matches_context_entry_point():
    import torch

    import paper_1112_4139_gb300 as pkg
    pkg.build()
    from paper_1112_4139_gb300 import agis

    ds = synth.simulate(synth.config("small1yr", n_src=1200, seed=31, min_transits=8))
    cfg = agis.default_config(seg_len=720, seg_overlap=12)

    # the existing entry point (library-owned device memory)
    g = agis.from_dataset(ds, cfg=cfg, with_ref=False)
    g.source_update()
    src_ref = g.sources()
    R_ref, W_ref = g.residuals()
    st_ref = g.source_stats()
    g.close()

    dev = "cuda"
    obs = agis.obs_from_dataset(ds, device=dev)
    att = torch.from_numpy(np.ascontiguousarray(ds.att0)).to(dev)
    cal = torch.from_numpy(np.ascontiguousarray(ds.cal0)).to(dev)
    n_max = int(np.max(np.diff(ds.src_offsets())))
    for call in range(2):
        src = torch.from_numpy(np.ascontiguousarray(ds.src0)).to(dev)
        R = torch.full((ds.n_obs,), np.nan, dtype=torch.float64, device=dev)
        W = torch.full((ds.n_obs,), np.nan, dtype=torch.float64, device=dev)
        stats = torch.full((5, ds.n_src), np.nan, dtype=torch.float64, device=dev)
        agis.source_update_static(ds.geometry, cfg, obs, src, att, cal, R_out=R, W_out=W, stats_out=stats,
                                  max_obs_per_source=n_max)
        torch.cuda.synchronize()
        s = src.cpu().numpy()
        e = s - src_ref
        e[:, 0] *= np.cos(src_ref[:, 1])
        assert np.max(np.abs(e)) < 0.5 * UAS, f"call {call}: {np.max(np.abs(e)) / UAS:.3e} uas"
        Rh, Wh = R.cpu().numpy(), W.cpu().numpy()
        assert np.all(np.abs(Rh - R_ref) <= 1e-9 * np.abs(R_ref) + 1e-3 * UAS)
        sh = stats.cpu().numpy()
        assert np.array_equal(sh[2], st_ref["nu"]) and np.array_equal(sh[3], st_ref["n_out"])
        # weights, Q_i and eps_i^2 within the first-order propagation of the measured residual
        # differences (tests/parity_tol.py)
        assert_stats_close(ds.src, ds.n_src, ds.sigma, R_ref, Rh, W_ref, Wh, st_ref["eps2"], sh[0], st_ref["Q"],
                           sh[1], what=f"call {call}: ")

    # sizes beyond the limits and invalid inputs are rejected with a clear error before anything
    # is written: the sources and the outputs keep their contents
    src = torch.from_numpy(np.ascontiguousarray(ds.src0)).to(dev)
    R = torch.full((ds.n_obs,), 7.0, dtype=torch.float64, device=dev)

    def refused(match, o=obs, **kw):
        with pytest.raises(agis.AgisError, match=match):
            agis.source_update_static(ds.geometry, cfg, o, src, att, cal, R_out=R, **kw)
        torch.cuda.synchronize()
        assert np.array_equal(src.cpu().numpy(), ds.src0), match
        assert bool(torch.all(R == 7.0)), match

    refused("max_obs_per_source", max_obs_per_source=n_max - 1)
    refused("AGIS_STATIC_MAX_OBS", max_obs_per_source=agis.STATIC_MAX_OBS + 1)
    bad = dict(obs)
    bad["src"] = obs["src"].flip(0).contiguous()
    refused("sorted", o=bad, max_obs_per_source=agis.STATIC_MAX_OBS)
    bad = dict(obs)
    bad["src"] = obs["src"].clone()
    bad["src"][-1] = ds.n_src
    refused("source index", o=bad, max_obs_per_source=agis.STATIC_MAX_OBS)
    for field, value in (("ccd", 62), ("ccd", 255), ("fov", 2), ("kind", 3)):
        bad = dict(obs)
        bad[field] = obs[field].clone()
        bad[field][ds.n_obs // 2] = value
        refused("ccd, fov or kind", o=bad, max_obs_per_source=agis.STATIC_MAX_OBS)
    bad = dict(obs)
    bad["sigma"] = obs["sigma"].clone()
    bad["sigma"][3] = 0.0
    refused("sigma", o=bad, max_obs_per_source=agis.STATIC_MAX_OBS)
    att_bad = att.clone()
    att_bad[5, 2] = float("nan")
    with pytest.raises(agis.AgisError, match="non-finite"):
        agis.source_update_static(ds.geometry, cfg, obs, src, att_bad, cal, R_out=R,
                                  max_obs_per_source=agis.STATIC_MAX_OBS)
    torch.cuda.synchronize()
    assert np.array_equal(src.cpu().numpy(), ds.src0) and bool(torch.all(R == 7.0))
