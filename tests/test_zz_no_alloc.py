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
        assert np.allclose(Wh, W_ref, rtol=1e-6, atol=0)
        sh = stats.cpu().numpy()
        assert np.array_equal(sh[2], st_ref["nu"]) and np.array_equal(sh[3], st_ref["n_out"])
        assert np.allclose(sh[0], st_ref["eps2"], rtol=1e-6, atol=1e-30)
        assert np.allclose(sh[1], st_ref["Q"], rtol=1e-6)

    # sizes beyond the limits are rejected with a clear error
    src = torch.from_numpy(np.ascontiguousarray(ds.src0)).to(dev)
    with pytest.raises(agis.AgisError, match="max_obs_per_source"):
        agis.source_update_static(ds.geometry, cfg, obs, src, att, cal, max_obs_per_source=n_max - 1)
    with pytest.raises(agis.AgisError, match="AGIS_STATIC_MAX_OBS"):
        agis.source_update_static(ds.geometry, cfg, obs, src, att, cal,
                                  max_obs_per_source=agis.STATIC_MAX_OBS + 1)
