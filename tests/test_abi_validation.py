"""Error behaviour of the C ABI that needs no GPU: agis_init checks its arguments before any
CUDA call and returns AGIS_E_INVALID with a message, and calls on a null context return
AGIS_E_INVALID.  Among the refusals: data of the full geometric calibration model (a
calibration vector that is not the per-day offsets), which the GPU library does not
implement."""
import ctypes as C

import numpy as np
import pytest

import synth
from paper_1112_4139_gb300 import agis

E_INVALID = -1   # AGIS_E_INVALID of include/agis.h


@pytest.fixture(scope="module")
def ds():
    return synth.simulate(synth.config("tiny"))


def _init(ds, cfg=None, geometry=None, cal0=None, att0=None):
    cfg = cfg if cfg is not None else agis.default_config()
    return agis.Agis(geometry if geometry is not None else ds.geometry, cfg, agis.obs_from_dataset(ds),
                     np.ascontiguousarray(ds.src0), np.ascontiguousarray(ds.att0 if att0 is None else att0),
                     np.ascontiguousarray(ds.cal0 if cal0 is None else cal0))


@pytest.mark.parametrize("case,match", [
    ("n_cal", "n_cal"),
    ("n_coef", "n_coef"),
    ("precision", "precision"),
    ("refresh", "refresh_every"),
    ("block_order", "block_order"),
    ("ccd_row", "ccd_row"),
    ("seg_len", "segmentation"),
    ("knot_dt", "non-positive"),
])
def test_init_rejects_invalid_arguments(ds, case, match):
    agis.load()
    kw = {}
    if case == "n_cal":
        kw["cal0"] = ds.cal0[:-1]
    elif case == "n_coef":
        kw["att0"] = ds.att0[:-1]
    elif case == "precision":
        kw["cfg"] = agis.default_config(precision=2)
    elif case == "refresh":
        kw["cfg"] = agis.default_config(precision=1, refresh_every=0)
    elif case == "block_order":
        kw["cfg"] = agis.default_config(block_order=3)
    elif case == "seg_len":
        kw["cfg"] = agis.default_config(seg_len=0)
    else:
        g = dict(ds.geometry)
        if case == "ccd_row":
            g["ccd_row"] = np.array(g["ccd_row"]).copy()
            g["ccd_row"][5] = 7
        else:
            g["knot_dt_ns"] = 0
        kw["geometry"] = g
    with pytest.raises(agis.AgisError, match=match) as e:
        _init(ds, **kw)
    assert e.value.code == E_INVALID


def test_full_calibration_data_are_refused():
    d = synth.simulate(synth.config("tiny", cal_generic=True, n_gate=2, cal_j_per_k=5, cal_col_bin=197))
    with pytest.raises(agis.AgisError, match="n_cal") as e:
        _init(d)
    assert e.value.code == E_INVALID


def test_calls_on_a_null_context():
    lib = agis.load()
    null = C.c_void_p()
    nb = C.c_int32(0)
    assert lib.agis_set_attnoise(null, 0) == E_INVALID
    assert lib.agis_get_attnoise(null, None, C.byref(nb)) == E_INVALID
    assert lib.agis_set_asi(null, 16, 0.9) == E_INVALID
    assert lib.agis_set_proposal(null, None, 5) == E_INVALID
    assert lib.agis_source_update(null, None) == E_INVALID
    assert lib.agis_iterate(null, 1, None, None) == E_INVALID
    lib.agis_destroy(null)   # a no-op
    # agis_asi_estimate checks its arguments before touching memory
    assert lib.agis_asi_estimate(None, None, 10, 1, 0.9, None, None, None) == E_INVALID
