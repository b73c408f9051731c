"""The launch-shape autotuner: it rates every candidate of every knob that applies to the
form, keeps the fastest, and leaves the solution unchanged bit for bit (every shaped kernel
gives each observation, source, knot interval or calibration parameter to one thread or warp
with the same arithmetic whatever the shape)."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

N_CAND = {0: dict(obs_pass=5, src_batch=6, mix_sums=0, mix_solve5=0, att_accum=4, cal_accum=5),
          1: dict(obs_pass=7, src_batch=0, mix_sums=6, mix_solve5=3, att_accum=4, cal_accum=5)}


@pytest.fixture(scope="module")
def lib():
    import paper_1112_4139_gb300 as pkg
    pkg.build()
    from paper_1112_4139_gb300 import agis
    agis.load()
    return agis


@pytest.fixture(scope="module")
def sky():
    # 5 years, 20k sources, 1-h knots: the mixed form iterates from the starting values
    return synth.simulate(synth.config("scale5yr", n_src=20_000, knot_dt_s=3600, seed=77))


def _state(g):
    return g.sources(), g.attitude(), g.calibration()


@pytest.mark.parametrize("precision", [0, 1])
def test_autotune_keeps_the_fastest_and_changes_nothing(lib, sky, precision):
    kw = dict(seg_len=720, seg_overlap=12, precision=precision)
    g = lib.from_dataset(sky, **kw)
    n_done, rep = g.autotune(20)
    g.iterate(3)
    tuned = _state(g)
    shapes = g.tuning()
    g.close()
    for name, n in N_CAND[precision].items():
        assert rep[name]["n_tried"] == n, (name, rep[name])
        if n:
            assert 0.0 < rep[name]["best_ms"] <= rep[name]["default_ms"]
        assert (shapes[name]["a"], shapes[name]["b"]) == (rep[name]["a"], rep[name]["b"])
    print("precision", precision, "iterations", n_done, {k: (v["a"], v["b"], round(v["best_ms"], 3),
                                                              round(v["default_ms"], 3)) for k, v in rep.items()})
    g = lib.from_dataset(sky, **kw)
    g.iterate(n_done + 3)
    plain = _state(g)
    g.close()
    for a, b in zip(tuned, plain):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("precision", [0, 1])
def test_extreme_shapes_change_nothing(lib, sky, precision):
    kw = dict(seg_len=720, seg_overlap=12, precision=precision)
    out = []
    for shapes in (None, dict(obs_pass=(128, 1), src_batch=(1, 0), mix_sums=(2, 1), mix_solve5=(64, 0),
                              att_accum=(0, 1), cal_accum=(128, 1)),
                   dict(obs_pass=(256, 64), src_batch=(32, 0), mix_sums=(8, 64), mix_solve5=(256, 0),
                        att_accum=(0, 64), cal_accum=(256, 64))):
        g = lib.from_dataset(sky, **kw)
        if shapes is not None:
            g.set_tuning(shapes)
        g.iterate(3)
        out.append(_state(g))
        g.close()
    for other in out[1:]:
        for a, b in zip(out[0], other):
            assert np.array_equal(a, b)


def test_invalid_shapes_are_rejected(lib, sky):
    g = lib.from_dataset(sky, seg_len=720, seg_overlap=12)
    before = g.tuning()
    for bad in (dict(obs_pass=(512, 8)), dict(obs_pass=(256, 0)), dict(mix_sums=(3, 8)), dict(src_batch=(33, 0)),
                dict(mix_solve5=(96, 0)), dict(cal_accum=(256, 65)), dict(att_accum=(0, -1))):
        with pytest.raises(lib.AgisError):
            g.set_tuning(bad)
    assert g.tuning() == before
    g.close()
