"""Source-partitioned iteration on the GPU (Sects. 4.6, 7.1): contexts holding parts of the
sources, their attitude and calibration normals and frame sums added over the parts
(paper_1112_4139_gb300/partition.py with the contexts of one process) and solved by every
context, against the one-context iteration (agis_iterate) on the same data.  The contexts run
one after the other on one GPU; no kernel waits on another context.
"""
import numpy as np
import pytest

import synth
from oracle import agis as OG
from oracle import model as OM
from oracle import quat as OQ

pytestmark = pytest.mark.gpu

UAS = synth.UAS


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


def _ctx(lib, ds, **kw):
    return lib.from_dataset(ds, seg_len=720, seg_overlap=12, **kw)


def test_one_part_is_the_iteration_bit_for_bit(lib, data):
    from paper_1112_4139_gb300 import partition
    ref = _ctx(lib, data)
    ref.iterate(2)
    g = _ctx(lib, data)
    partition.iterate([g], partition.LocalSum(), 2)
    assert np.array_equal(g.sources(), ref.sources())
    assert np.array_equal(g.attitude(), ref.attitude())
    assert np.array_equal(g.calibration(), ref.calibration())
    ref.close()
    g.close()


@pytest.mark.parametrize("n_parts", [2, 3])
def test_parts_reproduce_the_one_context_iteration(lib, data, n_parts):
    from paper_1112_4139_gb300 import partition
    n_iter = 2
    ref = _ctx(lib, data)
    it_ref = ref.iterate(n_iter)
    b = partition.split_sources(data.src_offsets(), n_parts)
    parts = [data.subset_sources(np.arange(b[i], b[i + 1])) for i in range(n_parts)]
    ctxs = [_ctx(lib, p) for p in parts]
    hist = partition.iterate(ctxs, partition.LocalSum(), n_iter)
    # every context solved the same sums: the same attitude and calibration bit for bit
    for c in ctxs[1:]:
        assert np.array_equal(c.attitude(), ctxs[0].attitude())
        assert np.array_equal(c.calibration(), ctxs[0].calibration())
    src = np.concatenate([c.sources() for c in ctxs])
    e = OG.source_errors(src, ref.sources())
    assert np.abs(e).max() < 0.5 * UAS, np.abs(e).max() / UAS
    P = OM.problem_from_dataset(data)
    ang = np.abs(OQ.diffrot(OM.attitude(P, ctxs[0].attitude(), data.t_ns)[0],
                            OM.attitude(P, ref.attitude(), data.t_ns)[0]))
    assert ang.max() < 0.5 * UAS
    assert np.abs(ctxs[0].calibration() - ref.calibration()).max() < 1e-3 * UAS
    # the statistics add up: chi^2 of the parts, rank defects of the shared solves
    for k in range(n_iter):
        chi2 = sum(s["chi2"] for s in hist[k]["s"])
        assert abs(chi2 / it_ref[k]["s"]["chi2"] - 1) < 1e-9
        from paper_1112_4139_gb300 import agis
        assert hist[k][agis.X_ATTITUDE][0]["rank_defect"] == it_ref[k]["a"]["rank_defect"]
        assert np.allclose(hist[k][agis.X_FRAME][0]["frame"], it_ref[k]["frame"], atol=1e-3 * UAS)
    for c in ctxs:
        c.close()
    ref.close()


def test_exchange_restrictions(lib, data):
    from paper_1112_4139_gb300.agis import AgisError
    g = _ctx(lib, data, precision=1)
    with pytest.raises(AgisError, match="FP64 form"):
        g.accumulate(lib.X_ATTITUDE)
    g.close()
    g = _ctx(lib, data)
    with pytest.raises(AgisError, match="source update first"):
        g.accumulate(lib.X_ATTITUDE)
    with pytest.raises(AgisError, match="no attitude sums"):
        g.solve_exchange(lib.X_ATTITUDE)
    g.close()
