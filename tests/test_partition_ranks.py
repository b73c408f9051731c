"""Host side of the source-partitioned iteration (paper_1112_4139_gb300/partition.py), on CPU:
the split of the sources by observation count, and the exchange of the partial sums between
two gloo ranks, each with stand-in contexts that record the calls (no GPU).  The GPU side,
contexts of the library solving the summed parts, is tests/test_gpu_partition.py."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1112_4139_gb300 import agis, partition

SIZES = {agis.X_ATTITUDE: 7, agis.X_CALIBRATION: 5, agis.X_FRAME: 27}


class FakeCtx:
    """Stand-in for a context: its partial sums depend on (process rank, local index, call), and
    it records the sums it is given back."""

    def __init__(self, rank, local):
        self.rank, self.local, self.calls, self.got = rank, local, [], {}
        self.k = 0

    def exchange_size(self, which):
        return SIZES[which]

    def source_update(self):
        self.calls.append("S")
        self.k += 1
        return {"chi2": float(self.rank)}

    def part(self, which):
        n = SIZES[which]
        return torch.arange(n, dtype=torch.float64) * (1 + self.rank) + 100.0 * self.local + 1000.0 * which + self.k

    def accumulate(self, which):
        self.calls.append(f"acc{which}")

    def get_exchange(self, which, out):
        out[...] = self.part(which)

    def set_exchange(self, which, buf):
        self.got[(self.k, which)] = buf.clone()

    def solve_exchange(self, which):
        self.calls.append(f"solve{which}")
        return {"rank_defect": 0}


def expected_total(which, k, world, n_local):
    n = SIZES[which]
    tot = torch.zeros(n, dtype=torch.float64)
    for r in range(world):
        for loc in range(n_local):
            tot += torch.arange(n, dtype=torch.float64) * (1 + r) + 100.0 * loc + 1000.0 * which + k
    return tot


def _worker(rank, world, port, n_local, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ctxs = [FakeCtx(rank, i) for i in range(n_local)]
        bufs = {w: [torch.zeros(SIZES[w], dtype=torch.float64) for _ in ctxs] for w in SIZES}
        partition.iterate(ctxs, partition.LocalSum(dist.group.WORLD), 2, bufs=bufs)
        ok = True
        for c in ctxs:
            assert c.calls == ["S", "acc0", "solve0", "acc1", "solve1", "acc2", "solve2"] * 2, c.calls
            for k in (1, 2):
                for w in SIZES:
                    ok &= bool(torch.equal(c.got[(k, w)], expected_total(w, k, world, n_local)))
        q.put((rank, ok))
    except Exception as e:  # report to the parent instead of hanging it
        q.put((rank, repr(e)))
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("n_local", [1, 2])
def test_two_ranks_exchange_the_summed_parts(n_local):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, n_local, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
    assert res == {0: True, 1: True}, res


def test_split_sources_balances_observations():
    rng = np.random.default_rng(3)
    counts = rng.integers(40, 250, 1000)
    off = np.concatenate([[0], np.cumsum(counts)])
    for parts in (1, 2, 3, 8):
        b = partition.split_sources(off, parts)
        assert b[0] == 0 and b[-1] == 1000 and np.all(np.diff(b) > 0)
        obs = off[b[1:]] - off[b[:-1]]
        assert obs.max() - obs.min() <= 2 * counts.max()
    # every source in exactly one part, and degenerate sizes
    assert list(partition.split_sources(np.array([0, 5, 9]), 2)) == [0, 1, 2]
    with pytest.raises(ValueError):
        partition.split_sources(off, 0)
