"""Source-partitioned iteration (Sects. 4.6 and 7.1 of Lindegren et al. 2012): orchestration only.

The sources are split into contiguous parts, one context per part (its own observations, the
whole attitude and calibration).  Per iteration every context runs its source update; the
attitude and calibration normals are sums over observations and the frame rotator's over
sources, so each context accumulates its part, the parts are added over all contexts (an
all-reduce, the role of the paper's accumulation servers, Sect. 7.1), and every context solves
the same sums.  The sums, solves and updates run in the library (agis_accumulate,
agis_get/set_exchange, agis_solve_exchange); this module only orders the calls and moves the
buffers.  The contexts of one process are summed in list order, then (with a process group)
across processes by torch.distributed.all_reduce, which hands every rank the same sums.
"""
from __future__ import annotations

import numpy as np

from . import agis

# exchange order within an iteration: S[AC] (A and C from the same source update), then the
# frame rotator
ORDER = (agis.X_ATTITUDE, agis.X_CALIBRATION)


def split_sources(src_offsets, n_parts):
    """Boundaries b[0..n_parts] of n_parts contiguous ranges of sources with about equal numbers
    of observations (src_offsets: start of every source's observations, length n_src + 1)."""
    off = np.asarray(src_offsets, dtype=np.int64)
    n_src = off.size - 1
    if n_parts < 1 or n_parts > max(1, n_src):
        raise ValueError("n_parts must be in 1..n_src")
    targets = off[-1] * np.arange(1, n_parts) / n_parts
    cuts = np.searchsorted(off, targets, side="left")
    b = np.concatenate([[0], np.clip(cuts, 1, n_src - 1) if n_src > 1 else cuts, [n_src]]).astype(np.int64)
    # strictly increasing boundaries (no empty part)
    for i in range(1, n_parts):
        b[i] = max(b[i], b[i - 1] + 1)
    for i in range(n_parts - 1, 0, -1):
        b[i] = min(b[i], b[i + 1] - 1)
    return b


class LocalSum:
    """Adds the buffers of the contexts of this process in list order and, with a process group,
    across processes (torch.distributed.all_reduce, SUM); every buffer then holds the total."""

    def __init__(self, group=None):
        self.group = group

    def __call__(self, which, bufs):
        total = bufs[0]
        if len(bufs) > 1:
            total = bufs[0].clone() if hasattr(bufs[0], "clone") else bufs[0].copy()
            for b in bufs[1:]:
                total += b
        if self.group is not None:
            import torch.distributed as dist
            dist.all_reduce(total, op=dist.ReduceOp.SUM, group=self.group)
        for b in bufs:
            if b is not total:
                b[...] = total


def make_buffers(ctxs, like=None):
    """One exchange buffer per context and kind (NumPy on the host, or torch tensors on the
    device of `like`)."""
    out = {}
    for which in ORDER + (agis.X_FRAME,):
        n = ctxs[0].exchange_size(which)
        if like is None:
            out[which] = [np.zeros(n) for _ in ctxs]
        else:
            import torch
            out[which] = [torch.zeros(n, dtype=torch.float64, device=like.device) for _ in ctxs]
    return out


def iterate(ctxs, reduce, n_iter, frame=True, bufs=None, sync=None):
    """n_iter S[AC] iterations of one problem split over the contexts `ctxs` of this process
    (and, through `reduce`, over other processes).  Returns per iteration the list of the
    contexts' source-update statistics and the attitude, calibration and frame results.
    sync: called before each reduction (e.g. torch.cuda.synchronize for device buffers)."""
    if bufs is None:
        bufs = make_buffers(ctxs)
    kinds = ORDER + ((agis.X_FRAME,) if frame else ())
    hist = []
    for _ in range(n_iter):
        rec = {"s": [c.source_update() for c in ctxs]}
        for which in kinds:
            for c, b in zip(ctxs, bufs[which]):
                c.accumulate(which)
                c.get_exchange(which, out=b)
            if sync is not None:
                sync()
            reduce(which, bufs[which])
            if sync is not None:
                sync()
            res = []
            for c, b in zip(ctxs, bufs[which]):
                c.set_exchange(which, b)
                res.append(c.solve_exchange(which))
            rec[which] = res
        hist.append(rec)
    return hist
