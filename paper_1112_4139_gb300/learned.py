"""Training data and training of the learned iteration proposal.

The network, its features and targets are defined in include/agis.h; every arithmetic step
(features, targets, forward, loss gradient, Adam) runs in libagis.so kernels on device
arrays.  This module only orchestrates: it runs the plain iteration of a training dataset,
keeps the features of each iteration and the state after its S block, iterates further to
a reference solution, and fits the network by Adam on random minibatches.
"""
from __future__ import annotations

import numpy as np

from . import agis

N_IN, N_OUT, N_PARAMS = agis.MLP_N_IN, agis.MLP_N_OUT, agis.MLP_N_PARAMS


def init_params(seed=0):
    """He initialisation (normal, std sqrt(2 / fan_in)), zero biases; layout of include/agis.h."""
    rng = np.random.default_rng(seed)
    parts = []
    for rows, cols in ((64, N_IN), (64, None), (64, 64), (64, None), (N_OUT, 64), (N_OUT, None)):
        if cols is None:
            parts.append(np.zeros(rows))
        else:
            parts.append(rng.normal(0.0, np.sqrt(2.0 / cols), size=rows * cols))
    return np.concatenate(parts).astype(np.float32)


def collect(ds, n_iter, ref_iter, first=3, stride=1, **cfg_over):
    """Plain iterations of a dataset.  After the S block of iterations first, first+stride, ...
    (< n_iter) the features of the last four updates and the sources are kept; the solution
    after ref_iter iterations is the reference of the targets.  Returns device tensors
    X (m x 22 FP32) and T (m x 5 FP32), m = rows kept, and the reference."""
    import torch
    g = agis.from_dataset(ds, **cfg_over)
    n = g.n_src
    feats, sigmas, states = [], [], []
    for k in range(n_iter):
        g.source_update()
        if k >= first and (k - first) % stride == 0:
            X = torch.empty((n, N_IN), dtype=torch.float32, device="cuda")
            s = torch.empty(n, dtype=torch.float64, device="cuda")
            x = torch.empty((n, 5), dtype=torch.float64, device="cuda")
            g.proposal_features(X, s)
            g.copy_sources_device(x)
            feats.append(X)
            sigmas.append(s)
            states.append(x)
        g.attitude_update()
        g.calibration_update()
        g.frame_rotate()
    if ref_iter > n_iter:
        g.iterate(ref_iter - n_iter)
    x_ref = torch.empty((n, 5), dtype=torch.float64, device="cuda")
    g.copy_sources_device(x_ref)
    g.close()
    Ts = []
    for s, x in zip(sigmas, states):
        T = torch.empty((n, N_OUT), dtype=torch.float32, device="cuda")
        agis.proposal_targets(x, x_ref, s, T)
        Ts.append(T)
    torch.cuda.synchronize()
    return torch.cat(feats), torch.cat(Ts), x_ref


def train(X, T, steps=3000, batch=8192, lr=1e-3, lr_final=1e-4, seed=0, max_target=100.0, params=None,
          val_frac=0.05, log_every=0):
    """Adam on random minibatches of the rows whose targets are finite and below max_target
    (a few sources with a vanishing update history have unbounded normalised targets).
    Returns (params as FP32 numpy, history of (step, train loss, validation loss))."""
    import torch
    rng = np.random.default_rng(seed)
    Th = T.cpu().numpy()
    ok = np.all(np.isfinite(Th), axis=1) & (np.max(np.abs(Th), axis=1) < max_target)
    rows = np.nonzero(ok)[0].astype(np.int32)
    rng.shuffle(rows)
    n_val = max(1, int(val_frac * rows.size))
    val = torch.from_numpy(rows[:n_val].copy()).cuda()
    tr = rows[n_val:]
    p = torch.from_numpy(init_params(seed) if params is None else np.asarray(params, np.float32)).cuda()
    m = torch.zeros_like(p)
    v = torch.zeros_like(p)
    grad = torch.empty_like(p)
    loss = torch.empty(1, dtype=torch.float32, device="cuda")
    hist = []
    for t in range(1, steps + 1):
        idx = torch.from_numpy(tr[rng.integers(0, tr.size, size=min(batch, tr.size))]).cuda()
        agis.mlp_loss_grad(p, X, T, grad, loss, idx=idx)
        lr_t = lr * (lr_final / lr) ** ((t - 1) / max(1, steps - 1))
        agis.mlp_adam(p, grad, m, v, t, lr_t)
        if log_every and (t % log_every == 0 or t == steps):
            tl = float(loss.item())
            agis.mlp_loss_grad(p, X, T, grad, loss, idx=val)
            hist.append((t, tl, float(loss.item())))
    torch.cuda.synchronize()
    return p.cpu().numpy(), hist


def validation_loss(params, X, T, rows=None):
    import torch
    p = torch.from_numpy(np.asarray(params, np.float32)).cuda()
    grad = torch.empty_like(p)
    loss = torch.empty(1, dtype=torch.float32, device="cuda")
    idx = None if rows is None else torch.from_numpy(np.asarray(rows, np.int32)).cuda()
    agis.mlp_loss_grad(p, X, T, grad, loss, idx=idx)
    return float(loss.item())
