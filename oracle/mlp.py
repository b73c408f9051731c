"""FP64 oracle of the learned iteration proposal (TEST INFRASTRUCTURE ONLY).

The learned proposal is not part of the paper.  Its analogue there is the accelerated simple
iteration of Sect. 4.7, which extrapolates the source updates with a factor estimated from
the ratio of successive updates; here a small network maps the last four updates of a
source to a correction towards the converged solution.  This module fixes that definition
in plain NumPy:

  features   22 inputs per source: the last four updates (oldest first, five parameters
             each, alpha* and delta as arcs, in the tangent units of the source update)
             divided by their RMS sigma; log10(n_obs) - 2.5; sin(ecliptic latitude)
  network    22 -> 64 -> 64 -> 5, ReLU hidden layers, linear output
  target     (x_ref - x_k) / sigma in the same tangent units; the correction applied is
             sigma * output
  loss       mean over rows of the sum of squared output errors
  Adam       Kingma & Ba (2015), with the bias corrections of that paper

The GPU forward multiplies on tensor cores with BF16 inputs, weights and hidden
activations and FP32 accumulation; `forward(..., bf16=True)` rounds at the same points
(round to nearest even of the FP32 value) so that the two can be compared closely, and the
gradients are those of the rounded forward with the rounding treated as the identity.

Parameter layout (flat vector, this order): W1[64][22], b1[64], W2[64][64], b2[64],
W3[5][64], b3[5]  (5957 values).
"""
import numpy as np

N_IN, N_H, N_OUT = 22, 64, 5
SHAPES = [("W1", (N_H, N_IN)), ("b1", (N_H,)), ("W2", (N_H, N_H)), ("b2", (N_H,)), ("W3", (N_OUT, N_H)),
          ("b3", (N_OUT,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SHAPES)


def unpack(p):
    out, o = {}, 0
    for name, shp in SHAPES:
        n = int(np.prod(shp))
        out[name] = np.asarray(p[o:o + n], dtype=np.float64).reshape(shp)
        o += n
    return out


def pack(d):
    return np.concatenate([np.asarray(d[name], dtype=np.float64).ravel() for name, _ in SHAPES])


def init_params(seed, scale=1.0):
    """He-style initialisation (normal, std sqrt(2 / fan_in)), zero biases."""
    rng = np.random.default_rng(seed)
    d = {}
    for name, shp in SHAPES:
        if name.startswith("W"):
            d[name] = rng.normal(0.0, scale * np.sqrt(2.0 / shp[1]), size=shp)
        else:
            d[name] = np.zeros(shp)
    return pack(d)


def bf16(x):
    """Round FP32 values to the nearest bfloat16 (ties to even), returned as float64."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) & 0xFFFF0000).astype(np.uint32)
    return r.view(np.float32).astype(np.float64)


def forward(p, X, bf16_round=False):
    """Outputs and the intermediate values (pre-activations and activations)."""
    w = unpack(p)
    X = np.asarray(X, dtype=np.float64)
    if bf16_round:
        X = bf16(X)
        W1, W2, W3 = bf16(w["W1"]), bf16(w["W2"]), bf16(w["W3"])
    else:
        W1, W2, W3 = w["W1"], w["W2"], w["W3"]
    Z1 = X @ W1.T + w["b1"]
    H1 = np.maximum(Z1, 0.0)
    if bf16_round:
        H1 = bf16(H1)
    Z2 = H1 @ W2.T + w["b2"]
    H2 = np.maximum(Z2, 0.0)
    if bf16_round:
        H2 = bf16(H2)
    Y = H2 @ W3.T + w["b3"]
    return Y, dict(X=X, W1=W1, W2=W2, W3=W3, Z1=Z1, H1=H1, Z2=Z2, H2=H2)


def loss(p, X, T, bf16_round=False):
    Y, _ = forward(p, X, bf16_round)
    return float(np.mean(np.sum((Y - np.asarray(T, dtype=np.float64)) ** 2, axis=1)))


def loss_grad(p, X, T, bf16_round=False):
    """Loss and its gradient with respect to the flat parameter vector (chain rule)."""
    Y, c = forward(p, X, bf16_round)
    n = Y.shape[0]
    dY = 2.0 * (Y - np.asarray(T, dtype=np.float64)) / n
    g = {}
    g["W3"] = dY.T @ c["H2"]
    g["b3"] = dY.sum(axis=0)
    dH2 = (dY @ c["W3"]) * (c["Z2"] > 0.0)
    g["W2"] = dH2.T @ c["H1"]
    g["b2"] = dH2.sum(axis=0)
    dH1 = (dH2 @ c["W2"]) * (c["Z1"] > 0.0)
    g["W1"] = dH1.T @ c["X"]
    g["b1"] = dH1.sum(axis=0)
    L = float(np.mean(np.sum((Y - T) ** 2, axis=1)))
    return L, pack(g)


def adam_step(p, g, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step (t counts from 1); returns new (p, m, v)."""
    m = b1 * m + (1.0 - b1) * g
    v = b2 * v + (1.0 - b2) * g * g
    mh = m / (1.0 - b1 ** t)
    vh = v / (1.0 - b2 ** t)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v


def tangent_diff(x, y):
    """x - y for source parameter arrays (alpha, delta, varpi, mu_a*, mu_d) in the tangent
    units of the source update: alpha difference wrapped and times cos(delta of y)."""
    e = np.asarray(x, dtype=np.float64) - np.asarray(y, dtype=np.float64)
    e[:, 0] = (np.mod(e[:, 0] + np.pi, 2 * np.pi) - np.pi) * np.cos(np.asarray(y)[:, 1])
    return e


def features(hist, n_obs, src, obliquity):
    """hist: [n, 4, 5] last four updates, oldest first.  Returns (X [n, 22], sigma [n])."""
    hist = np.asarray(hist, dtype=np.float64)
    n = hist.shape[0]
    sigma = np.sqrt(np.mean(hist.reshape(n, 20) ** 2, axis=1))
    safe = np.where(sigma > 0.0, sigma, 1.0)
    X = np.zeros((n, N_IN))
    X[:, :20] = hist.reshape(n, 20) / safe[:, None]
    X[:, 20] = np.log10(np.maximum(np.asarray(n_obs, dtype=np.float64), 1.0)) - 2.5
    a, d = np.asarray(src)[:, 0], np.asarray(src)[:, 1]
    r = np.stack([np.cos(d) * np.cos(a), np.cos(d) * np.sin(a), np.sin(d)], axis=1)
    pole = np.array([0.0, -np.sin(obliquity), np.cos(obliquity)])
    X[:, 21] = r @ pole
    return X, sigma


def targets(src_k, src_ref, sigma):
    safe = np.where(sigma > 0.0, sigma, 1.0)
    return tangent_diff(src_ref, src_k) / safe[:, None]


def apply_correction(src, Y, sigma):
    """src + sigma * Y in tangent units (alpha* turned back into alpha with cos(delta))."""
    c = np.asarray(Y, dtype=np.float64) * np.asarray(sigma, dtype=np.float64)[:, None]
    out = np.array(src, dtype=np.float64, copy=True)
    out[:, 0] += c[:, 0] / np.cos(out[:, 1])
    out[:, 1:] += c[:, 1:]
    return out
