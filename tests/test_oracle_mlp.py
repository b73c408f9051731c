"""Pins of the FP64 oracle of the learned proposal (oracle/mlp.py): the gradient against
central finite differences, bfloat16 rounding against the ties-to-even rule worked out by
hand, Adam against its closed form for a constant gradient, and the feature and target
definitions against invariances and closed forms."""
import numpy as np

from oracle import mlp as M


def _data(seed, n=40):
    rng = np.random.default_rng(seed)
    X = rng.normal(size=(n, M.N_IN))
    T = rng.normal(size=(n, M.N_OUT))
    p = M.init_params(seed) + 0.05 * rng.normal(size=M.N_PARAMS)   # non-zero biases too
    return p, X, T


def test_parameter_count_and_layout():
    assert M.N_PARAMS == 64 * 22 + 64 + 64 * 64 + 64 + 5 * 64 + 5 == 5957
    p = np.arange(M.N_PARAMS, dtype=np.float64)
    d = M.unpack(p)
    assert d["W1"][0, 1] == 1 and d["b1"][0] == 64 * 22 and d["b3"][-1] == M.N_PARAMS - 1
    assert np.array_equal(M.pack(d), p)


def test_gradient_matches_central_differences():
    p, X, T = _data(3)
    L, g = M.loss_grad(p, X, T)
    assert abs(L - M.loss(p, X, T)) < 1e-14 * max(1.0, L)
    rng = np.random.default_rng(0)
    idx = np.concatenate([rng.choice(M.N_PARAMS, 400, replace=False), np.arange(M.N_PARAMS - 5 - 64 * 5,
                                                                                   M.N_PARAMS)])
    for i in idx:
        h = 1e-6 * max(1.0, abs(p[i]))
        pp, pm = p.copy(), p.copy()
        pp[i] += h
        pm[i] -= h
        Yp, _ = M.forward(pp, X)
        Ym, _ = M.forward(pm, X)
        # L(p+h) - L(p-h) as sum (Y+ - Y-)(Y+ + Y- - 2T) / n: no cancellation of the losses
        fd = np.sum((Yp - Ym) * (Yp + Ym - 2.0 * T)) / X.shape[0] / (2 * h)
        # central differences are exact to O(h^2) away from the ReLU kinks
        assert abs(fd - g[i]) <= 1e-7 * max(1e-3, abs(g[i])), (i, fd, g[i])


def test_gradient_of_a_single_linear_layer_in_closed_form():
    # with W1, W2 the identity on the first channels and positive inputs the network is
    # linear: Y = X[:, :5] @ W3[:, :5].T + b3, whose gradient is 2 (Y - T)^T X / n
    d = {k: np.zeros(s) for k, s in M.SHAPES}
    d["W1"][:M.N_IN, :M.N_IN] = np.eye(M.N_IN)
    d["W2"][:] = np.eye(M.N_H)
    rng = np.random.default_rng(5)
    d["W3"] = rng.normal(size=(M.N_OUT, M.N_H))
    d["b3"] = rng.normal(size=M.N_OUT)
    X = rng.uniform(0.1, 1.0, size=(30, M.N_IN))
    T = rng.normal(size=(30, M.N_OUT))
    p = M.pack(d)
    Y, _ = M.forward(p, X)
    Yc = X @ d["W3"][:, :M.N_IN].T + d["b3"]
    assert np.allclose(Y, Yc, rtol=1e-14, atol=1e-14)
    _, g = M.loss_grad(p, X, T)
    gW3 = 2.0 * (Yc - T).T @ np.pad(X, ((0, 0), (0, M.N_H - M.N_IN))) / 30
    assert np.allclose(M.unpack(g)["W3"], gW3, rtol=1e-12, atol=1e-14)


def test_bf16_rounding_ties_to_even():
    u = 2.0 ** -7                      # bfloat16 spacing in [1, 2)
    cases = {1.0: 1.0, 1.0 + u / 2: 1.0, 1.0 + 3 * u / 2: 1.0 + 2 * u, 1.0 + u / 2 + 2.0 ** -20: 1.0 + u,
             -(1.0 + 3 * u / 2): -(1.0 + 2 * u), 0.0: 0.0, 3.0: 3.0}
    for x, r in cases.items():
        assert M.bf16(np.float32(x)) == r, (x, M.bf16(np.float32(x)), r)
    # nearest of the two neighbouring bfloat16 values, brute force over a sample
    rng = np.random.default_rng(1)
    x = rng.normal(size=2000).astype(np.float32)
    r = M.bf16(x)
    e = np.floor(np.log2(np.abs(x.astype(np.float64))))
    sp = 2.0 ** (e - 7)
    lo = np.floor(x / sp) * sp
    hi = lo + sp
    best = np.where(np.abs(x - lo) <= np.abs(hi - x), lo, hi)
    tie = np.isclose(np.abs(x - lo), np.abs(hi - x), rtol=0, atol=0)
    assert np.all((r == best) | tie)


def test_adam_constant_gradient_closed_form():
    # for a constant gradient the bias-corrected moments are exactly g and g^2, so every
    # step moves each parameter by lr * g / (|g| + eps)
    rng = np.random.default_rng(2)
    g = rng.normal(size=50)
    p0 = rng.normal(size=50)
    p, m, v = p0.copy(), np.zeros(50), np.zeros(50)
    lr, eps = 1e-3, 1e-8
    for t in range(1, 6):
        p, m, v = M.adam_step(p, g, m, v, t, lr, eps=eps)
        assert np.allclose(p, p0 - t * lr * g / (np.abs(g) + eps), rtol=0, atol=1e-15)


def test_features_scale_free_and_ecliptic_latitude():
    rng = np.random.default_rng(4)
    hist = rng.normal(size=(6, 4, 5)) * 1e-9
    src = np.zeros((6, 5))
    eps = np.deg2rad(23.4392911)
    # ecliptic north pole (alpha 270 deg, delta 90 deg - eps): sin(beta) = 1; equinox: 0
    src[0, :2] = [1.5 * np.pi, 0.5 * np.pi - eps]
    src[1, :2] = [0.0, 0.0]
    src[2:, :2] = rng.uniform(0.1, 1.0, size=(4, 2))
    n = np.array([100, 316, 1000, 50, 80, 250])
    X, s = M.features(hist, n, src, eps)
    X7, s7 = M.features(7.0 * hist, n, src, eps)
    assert np.allclose(X, X7, rtol=1e-14, atol=0) and np.allclose(s7, 7.0 * s, rtol=1e-14)
    assert np.allclose(np.mean(X[:, :20] ** 2, axis=1), 1.0, rtol=1e-12)
    assert abs(X[0, 21] - 1.0) < 1e-12 and abs(X[1, 21]) < 1e-15
    assert np.allclose(X[:, 20], np.log10(n) - 2.5)


def test_targets_and_correction_invert_each_other():
    rng = np.random.default_rng(6)
    src_k = np.column_stack([rng.uniform(0, 2 * np.pi, 20), rng.uniform(-1.4, 1.4, 20), rng.normal(size=(20, 3))])
    src_ref = src_k + rng.normal(size=(20, 5)) * 1e-7
    src_ref[:3, 0] += 2 * np.pi                   # the alpha difference is taken modulo 2 pi
    sigma = rng.uniform(1e-9, 1e-8, 20)
    T = M.targets(src_k, src_ref, sigma)
    back = M.apply_correction(src_k, T, sigma)
    d = back - src_ref
    d[:, 0] = np.mod(d[:, 0] + np.pi, 2 * np.pi) - np.pi
    assert np.max(np.abs(d)) < 1e-15
