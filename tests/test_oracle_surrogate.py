"""Pins of the surrogate network's oracle (FP64) against facts that do not
come from the oracle itself: the parameter count of a 30-256-256-1 network,
central finite differences of the loss, networks that reduce to closed forms,
the closed form of Adam's first step, and exactly known bfloat16 roundings."""
import numpy as np
import pytest

from oracle import surrogate as sg


def _theta(seed, scale=0.3):
    return np.random.default_rng(seed).normal(0.0, scale, sg.N_PARAMS)


def test_parameter_count():
    # (30 * 256 + 256) + (256 * 256 + 256) + (256 + 1)
    assert sg.N_PARAMS == 73_985


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(1)
    theta = _theta(2)
    X = rng.normal(size=(7, 30))
    t = rng.normal(size=7)
    g = sg.grad(theta, X, t)
    # every bias and output weight, and a spread of first- and second-layer weights
    layout, o = {}, 0
    for name, shape in sg.LAYOUT:
        layout[name] = (o, int(np.prod(shape)))
        o += int(np.prod(shape))
    idx = list(range(layout["b1"][0], layout["b1"][0] + 256, 17))
    idx += list(range(layout["b2"][0], layout["b2"][0] + 256, 13))
    idx += list(range(layout["w3"][0], layout["w3"][0] + 257))
    idx += list(rng.choice(layout["W1"][1], 40, replace=False))
    idx += list(layout["W2"][0] + rng.choice(layout["W2"][1], 60, replace=False))
    h = 1e-6
    for i in idx:
        e = np.zeros_like(theta)
        e[i] = h
        fd = (sg.loss(theta + e, X, t) - sg.loss(theta - e, X, t)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])


def test_forward_closed_forms():
    X = np.random.default_rng(3).normal(size=(5, 30))
    p = {name: np.zeros(shape) for name, shape in sg.LAYOUT}
    # W2 = 0: the output is b3 + w3 . relu(b2), whatever the input
    p["W1"] = np.random.default_rng(4).normal(size=(30, 256))
    p["b2"] = np.linspace(-1.0, 1.0, 256)
    p["w3"] = np.linspace(0.5, 2.0, 256)
    p["b3"] = np.array([0.25])
    y, _ = sg.forward(sg.pack(p), X)
    assert np.allclose(y, 0.25 + np.sum(np.linspace(0.5, 2.0, 256) * np.maximum(np.linspace(-1, 1, 256), 0)))
    # one path through the network: x0 -> unit 0 -> unit 0 -> y with positive weights is linear
    p = {name: np.zeros(shape) for name, shape in sg.LAYOUT}
    p["W1"][0, 0], p["W2"][0, 0], p["w3"][0], p["b3"][0] = 2.0, 3.0, 0.5, -1.0
    Xp = np.abs(X)
    y, _ = sg.forward(sg.pack(p), Xp)
    assert np.allclose(y, 3.0 * Xp[:, 0] - 1.0)
    # ... and zero through a negative first-layer input (the ReLU cuts it)
    y, _ = sg.forward(sg.pack(p), -Xp)
    assert np.allclose(y, -1.0)


def test_gradient_of_linear_path():
    # y = a x (one positive path, a = W1 W2 w3): dL/dw3 = mean 2 (y - t) h2
    p = {name: np.zeros(shape) for name, shape in sg.LAYOUT}
    p["W1"][0, 0], p["W2"][0, 0], p["w3"][0] = 2.0, 3.0, 0.5
    x = np.zeros((2, 30))
    x[:, 0] = [1.0, 2.0]
    t = np.array([1.0, 0.0])
    g = sg.unpack(sg.grad(sg.pack(p), x, t))
    y = 3.0 * x[:, 0]
    h2 = 6.0 * x[:, 0]
    assert np.isclose(g["w3"][0], np.mean(2 * (y - t) * h2))
    assert np.isclose(g["b3"][0], np.mean(2 * (y - t)))
    assert np.isclose(g["W1"][0, 0], np.mean(2 * (y - t) * 3.0 * 0.5 * x[:, 0]))


def test_adam_first_step_closed_form():
    g = np.array([0.3, -2.0, 1e-3, 0.0])
    theta = np.array([1.0, 1.0, 1.0, 1.0])
    new, m, v = sg.adam_step(theta, np.zeros(4), np.zeros(4), g, step=1, lr=1e-3)
    # after bias correction the first step is lr * g / (|g| + eps)
    assert np.allclose(new, theta - 1e-3 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-15)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)
    # a constant gradient keeps moving every weight by lr (m_hat = g, v_hat = g^2)
    th, mm, vv = theta, np.zeros(4), np.zeros(4)
    for s in range(1, 6):
        th, mm, vv = sg.adam_step(th, mm, vv, np.array([0.5, -0.5, 2.0, -2.0]), step=s, lr=0.01)
    assert np.allclose(th, theta - 0.05 * np.sign([0.5, -0.5, 2.0, -2.0]), atol=1e-7)


def test_bf16_round_known_values():
    u = 2.0 ** -8
    vals = np.array([1.0, 1.0 + u, 1.0 + 2 * u, 1.0 + 3 * u, -3.0 - 3 * u, 0.0, 2.0 ** -130, 65504.0])
    want = np.array([1.0, 1.0, 1.0 + 2 * u, 1.0 + 4 * u, -3.0 - 4 * u, 0.0, 2.0 ** -130, 65536.0])
    # 1 + u is a tie between 1 and 1 + 2u: to the even one (1); 1 + 3u: tie, to 1 + 4u (even)
    # -3 - 3u: spacing 4u above 2, so -3 - 3u rounds to the nearer -3 - 4u
    # 65504 = 2^16 - 32: spacing 256 above 2^15, so it rounds up to 2^16
    got = sg.bf16_round(vals)
    assert np.array_equal(got, want), (got, want)
    x = np.random.default_rng(5).normal(size=10000).astype(np.float32)
    r = sg.bf16_round(x)
    assert np.all(np.abs(r - x) <= np.abs(x) * 2.0 ** -8)
    assert np.all(r.astype(np.float32).view(np.uint32) & 0xFFFF == 0)


def test_feature_scaling():
    X = np.array([[1.0, 5.0, 2.0], [3.0, 5.0, 4.0], [5.0, 5.0, 9.0]])
    mean, std = sg.feature_scaling(X)
    assert np.allclose(mean, [3.0, 5.0, 5.0])
    assert np.allclose(std, [np.sqrt(8 / 3), 1.0, np.sqrt(26 / 3)])
