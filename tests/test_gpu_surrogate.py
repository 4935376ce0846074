"""Surrogate network kernels (forward, backward, Adam) against the FP64 oracle.

The GPU multiplies with the bfloat16 roundings of its FP32 master weights and
accumulates in FP32; the oracle gets the same rounded weights, so the only
differences are FP32 rounding: a 256-term FP32 dot product is within about
256 * 2^-24 ~ 1.5e-5 of its exact value relative to the sum of magnitudes,
and the tolerances below allow a few times that. The ReLU masks are decisions
taken from floating point: the gradient and Adam cases use weights (biases
of +-2, small weights) and inputs for which no pre-activation lies within 1e-3
of zero, where FP32 and FP64 could disagree (checked in the test).
"""
import numpy as np
import pytest
import torch

from oracle import surrogate as sg
from paper_2302_07084_gb300 import lne

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2302_07084_gb300 import build
    build.build()
    c = lne.Context(0)
    yield c
    c.close()


def _case(seed, rows, scale=0.08):
    rng = np.random.default_rng(seed)
    theta = rng.normal(0.0, scale, sg.N_PARAMS).astype(np.float32)
    mean = rng.normal(0.0, 1.0, 30).astype(np.float32)
    std = rng.uniform(0.5, 2.0, 30).astype(np.float32)
    X = (mean + std * rng.normal(size=(rows, 30))).astype(np.float32)
    t = rng.normal(size=rows).astype(np.float32)
    return theta, mean, std, X, t


def _gapped_case(seed, rows):
    """Weights whose pre-activations stay at least ~0.5 away from zero: biases
    of +-2 on alternating units and small weights, so every ReLU decision is
    the same in FP32 and FP64 (checked by the tests through _margin)."""
    theta, mean, std, X, t = _case(seed, rows, scale=0.005)
    p = sg.unpack(theta.astype(np.float64).copy())
    sign = np.where(np.arange(256) % 2 == 0, 1.0, -1.0)
    p["b1"][:] = 2.0 * sign
    p["b2"][:] = 2.0 * sign[::-1]
    p["W1"][:] *= 2.0
    p["w3"][:] = np.random.default_rng(seed + 100).normal(0.0, 0.1, 256)
    return sg.pack(p).astype(np.float32), mean, std, X, t


def _oracle_inputs(theta, mean, std, X):
    th = sg.bf16_round(theta)
    Xs = (X.astype(np.float64) - mean.astype(np.float64)) / std.astype(np.float64)
    return th, Xs


def _margin(th, Xs):
    _, (_, z1, _, z2, _) = sg.forward(th, Xs)
    return min(np.abs(z1).min(), np.abs(z2).min())


def test_forward_matches_oracle(ctx):
    theta, mean, std, X, _ = _case(1, 1000)     # 31 full 32-row tiles and a ragged tail of 8
    ctx.surrogate_set_params(theta, mean, std)
    y = ctx.surrogate_predict(torch.as_tensor(X).cuda()).cpu().numpy()
    th, Xs = _oracle_inputs(theta, mean, std, X)
    y_ref, _ = sg.forward(th, Xs)
    scale = np.abs(y_ref).max()
    assert np.max(np.abs(y - y_ref)) <= 1e-4 * scale, np.max(np.abs(y - y_ref)) / scale
    assert ctx.surrogate_predict(torch.zeros((0, 30), device="cuda")).numel() == 0


def test_gradient_matches_oracle(ctx):
    theta, mean, std, X, t = _gapped_case(2, 300)
    th, Xs = _oracle_inputs(theta, mean, std, X)
    assert _margin(th, Xs) > 1e-3
    ctx.surrogate_set_params(theta, mean, std)
    g, loss = ctx.surrogate_grad(torch.as_tensor(X).cuda(), torch.as_tensor(t).cuda())
    g = g.cpu().numpy().astype(np.float64)
    g_ref = sg.grad(th, Xs, t)
    assert abs(loss - sg.loss(th, Xs, t)) <= 1e-5 * sg.loss(th, Xs, t)
    parts, parts_ref = sg.unpack(g), sg.unpack(g_ref)
    for name, _ in sg.LAYOUT:
        a, b = parts[name], parts_ref[name]
        err = np.max(np.abs(a - b)) / max(np.abs(b).max(), 1e-30)
        assert err <= 2e-4, (name, err)


def test_adam_step_matches_oracle(ctx):
    theta, mean, std, X, t = _gapped_case(7, 256)
    th, Xs = _oracle_inputs(theta, mean, std, X)
    assert _margin(th, Xs) > 1e-3
    ctx.surrogate_set_params(theta, mean, std)
    ctx.surrogate_train(torch.as_tensor(X).cuda(), torch.as_tensor(t).cuda(), epochs=1, batch=256, lr=1e-3, seed=1)
    got, _, _ = ctx.surrogate_get_params()
    g_ref = sg.grad(th, Xs, t)
    want, _, _ = sg.adam_step(theta.astype(np.float64), np.zeros(sg.N_PARAMS), np.zeros(sg.N_PARAMS), g_ref, 1)
    diff = np.abs(got - want)
    # the first Adam step is lr * g / (|g| + eps): well-determined where |g| >> eps
    firm = np.abs(g_ref) > 1e-4 * np.abs(g_ref).max()
    assert diff[firm].max() <= 2e-6, diff[firm].max()
    assert diff.max() <= 2.1e-3


def test_training_fits_a_smooth_target(ctx):
    rng = np.random.default_rng(12)
    X = rng.normal(size=(4096, 30)).astype(np.float32) * 3.0 + 1.0
    Z = (X - 1.0) / 3.0
    t = (np.sin(Z[:, 0]) + 0.5 * Z[:, 1] * Z[:, 2] - 0.3 * Z[:, 3] ** 2).astype(np.float32)
    Xd, td = torch.as_tensor(X).cuda(), torch.as_tensor(t).cuda()
    ctx.surrogate_init(seed=5)
    ctx.surrogate_fit_scaling(Xd)
    _, mean, std = ctx.surrogate_get_params()
    m_ref, s_ref = sg.feature_scaling(X)
    assert np.allclose(mean, m_ref, rtol=1e-5, atol=1e-5) and np.allclose(std, s_ref, rtol=1e-5)
    loss0 = float(np.mean((ctx.surrogate_predict(Xd).cpu().numpy() - t) ** 2))
    loss = ctx.surrogate_train(Xd, td, epochs=40, batch=256, lr=1e-3, seed=3)
    print(f"MSE before {loss0:.4f} after {loss:.4f} (target variance {t.var():.4f})")
    assert loss < 0.1 * t.var() and loss < loss0
    # same seed, same data: bit-identical weights
    w1, _, _ = ctx.surrogate_get_params()
    ctx.surrogate_init(seed=5)
    ctx.surrogate_fit_scaling(Xd)
    ctx.surrogate_train(Xd, td, epochs=40, batch=256, lr=1e-3, seed=3)
    w2, _, _ = ctx.surrogate_get_params()
    assert np.array_equal(w1, w2)


def test_uninitialised_network_is_an_error():
    from paper_2302_07084_gb300 import build
    build.build()
    c = lne.Context(0)
    with pytest.raises(lne.LneError) as e:
        c.surrogate_predict(torch.zeros((4, 30), device="cuda"))
    assert e.value.code == -1
    c.close()
