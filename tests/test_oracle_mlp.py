"""Pins for the fp64 cost-model reference (no GPU): gradients against central
finite differences, Adam against its closed form after one and two steps, and
the network against an explicit affine composition where every ReLU is
active."""
from __future__ import annotations

import numpy as np
import pytest

from oracle import mlp
from paper_1304_7053_gb300 import inputs


def tiny(F=3, H=5, V=2, B=6, seed=0):
    p = mlp.init_params(F, H, V, inputs.uniform(seed, H * F + H * H + V * H))
    for j, name in enumerate(("b1", "b2", "b3")):
        p[name] = 0.1 * inputs.uniform(seed + 10 + j, p[name].size)
    X = inputs.uniform(seed + 1, B * F).reshape(B, F)
    T = inputs.uniform(seed + 2, B * V).reshape(B, V)
    mask = (inputs.splitmix64(seed + 3, B * V) % np.uint64(4) != 0).astype(np.float64).reshape(B, V)
    return p, X, T, mask


def test_gradients_match_central_differences():
    p, X, T, mask = tiny()
    Y, cache = mlp.forward(p, X)
    g = mlp.backward(p, cache, Y, T, mask)
    h = 1e-6
    for name in mlp.PARAM_NAMES:
        num = np.zeros_like(p[name])
        for idx in np.ndindex(*p[name].shape):
            old = p[name][idx]
            p[name][idx] = old + h
            lp = mlp.loss(mlp.forward(p, X)[0], T, mask)
            p[name][idx] = old - h
            lm = mlp.loss(mlp.forward(p, X)[0], T, mask)
            p[name][idx] = old
            num[idx] = (lp - lm) / (2 * h)
        np.testing.assert_allclose(g[name], num, rtol=1e-5, atol=1e-9, err_msg=name)


def test_masked_entries_do_not_contribute():
    p, X, T, mask = tiny(seed=4)
    Y, cache = mlp.forward(p, X)
    T2 = T.copy()
    T2[mask == 0] += 100.0
    g1 = mlp.backward(p, cache, Y, T, mask)
    g2 = mlp.backward(p, cache, Y, T2, mask)
    for name in mlp.PARAM_NAMES:
        np.testing.assert_array_equal(g1[name], g2[name])
    assert mlp.loss(Y, T, np.zeros_like(mask)) == 0.0


def test_affine_when_all_relus_active():
    """With every pre-activation positive the network is an affine map:
    Y = W3 (W2 (W1 x + b1) + b2) + b3."""
    p, X, T, mask = tiny(seed=7)
    p["b1"] = p["b1"] + 50.0
    p["b2"] = p["b2"] + 500.0
    Y, (X_, Z1, H1, Z2, H2) = mlp.forward(p, X)
    assert (Z1 > 0).all() and (Z2 > 0).all()
    for b in range(X.shape[0]):
        want = p["W3"] @ (p["W2"] @ (p["W1"] @ X[b] + p["b1"]) + p["b2"]) + p["b3"]
        np.testing.assert_allclose(Y[b], want, rtol=1e-12)


def test_adam_closed_form_two_steps():
    """Kingma & Ba, Algorithm 1, for a scalar parameter and gradients g1, g2."""
    lr, b1, b2, eps = 0.01, 0.9, 0.999, 1e-8
    p = {n: np.array([0.5]) for n in mlp.PARAM_NAMES}
    g1 = {n: np.array([0.2]) for n in mlp.PARAM_NAMES}
    g2 = {n: np.array([-0.3]) for n in mlp.PARAM_NAMES}
    st = {}
    mlp.adam_step(p, g1, st, lr, b1, b2, eps)
    # step 1: m_hat = g1, v_hat = g1^2  =>  theta -= lr * g1 / (|g1| + eps)
    theta1 = 0.5 - lr * 0.2 / (0.2 + eps)
    assert p["W1"][0] == pytest.approx(theta1, abs=1e-15)
    mlp.adam_step(p, g2, st, lr, b1, b2, eps)
    m2 = b1 * (1 - b1) * 0.2 + (1 - b1) * -0.3
    v2 = b2 * (1 - b2) * 0.04 + (1 - b2) * 0.09
    theta2 = theta1 - lr * (m2 / (1 - b1 ** 2)) / (np.sqrt(v2 / (1 - b2 ** 2)) + eps)
    assert p["b3"][0] == pytest.approx(theta2, abs=1e-15)
    assert st["t"] == 2


def test_adam_l2_penalty_closed_form():
    """With an L2 penalty (l2 / 2) p^2 the first step is the sign step of
    Algorithm 1 on g + l2 * p: theta -= lr * (g + l2 p) / (|g + l2 p| + eps);
    a gradient that the penalty exactly cancels leaves p in place, and
    l2 = 0 is plain Adam."""
    lr, eps, l2 = 0.01, 1e-8, 0.5
    p = {n: np.array([0.5]) for n in mlp.PARAM_NAMES}
    g = {n: np.array([-0.1]) for n in mlp.PARAM_NAMES}
    mlp.adam_step(p, g, {}, lr, 0.9, 0.999, eps, l2=l2)
    ge = -0.1 + l2 * 0.5
    assert p["W2"][0] == pytest.approx(0.5 - lr * ge / (abs(ge) + eps), abs=1e-15)
    p = {n: np.array([0.4]) for n in mlp.PARAM_NAMES}
    g = {n: np.array([-0.2]) for n in mlp.PARAM_NAMES}      # g + l2 p = 0
    mlp.adam_step(p, g, {}, lr, 0.9, 0.999, eps, l2=l2)
    assert p["b1"][0] == 0.4
    p0 = {n: np.array([0.3]) for n in mlp.PARAM_NAMES}
    p1 = {n: np.array([0.3]) for n in mlp.PARAM_NAMES}
    gz = {n: np.array([0.7]) for n in mlp.PARAM_NAMES}
    mlp.adam_step(p0, gz, {}, lr)
    mlp.adam_step(p1, gz, {}, lr, l2=0.0)
    assert p0["W3"][0] == p1["W3"][0]


def test_training_reduces_loss():
    """A few hundred full-batch Adam steps fit a smooth target."""
    F, H, V, B = 4, 16, 3, 64
    p = mlp.init_params(F, H, V, inputs.uniform(1, H * F + H * H + V * H))
    X = inputs.uniform(2, B * F).reshape(B, F)
    T = np.stack([X[:, 0] * X[:, 1], np.sin(X[:, 2]), X[:, 3] ** 2], axis=1)
    mask = np.ones_like(T)
    st = {}
    l0 = mlp.loss(mlp.forward(p, X)[0], T, mask)
    for _ in range(300):
        Y, cache = mlp.forward(p, X)
        mlp.adam_step(p, mlp.backward(p, cache, Y, T, mask), st, 0.01)
    l1 = mlp.loss(mlp.forward(p, X)[0], T, mask)
    assert l1 < 0.1 * l0
