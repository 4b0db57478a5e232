"""fp64 reference of the kernel-variant cost model (a 3-layer perceptron).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Network (hidden width H, F input features, V outputs = one predicted
log-time per kernel variant):
    Z1 = X W1^T + b1,  H1 = relu(Z1)        W1: H x F
    Z2 = H1 W2^T + b2, H2 = relu(Z2)        W2: H x H
    Y  = H2 W3^T + b3                        W3: V x H
Loss (masked mean squared error; a variant that was not timed for a shape
has mask 0):
    L = sum_{b,v} mask (Y - T)^2 / (2 M),   M = sum mask  (L = 0 if M = 0)
The gradients are the chain rule written out layer by layer (backprop),
with relu'(0) = 0.  The optimiser step is Adam as defined by Kingma & Ba,
"Adam: A method for stochastic optimization" (ICLR 2015), Algorithm 1.

Plain numpy matrix products serve as steps; nothing is fused or reordered.
"""
from __future__ import annotations

import numpy as np

PARAM_NAMES = ("W1", "b1", "W2", "b2", "W3", "b3")


def init_params(F: int, H: int, V: int, draws: np.ndarray) -> dict:
    """Deterministic init from a vector of uniform[-1, 1) draws: each weight
    matrix is scaled by sqrt(3 / fan_in) (unit-variance activations for
    unit-variance inputs), biases start at 0.  ``draws`` must hold at least
    H*F + H*H + V*H values."""
    d = np.asarray(draws, dtype=np.float64)
    n1, n2, n3 = H * F, H * H, V * H
    W1 = d[:n1].reshape(H, F) * np.sqrt(3.0 / F)
    W2 = d[n1:n1 + n2].reshape(H, H) * np.sqrt(3.0 / H)
    W3 = d[n1 + n2:n1 + n2 + n3].reshape(V, H) * np.sqrt(3.0 / H)
    return {"W1": W1, "b1": np.zeros(H), "W2": W2, "b2": np.zeros(H),
            "W3": W3, "b3": np.zeros(V)}


def forward(p: dict, X: np.ndarray):
    X = np.asarray(X, dtype=np.float64)
    Z1 = X @ p["W1"].T + p["b1"]
    H1 = np.maximum(Z1, 0.0)
    Z2 = H1 @ p["W2"].T + p["b2"]
    H2 = np.maximum(Z2, 0.0)
    Y = H2 @ p["W3"].T + p["b3"]
    return Y, (X, Z1, H1, Z2, H2)


def loss(Y: np.ndarray, T: np.ndarray, mask: np.ndarray) -> float:
    M = float(mask.sum())
    if M == 0.0:
        return 0.0
    r = (Y - T) * mask
    return float((r * r).sum() / (2.0 * M))


def backward(p: dict, cache, Y: np.ndarray, T: np.ndarray, mask: np.ndarray) -> dict:
    X, Z1, H1, Z2, H2 = cache
    M = float(mask.sum())
    dY = np.zeros_like(Y) if M == 0.0 else mask * (Y - T) / M
    g = {}
    g["W3"] = dY.T @ H2
    g["b3"] = dY.sum(axis=0)
    dH2 = dY @ p["W3"]
    dZ2 = dH2 * (Z2 > 0.0)
    g["W2"] = dZ2.T @ H1
    g["b2"] = dZ2.sum(axis=0)
    dH1 = dZ2 @ p["W2"]
    dZ1 = dH1 * (Z1 > 0.0)
    g["W1"] = dZ1.T @ X
    g["b1"] = dZ1.sum(axis=0)
    return g


def adam_step(p: dict, g: dict, state: dict, lr: float, beta1: float = 0.9,
              beta2: float = 0.999, eps: float = 1e-8, l2: float = 0.0) -> None:
    """One Adam update in place.  ``state`` holds t and the moment estimates.
    ``l2``: an L2 penalty (l2 / 2) |p|^2 added to the loss, so the moments
    see the gradient g + l2 * p."""
    t = state.get("t", 0) + 1
    state["t"] = t
    for name in PARAM_NAMES:
        m = state.setdefault("m_" + name, np.zeros_like(p[name]))
        v = state.setdefault("v_" + name, np.zeros_like(p[name]))
        gt = g[name] + l2 * p[name]
        m[...] = beta1 * m + (1.0 - beta1) * gt
        v[...] = beta2 * v + (1.0 - beta2) * gt * gt
        mhat = m / (1.0 - beta1 ** t)
        vhat = v / (1.0 - beta2 ** t)
        p[name] = p[name] - lr * mhat / (np.sqrt(vhat) + eps)
