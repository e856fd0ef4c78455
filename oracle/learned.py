"""CPU oracle of the learned position model's arithmetic — TEST INFRASTRUCTURE.

The model is the root of a two-layer recursive model index: a 1 -> H -> 1 multilayer perceptron with
saturating ReLU hidden units (a unit's output is capped at cap[h]; cap = inf gives plain ReLUs),

    y(u) = b2 + sum_h w2[h] * min(max(w1[h] * u + b1[h], 0), cap[h]),

fitted to the empirical CDF of the keys by mean squared error,

    L = (1/n) * sum_i (y(u_i) - t_i)^2.

This module writes the forward pass, the loss and its gradient out in float64 from these definitions
(plain numpy, no fusion), for checking the CUDA training kernels. Trained parameters are packed as
one vector ``theta = [w1 (H), b1 (H), w2 (H), b2]`` (3H + 1 values); the caps are fixed and passed
separately.

Pins (tests): central finite differences of the loss; zero gradient at the least-squares optimum that
``numpy.linalg.lstsq`` finds when every hidden unit is active (the model is then linear in w2, b2).
"""
from __future__ import annotations

import numpy as np


def unpack(theta, H: int = 16):
    theta = np.asarray(theta, dtype=np.float64)
    assert theta.size == 3 * H + 1
    return theta[:H], theta[H:2 * H], theta[2 * H:3 * H], theta[3 * H]


def _caps(cap, H):
    return np.full(H, np.inf) if cap is None else np.asarray(cap, dtype=np.float64)


def forward(theta, u, H: int = 16, cap=None):
    """y(u) for every input (float64)."""
    w1, b1, w2, b2 = unpack(theta, H)
    u = np.asarray(u, dtype=np.float64)
    z = np.outer(u, w1) + b1            # (n, H) pre-activations
    a = np.minimum(np.maximum(z, 0.0), _caps(cap, H))   # saturating ReLU
    return a @ w2 + b2


def loss(theta, u, t, H: int = 16, cap=None) -> float:
    y = forward(theta, u, H, cap)
    r = y - np.asarray(t, dtype=np.float64)
    return float(np.mean(r * r))


def grad(theta, u, t, H: int = 16, cap=None):
    """(loss, dL/dtheta) in float64, by the chain rule through the two layers."""
    w1, b1, w2, b2 = unpack(theta, H)
    c = _caps(cap, H)
    u = np.asarray(u, dtype=np.float64)
    t = np.asarray(t, dtype=np.float64)
    n = u.size
    z = np.outer(u, w1) + b1
    a = np.minimum(np.maximum(z, 0.0), c)
    y = a @ w2 + b2
    r = y - t
    dy = 2.0 * r / n                    # dL/dy_i
    g_w2 = a.T @ dy
    g_b2 = dy.sum()
    dz = np.outer(dy, w2) * ((z > 0.0) & (z < c))   # unit slope 1 inside (0, cap), else 0
    g_w1 = dz.T @ u
    g_b1 = dz.sum(axis=0)
    return float(np.mean(r * r)), np.concatenate([g_w1, g_b1, g_w2, [g_b2]])


def adam_step(theta, g, m, v, step: int, lr: float, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma and Ba, 2015), float64; returns (theta, m, v)."""
    m = beta1 * m + (1 - beta1) * g
    v = beta2 * v + (1 - beta2) * g * g
    mh = m / (1 - beta1 ** step)
    vh = v / (1 - beta2 ** step)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v
