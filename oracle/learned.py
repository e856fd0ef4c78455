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

The root's input may be given as an unevaluated sum of two floats, ``u + ulo`` (the training data
carries about 48 bits of the range-reduced key that way); every function below takes the optional
``ulo`` and works on the float64 sum.

Training fits the output layer in knot-value form: with unit input weights, fixed knots
c_0 < ... < c_H (b1[h] = -c_h) and caps c_{h+1} - c_h (the last unit uncapped), the network is the
linear spline through the points (c_h, v_h), with b2 = v_0 and w2[h] = (v_{h+1} - v_h) /
(c_{h+1} - c_h). ``knot_theta`` builds the weights from (v, c); ``knot_grad`` gives dL/dv by the
chain rule through those two relations; ``knot_adam_step`` is one Adam step on v.

Pins (tests): central finite differences of the loss, in theta and in v; zero gradient at the
least-squares optimum that ``numpy.linalg.lstsq`` finds when every hidden unit is active (the model
is then linear in w2, b2); ``numpy.interp`` for the knot-value spline; Adam's closed-form first step.
"""
from __future__ import annotations

import numpy as np


def unpack(theta, H: int = 16):
    theta = np.asarray(theta, dtype=np.float64)
    assert theta.size == 3 * H + 1
    return theta[:H], theta[H:2 * H], theta[2 * H:3 * H], theta[3 * H]


def _caps(cap, H):
    return np.full(H, np.inf) if cap is None else np.asarray(cap, dtype=np.float64)


def _input(u, ulo):
    u = np.asarray(u, dtype=np.float64)
    return u if ulo is None else u + np.asarray(ulo, dtype=np.float64)


def forward(theta, u, H: int = 16, cap=None, ulo=None):
    """y(u) for every input (float64)."""
    w1, b1, w2, b2 = unpack(theta, H)
    u = _input(u, ulo)
    z = np.outer(u, w1) + b1            # (n, H) pre-activations
    a = np.minimum(np.maximum(z, 0.0), _caps(cap, H))   # saturating ReLU
    return a @ w2 + b2


def loss(theta, u, t, H: int = 16, cap=None, ulo=None) -> float:
    y = forward(theta, u, H, cap, ulo)
    r = y - np.asarray(t, dtype=np.float64)
    return float(np.mean(r * r))


def grad(theta, u, t, H: int = 16, cap=None, ulo=None):
    """(loss, dL/dtheta) in float64, by the chain rule through the two layers."""
    w1, b1, w2, b2 = unpack(theta, H)
    c = _caps(cap, H)
    u = _input(u, ulo)
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


def knot_theta(v, c, H: int = 16, last_cap: float = 4.0):
    """(theta, cap) of the spline through (c_h, v_h), h = 0..H: unit input weights, b1 = -c_h,
    w2[h] = (v_{h+1} - v_h) / (c_{h+1} - c_h), b2 = v_0; caps c_{h+1} - c_h, except the last
    unit's, ``last_cap`` (it keeps rising past c_H)."""
    v = np.asarray(v, dtype=np.float64)
    c = np.asarray(c, dtype=np.float64)
    assert v.size == c.size == H + 1
    dc = np.diff(c)
    cap = dc.copy()
    cap[H - 1] = last_cap
    theta = np.concatenate([np.ones(H), -c[:H], np.diff(v) / dc, [v[0]]])
    return theta, cap


def knot_grad(v, c, u, t, H: int = 16, ulo=None, last_cap: float = 4.0):
    """(loss, dL/dv): the network's gradient carried to the knot values. v_j enters w2[j - 1]
    with weight +1 / (c_j - c_{j-1}), w2[j] with weight -1 / (c_{j+1} - c_j), and v_0 is b2."""
    theta, cap = knot_theta(v, c, H, last_cap)
    L, g = grad(theta, u, t, H, cap, ulo)
    g_w2, g_b2 = g[2 * H:3 * H], g[3 * H]
    dc = np.diff(np.asarray(c, dtype=np.float64))
    gv = np.zeros(H + 1)
    gv[1:] += g_w2 / dc
    gv[:-1] -= g_w2 / dc
    gv[0] += g_b2
    return L, gv


def knot_adam_step(v, m, q, step: int, c, u, t, lr: float, H: int = 16, ulo=None,
                   last_cap: float = 4.0):
    """One training step in knot-value form: the loss and dL/dv at v, then Adam on v (``step`` is
    the 1-based step number). Returns (v, m, q, loss at the old v)."""
    L, gv = knot_grad(v, c, u, t, H, ulo, last_cap)
    v1, m1, q1 = adam_step(np.asarray(v, dtype=np.float64), gv, m, q, step, lr)
    return v1, m1, q1, L
