"""Pins of the learned model's CPU oracle (oracle/learned.py) to facts outside it."""
import numpy as np
import pytest

from oracle import learned as L


@pytest.mark.parametrize("capped", [False, True])
def test_gradient_matches_central_differences(capped):
    rng = np.random.default_rng(1)
    H = 16
    theta = rng.normal(size=3 * H + 1)
    cap = rng.random(H) * 1.5 + 0.05 if capped else None
    u = rng.random(500)
    t = np.sort(rng.random(500))
    _, g = L.grad(theta, u, t, H, cap)
    eps = 1e-6
    for k in range(theta.size):
        d = np.zeros_like(theta)
        d[k] = eps
        num = (L.loss(theta + d, u, t, H, cap) - L.loss(theta - d, u, t, H, cap)) / (2 * eps)
        assert abs(num - g[k]) <= 1e-6 * max(1.0, abs(num)), k


def test_capped_units_give_the_linear_spline_through_knots():
    """Unit slopes, knots c_h, caps c_{h+1} - c_h, output weights the segment slopes: the network is
    the linear interpolation through (c_h, v_h) — the same values as numpy.interp."""
    rng = np.random.default_rng(4)
    H = 16
    c = np.sort(rng.random(H + 1))
    v = np.sort(rng.random(H + 1))
    s = np.diff(v) / np.diff(c)
    theta = np.concatenate([np.ones(H), -c[:H], s, [v[0]]])
    u = rng.uniform(c[0], c[-1], 1000)
    assert np.allclose(L.forward(theta, u, H, np.diff(c)), np.interp(u, c, v), atol=1e-12)


def test_zero_gradient_at_least_squares_optimum():
    """With every hidden unit active (w1 > 0, b1 > 0, u >= 0) the model is linear in (w2, b2);
    at numpy's least-squares solution their gradient vanishes."""
    rng = np.random.default_rng(2)
    H = 16
    u = rng.random(2000)
    t = np.sqrt(u) + 0.01 * rng.normal(size=u.size)
    w1 = rng.random(H) + 0.1
    b1 = rng.random(H) + 0.1
    A = np.column_stack([np.outer(u, w1) + b1, np.ones(u.size)])
    sol, *_ = np.linalg.lstsq(A, t, rcond=None)
    theta = np.concatenate([w1, b1, sol[:H], [sol[H]]])
    _, g = L.grad(theta, u, t, H)
    assert np.max(np.abs(g[2 * H:])) < 1e-9
    # and moving w2 away from the optimum raises the loss
    theta2 = theta.copy()
    theta2[2 * H] += 1e-3
    assert L.loss(theta2, u, t, H) > L.loss(theta, u, t, H)


def test_relu_derivative_is_zero_for_inactive_units():
    H = 16
    theta = np.zeros(3 * H + 1)
    theta[:H] = 1.0
    theta[H:2 * H] = -2.0           # z = u - 2 < 0 for u in [0, 1): every unit inactive
    theta[2 * H:3 * H] = 5.0
    u = np.linspace(0, 0.99, 50)
    t = u
    _, g = L.grad(theta, u, t, H)
    assert np.all(g[:2 * H] == 0) and np.all(g[2 * H:3 * H] == 0)
    assert abs(g[-1] - 2 * np.mean(0 - t)) < 1e-12


def test_adam_matches_closed_form_first_step():
    """Adam's first step moves every parameter by lr * sign(g) (bias-corrected moments)."""
    g = np.array([0.5, -2.0, 1e-3])
    th, m, v = L.adam_step(np.zeros(3), g, np.zeros(3), np.zeros(3), 1, lr=0.1, eps=0.0)
    assert np.allclose(th, -0.1 * np.sign(g))
