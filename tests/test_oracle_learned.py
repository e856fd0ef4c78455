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


def test_two_float_input_is_the_sum():
    """A float64 input split into a float32 and the float32 rest gives the same network output and
    gradient as the input itself (to float64 rounding): the split carries the value."""
    rng = np.random.default_rng(11)
    H = 16
    theta = rng.normal(size=3 * H + 1)
    cap = rng.random(H) + 0.05
    x = rng.random(300)
    hi = x.astype(np.float32).astype(np.float64)
    lo = (x - hi).astype(np.float32).astype(np.float64)
    assert np.all(hi + lo == x) or np.max(np.abs(hi + lo - x)) < 1e-15
    t = np.sort(rng.random(300))
    assert np.allclose(L.forward(theta, hi, H, cap, ulo=lo), L.forward(theta, x, H, cap),
                       rtol=0, atol=1e-13)
    l1, g1 = L.grad(theta, hi, t, H, cap, ulo=lo)
    l0, g0 = L.grad(theta, x, t, H, cap)
    assert abs(l1 - l0) < 1e-13 and np.max(np.abs(g1 - g0)) < 1e-12
    # the low part matters: dropping it changes the output where the input is steep
    assert np.max(np.abs(lo)) > 0


def test_two_float_gradient_matches_central_differences():
    rng = np.random.default_rng(12)
    H = 16
    theta = rng.normal(size=3 * H + 1)
    cap = rng.random(H) * 1.5 + 0.05
    u = rng.random(400)
    ulo = rng.normal(size=400) * 1e-4
    t = np.sort(rng.random(400))
    _, g = L.grad(theta, u, t, H, cap, ulo=ulo)
    eps = 1e-6
    for k in range(theta.size):
        d = np.zeros_like(theta)
        d[k] = eps
        num = (L.loss(theta + d, u, t, H, cap, ulo=ulo)
               - L.loss(theta - d, u, t, H, cap, ulo=ulo)) / (2 * eps)
        assert abs(num - g[k]) <= 1e-6 * max(1.0, abs(num)), k


def knots_and_data(seed, n=3000):
    rng = np.random.default_rng(seed)
    H = 16
    u = np.sort(rng.random(n) ** 2)                 # a CDF far from linear
    c = np.quantile(u, np.linspace(0, 1, H + 1))
    c = np.maximum.accumulate(c + np.arange(H + 1) * 1e-9)
    v = np.sort(rng.random(H + 1))
    t = (np.arange(n) + 0.5) / n
    return H, u, c, v, t


def test_knot_theta_is_the_interpolating_spline():
    """knot_theta's network equals numpy.interp through (c_h, v_h) on [c_0, c_H]."""
    H, u, c, v, _ = knots_and_data(13)
    theta, cap = L.knot_theta(v, c, H)
    x = np.random.default_rng(14).uniform(c[0], c[-1], 2000)
    assert np.allclose(L.forward(theta, x, H, cap), np.interp(x, c, v), rtol=0, atol=1e-12)


def test_knot_gradient_matches_central_differences():
    """dL/dv by the chain rule equals central differences of L(v) = loss(knot_theta(v))."""
    H, u, c, v, t = knots_and_data(15)
    ulo = np.random.default_rng(16).normal(size=u.size) * 1e-7
    _, gv = L.knot_grad(v, c, u, t, H, ulo=ulo)
    eps = 1e-7
    for k in range(H + 1):
        d = np.zeros(H + 1)
        d[k] = eps
        th_p, cap = L.knot_theta(v + d, c, H)
        th_m, _ = L.knot_theta(v - d, c, H)
        num = (L.loss(th_p, u, t, H, cap, ulo=ulo) - L.loss(th_m, u, t, H, cap, ulo=ulo)) / (2 * eps)
        assert abs(num - gv[k]) <= 1e-6 * max(1.0, abs(num)), k


def test_knot_gradient_vanishes_at_the_least_squares_values():
    """For fixed knots the spline is linear in v: numpy's least-squares v (basis: the hat
    functions, obtained as the spline of each unit vector) has zero knot gradient."""
    H, u, c, _, t = knots_and_data(17)
    B = np.column_stack([np.interp(u, c, np.eye(H + 1)[k]) for k in range(H + 1)])
    v_opt, *_ = np.linalg.lstsq(B, t, rcond=None)
    _, gv = L.knot_grad(v_opt, c, u, t, H)
    assert np.max(np.abs(gv)) < 1e-10


def test_knot_adam_first_step_closed_form():
    """Adam's first step on v moves each knot value by lr against the sign of its gradient
    (bias-corrected moments; eps negligible), and the step lowers the loss for small lr."""
    H, u, c, v, t = knots_and_data(18)
    L0, gv = L.knot_grad(v, c, u, t, H)
    lr = 1e-3
    v1, m1, q1, l_at_v = L.knot_adam_step(v, np.zeros(H + 1), np.zeros(H + 1), 1, c, u, t, lr, H)
    assert l_at_v == L0
    # eps = 1e-8 against |dL/dv| >= 1e-4 moves the step by at most 1e-4 of lr
    assert np.min(np.abs(gv)) > 1e-4
    assert np.allclose(v1, v - lr * np.sign(gv), rtol=0, atol=1e-4 * lr)
    assert np.allclose(m1, 0.1 * gv) and np.allclose(q1, 0.001 * gv * gv)
    th1, cap = L.knot_theta(v1, c, H)
    assert L.loss(th1, u, t, H, cap) < L0
