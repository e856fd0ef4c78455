"""GPU tests of the learned position model: the library's forward and gradient kernels against the
float64 CPU oracle (oracle/learned.py), and what the trained root gains over the untrained one."""
import numpy as np
import pytest

import oracle
from oracle import learned as OL
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2604_14650_gb300 as pb  # noqa: E402

H = 16


@pytest.fixture(scope="module", autouse=True)
def built():
    pb.build()


def weights(rng):
    """65 floats: the 49 trained parameters (w1, b1, w2, b2), then the 16 saturation caps."""
    return np.concatenate([rng.normal(size=H), rng.normal(size=H) * 0.5, rng.normal(size=H),
                           [rng.normal()], rng.random(H) * 1.5 + 0.05]).astype(np.float32)


def split(w):
    return w[:3 * H + 1].astype(np.float64), w[3 * H + 1:].astype(np.float64)


@pytest.mark.parametrize("n", [1, 1000, 300_001])
def test_forward_matches_oracle(n):
    rng = np.random.default_rng(n)
    w = weights(rng)
    u = rng.random(n).astype(np.float32)
    y = pb.mlp_forward(torch.from_numpy(u).cuda(), w)
    torch.cuda.synchronize()
    th, cap = split(w)
    ref = OL.forward(th, u.astype(np.float64), H, cap)
    # 16 fused multiply-adds in FP32 on O(1) values: a few units in the last place of O(10)
    assert np.max(np.abs(y.cpu().numpy() - ref)) <= 1e-5 * max(1.0, np.max(np.abs(ref)))


@pytest.mark.parametrize("n,seed", [(1, 1), (777, 2), (200_000, 3), (1_000_003, 4)])
def test_gradient_matches_oracle(n, seed):
    """The training kernels' full-batch gradient equals the float64 chain rule: FP32 sums of n
    terms carry a relative error of order 1e-6 of the summed magnitudes; the bound below is
    1e-4 of the largest gradient component."""
    rng = np.random.default_rng(seed)
    w = weights(rng)
    u = rng.random(n).astype(np.float32)
    t = np.sort(rng.random(n)).astype(np.float32)
    loss, g = pb.mlp_grad(torch.from_numpy(u).cuda(), torch.from_numpy(t).cuda(), w)
    th, cap = split(w)
    ref_loss, ref = OL.grad(th, u.astype(np.float64), t.astype(np.float64), H, cap)
    assert abs(loss - ref_loss) <= 1e-5 * max(ref_loss, 1e-12)
    tol = 1e-4 * np.max(np.abs(ref)) + 1e-7
    assert np.max(np.abs(g - ref)) <= tol, (np.max(np.abs(g - ref)), tol)


def split_input(x):
    """float64 values in [0, 1) as the two-float input the training feeds: (float32 of x, float32
    of the rest)."""
    u = x.astype(np.float32)
    return u, (x - u.astype(np.float64)).astype(np.float32)


@pytest.mark.parametrize("n,seed", [(777, 21), (200_000, 22), (1_000_003, 23)])
def test_gradient_split_input_matches_oracle(n, seed):
    """The gradient kernel on the two-float input u + ulo (the form the table build trains on)
    equals the float64 chain rule on the summed input, within the FP32 summation bound above."""
    rng = np.random.default_rng(seed)
    w = weights(rng)
    x = np.sort(rng.random(n) ** 2)
    u, ulo = split_input(x)
    assert np.any(ulo != 0)
    t = ((np.arange(n) + 0.5) / n).astype(np.float32)
    loss, g = pb.mlp_grad_split(torch.from_numpy(u).cuda(), torch.from_numpy(ulo).cuda(),
                                torch.from_numpy(t).cuda(), w)
    th, cap = split(w)
    ref_loss, ref = OL.grad(th, u, t.astype(np.float64), H, cap, ulo=ulo)
    assert abs(loss - ref_loss) <= 1e-5 * max(ref_loss, 1e-12)
    tol = 1e-4 * np.max(np.abs(ref)) + 1e-7
    assert np.max(np.abs(g - ref)) <= tol, (np.max(np.abs(g - ref)), tol)


@pytest.mark.parametrize("n,seed", [(100_000, 2), (1_000_003, 5)])
def test_knot_step_matches_oracle(n, seed):
    """Five training iterations by the library's kernels (gradient, then Adam on the knot values
    through the chain rule) track five float64 steps of the oracle's knot-value Adam: the moments
    within FP32 gradient accuracy (1e-4 of the largest), the knot values within 1e-3 of the
    learning rate per step (every |dL/dv| is above 0.1 of the largest at the start, so no step
    can change sign), and the returned weights are the spline of the returned knot values."""
    rng = np.random.default_rng(seed)
    x = np.sort(rng.random(n) ** 2)
    u, ulo = split_input(x)
    t = ((np.arange(n) + 0.5) / n).astype(np.float32)
    idx = np.minimum(n - 1, (np.arange(H + 1) * n) // H)
    c = (u[idx].astype(np.float64) + ulo[idx]).astype(np.float32)
    for h in range(1, H + 1):
        if not c[h] > c[h - 1]:
            c[h] = np.nextafter(c[h - 1], np.float32(2))
    v = (t[idx] + 0.05 * rng.choice([-1, 1], H + 1)).astype(np.float32)
    th0, cap = OL.knot_theta(v.astype(np.float64), c.astype(np.float64), H)
    w = np.concatenate([th0, cap]).astype(np.float32)
    _, gv0 = OL.knot_grad(v.astype(np.float64), c.astype(np.float64), u, t, H, ulo=ulo)
    assert np.min(np.abs(gv0)) > 0.1 * np.max(np.abs(gv0))
    du, dl, dt = (torch.from_numpy(a).cuda() for a in (u, ulo, t))
    lr = 1e-3
    m = q = np.zeros(H + 1, np.float32)
    rv, rm, rq = v.astype(np.float64), np.zeros(H + 1), np.zeros(H + 1)
    for step in range(5):
        loss, w, v, m, q = pb.mlp_knot_step(du, dl, dt, w, c, v, m, q, step, lr)
        rv, rm, rq, rloss = OL.knot_adam_step(rv, rm, rq, step + 1, c.astype(np.float64), u, t,
                                              lr, H, ulo=ulo)
        assert abs(loss - rloss) <= 1e-5 * rloss + 1e-12, step
        assert np.max(np.abs(m - rm)) <= 1e-4 * np.max(np.abs(rm)) + 1e-9, step
        assert np.max(np.abs(q - rq)) <= 2e-4 * np.max(np.abs(rq)) + 1e-12, step
        assert np.max(np.abs(v - rv)) <= 1e-3 * lr * (step + 1) + 2e-7, step
        th, _ = OL.knot_theta(v.astype(np.float64), c.astype(np.float64), H)
        assert np.allclose(w[2 * H:3 * H + 1], th[2 * H:], rtol=1e-5, atol=1e-6), step


def test_gradient_descent_direction():
    """A small step against the library's gradient lowers the oracle's loss."""
    rng = np.random.default_rng(5)
    w = weights(rng)
    u = rng.random(50_000).astype(np.float32)
    t = np.sort(rng.random(50_000)).astype(np.float32)
    _, g = pb.mlp_grad(torch.from_numpy(u).cuda(), torch.from_numpy(t).cuda(), w)
    th, cap = split(w)
    l0 = OL.loss(th, u, t, H, cap)
    l1 = OL.loss(th - 1e-3 * g / np.linalg.norm(g), u, t, H, cap)
    assert l1 < l0


def skewed_fib():
    """150,000 prefixes spread over 2000::/3 plus 50,000 packed into one /24 (2a00:0100::/24): a key
    distribution whose CDF is far from linear, as dense regional allocations make real tables."""
    a = synth.gen_fib(150_000, seed=2604, nh_max=4095, default=False)
    b = synth.gen_fib(50_000, seed=2605, nh_max=4095, root_prefix_bits=24,
                      root_prefix_value=0x2A0001)
    return synth.Fib(np.concatenate([a.hi, b.hi]), np.concatenate([a.lo, b.lo]),
                     np.concatenate([a.len, b.len]), np.concatenate([a.nh, b.nh]), 0)


def test_trained_root_gains_over_untrained():
    """Same table, same leaf count: the untrained root is the identity (plain linear range
    reduction); training it on the GPU to the key CDF routes keys evenly over the leaves, so more
    keys land in leaves whose error window is within the limit and the mean window shrinks.
    Lookups are exact either way."""
    f = skewed_fib()
    xh, xl = synth.gen_trace(f, 2_000_000, seed=9)
    want = oracle.Trie(f.hi, f.lo, f.len, f.nh).lookup(xh, xl)
    stats = {}
    for iters in (0, 2000):
        with pb.Fib(f.hi, f.lo, f.len, f.nh, kernel="learned", model_iters=iters) as fib:
            st = fib.stats()
            stats[iters] = st
            out = fib.lookup(torch.from_numpy(xh.view(np.int64)).cuda(),
                             torch.from_numpy(xl.view(np.int64)).cuda())
            torch.cuda.synchronize()
            assert np.array_equal(out.cpu().numpy().view(np.uint16), want)
    a, b = stats[0], stats[2000]
    print("untrained", {k: a[k] for k in a if k.startswith("model")})
    print("trained", {k: b[k] for k in b if k.startswith("model")})
    assert b["model_iters"] >= 2000 and a["model_iters"] == 0
    assert b["model_loss"] < 0.1 * a["model_loss0"]
    assert b["model_covered"] > a["model_covered"]
    assert b["model_covered"] > 0.9
