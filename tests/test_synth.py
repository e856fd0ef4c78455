"""The seeded generator produces the stated workload shape, deterministically."""
import numpy as np

import synth


def test_length_mix_and_default_route():
    fib = synth.gen_fib(20_000, seed=1, nh_max=4095)
    assert fib.n == 20_001 and fib.len[-1] == 0 and fib.nh[-1] == 0
    L = fib.len[:-1].astype(int)
    for length, share in synth.LENGTH_MIX:
        extra = 0.14 / 49 if 16 <= length <= 64 else 0.0
        assert abs(np.mean(L == length) - (share + extra)) < 0.015, length
    assert L.min() >= 16 and set(np.unique(L)) <= set(range(16, 65)) | {128}
    assert fib.nh[:-1].min() >= 1 and fib.nh[:-1].max() <= 4095
    keys = set(zip(fib.hi.tolist(), fib.lo.tolist(), fib.len.tolist()))
    assert len(keys) == fib.n                                  # distinct (prefix, length)
    mh, ml = synth.top_mask(fib.len)
    assert np.all(fib.hi & ~mh == 0) and np.all(fib.lo & ~ml == 0)   # canonical


def test_nesting_share():
    fib = synth.gen_fib(3000, seed=2)
    hi, lo, L = fib.hi[:-1], fib.lo[:-1], fib.len[:-1].astype(int)
    nested = 0
    for i in range(L.size):
        mh, ml = synth.top_mask(L)                               # masks of every candidate parent
        inside = (L < L[i]) & ((hi[i] & mh) == hi) & ((lo[i] & ml) == lo)
        nested += bool(inside.any())
    assert 0.25 < nested / L.size < 0.40


def test_trace_deterministic_under_chunking():
    fib = synth.gen_fib(500, seed=3)
    a = synth.gen_trace(fib, 100_000, seed=9, threads=1, chunk=1 << 20)
    b = synth.gen_trace(fib, 100_000, seed=9, threads=4, chunk=7_777)
    c = synth.gen_trace(fib, 50_000, seed=9, start=50_000)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    assert np.array_equal(a[0][50_000:], c[0]) and np.array_equal(a[1][50_000:], c[1])


def test_zipf_trace_is_skewed():
    fib = synth.gen_fib(2000, seed=4)
    h, _ = synth.gen_trace_zipf(fib, 200_000, seed=5, hot=10_000)
    _, counts = np.unique(h, return_counts=True)
    counts = np.sort(counts)[::-1]
    assert counts[0] > 20 * np.median(counts)
