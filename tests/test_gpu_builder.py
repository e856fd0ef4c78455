"""GPU tests of the device builder (build steps a1-a4 on the GPU: radix sorts, the bracket-matching
scan that replaces Algorithm 2's stack, closed-form layout fill).

* Its intervals satisfy the oracle's interval invariants and equal the host builder's, on seeded
  FIBs and on the degenerate tables (empty, ::/0 alone, /128 at both ends of the space, duplicates,
  prefixes nested on one start or one end, host bits set).
* A table it builds is the host builder's table byte for byte (node arrays, index, next hops) in
  every format, and its lookups equal the oracle's.
* Rebuilds by planb_update with the device builder match the host builder after the same batches.
"""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2604_14650_gb300 as pb  # noqa: E402

U = np.uint64


@pytest.fixture(scope="module", autouse=True)
def built():
    pb.build()


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a).view(np.int64)).cuda()


def arrays(h, l, L, n):
    return (np.array(h, U), np.array(l, U), np.array(L, np.uint8), np.array(n, np.uint16))


EDGE = {
    "empty": arrays([], [], [], []),
    "default_only": arrays([0], [0], [0], [7]),
    "top_128": arrays([0xFFFFFFFFFFFFFFFF], [0xFFFFFFFFFFFFFFFF], [128], [3]),
    "zero_128": arrays([0], [0], [128], [3]),
    "default_and_128s": arrays([0, 0, 0xFFFFFFFFFFFFFFFF], [0, 0, 0xFFFFFFFFFFFFFFFF], [0, 128, 128],
                               [1, 2, 3]),
    "duplicates_last_wins": arrays([0x20010DB800000000] * 3, [0] * 3, [32] * 3, [1, 2, 3]),
    "nested_same_start": arrays([0x2001 << 48] * 3, [0] * 3, [16, 32, 48], [1, 2, 3]),
    "nested_same_end": arrays([0x2001FFFF00000000, 0x2001FFFFFFFF0000, 0x2001 << 48], [0] * 3,
                              [32, 48, 16], [1, 2, 3]),
    "top_half_chain": arrays([1 << 63, 3 << 62, 7 << 61], [0] * 3, [1, 2, 3], [5, 6, 5]),
    "host_bits_set": arrays([0x2001FFFFFFFFFFFF], [0xFFFF], [16], [9]),
    "long_prefixes": arrays([0x2001 << 48] * 4, [0, 1 << 63, 0xFFFF, 0xFFFFFFFFFFFFFFFF],
                            [64, 65, 112, 128], [1, 2, 3, 4]),
}


def random_nested(seed, n=3000):
    r = np.random.default_rng(seed)
    hi = r.integers(0, 2**63, size=n, dtype=U) * U(2)
    lo = r.integers(0, 2**63, size=n, dtype=U)
    idx = r.integers(0, n, size=n // 2)
    hi[: n // 2] = hi[idx]
    lo[: n // 2] = lo[idx]
    L = r.integers(0, 129, size=n).astype(np.uint8)
    nh = r.integers(0, 6, size=n).astype(np.uint16)
    return hi, lo, L, nh


def cases():
    out = dict(EDGE)
    for s in range(3):
        f = synth.gen_fib(20_000, seed=300 + s, nh_max=4095)
        out[f"fib{s}"] = (f.hi, f.lo, f.len, f.nh)
        out[f"nested{s}"] = random_nested(310 + s)
    return out


CASES = cases()


@pytest.mark.parametrize("name", sorted(CASES))
@pytest.mark.parametrize("merge", [False, True])
def test_device_intervals_equal_host_and_pass_oracle_checks(name, merge):
    h, l, L, n = CASES[name]
    d = pb.intervals(h, l, L, n, merge, device=True)
    c = pb.intervals(h, l, L, n, merge)
    assert oracle.check_intervals(h, l, L, n, *d, merged=merge) is None
    for x, y in zip(d, c):
        assert np.array_equal(x, y)


VARIANTS = [("f8x128", "hybrid"), ("f8x128", "coop"), ("f8x128", "flat"), ("f8v7", "hybrid"),
            ("f16hi", "coop"), ("f16hi", "hybrid")]


@pytest.mark.parametrize("fmt,kernel", VARIANTS)
@pytest.mark.parametrize("n_prefixes", [0, 1, 700, 60_000])
def test_device_built_table_is_the_host_table(fmt, kernel, n_prefixes):
    if n_prefixes:
        f = synth.gen_fib(n_prefixes, seed=320 + n_prefixes, nh_max=4095)
        h, l, L, n = f.hi, f.lo, f.len, f.nh
    else:
        h, l, L, n = EDGE["empty"]
    kw = dict(format=fmt, kernel=kernel)
    with pb.Fib(h, l, L, n, builder="host", **kw) as a, pb.Fib(h, l, L, n, builder="device",
                                                                 **kw) as b:
        sa, sb = a.stats(), b.stats()
        assert sa["builder"] == 0 and sb["builder"] == 1
        for k in ("n_prefixes", "n_intervals", "depth", "smem_levels", "leaf_nodes", "kernel"):
            assert sa[k] == sb[k], k
        assert np.array_equal(a.table_dump(), b.table_dump())
        if n_prefixes == 0:
            xh = np.array([0, 0xFFFFFFFFFFFFFFFF], U)
            xl = np.array([0, 0xFFFFFFFFFFFFFFFF], U)
            want = np.zeros(2, np.uint16)
        else:
            xh, xl = synth.gen_trace(synth.Fib(h, l, L, n, 0), 200_000, seed=321)
            want = oracle.Trie(h, l, L, n).lookup(xh, xl)
        out = b.lookup(dev(xh), dev(xl))
        torch.cuda.synchronize()
        assert np.array_equal(out.cpu().numpy().view(np.uint16), want)


@pytest.mark.parametrize("name", ["default_and_128s", "nested_same_end", "long_prefixes",
                                  "top_half_chain"])
def test_device_built_edge_tables(name):
    h, l, L, n = EDGE[name]
    with pb.Fib(h, l, L, n, builder="host") as a, pb.Fib(h, l, L, n, builder="device") as b:
        assert np.array_equal(a.table_dump(), b.table_dump())


def test_device_builder_merge_equal_next_hops():
    f = synth.gen_fib(30_000, seed=330, nh_max=3)   # few next hops: many merges
    with pb.Fib(f.hi, f.lo, f.len, f.nh, merge=True, builder="host") as a, \
            pb.Fib(f.hi, f.lo, f.len, f.nh, merge=True, builder="device") as b:
        assert b.stats()["n_intervals"] < pb.intervals(f.hi, f.lo, f.len, f.nh)[0].size
        assert np.array_equal(a.table_dump(), b.table_dump())


def test_device_builder_learned_kernel_matches_oracle():
    f = synth.gen_fib(40_000, seed=340, nh_max=4095)
    xh, xl = synth.gen_trace(f, 300_000, seed=341)
    with pb.Fib(f.hi, f.lo, f.len, f.nh, kernel="learned", builder="device") as b:
        out = b.lookup(dev(xh), dev(xl))
        torch.cuda.synchronize()
        assert np.array_equal(out.cpu().numpy().view(np.uint16),
                              oracle.Trie(f.hi, f.lo, f.len, f.nh).lookup(xh, xl))


@pytest.mark.parametrize("fmt", ["f8x128", "f8v7"])
def test_device_builder_updates_track_host_builder(fmt):
    f = synth.gen_fib(20_000, seed=350, nh_max=4095)
    with pb.Fib(f.hi, f.lo, f.len, f.nh, format=fmt, builder="host") as a, \
            pb.Fib(f.hi, f.lo, f.len, f.nh, format=fmt, builder="device") as b:
        for batch in range(4):
            upd = synth.gen_updates(f, 700 * (batch + 1), seed=351, start=batch * 10_000)
            a.update(*upd)
            b.update(*upd)
            sa, sb = a.stats(), b.stats()
            assert sa["version"] == sb["version"] == batch + 2
            assert sa["withdraw_absent"] == sb["withdraw_absent"]
            assert sb["builder"] == 1
            assert np.array_equal(a.table_dump(), b.table_dump())


def test_device_builder_million_prefixes():
    f = synth.gen_fib(1_000_000, seed=360)
    with pb.Fib(f.hi, f.lo, f.len, f.nh, builder="host") as a, \
            pb.Fib(f.hi, f.lo, f.len, f.nh, builder="device") as b:
        assert np.array_equal(a.table_dump(), b.table_dump())
