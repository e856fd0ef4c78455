"""GPU parity: libplanb's lookup kernels against the CPU oracle, bit-exact, through the C ABI.

Expected next hops always come from ``oracle`` (O2 trie, cross-checked with O1 brute force on
samples); inputs come from ``synth``. Boundary probes are derived from the oracle-independent
product intervals only as *addresses* to look up, never as expected values.
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

M64 = (1 << 64) - 1


@pytest.fixture(scope="module", autouse=True)
def built():
    pb.build()


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a).view(np.int64)).cuda()


def gpu_lookup(fib, xh, xl, stream=None):
    out = fib.lookup(dev(xh), dev(xl), stream=stream)
    torch.cuda.synchronize()
    return out.cpu().numpy().view(np.uint16)


def expected(f, xh, xl):
    return oracle.Trie(f.hi, f.lo, f.len, f.nh).lookup(xh, xl)


def boundary_probes(f):
    """Every interval start, start - 1, start + 1, plus 0 and all-ones."""
    sh, sl, _ = pb.intervals(f.hi, f.lo, f.len, f.nh)
    s = [(int(h) << 64) | int(l) for h, l in zip(sh, sl)]
    vals = set()
    for v in s:
        for d in (-1, 0, 1):
            vals.add((v + d) % (1 << 128))
    vals |= {0, (1 << 128) - 1}
    vals = sorted(vals)
    return (np.array([v >> 64 for v in vals], np.uint64),
            np.array([v & M64 for v in vals], np.uint64))


FORMATS = ["f8x128", "f16hi"]
# (node format, kernel) pairs: every lookup kernel of the library
VARIANTS = [("f8v7", "hybrid"), ("f8v7", "learned"), ("f8x128", "hybrid"), ("f8x128", "learned"),
            ("f8x128", "coop"), ("f8x128", "flat"), ("f16hi", "coop"), ("f16hi", "hybrid")]
VIDS = [f"{f}-{k}" for f, k in VARIANTS]


def make(f, which, **kw):
    fmt, kernel = which
    return pb.Fib(f.hi, f.lo, f.len, f.nh, format=fmt, kernel=kernel, **kw)


@pytest.mark.parametrize("variant", VARIANTS, ids=VIDS)
@pytest.mark.parametrize("smem", [-1, 0, 1, 2, 3, 99])
def test_config_small_parity(variant, smem):
    """1,000 prefixes (+ ::/0), 10^6 addresses (70 % covered), every shared-memory depth."""
    f = synth.gen_fib(1000, seed=101, nh_max=255)
    xh, xl = synth.gen_trace(f, 1_000_000, seed=102)
    with make(f, variant, smem_levels=smem) as fib:
        got = gpu_lookup(fib, xh, xl)
        want = expected(f, xh, xl)
        assert np.array_equal(got, want)
        sub = slice(0, 20_000)
        assert np.array_equal(want[sub], oracle.brute_lookup(f.hi, f.lo, f.len, f.nh, xh[sub], xl[sub]))
        bh, bl = boundary_probes(f)
        assert np.array_equal(gpu_lookup(fib, bh, bl), expected(f, bh, bl))


@pytest.mark.parametrize("variant", VARIANTS, ids=VIDS)
@pytest.mark.parametrize("n", [0, 1, 5, 31, 32, 33, 1000, 123_457])
def test_ragged_batches_and_tables(variant, n):
    f = synth.gen_fib(max(n, 1) if n < 1000 else 3000, seed=200 + n, nh_max=4095)
    xh, xl = synth.gen_trace(f, n, seed=7)
    with make(f, variant) as fib:
        got = gpu_lookup(fib, xh, xl) if n else np.zeros(0, np.uint16)
        assert np.array_equal(got, expected(f, xh, xl))


@pytest.mark.parametrize("variant", VARIANTS, ids=VIDS)
def test_degenerate_tables(variant):
    probes_h = np.array([0, M64, 0x2001_0DB8 << 32, 0xFFFF << 48, 1], np.uint64)
    probes_l = np.array([0, M64, 0, 5, M64], np.uint64)
    tables = {
        "empty": ([], [], [], []),
        "default_only": ([0], [0], [0], [77]),
        "host_routes_at_ends": ([0, M64], [0, M64], [128, 128], [5, 6]),
        "top_of_space": ([0xFFFF << 48], [0], [16], [9]),
        "chain": ([0x2001_0DB8_1234_5678] * 129, [0x9ABC_DEF0_1234_5678] * 129, list(range(129)),
                  [L + 1 for L in range(129)]),
        "duplicates": ([0x2001_0DB8 << 32] * 3, [0, 1, 2], [32, 32, 32], [1, 2, 3]),
    }
    for name, (h, l, L, nh) in tables.items():
        f = synth.Fib(np.array(h, np.uint64), np.array(l, np.uint64), np.array(L, np.uint8),
                      np.array(nh, np.uint16), 0)
        with make(f, variant) as fib:
            bh, bl = boundary_probes(f)
            xh = np.concatenate([probes_h, bh])
            xl = np.concatenate([probes_l, bl])
            assert np.array_equal(gpu_lookup(fib, xh, xl), expected(f, xh, xl)), name


@pytest.mark.parametrize("variant", VARIANTS, ids=VIDS)
def test_merge_flag_keeps_results(variant):
    f = synth.gen_fib(20_000, seed=31, nh_max=3)   # few next hops: many equal neighbours
    xh, xl = synth.gen_trace(f, 300_000, seed=32)
    with make(f, variant, merge=True) as a, make(f, variant) as b:
        assert a.stats()["n_intervals"] < b.stats()["n_intervals"]
        want = expected(f, xh, xl)
        assert np.array_equal(gpu_lookup(a, xh, xl), want)
        assert np.array_equal(gpu_lookup(b, xh, xl), want)


def test_bounds_checked_build_reports_clean():
    f = synth.gen_fib(5000, seed=41, nh_max=4095)
    xh, xl = synth.gen_trace(f, 200_000, seed=42)
    for v in VARIANTS:
        with make(f, v, variant="libplanb_checked.so") as fib:
            assert np.array_equal(gpu_lookup(fib, xh, xl), expected(f, xh, xl))
            assert fib.device_status() == (0, 0)


def test_zipf_trace_parity():
    f = synth.gen_fib(20_000, seed=51, nh_max=4095)
    xh, xl = synth.gen_trace_zipf(f, 500_000, seed=52, hot=10_000)
    want = expected(f, xh, xl)
    for v in VARIANTS:
        with make(f, v) as fib:
            assert np.array_equal(gpu_lookup(fib, xh, xl), want), v


def test_lookup_host_matches_device_path():
    f = synth.gen_fib(5000, seed=61, nh_max=4095)
    n = (1 << 21) * 2 + 12345                 # more than two host-pipeline chunks, ragged
    xh, xl = synth.gen_trace(f, n, seed=62)
    with pb.Fib(f.hi, f.lo, f.len, f.nh) as fib:
        got = fib.lookup_host(xh, xl)
        assert np.array_equal(got, expected(f, xh, xl))
        pin_h = torch.from_numpy(xh.view(np.int64)).pin_memory()
        pin_l = torch.from_numpy(xl.view(np.int64)).pin_memory()
        out = torch.empty(n, dtype=torch.int16).pin_memory()
        fib.lookup_host(pin_h, pin_l, out=out)       # all pinned: the kernel reads host memory
        assert np.array_equal(out.numpy().view(np.uint16), got)
        mixed = np.zeros(n, np.uint16)               # pageable result buffer: the copy pipeline
        fib.lookup_host(pin_h, pin_l, out=mixed)
        assert np.array_equal(mixed, got)


def test_api_errors():
    f = synth.gen_fib(100, seed=71)
    with pytest.raises(pb.PlanbError):
        pb.Fib(f.hi, f.lo, np.full(f.n, 129, np.uint8), f.nh)
    with pb.Fib(f.hi, f.lo, f.len, f.nh) as fib:
        x = dev(np.zeros(8, np.uint64))
        with pytest.raises(pb.PlanbError):      # misaligned device pointer
            fib.lookup_ptr(x.data_ptr() + 4, x.data_ptr(), 1, x.data_ptr())
        fib.lookup_ptr(x.data_ptr(), x.data_ptr(), 0, x.data_ptr())   # n = 0 is a no-op


@pytest.fixture(scope="module")
def backbone():
    """200,000 prefixes (next hops in [1, 4095]) and 2^28 addresses: the benchmark's workload;
    the oracle's answer for all 2^28 addresses is computed once."""
    import os
    f = synth.gen_fib(200_000, seed=2604, nh_max=4095)
    n = 1 << 28
    xh, xl = synth.gen_trace(f, n, seed=2605)
    want = oracle.Trie(f.hi, f.lo, f.len, f.nh).lookup(xh, xl, threads=os.cpu_count())
    return f, xh, xl, want


@pytest.mark.parametrize("variant", VARIANTS, ids=VIDS)
def test_backbone_full_size_parity(backbone, variant):
    """Every one of the 2^28 next hops equals the oracle's, in the launch configuration the
    benchmark times (default grid, block and shared-memory depth)."""
    f, xh, xl, want = backbone
    with make(f, variant) as fib:
        dh, dl = dev(xh), dev(xl)
        out = fib.lookup(dh, dl)
        torch.cuda.synchronize()
        got = out.cpu().numpy().view(np.uint16)
        del dh, dl, out
    bad = np.count_nonzero(got != want)
    assert bad == 0, f"{bad} of {want.size} differ"


@pytest.mark.parametrize("variant", VARIANTS, ids=VIDS)
def test_shared_high_halves(variant):
    """Many boundaries that differ only in their low 64 bits (clusters of /128 and /65../127 routes
    inside single /64s): exercises every high-half tie path of the kernels."""
    f = synth.gen_fib(20_000, seed=301, nh_max=4095)
    rng = np.random.default_rng(302)
    base = rng.choice(np.nonzero(f.len == 48)[0], 400, replace=False)
    eh, el, eL, en = [], [], [], []
    for i, b in enumerate(base):
        h = np.uint64(f.hi[b] | np.uint64(i))                 # a /64 inside the /48
        for k in range(6):
            eh.append(h)
            el.append(np.uint64(rng.integers(0, 2 ** 63)) * np.uint64(2))
            eL.append(128 if k < 4 else int(rng.integers(65, 128)))
            en.append(int(rng.integers(1, 4096)))
    g = synth.Fib(np.concatenate([f.hi, np.array(eh, np.uint64)]),
                  np.concatenate([f.lo, np.array(el, np.uint64)]),
                  np.concatenate([f.len, np.array(eL, np.uint8)]),
                  np.concatenate([f.nh, np.array(en, np.uint16)]), 0)
    bh, bl = boundary_probes(g)
    xh, xl = synth.gen_trace(g, 200_000, seed=303)
    xh = np.concatenate([bh, xh, np.array(eh, np.uint64)])
    xl = np.concatenate([bl, xl, np.array(el, np.uint64)])
    with make(g, variant) as fib:
        assert np.array_equal(gpu_lookup(fib, xh, xl), expected(g, xh, xl))


def test_tables_sharing_a_kernel_with_different_shared_memory():
    """Two live tables that use the same kernel instantiation but need different amounts of shared
    memory (the whole key index of each sits in shared memory), the larger built first: lookups on
    both stay correct (the kernel's shared-memory limit must not follow the last table built)."""
    big = synth.gen_fib(5000, seed=401, nh_max=4095)
    small = synth.gen_fib(1500, seed=402, nh_max=4095)
    with pb.Fib(big.hi, big.lo, big.len, big.nh) as fb, \
            pb.Fib(small.hi, small.lo, small.len, small.nh) as fs:
        assert fb.stats()["smem_levels"] == fb.stats()["depth"]       # index holds every key
        assert fb.stats()["smem_bytes"] > 48 * 1024 > fs.stats()["smem_bytes"]
        for f, fib in ((big, fb), (small, fs)):
            xh, xl = synth.gen_trace(f, 100_000, seed=403)
            assert np.array_equal(gpu_lookup(fib, xh, xl), expected(f, xh, xl))


@pytest.mark.parametrize("kernel", ["coop", "hybrid"])
@pytest.mark.parametrize("builder", ["host", "device"])
def test_f16hi_next_hop_words(kernel, builder):
    """The F16HI next-hop words at the end of the table image: the next hop of interval i, plus
    bit 16 exactly when interval i + 1 starts at a nonzero low half (interval i's key then has a
    low half other than all-ones), from the intervals the host builder reports."""
    f = synth.gen_fib(30_000, seed=921, nh_max=65535)
    sh, sl, snh = pb.intervals(f.hi, f.lo, f.len, f.nh)
    m = sh.size
    want = snh.astype(np.uint32)
    want[:-1] |= (sl[1:] != 0).astype(np.uint32) << 16
    assert 0 < np.count_nonzero(want >> 16) < m // 4      # the /128s (and nothing else) flag
    with pb.Fib(f.hi, f.lo, f.len, f.nh, format="f16hi", kernel=kernel, builder=builder) as fib:
        assert fib.stats()["value_bytes"] == 4 * m
        img = fib.table_dump()
        assert np.array_equal(img[-4 * m:].view(np.uint32), want)


def test_f16hi_without_long_prefixes_sets_no_flag():
    """With no prefix longer than /64 every boundary has an all-ones low half below it, no
    next-hop word carries the flag, and the high-half-only lookup (the paper's 64-bit key scheme)
    is the whole lookup: still equal to the oracle, at every boundary and its neighbours."""
    f = synth.gen_fib(30_000, seed=941, nh_max=4095)
    keep = f.len <= 64
    g = synth.Fib(f.hi[keep], f.lo[keep], f.len[keep], f.nh[keep], 0)
    m = pb.intervals(g.hi, g.lo, g.len, g.nh)[0].size
    bh, bl = boundary_probes(g)
    xh, xl = synth.gen_trace(g, 200_000, seed=942)
    xh, xl = np.concatenate([bh, xh]), np.concatenate([bl, xl])
    for kernel in ("hybrid", "coop"):
        with pb.Fib(g.hi, g.lo, g.len, g.nh, format="f16hi", kernel=kernel) as fib:
            assert not np.any(fib.table_dump()[-4 * m:].view(np.uint32) >> 16)
            assert np.array_equal(gpu_lookup(fib, xh, xl), expected(g, xh, xl))


@pytest.mark.parametrize("variant", VARIANTS, ids=VIDS)
def test_long_runs_of_shared_high_halves(variant):
    """One /64 holding 3,000 /128 routes and nested /80../127 prefixes (thousands of keys with one
    high half, spanning many leaves and index entries): the F16HI count over them is settled by
    doubling and halving steps; every kernel agrees with the oracle on each route's address, its
    neighbours and random addresses of the /64."""
    f = synth.gen_fib(20_000, seed=931, nh_max=4095)
    rng = np.random.default_rng(932)
    h64 = np.uint64(f.hi[np.nonzero(f.len == 48)[0][0]] | np.uint64(0x1234))
    lo128 = np.unique(rng.integers(0, 2 ** 63, size=3000, dtype=np.uint64) * np.uint64(2))
    nest_len = rng.integers(80, 128, size=300)
    nest_lo = rng.integers(0, 2 ** 63, size=300, dtype=np.uint64) * np.uint64(2)
    eh = np.full(lo128.size + 300 + 1, h64, np.uint64)
    el = np.concatenate([lo128, nest_lo, np.zeros(1, np.uint64)])
    eL = np.concatenate([np.full(lo128.size, 128), nest_len, [64]]).astype(np.uint8)
    en = rng.integers(1, 4096, size=eh.size).astype(np.uint16)
    g = synth.Fib(np.concatenate([f.hi, eh]), np.concatenate([f.lo, el]),
                  np.concatenate([f.len, eL]), np.concatenate([f.nh, en]), 0)
    xl = np.concatenate([lo128, lo128 - np.uint64(1), lo128 + np.uint64(1),
                         rng.integers(0, 2 ** 63, size=20_000, dtype=np.uint64) * np.uint64(2),
                         np.array([0, M64], np.uint64)])
    xh = np.full(xl.size, h64, np.uint64)
    bh, bl = boundary_probes(g)
    xh = np.concatenate([xh, bh])
    xl = np.concatenate([xl, bl])
    with make(g, variant) as fib:
        assert np.array_equal(gpu_lookup(fib, xh, xl), expected(g, xh, xl))


@pytest.mark.parametrize("fmt", ["f8x128", "f8v7", "f16hi"])
def test_mapped_lookup_formats_and_ties(fmt):
    """The low half is read only on a tie of high halves: addresses inside /64 and longer prefixes
    (and the 30 % uniform ones) exercise both the tie path and the plain path."""
    f = synth.gen_fib(40_000, seed=911, nh_max=4095)
    xh, xl = synth.gen_trace(f, 700_001, seed=912)
    want = oracle.Trie(f.hi, f.lo, f.len, f.nh).lookup(xh, xl)
    with pb.Fib(f.hi, f.lo, f.len, f.nh, format=fmt) as fib:
        ph = torch.from_numpy(xh.view(np.int64)).pin_memory()
        pl = torch.from_numpy(xl.view(np.int64)).pin_memory()
        po = torch.full((xh.size,), -1, dtype=torch.int16).pin_memory()
        s = torch.cuda.Stream()
        fib.lookup_mapped(ph, pl, po, s)
        s.synchronize()
        assert np.array_equal(po.numpy().view(np.uint16), want)


def test_mapped_lookup_on_pinned_host_buffers():
    """planb_lookup_mapped: the kernel reads pinned host addresses and writes pinned host results
    directly; unpinned buffers are refused before anything is launched."""
    import ctypes
    f = synth.gen_fib(30_000, seed=901, nh_max=4095)
    xh, xl = synth.gen_trace(f, 1_000_003, seed=902)
    want = oracle.Trie(f.hi, f.lo, f.len, f.nh).lookup(xh, xl)
    with pb.Fib(f.hi, f.lo, f.len, f.nh) as fib:
        ph = torch.from_numpy(xh.view(np.int64)).pin_memory()
        pl = torch.from_numpy(xl.view(np.int64)).pin_memory()
        po = torch.full((xh.size,), -1, dtype=torch.int16).pin_memory()
        s = torch.cuda.Stream()
        fib.lookup_mapped(ph, pl, po, s)
        s.synchronize()
        assert np.array_equal(po.numpy().view(np.uint16), want)
        # a slice at an offset inside the pinned buffers
        k0, k1 = 12_345, 600_001
        po2 = torch.full((k1 - k0,), -1, dtype=torch.int16).pin_memory()
        fib.lookup_mapped(ph[k0:k1], pl[k0:k1], po2, s)
        s.synchronize()
        assert np.array_equal(po2.numpy().view(np.uint16), want[k0:k1])
        # pageable memory: refused by the library itself
        hh, hl = np.ascontiguousarray(xh[:1000]), np.ascontiguousarray(xl[:1000])
        out = np.zeros(1000, np.uint16)
        rc = fib._lib.planb_lookup_mapped(fib._h, ctypes.c_void_p(hh.ctypes.data),
                                          ctypes.c_void_p(hl.ctypes.data), 1000,
                                          ctypes.c_void_p(out.ctypes.data), None)
        assert rc == -1   # PLANB_EINVAL
        assert np.all(out == 0)


@pytest.mark.parametrize("fmt", ["f8x128", "f16hi"])
def test_small_and_large_launches_agree(fmt):
    """Launches with under two 32-address tiles per warp search the index in global memory, larger
    ones stage it in shared memory; both give the oracle's answers, at sizes on both sides."""
    f = synth.gen_fib(200_000, seed=921, nh_max=4095)
    xh, xl = synth.gen_trace(f, 3_000_000, seed=922)
    want = oracle.Trie(f.hi, f.lo, f.len, f.nh).lookup(xh, xl)
    with pb.Fib(f.hi, f.lo, f.len, f.nh, format=fmt, kernel="hybrid") as fib:
        dh, dl = dev(xh), dev(xl)
        for k in (1, 31, 4096, 65_536, 300_000, 3_000_000):
            out = fib.lookup(dh[:k], dl[:k])
            torch.cuda.synchronize()
            assert np.array_equal(out.cpu().numpy().view(np.uint16), want[:k]), k


@pytest.mark.parametrize("spread", [False, True], ids=["dense", "sparse_wide"])
def test_f16hi_index_clusters_in_one_bucket(spread):
    """A cluster of 100 /64 routes whose high halves differ only in their low 8 bits (with /128
    routes inside some of them) puts many index entries into one radix-directory bucket, in a
    dense table and in a small table spread over the whole space (buckets tens of bits wide);
    every boundary, its neighbours and random addresses of the cluster are looked up in a launch
    large enough to stage the index in shared memory."""
    rng = np.random.default_rng(951)
    H = np.uint64(0x2001_0DB8_0000_0000)                      # 256-aligned high half
    ch = H + np.arange(100, dtype=np.uint64) * np.uint64(2)
    cl = np.zeros(100, np.uint64)
    cL = np.full(100, 64, np.uint8)
    # /128 routes inside a few of the /64s (flagged keys sharing the address's high half)
    hh = ch[::10]
    hl = rng.integers(1, 2 ** 63, size=hh.size, dtype=np.uint64)
    if spread:
        far = synth.gen_fib(12, seed=952, nh_max=4095, default=False)
    else:
        far = synth.gen_fib(20_000, seed=953, nh_max=4095, default=False)
    z64 = np.zeros(1, np.uint64)
    hi = np.concatenate([far.hi, ch, hh, z64])
    lo = np.concatenate([far.lo, cl, hl, z64])
    ln = np.concatenate([far.len, cL, np.full(hh.size, 128, np.uint8), np.zeros(1, np.uint8)])
    nh = rng.integers(1, 4096, size=hi.size).astype(np.uint16)
    g = synth.Fib(hi, lo, ln, nh, 0)
    bh, bl = boundary_probes(g)
    k = 400_000                                               # large enough to stage the index
    ih = H + rng.integers(0, 256, size=k // 2, dtype=np.uint64)
    il = rng.integers(0, 2 ** 63, size=k // 2, dtype=np.uint64) * np.uint64(2)
    th, tl = synth.gen_trace(g, k // 2, seed=954)
    xh = np.concatenate([bh, ih, th])
    xl = np.concatenate([bl, il, tl])
    with pb.Fib(g.hi, g.lo, g.len, g.nh, format="f16hi", kernel="hybrid") as fib:
        assert fib.stats()["smem_levels"] >= 1
        assert np.array_equal(gpu_lookup(fib, xh, xl), expected(g, xh, xl))
