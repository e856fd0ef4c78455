"""Multi-table (VRF) lookups: each address carries a u8 table id. When every table is an F16HI
hybrid table, one persistent launch looks the batch up in input order (the direct form); else one
captured graph buckets the batch by table, looks every group up — in one persistent launch when
every table uses the hybrid kernel, else one launch per table — and gathers results back into
input order. Checked bit-exactly against the oracle of each table, in every form, captured and
launched directly."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2604_14650_gb300 as pb  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def built():
    pb.build()


def dev(a, dtype=np.int64):
    return torch.from_numpy(np.ascontiguousarray(a).view(dtype)).cuda()


def workload(sizes, n, seed, invalid=0.01):
    fibs = [synth.gen_fib(s, seed=seed + t, nh_max=4095) for t, s in enumerate(sizes)]
    rng = np.random.default_rng(seed)
    p = np.array(sizes, float) / sum(sizes)
    tid = rng.choice(len(sizes), size=n, p=p).astype(np.uint8)
    bad = rng.random(n) < invalid
    tid[bad] = rng.integers(len(sizes), 256, size=int(bad.sum()), dtype=np.uint8)
    xh = np.empty(n, np.uint64)
    xl = np.empty(n, np.uint64)
    for t, f in enumerate(fibs):
        idx = np.nonzero(tid == t)[0]
        h, l = synth.gen_trace(f, idx.size, seed=seed + 100 + t)
        xh[idx], xl[idx] = h, l
    idx = np.nonzero(tid >= len(sizes))[0]
    xh[idx] = rng.integers(0, 2 ** 63, idx.size, dtype=np.uint64)
    xl[idx] = rng.integers(0, 2 ** 63, idx.size, dtype=np.uint64)
    return fibs, tid, xh, xl


def expected(fibs, tid, xh, xl):
    want = np.zeros(tid.size, np.uint16)
    for t, f in enumerate(fibs):
        idx = np.nonzero(tid == t)[0]
        want[idx] = oracle.Trie(f.hi, f.lo, f.len, f.nh).lookup(xh[idx], xl[idx])
    return want


@pytest.mark.parametrize("per_table", [False, True])
@pytest.mark.parametrize("graph", [False, True])
@pytest.mark.parametrize("kinds", [("f8x128", "hybrid"), ("f8v7", "hybrid"), ("f16hi", "hybrid"),
                                   ("mixed_hybrid", None), ("mixed", None)])
def test_multi_table_parity_and_replay(kinds, graph, per_table):
    sizes = [500, 3000, 20_000, 1000, 60_000, 7, 12_000, 2500]
    fibs_in, tid, xh, xl = workload(sizes, 600_000, seed=41)
    want = expected(fibs_in, tid, xh, xl)
    choices = [("f8x128", "hybrid"), ("f8v7", "hybrid"), ("f16hi", "hybrid"), ("f8x128", "coop"),
               ("f8x128", "flat"), ("f16hi", "coop")]
    fibs = []
    for t, f in enumerate(fibs_in):
        if kinds[0] == "mixed":
            fmt, ker = choices[t % len(choices)]
        elif kinds[0] == "mixed_hybrid":          # every hybrid format, several index depths
            fmt, ker = choices[t % 3]
        else:
            fmt, ker = kinds
        smem = {2: 0, 5: 1}.get(t, -1) if kinds[0] == "mixed_hybrid" else -1
        fibs.append(pb.Fib(f.hi, f.lo, f.len, f.nh, format=fmt, kernel=ker, smem_levels=smem))
    with pb.MultiFib(fibs, max_batch=1 << 20, graph=graph, per_table=per_table) as mt:
        dh, dl, dt = dev(xh), dev(xl), dev(tid, np.uint8)
        out = torch.empty(tid.size, dtype=torch.int16, device="cuda")
        for _ in range(3):                     # first call captures the graph, the others replay
            out.fill_(-1)
            mt.lookup(dh, dl, dt, out=out)
            torch.cuda.synchronize()
            assert np.array_equal(out.cpu().numpy().view(np.uint16), want)
        # every table on the hybrid kernel shares the single persistent launch unless asked not to
        assert mt.persistent == (kinds[0] != "mixed" and not per_table)
        # a smaller batch (new capture) and an empty one
        k = 12_345
        small = mt.lookup(dh[:k], dl[:k], dt[:k])
        torch.cuda.synchronize()
        assert np.array_equal(small.cpu().numpy().view(np.uint16), want[:k])
        mt.lookup(dh[:0], dl[:0], dt[:0])
    for f in fibs:
        f.close()


@pytest.mark.parametrize("fmt", ["f8x128", "f16hi"])
@pytest.mark.parametrize("per_table", [False, True])
def test_multi_table_sees_updates(per_table, fmt):
    sizes = [5000, 20_000, 800]
    fibs_in, tid, xh, xl = workload(sizes, 300_000, seed=51)
    fibs = [pb.Fib(f.hi, f.lo, f.len, f.nh, format=fmt) for f in fibs_in]
    with pb.MultiFib(fibs, max_batch=300_000, per_table=per_table) as mt:
        dh, dl, dt = dev(xh), dev(xl), dev(tid, np.uint8)
        out = mt.lookup(dh, dl, dt)
        torch.cuda.synchronize()
        assert np.array_equal(out.cpu().numpy().view(np.uint16), expected(fibs_in, tid, xh, xl))
        # withdraw every prefix of table 1 except the default: its addresses then all get 0
        before = mt.captures
        f1 = fibs_in[1]
        keep = f1.len == 0
        fibs[1].update(wd_hi=f1.hi[~keep], wd_lo=f1.lo[~keep], wd_len=f1.len[~keep])
        fibs_in[1] = synth.Fib(f1.hi[keep], f1.lo[keep], f1.len[keep], f1.nh[keep], 0)
        out = mt.lookup(dh, dl, dt, out=out)
        torch.cuda.synchronize()
        got = out.cpu().numpy().view(np.uint16)
        assert np.array_equal(got, expected(fibs_in, tid, xh, xl))
        assert np.all(got[tid == 1] == 0)
        # a swapped table reaches the single persistent launch through its descriptors (no new
        # capture while the launch keeps its shape); per-table launches are captured again
        if not per_table:
            assert mt.captures == before
        else:
            assert mt.captures == before + 1
        # and again: a second update of another table, replayed
        f0 = fibs_in[0]
        upd = synth.gen_updates(f0, 500, seed=52)
        fibs[0].update(*upd)
        ref = {}
        for h, l, L, n_ in zip(f0.hi, f0.lo, f0.len, f0.nh):
            mh, ml = synth.top_mask(np.array([L]))
            ref[(int(h & mh[0]), int(l & ml[0]), int(L))] = int(n_)
        ih, il, iL, inh, wh, wl, wL = upd
        for h, l, L in zip(wh, wl, wL):
            mh, ml = synth.top_mask(np.array([L]))
            ref.pop((int(h & mh[0]), int(l & ml[0]), int(L)), None)
        for h, l, L, n_ in zip(ih, il, iL, inh):
            mh, ml = synth.top_mask(np.array([L]))
            ref[(int(h & mh[0]), int(l & ml[0]), int(L))] = int(n_)
        ks = list(ref)
        fibs_in[0] = synth.Fib(np.array([k[0] for k in ks], np.uint64),
                               np.array([k[1] for k in ks], np.uint64),
                               np.array([k[2] for k in ks], np.uint8),
                               np.array([ref[k] for k in ks], np.uint16), 0)
        out = mt.lookup(dh, dl, dt, out=out)
        torch.cuda.synchronize()
        assert np.array_equal(out.cpu().numpy().view(np.uint16), expected(fibs_in, tid, xh, xl))
    for f in fibs:
        f.close()


@pytest.mark.parametrize("fmt,kernel", [("f8x128", "learned"), ("f8v7", "learned")])
def test_tables_without_a_multi_form_cannot_join(fmt, kernel):
    f = synth.gen_fib(2000, seed=3)
    with pb.Fib(f.hi, f.lo, f.len, f.nh, format=fmt, kernel=kernel) as fib:
        with pytest.raises(pb.PlanbError):
            pb.MultiFib([fib], max_batch=1000)


@pytest.mark.parametrize("fmt", ["f8x128", "f16hi"])
@pytest.mark.parametrize("n", [1, 31, 33, 1000])
def test_multi_table_tiny_batches(n, fmt):
    """Batches smaller than the persistent grid: most CTAs get no addresses."""
    sizes = [3000, 40_000, 100]
    fibs_in, tid, xh, xl = workload(sizes, n, seed=61)
    fibs = [pb.Fib(f.hi, f.lo, f.len, f.nh, format=fmt) for f in fibs_in]
    with pb.MultiFib(fibs, max_batch=4096) as mt:
        out = mt.lookup(dev(xh), dev(xl), dev(tid, np.uint8))
        torch.cuda.synchronize()
        assert mt.persistent
        assert np.array_equal(out.cpu().numpy().view(np.uint16), expected(fibs_in, tid, xh, xl))
    for f in fibs:
        f.close()


def test_autotuned_group_is_exact_and_persistent(tmp_path):
    from paper_2604_14650_gb300.autotune import Autotuner
    sizes = [2000, 30_000, 9000]
    fibs_in, tid, xh, xl = workload(sizes, 200_000, seed=71)
    tuner = Autotuner(cache_path=str(tmp_path / "tune.json"), warmup=1, reps=2, persistent=True)
    fibs = []
    for t, f in enumerate(fibs_in):
        sel = tid == t
        opts = tuner.best(f.hi, f.lo, f.len, f.nh, dev(xh[sel]), dev(xl[sel]))
        assert opts["kernel"] == "hybrid" and opts["format"] in ("f8x128", "f8v7", "f16hi")
        fibs.append(pb.Fib(f.hi, f.lo, f.len, f.nh, **opts))
    # a second tuner on the same cache answers from it
    again = Autotuner(cache_path=str(tmp_path / "tune.json"), persistent=True)
    assert again.best(fibs_in[1].hi, fibs_in[1].lo, fibs_in[1].len, fibs_in[1].nh, None, None) == \
        tuner.best(fibs_in[1].hi, fibs_in[1].lo, fibs_in[1].len, fibs_in[1].nh, None, None)
    with pb.MultiFib(fibs, max_batch=200_000) as mt:
        out = mt.lookup(dev(xh), dev(xl), dev(tid, np.uint8))
        torch.cuda.synchronize()
        assert mt.persistent
        assert np.array_equal(out.cpu().numpy().view(np.uint16), expected(fibs_in, tid, xh, xl))
    for f in fibs:
        f.close()


def test_large_index_is_searched_in_place():
    """An F16HI table built for the single-table kernel (index over its leaves, about 160 KB of
    shared memory) joins the single persistent launch beside small tables: its index is searched in
    place in global memory rather than staged, and every result stays exact."""
    sizes = [160_000, 2000, 30_000]
    fibs_in, tid, xh, xl = workload(sizes, 400_000, seed=81)
    fibs = [pb.Fib(f.hi, f.lo, f.len, f.nh, format="f16hi") for f in fibs_in]
    assert fibs[0].stats()["smem_bytes"] > 96 * 1024 > fibs[1].stats()["smem_bytes"]
    with pb.MultiFib(fibs, max_batch=400_000, bucketed=True) as mt:
        out = mt.lookup(dev(xh), dev(xl), dev(tid, np.uint8))
        torch.cuda.synchronize()
        assert mt.persistent and mt.mode == "bucketed"
        assert np.array_equal(out.cpu().numpy().view(np.uint16), expected(fibs_in, tid, xh, xl))
    for f in fibs:
        f.close()


@pytest.mark.parametrize("graph", [False, True])
def test_direct_form_matches_oracle_and_bucketed(graph):
    """The direct form over F16HI tables of every shape it meets: a table of the default route
    alone (no index), tiny tables whose index holds every key (nothing below it), tables whose
    top-of-tree index sits right above the leaves, and tables whose index sits two or more levels
    higher (forced by smem_levels), which the direct form searches through their extra leaf-level
    index. Ids beyond the tables give 0; batch sizes that end mid-warp; the bucketed form of the
    same group gives the same results."""
    sizes = [1, 7, 500, 3000, 20_000, 60_000, 160_000, 12_000, 2500]
    smem = {4: 0, 5: 1, 7: 2}          # index levels forced shallow: leaf index built
    fibs_in, tid, xh, xl = workload(sizes, 700_001, seed=91)
    want = expected(fibs_in, tid, xh, xl)
    fibs = [pb.Fib(f.hi, f.lo, f.len, f.nh, format="f16hi", smem_levels=smem.get(t, -1))
            for t, f in enumerate(fibs_in)]
    assert any(f.stats()["depth"] - f.stats()["smem_levels"] >= 2 for f in fibs)
    dh, dl, dt = dev(xh), dev(xl), dev(tid, np.uint8)
    for bucketed in (False, True):
        with pb.MultiFib(fibs, max_batch=1 << 20, graph=graph, bucketed=bucketed) as mt:
            for k in (tid.size, 33, 1):
                out = torch.full((k,), -1, dtype=torch.int16, device="cuda")
                mt.lookup(dh[:k], dl[:k], dt[:k], out=out)
                torch.cuda.synchronize()
                assert np.array_equal(out.cpu().numpy().view(np.uint16), want[:k]), (bucketed, k)
            assert mt.persistent and mt.mode == ("bucketed" if bucketed else "direct")
    for f in fibs:
        f.close()


def test_direct_form_needs_every_table_f16hi():
    """One F8X128 table in the group: the batch is bucketed (the direct form reads F16HI nodes)."""
    sizes = [3000, 20_000]
    fibs_in, tid, xh, xl = workload(sizes, 100_000, seed=93)
    fibs = [pb.Fib(fibs_in[0].hi, fibs_in[0].lo, fibs_in[0].len, fibs_in[0].nh, format="f16hi"),
            pb.Fib(fibs_in[1].hi, fibs_in[1].lo, fibs_in[1].len, fibs_in[1].nh, format="f8x128")]
    with pb.MultiFib(fibs, max_batch=100_000) as mt:
        out = mt.lookup(dev(xh), dev(xl), dev(tid, np.uint8))
        torch.cuda.synchronize()
        assert mt.mode == "bucketed"
        assert np.array_equal(out.cpu().numpy().view(np.uint16), expected(fibs_in, tid, xh, xl))
    for f in fibs:
        f.close()
