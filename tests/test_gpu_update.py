"""GPU tests of planb_update (rebuild-and-swap, Section 3.6): after every batch the GPU answers equal
the oracle rebuilt from scratch on the updated prefix set; the swap is stream-ordered; a failed
rebuild (host-side fault injection) leaves the previous table current and correct."""
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


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a).view(np.int64)).cuda()


def masked(h, l, L):
    mh, ml = synth.top_mask(np.array([L]))
    return int(np.uint64(h) & mh[0]), int(np.uint64(l) & ml[0]), int(L)


class RefTable:
    """The expected prefix set: a dict (prefix, len) -> next hop, updated by the documented rules."""

    def __init__(self, f):
        self.d = {}
        for h, l, L, n in zip(f.hi, f.lo, f.len, f.nh):
            self.d[masked(h, l, L)] = int(n)

    def apply(self, upd):
        ih, il, iL, inh, wh, wl, wL = upd
        absent = 0
        for h, l, L in zip(wh, wl, wL):
            k = masked(h, l, L)
            if k in self.d:
                del self.d[k]
            else:
                absent += 1
        for h, l, L, n in zip(ih, il, iL, inh):
            self.d[masked(h, l, L)] = int(n)
        return absent

    def arrays(self):
        ks = list(self.d)
        return (np.array([k[0] for k in ks], np.uint64), np.array([k[1] for k in ks], np.uint64),
                np.array([k[2] for k in ks], np.uint8), np.array([self.d[k] for k in ks], np.uint16))


def oracle_answer(ref, xh, xl):
    h, l, L, n = ref.arrays()
    return oracle.Trie(h, l, L, n).lookup(xh, xl)


@pytest.mark.parametrize("fmt,kernel", [("f8v7", "hybrid"), ("f8x128", "hybrid"),
                                        ("f8x128", "coop"), ("f16hi", "coop")])
def test_update_batches_match_oracle_rebuild(fmt, kernel):
    f = synth.gen_fib(20_000, seed=81, nh_max=4095)
    xh, xl = synth.gen_trace(f, 400_000, seed=82)
    ref = RefTable(f)
    absent_total = 0
    with pb.Fib(f.hi, f.lo, f.len, f.nh, format=fmt, kernel=kernel) as fib:
        dh, dl = dev(xh), dev(xl)
        for batch in range(6):
            upd = synth.gen_updates(f, 500 * (batch + 1), seed=83, start=batch * 10_000)
            if batch == 3:   # withdraw prefixes that are not present, and re-insert one as a modify
                upd = upd[:4] + (np.concatenate([upd[4], [np.uint64(0x3FFF << 48)]]),
                                 np.concatenate([upd[5], [np.uint64(0)]]),
                                 np.concatenate([upd[6], [np.uint8(16)]]))
            absent_total += ref.apply(upd)
            fib.update(*upd)
            st = fib.stats()
            assert st["version"] == batch + 2
            assert st["withdraw_absent"] == absent_total
            out = fib.lookup(dh, dl)
            torch.cuda.synchronize()
            assert np.array_equal(out.cpu().numpy().view(np.uint16), oracle_answer(ref, xh, xl))


def test_swap_is_stream_ordered():
    f = synth.gen_fib(50_000, seed=91, nh_max=4095)
    n = 1 << 23
    xh, xl = synth.gen_trace(f, n, seed=92)
    ref = RefTable(f)
    old_want = oracle_answer(ref, xh, xl)
    upd = synth.gen_updates(f, 5000, seed=93, withdraw_frac=0.8)
    ref.apply(upd)
    new_want = oracle_answer(ref, xh, xl)
    assert not np.array_equal(old_want, new_want)
    s = torch.cuda.Stream()
    with pb.Fib(f.hi, f.lo, f.len, f.nh) as fib:
        dh, dl = dev(xh), dev(xl)
        torch.cuda.synchronize()
        with torch.cuda.stream(s):
            before = torch.empty(n, dtype=torch.int16, device="cuda")
            after = torch.empty(n, dtype=torch.int16, device="cuda")
            torch.cuda._sleep(50_000_000)       # keep the stream busy so the swap lands mid-queue
            for _ in range(4):
                fib.lookup(dh, dl, out=before, stream=s)
            fib.update(*upd, stream=s)           # swaps while the lookups above are still queued
            fib.lookup(dh, dl, out=after, stream=s)
        s.synchronize()
        assert np.array_equal(before.cpu().numpy().view(np.uint16), old_want)
        assert np.array_equal(after.cpu().numpy().view(np.uint16), new_want)


@pytest.mark.parametrize("point", [1, 2])
def test_failed_rebuild_keeps_old_table(point):
    f = synth.gen_fib(10_000, seed=95, nh_max=4095)
    xh, xl = synth.gen_trace(f, 200_000, seed=96)
    want = oracle_answer(RefTable(f), xh, xl)
    with pb.Fib(f.hi, f.lo, f.len, f.nh) as fib:
        upd = synth.gen_updates(f, 1000, seed=97)
        pb.debug_inject(point)
        with pytest.raises(pb.PlanbError):
            fib.update(*upd)
        assert fib.stats()["version"] == 1
        out = fib.lookup(dev(xh), dev(xl))
        torch.cuda.synchronize()
        assert np.array_equal(out.cpu().numpy().view(np.uint16), want)
        fib.update(*upd)                          # the hook fired once; the next rebuild succeeds
        assert fib.stats()["version"] == 2
