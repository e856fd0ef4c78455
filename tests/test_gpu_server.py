"""The serving engine: requests from several threads, many tables, continuous batching. Each
request's result is the same as the same request run alone (planb_lookup_host on its table) and as
the oracle's; tables are admitted against a device-memory budget; route updates applied while
serving are seen by later requests."""
import threading

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu, pytest.mark.timeout(180)]
WAIT_US = 20_000_000     # no request may take 20 s

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2604_14650_gb300 as pb  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def built():
    pb.build()


@pytest.mark.parametrize("fmt,bucketed", [("f8x128", False), ("f16hi", False), ("f16hi", True)],
                         ids=["f8x128", "f16hi-direct", "f16hi-bucketed"])
def test_requests_in_the_mix_equal_alone(fmt, bucketed):
    """Requests batched by the serving loop get the results they get alone and the oracle's; the
    slots' batches of F16HI tables take the direct multi-table form (or, asked, the grouped one),
    with the batch size read from device memory."""
    sizes = [3000, 40_000, 700, 12_000, 90_000, 5000]
    fibs_in = [synth.gen_fib(s, seed=600 + t, nh_max=4095) for t, s in enumerate(sizes)]
    fibs = [pb.Fib(f.hi, f.lo, f.len, f.nh, format=fmt) for f in fibs_in]
    rng = np.random.default_rng(7)
    reqs = []
    for i in range(240):
        t = int(rng.integers(len(sizes)))
        n = int(np.exp(rng.uniform(np.log(32), np.log(65536))))
        xh, xl = synth.gen_trace(fibs_in[t], n, seed=10_000 + i)
        reqs.append((t, xh, xl, np.zeros(n, np.uint16)))
    with pb.Server(slots=3, max_batch=1 << 18, bucketed=bucketed) as srv:
        ids = [srv.add_table(f) for f in fibs]
        assert ids == list(range(len(sizes)))
        tickets = [None] * len(reqs)

        def producer(k):
            for i in range(k, len(reqs), 4):
                t, xh, xl, out = reqs[i]
                tickets[i] = srv.submit(t, xh, xl, out)

        th = [threading.Thread(target=producer, args=(k,)) for k in range(4)]
        for x in th:
            x.start()
        for x in th:
            x.join()
        for tk in tickets:
            srv.wait(tk, WAIT_US)
        st = srv.stats()
        assert st["requests"] == len(reqs)
        assert st["batches"] < len(reqs)             # requests were batched together
        assert st["last_error"] == 0
    for t, xh, xl, out in reqs:
        alone = fibs[t].lookup_host(xh, xl)
        assert np.array_equal(out, alone)
        assert np.array_equal(out, oracle.Trie(fibs_in[t].hi, fibs_in[t].lo, fibs_in[t].len,
                                               fibs_in[t].nh).lookup(xh, xl))
    for f in fibs:
        f.close()


def test_admission_by_memory_budget():
    a = synth.gen_fib(20_000, seed=1)
    b = synth.gen_fib(20_000, seed=2)
    with pb.Fib(a.hi, a.lo, a.len, a.nh) as fa, pb.Fib(b.hi, b.lo, b.len, b.nh) as fb:
        need = fa.stats()["node_bytes"] + fa.stats()["value_bytes"]
        with pb.Server(slots=1, max_batch=1 << 16, mem_budget=int(need * 1.5)) as srv:
            assert srv.add_table(fa) == 0
            with pytest.raises(pb.PlanbError):        # the second table does not fit
                srv.add_table(fb)
            assert srv.stats()["tables"] == 1


@pytest.mark.parametrize("fmt", ["f8x128", "f16hi"])
def test_updates_while_serving_are_seen(fmt):
    f = synth.gen_fib(30_000, seed=77, nh_max=4095)
    xh, xl = synth.gen_trace(f, 20_000, seed=78)
    with pb.Fib(f.hi, f.lo, f.len, f.nh, format=fmt) as fib, \
            pb.Server(slots=2, update_period_us=2000) as srv:
        t = srv.add_table(fib)
        out = np.zeros(xh.size, np.uint16)
        srv.wait(srv.submit(t, xh, xl, out), WAIT_US)
        assert np.array_equal(out, oracle.Trie(f.hi, f.lo, f.len, f.nh).lookup(xh, xl))
        keep = f.len == 0                              # withdraw everything but the default
        srv.update(t, wd_hi=f.hi[~keep], wd_lo=f.lo[~keep], wd_len=f.len[~keep])
        for _ in range(400):                           # the updater applies it within a period
            if srv.stats()["update_batches"]:
                break
            threading.Event().wait(0.005)
        assert srv.stats()["update_batches"] == 1
        srv.wait(srv.submit(t, xh, xl, out), WAIT_US)
        assert np.all(out == 0)
