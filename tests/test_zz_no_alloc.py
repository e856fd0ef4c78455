"""planb_lookup_host_noalloc: the host-buffer lookup for callers that must not allocate device
memory (a packet-forwarding thread cannot wait on cudaMalloc; a process whose device memory is
owned by another allocator's pool cannot take more). It stages through a fixed device array
instead of allocated buffers. Checked through the C ABI against the O2 trie oracle and against
planb_lookup_host, bit-exactly, on two calls in a row, and from two threads on two streams at once
(the library serialises them on its lock); sizes above the array's limit are refused."""
import ctypes as C
import threading

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2604_14650_gb300 as pb  # noqa: E402

MAX_KEYS = 262144   # PLANB_NOALLOC_MAX_KEYS


def _entry():
    pb.build()
    fn = pb.load().planb_lookup_host_noalloc
    fn.restype = C.c_int
    fn.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p]
    return fn


def test_noalloc_matches_oracle_and_lookup_host_on_two_calls():
    fn = _entry()
    f = synth.gen_fib(200_000, seed=2604, nh_max=4095)
    trie = oracle.Trie(f.hi, f.lo, f.len, f.nh)
    with pb.Fib(f.hi, f.lo, f.len, f.nh, format="f16hi") as fib:
        for n, seed in ((MAX_KEYS, 11), (123_457, 12)):      # two calls in a row
            xh, xl = synth.gen_trace(f, n, seed=seed)
            want = trie.lookup(xh, xl)
            got = np.full(n, 0xFFFF, dtype=np.uint16)
            rc = fn(fib._h, xh.ctypes.data, xl.ctypes.data, n, got.ctypes.data, None)
            assert rc == 0, pb.binding._strerror(rc)
            assert np.array_equal(got, want)
            assert np.array_equal(got, fib.lookup_host(xh, xl))  # the existing entry point
        too_many = np.zeros(MAX_KEYS + 1, dtype=np.uint64)
        out = np.zeros(MAX_KEYS + 1, dtype=np.uint16)
        assert fn(fib._h, too_many.ctypes.data, too_many.ctypes.data, MAX_KEYS + 1,
                  out.ctypes.data, None) == -1                 # PLANB_EINVAL


def test_noalloc_two_threads_two_streams():
    """Two threads, each on its own stream with its own trace and size, call the entry point in a
    loop; ctypes drops the GIL, so the calls really contend for the one staging array."""
    fn = _entry()
    f = synth.gen_fib(50_000, seed=2605, nh_max=4095)
    trie = oracle.Trie(f.hi, f.lo, f.len, f.nh)
    jobs = []
    for n, seed in ((MAX_KEYS, 21), (77_777, 22)):
        xh, xl = synth.gen_trace(f, n, seed=seed)
        jobs.append((xh, xl, trie.lookup(xh, xl)))
    with pb.Fib(f.hi, f.lo, f.len, f.nh) as fib:
        bad = []

        def worker(k):
            xh, xl, want = jobs[k]
            s = torch.cuda.Stream()
            for _ in range(8):
                got = np.full(want.size, 0xFFFF, dtype=np.uint16)
                rc = fn(fib._h, xh.ctypes.data, xl.ctypes.data, want.size, got.ctypes.data,
                        s.cuda_stream)
                if rc != 0 or not np.array_equal(got, want):
                    bad.append((k, rc))
            fib.forget_stream(s)

        ts = [threading.Thread(target=worker, args=(k,)) for k in range(2)]
        for t in ts:
            t.start()
        for t in ts:
            t.join()
        assert not bad
