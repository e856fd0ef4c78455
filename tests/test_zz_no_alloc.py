"""planb_lookup_host_noalloc: the host-buffer lookup for callers that must not allocate device
memory (a packet-forwarding thread cannot wait on cudaMalloc; a process whose device memory is
owned by another allocator's pool cannot take more). It stages through a fixed device array
instead of allocated buffers. Checked through the C ABI against planb_lookup_host, bit-exactly,
on two calls in a row; sizes above the array's limit are refused."""
import ctypes as C

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2604_14650_gb300 as pb  # noqa: E402

MAX_KEYS = 262144   # PLANB_NOALLOC_MAX_KEYS


def test_noalloc_matches_lookup_host_on_two_calls():
    pb.build()
    fn = pb.load().planb_lookup_host_noalloc
    fn.restype = C.c_int
    fn.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p]
    f = synth.gen_fib(200_000, seed=2604, nh_max=4095)
    with pb.Fib(f.hi, f.lo, f.len, f.nh) as fib:
        for n, seed in ((MAX_KEYS, 11), (123_457, 12)):      # two calls in a row
            xh, xl = synth.gen_trace(f, n, seed=seed)
            want = fib.lookup_host(xh, xl)                     # the existing entry point
            got = np.full(n, 0xFFFF, dtype=np.uint16)
            rc = fn(fib._h, xh.ctypes.data, xl.ctypes.data, n, got.ctypes.data, None)
            assert rc == 0, pb.binding._strerror(rc)
            assert np.array_equal(got, want)
        too_many = np.zeros(MAX_KEYS + 1, dtype=np.uint64)
        out = np.zeros(MAX_KEYS + 1, dtype=np.uint16)
        assert fn(fib._h, too_many.ctypes.data, too_many.ctypes.data, MAX_KEYS + 1,
                  out.ctypes.data, None) == -1                 # PLANB_EINVAL
