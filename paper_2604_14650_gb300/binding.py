"""Python binding of libplanb.so (include/planb.h): argument marshalling only.

Every step of a lookup runs in the library's CUDA kernels; the table build runs in its C++ host
code. PyTorch supplies device memory and streams: device arrays are CUDA tensors (addresses as
int64 holding the u64 bits, next hops as int16 holding the u16 bits) and a stream is a
``torch.cuda.Stream``. If the compiled library is missing, every call raises — there is no Python
or CPU fallback.
"""
from __future__ import annotations

import atexit
import ctypes as C
import os
import platform
import weakref

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_DIR = os.path.join(HERE, "_build", platform.machine())

PLANB_OK = 0
ERRORS = {-1: "EINVAL", -2: "ENOMEM", -3: "ECUDA", -4: "EDEVICE", -5: "ENODEV", -6: "ETIMEOUT"}
FORMATS = {"f8x128": 0, "f16hi": 1, "f8v7": 2}
KERNELS = {"auto": 0, "coop": 1, "hybrid": 2, "flat": 3, "learned": 4}
BUILDERS = {"host": 0, "device": 1}


class PlanbError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        detail = ""
        try:
            detail = load().planb_last_error().decode()
        except Exception:
            pass
        super().__init__(f"{where}: {ERRORS.get(code, code)} ({_strerror(code)})"
                         + (f" [{detail}]" if detail else ""))


class Opts(C.Structure):
    _fields_ = [("struct_size", C.c_uint32), ("format", C.c_int32), ("merge_equal_nh", C.c_int32),
                ("smem_levels", C.c_int32), ("device", C.c_int32), ("block_threads", C.c_int32),
                ("ctas_per_sm", C.c_int32), ("kernel", C.c_int32), ("model_leaves", C.c_int32),
                ("model_iters", C.c_int32), ("builder", C.c_int32), ("reserved", C.c_int32 * 4)]


class Stats(C.Structure):
    _fields_ = [("n_input", C.c_uint64), ("n_prefixes", C.c_uint64), ("n_intervals", C.c_uint64),
                ("depth", C.c_uint32), ("keys_per_node", C.c_uint32), ("fanout", C.c_uint32),
                ("smem_levels", C.c_uint32), ("format", C.c_uint32), ("device", C.c_uint32),
                ("internal_nodes", C.c_uint64), ("leaf_nodes", C.c_uint64),
                ("node_bytes", C.c_uint64), ("value_bytes", C.c_uint64), ("version", C.c_uint64),
                ("withdraw_absent", C.c_uint64), ("build_ms", C.c_double),
                ("upload_ms", C.c_double), ("kernel", C.c_uint32), ("threads", C.c_uint32),
                ("ctas", C.c_uint32), ("smem_bytes", C.c_uint32), ("model_leaves", C.c_uint32),
                ("model_iters", C.c_uint32), ("model_max_err", C.c_uint32),
                ("builder", C.c_uint32), ("model_loss0", C.c_double), ("model_loss", C.c_double),
                ("model_covered", C.c_double), ("model_mean_err", C.c_double),
                ("model_train_ms", C.c_double)]


class LayoutT(C.Structure):
    _fields_ = [("keys_per_node", C.c_uint32), ("fanout", C.c_uint32), ("depth", C.c_uint32),
                ("reserved", C.c_uint32), ("n_keys", C.c_uint64), ("internal_nodes", C.c_uint64),
                ("leaf_capacity", C.c_uint64), ("key_capacity", C.c_uint64),
                ("level_start", C.c_uint64 * 16)]


# planb_route {u64 hi, lo; u8 len; u16 nexthop} and planb_prefix {u64 hi, lo; u8 len} in C layout
ROUTE_DTYPE = np.dtype({"names": ["hi", "lo", "len", "nexthop"],
                        "formats": [np.uint64, np.uint64, np.uint8, np.uint16],
                        "offsets": [0, 8, 16, 18], "itemsize": 24})
PREFIX_DTYPE = np.dtype({"names": ["hi", "lo", "len"], "formats": [np.uint64, np.uint64, np.uint8],
                         "offsets": [0, 8, 16], "itemsize": 24})

_libs: dict = {}

_vp = C.c_void_p
_sz = C.c_size_t
_SIGS = {
    "planb_opts_default": (None, [_vp]),
    "planb_strerror": (C.c_char_p, [C.c_int]),
    "planb_last_error": (C.c_char_p, []),
    "planb_version": (C.c_uint32, []),
    "planb_build": (C.c_int, [_vp, _vp, _vp, _vp, _sz, _vp, C.POINTER(_vp)]),
    "planb_lookup": (C.c_int, [_vp, _vp, _vp, _sz, _vp, _vp]),
    "planb_lookup_host": (C.c_int, [_vp, _vp, _vp, _sz, _vp]),
    "planb_update": (C.c_int, [_vp, _vp, _sz, _vp, _sz, _vp]),
    "planb_forget_stream": (C.c_int, [_vp, _vp]),
    "planb_lookup_mapped": (C.c_int, [_vp, _vp, _vp, _sz, _vp, _vp]),
    "planb_stats": (C.c_int, [_vp, _vp]),
    "planb_device_status": (C.c_int, [_vp, C.POINTER(C.c_uint32)]),
    "planb_destroy": (None, [_vp]),
    "planb_intervals": (C.c_int, [_vp, _vp, _vp, _vp, _sz, C.c_int, _vp, _vp, _vp, _sz,
                                  C.POINTER(_sz)]),
    "planb_layout_info": (C.c_int, [C.c_uint32, C.c_uint64, C.c_uint32, _vp]),
    "planb_child_index": (C.c_uint64, [C.c_uint32, C.c_uint32, C.c_uint64, C.c_uint32]),
    "planb_debug_inject": (C.c_int, [C.c_int]),
    "planb_debug_kernel_info": (C.c_int, [_vp, C.c_int, _vp]),
    "planb_debug_table_dump": (C.c_int, [_vp, _vp, _sz, C.POINTER(_sz)]),
    "planb_intervals_device": (C.c_int, [_vp, _vp, _vp, _vp, _sz, C.c_int, _vp, _vp, _vp, _sz,
                                         C.POINTER(_sz)]),
    "planb_mlp_grad": (C.c_int, [_vp, _vp, _sz, _vp, _vp, C.POINTER(C.c_double), _vp]),
    "planb_mlp_forward": (C.c_int, [_vp, _sz, _vp, _vp, _vp]),
    "planb_mlp_grad_split": (C.c_int, [_vp, _vp, _vp, _sz, _vp, _vp, C.POINTER(C.c_double), _vp]),
    "planb_mlp_knot_step": (C.c_int, [_vp, _vp, _vp, _sz, _vp, _vp, _vp, _vp, _vp, C.c_int32,
                                      C.c_float, C.POINTER(C.c_double), _vp]),
    "planb_multi_create": (C.c_int, [_vp, C.c_uint32, _sz, C.c_uint32, C.POINTER(_vp)]),
    "planb_multi_lookup": (C.c_int, [_vp, _vp, _vp, _vp, _sz, _vp, _vp]),
    "planb_multi_destroy": (None, [_vp]),
    "planb_multi_persistent": (C.c_int, [_vp]),
    "planb_multi_mode": (C.c_int, [_vp]),
    "planb_multi_captures": (C.c_uint64, [_vp]),
    "planb_multi_lookup_devn": (C.c_int, [_vp, _vp, _vp, _vp, _vp, _sz, _vp, _vp]),
    "planb_server_opts_default": (None, [_vp]),
    "planb_server_create": (C.c_int, [_vp, C.POINTER(_vp)]),
    "planb_server_add_table": (C.c_int, [_vp, _vp, C.POINTER(C.c_uint32)]),
    "planb_server_submit": (C.c_int, [_vp, C.c_uint32, _vp, _vp, _sz, _vp,
                                      C.POINTER(C.c_uint64)]),
    "planb_server_wait": (C.c_int, [_vp, C.c_uint64, C.c_uint32]),
    "planb_server_update": (C.c_int, [_vp, C.c_uint32, _vp, _sz, _vp, _sz]),
    "planb_server_stats": (C.c_int, [_vp, _vp]),
    "planb_server_reset_stats": (None, [_vp]),
    "planb_server_error_detail": (C.c_int, [_vp, C.c_char_p, _sz]),
    "planb_server_destroy": (None, [_vp]),
}


def library_path(variant: str = "libplanb.so") -> str:
    return os.path.join(LIB_DIR, variant)


def load(variant: str = "libplanb.so"):
    """Loads (once) and returns the ctypes handle of a compiled library variant."""
    if variant in _libs:
        return _libs[variant]
    path = library_path(variant)
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with paper_2604_14650_gb300.build()")
    lib = C.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _libs[variant] = lib
    return lib


def _strerror(code: int) -> str:
    try:
        return load().planb_strerror(code).decode()
    except Exception:
        return "?"


def _check(rc: int, where: str):
    if rc != PLANB_OK:
        raise PlanbError(rc, where)


def _np(a, dtype):
    a = np.ascontiguousarray(a)
    if a.dtype != dtype:
        if a.dtype.itemsize == np.dtype(dtype).itemsize and a.dtype.kind in "iu":
            a = a.view(dtype)
        else:
            a = a.astype(dtype)
    return a


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p) if a.size else None


def _stream_handle(stream):
    if stream is None:
        import torch
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return C.c_void_p(stream)
    return C.c_void_p(stream.cuda_stream)


def version() -> int:
    return int(load().planb_version())


def intervals(hi, lo, ln, nh, merge: bool = False, variant: str = "libplanb.so",
              device: bool = False):
    """Elementary intervals of a prefix table: (start_hi, start_lo, nh) arrays. device=False runs
    the host builder (no GPU needed), device=True the GPU builder on the current device."""
    lib = load(variant)
    entry = lib.planb_intervals_device if device else lib.planb_intervals
    hi, lo, ln, nh = _np(hi, np.uint64), _np(lo, np.uint64), _np(ln, np.uint8), _np(nh, np.uint16)
    n = hi.size
    m = _sz(0)
    cap = 2 * n + 1
    sh = np.empty(cap, np.uint64)
    sl = np.empty(cap, np.uint64)
    snh = np.empty(cap, np.uint16)
    _check(entry(_ptr(hi), _ptr(lo), _ptr(ln), _ptr(nh), n, int(merge), _ptr(sh), _ptr(sl),
                 _ptr(snh), cap, C.byref(m)),
           "planb_intervals_device" if device else "planb_intervals")
    k = m.value
    return sh[:k].copy(), sl[:k].copy(), snh[:k].copy()


def layout_info(keys_per_node: int, n_keys: int, depth: int = 0) -> dict:
    t = LayoutT()
    _check(load().planb_layout_info(keys_per_node, n_keys, depth, C.byref(t)), "planb_layout_info")
    d = {f: getattr(t, f) for f, _ in LayoutT._fields_ if f not in ("reserved", "level_start")}
    d["level_start"] = list(t.level_start)[: t.depth]
    return d


def child_index(keys_per_node: int, d: int, j: int, c: int) -> int:
    return int(load().planb_child_index(keys_per_node, d, j, c))


def debug_inject(point: int):
    _check(load().planb_debug_inject(point), "planb_debug_inject")


def mlp_grad(u, t, w, stream=None):
    """Root-MLP loss and gradient by the library's training kernels (CUDA float32 tensors u, t;
    w: 65 floats w1, b1, w2, b2, cap). Returns (loss, grad of the 49 trained parameters)."""
    wv = np.ascontiguousarray(w, dtype=np.float32)
    if wv.size != 65:
        raise ValueError("w holds 65 floats: w1, b1, w2, b2, cap")
    g = np.zeros(49, dtype=np.float32)
    loss = C.c_double(0.0)
    _check(load().planb_mlp_grad(C.c_void_p(u.data_ptr()), C.c_void_p(t.data_ptr()), u.numel(),
                                 _ptr(wv), _ptr(g), C.byref(loss), _stream_handle(stream)),
           "planb_mlp_grad")
    return loss.value, g


def mlp_grad_split(u, ulo, t, w, stream=None):
    """mlp_grad on the two-float input u + ulo (CUDA float32 tensors u, ulo, t)."""
    wv = np.ascontiguousarray(w, dtype=np.float32)
    if wv.size != 65:
        raise ValueError("w holds 65 floats: w1, b1, w2, b2, cap")
    g = np.zeros(49, dtype=np.float32)
    loss = C.c_double(0.0)
    _check(load().planb_mlp_grad_split(C.c_void_p(u.data_ptr()), C.c_void_p(ulo.data_ptr()),
                                       C.c_void_p(t.data_ptr()), u.numel(), _ptr(wv), _ptr(g),
                                       C.byref(loss), _stream_handle(stream)),
           "planb_mlp_grad_split")
    return loss.value, g


def mlp_knot_step(u, ulo, t, w, knots, v, m, q, step: int, lr: float, stream=None):
    """One training iteration in knot-value form by the library's kernels (gradient, then Adam on
    the knot values). u, ulo (or None), t: CUDA float32 tensors; w (65), knots, v, m, q (17):
    host arrays. Returns (loss before the step, new w, new v, new m, new q) as float32 arrays."""
    wv = np.array(w, dtype=np.float32)
    kv = np.ascontiguousarray(knots, dtype=np.float32)
    vv, mv, qv = (np.array(a, dtype=np.float32) for a in (v, m, q))
    if wv.size != 65 or kv.size != 17 or vv.size != 17 or mv.size != 17 or qv.size != 17:
        raise ValueError("w holds 65 floats; knots, v, m, q 17 each")
    loss = C.c_double(0.0)
    _check(load().planb_mlp_knot_step(C.c_void_p(u.data_ptr()),
                                      C.c_void_p(ulo.data_ptr()) if ulo is not None else None,
                                      C.c_void_p(t.data_ptr()), u.numel(), _ptr(wv), _ptr(kv),
                                      _ptr(vv), _ptr(mv), _ptr(qv), int(step), float(lr),
                                      C.byref(loss), _stream_handle(stream)),
           "planb_mlp_knot_step")
    return loss.value, wv, vv, mv, qv


def mlp_forward(u, w, out=None, stream=None):
    """y = root(u) by the library's inference kernel (CUDA float32 tensors; w: 65 floats)."""
    import torch
    wv = np.ascontiguousarray(w, dtype=np.float32)
    if wv.size != 65:
        raise ValueError("w holds 65 floats: w1, b1, w2, b2, cap")
    if out is None:
        out = torch.empty_like(u)
    _check(load().planb_mlp_forward(C.c_void_p(u.data_ptr()), u.numel(), _ptr(wv),
                                    C.c_void_p(out.data_ptr()), _stream_handle(stream)),
           "planb_mlp_forward")
    return out


class Fib:
    """One lookup table on a GPU (a planb_fib)."""

    def __init__(self, hi, lo, ln, nh, *, format: str = "f8x128", merge: bool = False,
                 smem_levels: int = -1, device: int | None = None, block_threads: int = 0,
                 ctas_per_sm: int = 0, kernel: str = "auto", model_leaves: int = 0,
                 model_iters: int = -1, builder: str = "host", variant: str = "libplanb.so"):
        self._lib = load(variant)
        self._h = None
        hi, lo, ln, nh = _np(hi, np.uint64), _np(lo, np.uint64), _np(ln, np.uint8), _np(nh, np.uint16)
        if not (hi.shape == lo.shape == ln.shape == nh.shape):
            raise ValueError("prefix arrays differ in length")
        o = Opts()
        self._lib.planb_opts_default(C.byref(o))
        o.format = FORMATS[format]
        o.merge_equal_nh = int(merge)
        o.smem_levels = smem_levels
        o.device = -1 if device is None else device
        o.block_threads = block_threads
        o.ctas_per_sm = ctas_per_sm
        o.kernel = KERNELS[kernel]
        o.model_leaves = model_leaves
        o.model_iters = model_iters
        o.builder = BUILDERS[builder]
        h = C.c_void_p()
        _check(self._lib.planb_build(_ptr(hi), _ptr(lo), _ptr(ln), _ptr(nh), hi.size, C.byref(o),
                                     C.byref(h)), "planb_build")
        self._h = h
        self.device = self.stats()["device"]

    # -- lookups ---------------------------------------------------------------------------
    def lookup(self, addr_hi, addr_lo, out=None, stream=None):
        """Next hops of CUDA tensors of addresses (int64 bits of u64); returns an int16 tensor."""
        import torch
        if not (addr_hi.is_cuda and addr_lo.is_cuda):
            raise ValueError("addresses must be CUDA tensors (use lookup_host for host arrays)")
        if addr_hi.dtype not in (torch.int64, torch.uint64) or addr_lo.dtype != addr_hi.dtype:
            raise ValueError("addresses must be int64 (u64 bits)")
        if not (addr_hi.is_contiguous() and addr_lo.is_contiguous()):
            raise ValueError("addresses must be contiguous")
        n = addr_hi.numel()
        if addr_lo.numel() != n:
            raise ValueError("hi and lo differ in length")
        if out is None:
            out = torch.empty(n, dtype=torch.int16, device=addr_hi.device)
        elif out.numel() != n or out.element_size() != 2 or not out.is_contiguous():
            raise ValueError("out must be a contiguous 2-byte tensor of n elements")
        _check(self._lib.planb_lookup(self._h, C.c_void_p(addr_hi.data_ptr()),
                                      C.c_void_p(addr_lo.data_ptr()), n,
                                      C.c_void_p(out.data_ptr()), _stream_handle(stream)),
               "planb_lookup")
        return out

    def lookup_ptr(self, hi_ptr: int, lo_ptr: int, n: int, out_ptr: int, stream=None):
        """Same as lookup on raw device pointers (for timing loops)."""
        _check(self._lib.planb_lookup(self._h, C.c_void_p(hi_ptr), C.c_void_p(lo_ptr), n,
                                      C.c_void_p(out_ptr), _stream_handle(stream)), "planb_lookup")

    def lookup_mapped(self, addr_hi, addr_lo, out, stream=None):
        """Lookups on pinned host tensors read and written directly by the kernel (no copies);
        asynchronous on `stream`."""
        for t in (addr_hi, addr_lo, out):
            if t.is_cuda or not t.is_pinned() or not t.is_contiguous():
                raise ValueError("lookup_mapped takes contiguous pinned host tensors")
        n = addr_hi.numel()
        if addr_lo.numel() != n or out.numel() != n or out.element_size() != 2:
            raise ValueError("buffer sizes differ")
        _check(self._lib.planb_lookup_mapped(self._h, C.c_void_p(addr_hi.data_ptr()),
                                             C.c_void_p(addr_lo.data_ptr()), n,
                                             C.c_void_p(out.data_ptr()), _stream_handle(stream)),
               "planb_lookup_mapped")
        return out

    def lookup_host(self, addr_hi, addr_lo, out=None):
        """Next hops of host arrays (numpy, or CPU tensors — pinned for full speed); synchronous."""
        hp, lp, n, keep = _host_ptrs(addr_hi, addr_lo)
        if out is None:
            out = np.empty(n, dtype=np.uint16)
        op = out.data_ptr() if hasattr(out, "data_ptr") else out.ctypes.data
        _check(self._lib.planb_lookup_host(self._h, C.c_void_p(hp), C.c_void_p(lp), n,
                                           C.c_void_p(op)), "planb_lookup_host")
        del keep
        return out

    # -- updates ---------------------------------------------------------------------------
    def update(self, ins_hi=(), ins_lo=(), ins_len=(), ins_nh=(), wd_hi=(), wd_lo=(), wd_len=(),
               stream=None):
        """Rebuild-and-swap with a batch of inserts (or modifies) and withdraws."""
        ins = np.zeros(len(ins_hi), dtype=ROUTE_DTYPE)
        ins["hi"], ins["lo"], ins["len"], ins["nexthop"] = ins_hi, ins_lo, ins_len, ins_nh
        wd = np.zeros(len(wd_hi), dtype=PREFIX_DTYPE)
        wd["hi"], wd["lo"], wd["len"] = wd_hi, wd_lo, wd_len
        st = _stream_handle(stream) if stream is not None else C.c_void_p(0)
        _check(self._lib.planb_update(self._h, _ptr(ins), ins.size, _ptr(wd), wd.size, st),
               "planb_update")

    # -- introspection ---------------------------------------------------------------------
    def stats(self) -> dict:
        s = Stats()
        _check(self._lib.planb_stats(self._h, C.byref(s)), "planb_stats")
        return {f: getattr(s, f) for f, _ in Stats._fields_}

    def kernel_info(self, multi: bool = False) -> dict:
        a = (C.c_int * 6)()
        _check(self._lib.planb_debug_kernel_info(self._h, int(multi), a), "planb_debug_kernel_info")
        return dict(zip(("regs", "max_threads", "max_dyn_smem", "local", "static_smem", "const"), a))

    def forget_stream(self, stream):
        """Before destroying a stream used with this table: waits for it and stops fencing on it."""
        _check(self._lib.planb_forget_stream(self._h, _stream_handle(stream)),
               "planb_forget_stream")

    def table_dump(self) -> np.ndarray:
        """The current table's device image (node arrays, index, next hops) as bytes."""
        nb = _sz(0)
        self._lib.planb_debug_table_dump(self._h, None, 0, C.byref(nb))
        buf = np.empty(nb.value, dtype=np.uint8)
        _check(self._lib.planb_debug_table_dump(self._h, _ptr(buf), buf.size, C.byref(nb)),
               "planb_debug_table_dump")
        return buf

    def device_status(self):
        w = C.c_uint32(0)
        rc = self._lib.planb_device_status(self._h, C.byref(w))
        return rc, w.value

    def close(self):
        if self._h:
            self._lib.planb_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _host_ptrs(hi, lo):
    if hasattr(hi, "data_ptr"):
        if hi.is_cuda or lo.is_cuda:
            raise ValueError("lookup_host takes host arrays")
        if not (hi.is_contiguous() and lo.is_contiguous()) or hi.element_size() != 8:
            raise ValueError("host tensors must be contiguous 8-byte integers")
        return hi.data_ptr(), lo.data_ptr(), hi.numel(), (hi, lo)
    hi, lo = _np(hi, np.uint64), _np(lo, np.uint64)
    if hi.size != lo.size:
        raise ValueError("hi and lo differ in length")
    return hi.ctypes.data, lo.ctypes.data, hi.size, (hi, lo)


class MultiFib:
    """Several tables (VRFs) looked up by one captured graph; each address carries a table id."""

    MODES = ("per_table", "bucketed", "direct")   # planb_multi_mode's values, in order

    def __init__(self, fibs, max_batch: int, graph: bool = True, per_table: bool = False,
                 bucketed: bool = False, direct: bool = False):
        self._lib = fibs[0]._lib
        self._h = None
        self.fibs = list(fibs)                 # keep the tables alive while the group exists
        arr = (C.c_void_p * len(fibs))(*[f._h.value for f in fibs])
        h = C.c_void_p()
        flags = ((0 if graph else 1) | (2 if per_table else 0) | (4 if bucketed else 0) |
                 (8 if direct else 0))
        _check(self._lib.planb_multi_create(arr, len(fibs), max_batch, flags, C.byref(h)),
               "planb_multi_create")
        self._h = h

    def lookup(self, addr_hi, addr_lo, table, out=None, stream=None):
        """CUDA tensors: addresses int64 (u64 bits), table ids uint8; returns int16 (u16 bits)."""
        import torch
        n = addr_hi.numel()
        if addr_lo.numel() != n or table.numel() != n or table.element_size() != 1:
            raise ValueError("addresses and table ids differ in length, or ids are not bytes")
        if out is None:
            out = torch.empty(n, dtype=torch.int16, device=addr_hi.device)
        _check(self._lib.planb_multi_lookup(self._h, C.c_void_p(addr_hi.data_ptr()),
                                            C.c_void_p(addr_lo.data_ptr()),
                                            C.c_void_p(table.data_ptr()), n,
                                            C.c_void_p(out.data_ptr()), _stream_handle(stream)),
               "planb_multi_lookup")
        return out

    @property
    def captures(self) -> int:
        """Graph captures so far (the first lookup, then changes of buffers or launch shape)."""
        return int(self._lib.planb_multi_captures(self._h))

    @property
    def persistent(self) -> bool:
        """True when the lookups run as the single persistent launch over all tables."""
        rc = self._lib.planb_multi_persistent(self._h)
        if rc < 0:
            _check(rc, "planb_multi_persistent")
        return rc == 1

    @property
    def mode(self) -> str:
        """The form of the last lookup: "direct" (input order, no bucketing), "bucketed" (grouped
        by table, one persistent launch) or "per_table" (also before the first lookup)."""
        rc = self._lib.planb_multi_mode(self._h)
        if rc < 0:
            _check(rc, "planb_multi_mode")
        return self.MODES[rc]

    def lookup_ptr(self, hi_ptr: int, lo_ptr: int, tid_ptr: int, n: int, out_ptr: int, stream=None):
        _check(self._lib.planb_multi_lookup(self._h, C.c_void_p(hi_ptr), C.c_void_p(lo_ptr),
                                            C.c_void_p(tid_ptr), n, C.c_void_p(out_ptr),
                                            _stream_handle(stream)), "planb_multi_lookup")

    def close(self):
        if self._h:
            self._lib.planb_multi_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class ServerOpts(C.Structure):
    _fields_ = [("struct_size", C.c_uint32), ("slots", C.c_uint32), ("max_batch", C.c_uint32),
                ("max_request", C.c_uint32), ("mem_budget", C.c_uint64),
                ("update_period_us", C.c_uint32), ("device", C.c_int32),
                ("multi_flags", C.c_uint32), ("reserved", C.c_uint32 * 5)]


class ServerStats(C.Structure):
    _fields_ = [("requests", C.c_uint64), ("lookups", C.c_uint64), ("batches", C.c_uint64),
                ("updates", C.c_uint64), ("update_batches", C.c_uint64), ("tables", C.c_uint64),
                ("table_bytes", C.c_uint64), ("queued", C.c_uint64), ("p50_us", C.c_double),
                ("p99_us", C.c_double), ("max_us", C.c_double), ("mean_batch", C.c_double),
                ("rebuild_ms_mean", C.c_double), ("last_error", C.c_int32),
                ("reserved", C.c_int32), ("batch_p50_us", C.c_double),
                ("batch_p99_us", C.c_double), ("batch_max_us", C.c_double),
                ("recaptures", C.c_uint64)]


_live_servers = weakref.WeakSet()


@atexit.register
def _close_live_servers():
    # an engine's threads must stop before the CUDA runtime is torn down at process exit
    for srv in list(_live_servers):
        try:
            srv.close()
        except Exception:
            pass


class Server:
    """The serving engine (planb_server): continuous batching of host-buffer requests over tables."""

    def __init__(self, slots: int = 4, max_batch: int = 1 << 18, max_request: int = 1 << 16,
                 mem_budget: int = 0, update_period_us: int = 10_000, device: int | None = None,
                 per_table: bool = False, bucketed: bool = False):
        self._lib = load()
        self._h = None
        o = ServerOpts()
        self._lib.planb_server_opts_default(C.byref(o))
        o.slots, o.max_batch, o.max_request = slots, max_batch, max_request
        o.mem_budget, o.update_period_us = mem_budget, update_period_us
        o.device = -1 if device is None else device
        o.multi_flags = (2 if per_table else 0) | (4 if bucketed else 0)
        h = C.c_void_p()
        _check(self._lib.planb_server_create(C.byref(o), C.byref(h)), "planb_server_create")
        self._h = h
        self.tables = []
        _live_servers.add(self)

    def add_table(self, fib: Fib) -> int:
        tid = C.c_uint32()
        _check(self._lib.planb_server_add_table(self._h, fib._h, C.byref(tid)),
               "planb_server_add_table")
        self.tables.append(fib)
        return tid.value

    def submit(self, table: int, hi: np.ndarray, lo: np.ndarray, out: np.ndarray) -> int:
        """Queues a request; the arrays must stay alive until wait() returns for its ticket."""
        t = C.c_uint64()
        _check(self._lib.planb_server_submit(self._h, table, hi.ctypes.data, lo.ctypes.data,
                                             hi.size, out.ctypes.data, C.byref(t)),
               "planb_server_submit")
        return t.value

    def wait(self, ticket: int, timeout_us: int = 60_000_000):
        _check(self._lib.planb_server_wait(self._h, ticket, timeout_us), "planb_server_wait")

    def update(self, table: int, ins_hi=(), ins_lo=(), ins_len=(), ins_nh=(), wd_hi=(), wd_lo=(),
               wd_len=()):
        ins = np.zeros(len(ins_hi), dtype=ROUTE_DTYPE)
        ins["hi"], ins["lo"], ins["len"], ins["nexthop"] = ins_hi, ins_lo, ins_len, ins_nh
        wd = np.zeros(len(wd_hi), dtype=PREFIX_DTYPE)
        wd["hi"], wd["lo"], wd["len"] = wd_hi, wd_lo, wd_len
        _check(self._lib.planb_server_update(self._h, table, _ptr(ins), ins.size, _ptr(wd),
                                             wd.size), "planb_server_update")

    def stats(self) -> dict:
        s = ServerStats()
        _check(self._lib.planb_server_stats(self._h, C.byref(s)), "planb_server_stats")
        return {f: getattr(s, f) for f, _ in ServerStats._fields_ if f != "reserved"}

    def error_detail(self) -> str:
        buf = C.create_string_buffer(256)
        _check(self._lib.planb_server_error_detail(self._h, buf, 256), "planb_server_error_detail")
        return buf.value.decode(errors="replace")

    def reset_stats(self):
        self._lib.planb_server_reset_stats(self._h)

    def close(self):
        if self._h:
            self._lib.planb_server_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
