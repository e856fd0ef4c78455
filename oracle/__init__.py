"""CPU oracle for batched IPv6 longest-prefix-match — TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may import this
package. It shares no code with the CUDA lookup library (``paper_2604_14650_gb300``) and neither imports
the other; both take their inputs from ``synth``.

It wraps ``planb_oracle.c`` (plain C, compiled with gcc into ``oracle/_build/liboracle.so``):

* ``brute_lookup`` (O1): scan of every prefix per address — the plain LPM definition (Section 3.1:
  the longest prefix whose top bits equal the address's gives the next hop; no match gives 0).
* ``Trie`` (O2): binary trie walked MSB first, remembering the last next hop seen.
* ``check_intervals`` (O3): the elementary-interval invariants of Section 3.1 (partition of the
  128-bit space, at most 2N+1 intervals, every prefix boundary is a boundary, every point of an
  interval has that interval's LPM next hop).

Every function is exact integer work; there is no tolerance anywhere.
"""
from __future__ import annotations

import ctypes as C
import os
import platform
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "planb_oracle.c")
_OUT = os.path.join(_HERE, "_build", platform.machine(), "liboracle.so")
_lib = None

_u64p = np.ctypeslib.ndpointer(dtype=np.uint64, flags="C_CONTIGUOUS")
_u16p = np.ctypeslib.ndpointer(dtype=np.uint16, flags="C_CONTIGUOUS")
_u8p = np.ctypeslib.ndpointer(dtype=np.uint8, flags="C_CONTIGUOUS")


def build(force: bool = False) -> str:
    """Compiles liboracle.so with gcc (no-op when it is newer than the source)."""
    os.makedirs(os.path.dirname(_OUT), exist_ok=True)
    if (not force and os.path.exists(_OUT)
            and os.path.getmtime(_OUT) >= os.path.getmtime(_SRC)):
        return _OUT
    tmp = _OUT + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-pthread",
                           "-o", tmp, _SRC])
    os.replace(tmp, _OUT)
    return _OUT


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        L = _lib
        L.orc_brute_lookup.argtypes = [C.c_size_t, _u64p, _u64p, _u8p, _u16p, C.c_size_t, _u64p,
                                       _u64p, _u16p, C.c_int]
        L.orc_brute_lookup.restype = C.c_int
        L.orc_trie_new.argtypes = [C.c_size_t, _u64p, _u64p, _u8p, _u16p]
        L.orc_trie_new.restype = C.c_void_p
        L.orc_trie_free.argtypes = [C.c_void_p]
        L.orc_trie_free.restype = None
        L.orc_trie_nodes.argtypes = [C.c_void_p]
        L.orc_trie_nodes.restype = C.c_size_t
        L.orc_trie_lookup.argtypes = [C.c_void_p, C.c_size_t, _u64p, _u64p, _u16p, C.c_int]
        L.orc_trie_lookup.restype = C.c_int
        L.orc_check_intervals.argtypes = [C.c_size_t, _u64p, _u64p, _u8p, _u16p, C.c_size_t, _u64p,
                                          _u64p, _u16p, C.c_int, C.c_char_p, C.c_size_t]
        L.orc_check_intervals.restype = C.c_int
    return _lib


def _prefixes(hi, lo, ln, nh):
    hi = np.ascontiguousarray(hi, dtype=np.uint64)
    lo = np.ascontiguousarray(lo, dtype=np.uint64)
    ln = np.ascontiguousarray(ln, dtype=np.uint8)
    nh = np.ascontiguousarray(nh, dtype=np.uint16)
    if not (hi.shape == lo.shape == ln.shape == nh.shape):
        raise ValueError("prefix arrays differ in length")
    return hi, lo, ln, nh


def threads_default() -> int:
    return os.cpu_count() or 1


def brute_lookup(hi, lo, ln, nh, xhi, xlo, threads: int | None = None) -> np.ndarray:
    """O1: next hop of every address by scanning every prefix."""
    hi, lo, ln, nh = _prefixes(hi, lo, ln, nh)
    xhi = np.ascontiguousarray(xhi, dtype=np.uint64)
    xlo = np.ascontiguousarray(xlo, dtype=np.uint64)
    out = np.empty(xhi.shape[0], dtype=np.uint16)
    rc = lib().orc_brute_lookup(hi.size, hi, lo, ln, nh, xhi.size, xhi, xlo, out,
                                threads or threads_default())
    if rc < 0:
        raise ValueError("prefix length above 128")
    return out


class Trie:
    """O2: binary trie over the prefix table (input order; a later duplicate overwrites)."""

    def __init__(self, hi, lo, ln, nh):
        hi, lo, ln, nh = _prefixes(hi, lo, ln, nh)
        self._h = lib().orc_trie_new(hi.size, hi, lo, ln, nh)
        if not self._h:
            raise ValueError("trie build failed (length above 128 or out of memory)")

    @property
    def nodes(self) -> int:
        return int(lib().orc_trie_nodes(self._h))

    def lookup(self, xhi, xlo, threads: int | None = None, out: np.ndarray | None = None):
        xhi = np.ascontiguousarray(xhi, dtype=np.uint64)
        xlo = np.ascontiguousarray(xlo, dtype=np.uint64)
        if out is None:
            out = np.empty(xhi.shape[0], dtype=np.uint16)
        self.last_threads = lib().orc_trie_lookup(self._h, xhi.size, xhi, xlo, out,
                                                  threads or threads_default())
        return out

    def close(self):
        if getattr(self, "_h", None):
            lib().orc_trie_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def check_intervals(hi, lo, ln, nh, start_hi, start_lo, start_nh, merged: bool = False):
    """O3: returns None when the interval array satisfies every invariant, else the failure message."""
    hi, lo, ln, nh = _prefixes(hi, lo, ln, nh)
    shi = np.ascontiguousarray(start_hi, dtype=np.uint64)
    slo = np.ascontiguousarray(start_lo, dtype=np.uint64)
    snh = np.ascontiguousarray(start_nh, dtype=np.uint16)
    buf = C.create_string_buffer(256)
    rc = lib().orc_check_intervals(hi.size, hi, lo, ln, nh, shi.size, shi, slo, snh, int(merged),
                                   buf, 256)
    return None if rc == 0 else buf.value.decode()
