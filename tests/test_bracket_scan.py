"""The GPU builder's replacement for Algorithm 2's stack, restated in numpy and checked on the CPU.

The device builder finds the top of the stack after every event without a stack: the nesting depth
is a prefix sum of +1 (start) / -1 (end), and the top after event e is the latest start s <= e whose
depth equals e's. This module walks the same steps (stable sorts, prefix sum, depth grouping,
segmented running maximum) with numpy and requires the result to pass the oracle's interval checker
and to equal the host builder's intervals (planb_intervals, no GPU) on seeded and degenerate tables.
It checks the reading, not the CUDA code (tests/test_gpu_builder.py does that on the GPU).
"""
import numpy as np
import pytest

import oracle
import synth

pb = pytest.importorskip("paper_2604_14650_gb300")

U = np.uint64
M64 = (1 << 64) - 1


def bracket_intervals(hi, lo, ln, nh, merge):
    L = np.asarray(ln, np.int64)
    mh, ml = synth.top_mask(L)
    h, l = np.asarray(hi, U) & mh, np.asarray(lo, U) & ml
    n = h.size
    # a1: (prefix, len, input order), last of each (prefix, len) run
    order = np.arange(n)
    for key in (L, l, h):
        order = order[np.argsort(key[order], kind="stable")]
    keep = np.ones(n, bool)
    if n:
        a, b = order[:-1], order[1:]
        keep[:-1] = (h[a] != h[b]) | (l[a] != l[b]) | (L[a] != L[b])
    sel = order[keep]
    ch, cl, cL, cn = h[sel], l[sel], L[sel], np.asarray(nh, np.uint16)[sel]
    # a2: events 2j (start) and 2j+1 (end below 2^128), sorted by (address, kind, length)
    N = sel.size
    eh, el = np.zeros(2 * N, U), np.zeros(2 * N, U)
    ek = np.zeros(2 * N, np.int64)
    valid = np.zeros(2 * N, bool)
    for j in range(N):
        p = (int(ch[j]) << 64) | int(cl[j])
        eh[2 * j], el[2 * j], ek[2 * j], valid[2 * j] = ch[j], cl[j], 256 | int(cL[j]), True
        e = (p + (1 << (128 - int(cL[j])))) % (1 << 128) if cL[j] > 0 else 0
        eh[2 * j + 1], el[2 * j + 1], ek[2 * j + 1] = e >> 64, e & M64, int(cL[j])
        valid[2 * j + 1] = cL[j] > 0 and e != 0
    ev = np.nonzero(valid)[0]
    for key in (ek, el, eh):
        ev = ev[np.argsort(key[ev], kind="stable")]
    E = ev.size
    # a3: depth, grouping by depth, segmented running max of start positions
    depth = np.cumsum(np.where(ek[ev] >> 8, 1, -1))
    gpos = np.argsort(depth, kind="stable")
    top = np.zeros(E, np.int64)
    run = 0
    for i in range(E):
        p = gpos[i]
        v = p + 1 if ek[ev[p]] >> 8 else 0
        run = v if (i == 0 or depth[gpos[i]] != depth[gpos[i - 1]]) else max(run, v)
        top[p] = run
    sh, sl, sn = [], [], []
    for i in range(E):
        a = ev[i]
        if i + 1 < E and eh[a] == eh[ev[i + 1]] and el[a] == el[ev[i + 1]]:
            continue                       # not the last event at this address
        v = int(cn[ev[top[i] - 1] >> 1]) if depth[i] > 0 and top[i] > 0 else 0
        sh.append(int(eh[a]))
        sl.append(int(el[a]))
        sn.append(v)
    if not sh or sh[0] != 0 or sl[0] != 0:
        sh, sl, sn = [0] + sh, [0] + sl, [0] + sn
    out = [(a, b, c) for i, (a, b, c) in enumerate(zip(sh, sl, sn))
           if i == 0 or not merge or c != sn[i - 1]]
    return (np.array([o[0] for o in out], U), np.array([o[1] for o in out], U),
            np.array([o[2] for o in out], np.uint16))


def arrays(h, l, L, n):
    return (np.array(h, U), np.array(l, U), np.array(L, np.uint8), np.array(n, np.uint16))


EDGE = {
    "empty": arrays([], [], [], []),
    "default_only": arrays([0], [0], [0], [7]),
    "top_128": arrays([M64], [M64], [128], [3]),
    "zero_128": arrays([0], [0], [128], [3]),
    "duplicates": arrays([0x20010DB800000000] * 3, [0] * 3, [32] * 3, [1, 2, 3]),
    "nested_same_start": arrays([0x2001 << 48] * 3, [0] * 3, [16, 32, 48], [1, 2, 3]),
    "nested_same_end": arrays([0x2001FFFF00000000, 0x2001FFFFFFFF0000, 0x2001 << 48], [0] * 3,
                              [32, 48, 16], [1, 2, 3]),
    "host_bits": arrays([0x2001FFFFFFFFFFFF], [0xFFFF], [16], [9]),
}


def random_nested(seed, n=1500):
    r = np.random.default_rng(seed)
    hi = r.integers(0, 2**63, size=n, dtype=U) * U(2)
    lo = r.integers(0, 2**63, size=n, dtype=U)
    idx = r.integers(0, n, size=n // 2)
    hi[: n // 2], lo[: n // 2] = hi[idx], lo[idx]
    return hi, lo, r.integers(0, 129, size=n).astype(np.uint8), \
        r.integers(0, 6, size=n).astype(np.uint16)


def all_cases():
    c = dict(EDGE)
    c["fib"] = (lambda f: (f.hi, f.lo, f.len, f.nh))(synth.gen_fib(2000, seed=5))
    c["nested"] = random_nested(6)
    return c


CASES = all_cases()


@pytest.mark.parametrize("name", sorted(CASES))
@pytest.mark.parametrize("merge", [False, True])
def test_bracket_scan_gives_the_stack_result(name, merge):
    h, l, L, n = CASES[name]
    got = bracket_intervals(h, l, L, n, merge)
    assert oracle.check_intervals(h, l, L, n, *got, merged=merge) is None
    want = pb.intervals(h, l, L, n, merge)
    for x, y in zip(got, want):
        assert np.array_equal(x, y)


def test_hand_worked_nesting():
    """2001::/16 (next hop 1) holding 2001:1::/32 (next hop 2): after the /32 ends the /16 is on top
    again. A running maximum over starts of every depth would answer 2 there; grouping by depth
    answers 1. Worked by hand: depths 1, 2, 1, 0 after the four events."""
    got = bracket_intervals(*arrays([0x2001 << 48, 0x2001000100000000], [0, 0], [16, 32], [1, 2]),
                            False)
    assert [int(x) for x in got[0]] == [0, 0x2001 << 48, 0x2001000100000000, 0x2001000200000000,
                                        0x2002 << 48]
    assert list(got[1]) == [0] * 5
    assert list(got[2]) == [0, 1, 2, 1, 0]
