"""Pins of the CPU oracle (O1 brute force, O2 trie, O3 interval checker) to facts fixed outside it.

Each expected value here comes from the paper's worked example, a closed form, a standard-library
routine (``ipaddress``, ``bisect``) or brute force on a tiny universe — never from the oracle itself
and never from the CUDA path.
"""
import bisect
import ipaddress
import os
import random

import numpy as np
import pytest

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
M64 = (1 << 64) - 1
ALL128 = (1 << 128) - 1


def split(v: int):
    return v >> 64, v & M64


def arrays(prefixes):
    """[(int prefix, len, nh)] -> oracle argument arrays."""
    hi = np.array([p >> 64 for p, _, _ in prefixes], dtype=np.uint64)
    lo = np.array([p & M64 for p, _, _ in prefixes], dtype=np.uint64)
    ln = np.array([L for _, L, _ in prefixes], dtype=np.uint8)
    nh = np.array([h for _, _, h in prefixes], dtype=np.uint16)
    return hi, lo, ln, nh


def addrs(values):
    return (np.array([v >> 64 for v in values], dtype=np.uint64),
            np.array([v & M64 for v in values], dtype=np.uint64))


def both(prefixes, values):
    hi, lo, ln, nh = arrays(prefixes)
    xh, xl = addrs(values)
    b = oracle.brute_lookup(hi, lo, ln, nh, xh, xl, threads=2)
    t = oracle.Trie(hi, lo, ln, nh).lookup(xh, xl, threads=2)
    return b, t


def lpm_ipaddress(prefixes, v):
    """LPM by the standard library: membership of an address in an IPv6Network, longest wins,
    later duplicates win."""
    a = ipaddress.IPv6Address(v)
    best, best_len = 0, -1
    for p, L, h in prefixes:
        net = ipaddress.IPv6Network((p, L), strict=False)
        if a in net and L >= best_len:
            best, best_len = h, L
    return best


# ------------------------------------------------------------------------- worked example

def read_golden(name):
    out = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                k, v = line.split(None, 1)
                out[k] = v
    return out


def test_worked_example_range_and_byte_order():
    g = read_golden("worked_example_2001_db8.txt")
    net = ipaddress.IPv6Network(g["prefix"])
    start = int(ipaddress.IPv6Address(g["start"]))
    end = int(ipaddress.IPv6Address(g["end"]))
    assert int(net.network_address) == start and int(net.broadcast_address) == end
    # the (hi, lo) convention: hi is the first 8 bytes read big-endian
    assert split(start) == (0x20010DB800000000, 0)
    pfx = [(start, net.prefixlen, 7), (0, 0, 3)]
    probes = [start, end, start - 1, end + 1, (start + end) // 2]
    b, t = both(pfx, probes)
    assert list(b) == [7, 7, 3, 3, 7]
    assert list(t) == [7, 7, 3, 3, 7]


# ------------------------------------------------------------------------- closed forms

def test_nested_chain_closed_form():
    """Prefixes of every length 0..128 along one address A: the LPM length of x is the number of
    leading bits x shares with A (128 when x == A)."""
    rng = random.Random(11)
    A = rng.getrandbits(128)
    pfx = [(A, L, L + 1) for L in range(129)]
    probes = [A, 0, ALL128] + [A ^ (1 << (127 - k)) for k in range(128)]
    probes += [rng.getrandbits(128) for _ in range(300)]
    probes += [A ^ rng.getrandbits(128 - k) for k in range(1, 128) for _ in range(2)]
    b, t = both(pfx, probes)
    for v, rb, rt in zip(probes, b, t):
        common = 128 - (A ^ v).bit_length()
        assert rb == common + 1 and rt == common + 1, hex(v)


def test_only_default_and_empty():
    probes = [0, ALL128, 1 << 127, 12345]
    b, t = both([(0, 0, 42)], probes)
    assert set(b) == {42} and set(t) == {42}
    hi = np.zeros(0, np.uint64)
    xh, xl = addrs(probes)
    assert set(oracle.brute_lookup(hi, hi, np.zeros(0, np.uint8), np.zeros(0, np.uint16), xh, xl)) == {0}
    assert set(oracle.Trie(hi, hi, np.zeros(0, np.uint8), np.zeros(0, np.uint16)).lookup(xh, xl)) == {0}


def test_disjoint_prefixes_match_bisect():
    """Disjoint prefixes: the answer is the one range (from ipaddress) that contains x, found by
    bisect over the sorted range starts."""
    rng = random.Random(5)
    nets = set()
    while len(nets) < 300:
        L = rng.choice([16, 24, 32, 40, 48, 56, 64, 96, 128])
        nets.add(ipaddress.IPv6Network((rng.getrandbits(128), L), strict=False))
    nets = sorted(nets, key=lambda n: (int(n.network_address), n.prefixlen))
    disjoint = []
    for n in nets:
        if disjoint and n.overlaps(disjoint[-1]):
            continue
        disjoint.append(n)
    pfx = [(int(n.network_address), n.prefixlen, 1 + i % 4000) for i, n in enumerate(disjoint)]
    starts = [int(n.network_address) for n in disjoint]
    ends = [int(n.broadcast_address) for n in disjoint]
    probes = [0, ALL128]
    for s, e in zip(starts, ends):
        probes += [s, e, max(s - 1, 0), min(e + 1, ALL128), rng.randint(s, e)]
    probes += [rng.getrandbits(128) for _ in range(2000)]
    b, t = both(pfx, probes)
    for v, rb, rt in zip(probes, b, t):
        i = bisect.bisect_right(starts, v) - 1
        want = pfx[i][2] if i >= 0 and v <= ends[i] else 0
        assert rb == want and rt == want


# ------------------------------------------------------------------------- edge cases

def test_edges_top_of_space_and_host_routes():
    pfx = [
        (0xFFFF << 112, 16, 5),          # ffff::/16: its end is 2^128
        (ALL128, 128, 6),                # ffff:...:ffff/128
        (0, 128, 7),                     # ::/128
        (0, 0, 1),                       # default
        (0x2001_0DB8 << 96, 32, 8),      # shared start with the /48 below
        (0x2001_0DB8 << 96, 48, 9),
        ((0x2001_0DB8 << 96) | (1 << 80), 48, 10),   # adjacent /48 (one's end = next start)
    ]
    probes = [0, 1, ALL128, ALL128 - 1, 0xFFFF << 112, (0xFFFF << 112) - 1,
              0x2001_0DB8 << 96, (0x2001_0DB8 << 96) + (1 << 80) - 1, (0x2001_0DB8 << 96) + (1 << 80),
              (0x2001_0DB8 << 96) + (2 << 80), (0x2001_0DB9 << 96) - 1, 0x2001_0DB9 << 96]
    b, t = both(pfx, probes)
    want = [lpm_ipaddress(pfx, v) for v in probes]
    assert list(b) == want and list(t) == want
    assert want[:4] == [7, 1, 6, 5]


def test_duplicates_last_wins_and_host_bits_masked():
    base = 0x2001_0DB8 << 96
    pfx = [(base, 32, 3), (base | 0xABCDEF, 32, 4), (0, 0, 1)]   # same /32, host bits set on the 2nd
    b, t = both(pfx, [base, base + 99])
    assert list(b) == [4, 4] and list(t) == [4, 4]
    pfx = [(base | 0xABCDEF, 32, 4), (base, 32, 3)]
    b, t = both(pfx, [base])
    assert list(b) == [3] and list(t) == [3]


def test_length_above_128_rejected():
    hi, lo, ln, nh = arrays([(0, 129, 1)])
    with pytest.raises(ValueError):
        oracle.brute_lookup(hi, lo, ln, nh, hi, lo)
    with pytest.raises(ValueError):
        oracle.Trie(hi, lo, ln, nh)


# ------------------------------------------------------------------------- toy universe

@pytest.mark.parametrize("seed", [1, 2, 3])
def test_toy_universe_exhaustive(seed):
    """All prefixes live in the top 12 bits (lengths 0..12) plus a few longer ones; every one of the
    4096 top-12-bit classes is probed (at its first, last and a random address), and the result is
    checked against the standard-library LPM, with O1 and O2 agreeing."""
    rng = random.Random(seed)
    pfx = [(0, 0, 1)]
    for _ in range(60):
        L = rng.randint(1, 12)
        pfx.append((rng.getrandbits(12) << 116, L, rng.randint(1, 65535)))
    for _ in range(10):                          # crafted longer prefixes inside the toy space
        L = rng.choice([13, 20, 64, 65, 127, 128])
        pfx.append((rng.getrandbits(128), L, rng.randint(1, 65535)))
    probes = []
    for c in range(4096):
        lo = c << 116
        hi = lo | ((1 << 116) - 1)
        probes += [lo, hi, rng.randint(lo, hi)]
    for p, L, _ in pfx[61:]:
        net = ipaddress.IPv6Network((p, L), strict=False)
        s, e = int(net.network_address), int(net.broadcast_address)
        probes += [s, e, max(s - 1, 0), min(e + 1, ALL128)]
    b, t = both(pfx, probes)
    assert np.array_equal(b, t)
    sample = rng.sample(range(len(probes)), 1500)
    for i in sample:
        assert b[i] == lpm_ipaddress(pfx, probes[i])


def test_o1_equals_o2_on_synthetic_table():
    fib = synth.gen_fib(2000, seed=3, nh_max=4095)
    xh, xl = synth.gen_trace(fib, 50_000, seed=4)
    b = oracle.brute_lookup(fib.hi, fib.lo, fib.len, fib.nh, xh, xl, threads=4)
    t = oracle.Trie(fib.hi, fib.lo, fib.len, fib.nh).lookup(xh, xl, threads=4)
    assert np.array_equal(b, t)
    # the covered share really lands in prefixes, the uniform share mostly on the default
    assert 0.6 < np.mean(b != 0) < 0.8


# ------------------------------------------------------------------------- O3 checker

def iv(items):
    """[(int start, nh)] -> (hi, lo, nh) arrays."""
    return (np.array([s >> 64 for s, _ in items], np.uint64),
            np.array([s & M64 for s, _ in items], np.uint64),
            np.array([h for _, h in items], np.uint16))


def check(pfx, items, merged=False):
    hi, lo, ln, nh = arrays(pfx)
    return oracle.check_intervals(hi, lo, ln, nh, *iv(items), merged=merged)


def test_o3_accepts_hand_built_partition_and_rejects_mistakes():
    A = 0x2001_0DB8 << 96
    pfx = [(A, 32, 7), (0, 0, 3)]
    good = [(0, 3), (A, 7), (A + (1 << 96), 3)]
    assert check(pfx, good) is None
    assert check(pfx, [(0, 3), (A, 7)]) is not None                            # end boundary dropped
    assert check(pfx, [(0, 3), (A, 8), (A + (1 << 96), 3)]) is not None        # wrong next hop
    assert check(pfx, [(0, 3), (A, 7), (A + 5, 7), (A + (1 << 96), 3)]) is not None   # extra boundary
    assert check(pfx, [(1, 3), (A, 7), (A + (1 << 96), 3)]) is not None        # not starting at 0
    assert check(pfx, [(0, 3), (A + (1 << 96), 3), (A, 7)]) is not None        # not sorted
    assert check(pfx, [(0, 3), (A - 1, 7), (A + (1 << 96), 3)]) is not None    # off by one
    assert check(pfx, [(0, 3), (A, 7), (A + (1 << 96) - 1, 3)]) is not None    # inclusive end used


def test_o3_top_of_space_has_no_end_boundary():
    T = 0xFFFF << 112
    pfx = [(T, 16, 5)]
    assert check(pfx, [(0, 0), (T, 5)]) is None
    assert check(pfx, [(0, 0), (T, 5), (ALL128, 5)]) is not None


def test_o3_merge_mode():
    A = 0x2001_0DB8 << 96
    pfx = [(A, 33, 7), (A | (1 << 95), 33, 7), (0, 0, 0)]
    plain = [(0, 0), (A, 7), (A + (1 << 95), 7), (A + (1 << 96), 0)]
    merged = [(0, 0), (A, 7), (A + (1 << 96), 0)]
    assert check(pfx, plain) is None
    assert check(pfx, merged) is not None
    assert check(pfx, merged, merged=True) is None
    assert check(pfx, plain, merged=True) is not None
    assert check(pfx, [(0, 0), (A, 7), (A + (1 << 96), 7)], merged=True) is not None


def test_o3_chain_partition_from_ipaddress():
    """The nested chain along A: the boundaries are the ipaddress ranges' starts and (last + 1)
    values, and each interval's next hop is the standard-library LPM of its first address."""
    rng = random.Random(9)
    A = rng.getrandbits(128)
    pfx = [(A, L, L + 1) for L in range(0, 129, 4)] + [(A, 128, 200)]
    bset = {0}
    for p, L, _ in pfx:
        net = ipaddress.IPv6Network((p, L), strict=False)
        bset.add(int(net.network_address))
        if int(net.broadcast_address) < ALL128:
            bset.add(int(net.broadcast_address) + 1)
    starts = sorted(bset)
    items = [(s, lpm_ipaddress(pfx, s)) for s in starts]
    assert check(pfx, items) is None
    assert len(items) <= 2 * len(pfx) + 1
    bad = list(items)
    k = len(bad) // 2
    bad[k] = (bad[k][0], (bad[k][1] + 1) % 65536)
    assert check(pfx, bad) is not None


def test_o3_interval_count_bound_counts_distinct_prefixes():
    """Section 3.1: N prefixes give at most 2N+1 elementary intervals. N disjoint, non-adjacent
    prefixes with no default reach the bound exactly (each adds its start and its end), which O3
    accepts; an array one entry longer fails on the bound itself, and N counts distinct
    (prefix, length) pairs, so repeating a prefix in the input does not loosen it."""
    A = 0x2001_0DB8 << 96
    pfx = [(A + (2 * j) * (1 << 96), 32, 10 + j) for j in range(3)]
    tight = [(0, 0)]
    for p, L, h in pfx:
        tight += [(p, h), (p + (1 << (128 - L)), 0)]
    assert len(tight) == 2 * len(pfx) + 1
    assert check(pfx, tight) is None
    over = tight + [(ALL128 - 5, 0)]
    msg = check(pfx, over)
    assert msg is not None and msg.startswith("more than 2N+1 intervals")
    msg = check(pfx + [pfx[0], pfx[1]], over)          # five input rows, still N = 3
    assert msg is not None and msg.startswith("more than 2N+1 intervals")
