"""Host-side build steps (a1-a4) of libplanb, checked on the CPU against the oracle's interval
invariants (O3) and the paper's closed forms; plus the exported C ABI. No GPU is used."""
import ctypes
import re
import os

import numpy as np
import pytest

import oracle
import synth
import paper_2604_14650_gb300 as pb

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built():
    pb.build()


def test_library_exports_every_declared_symbol():
    hdr = open(os.path.join(ROOT, "include", "planb.h")).read()
    names = set(re.findall(r"^\s*(?:[\w\s\*]+?)\b(planb_\w+)\s*\(", hdr, re.M))
    assert {"planb_build", "planb_lookup", "planb_update", "planb_destroy"} <= names
    for variant in ("libplanb.so", "libplanb_checked.so"):
        lib = ctypes.CDLL(pb.library_path(variant))
        for n in sorted(names):
            assert hasattr(lib, n), (variant, n)
    assert pb.version() >> 16 == 1


@pytest.mark.parametrize("n,seed,merge", [(0, 1, False), (1, 2, False), (50, 3, False),
                                          (1000, 4, False), (1000, 5, True), (20000, 6, False)])
def test_intervals_satisfy_oracle_invariants(n, seed, merge):
    fib = synth.gen_fib(n, seed=seed, nh_max=4095 if n > 1000 else 3)
    sh, sl, snh = pb.intervals(fib.hi, fib.lo, fib.len, fib.nh, merge=merge)
    msg = oracle.check_intervals(fib.hi, fib.lo, fib.len, fib.nh, sh, sl, snh, merged=merge)
    assert msg is None, msg


def test_intervals_edge_tables():
    M = (1 << 64) - 1
    cases = [
        # ffff::/16 (end = 2^128), ::/128 and ffff..ff/128, duplicates with host bits, shared starts
        [(0xFFFF << 48, 0, 16, 5), (0, 0, 128, 7), (M, M, 128, 6), (0x20010DB8 << 32, 0, 32, 3),
         (0x20010DB8 << 32, 0xABC, 32, 4), (0x20010DB8 << 32, 0, 48, 9), (0, 0, 0, 1)],
        # a full nested chain /0 .. /128 along one address
        [(0x20010DB812345678, 0x9ABCDEF012345678, L, L + 1) for L in range(129)],
        # no default route, adjacent prefixes
        [(0x2001 << 48, 0, 16, 1), (0x2002 << 48, 0, 16, 2), (0x2003 << 48, 0, 17, 3)],
    ]
    for pf in cases:
        hi = np.array([p[0] for p in pf], np.uint64)
        lo = np.array([p[1] for p in pf], np.uint64)
        ln = np.array([p[2] for p in pf], np.uint8)
        nh = np.array([p[3] for p in pf], np.uint16)
        for merge in (False, True):
            iv = pb.intervals(hi, lo, ln, nh, merge=merge)
            assert oracle.check_intervals(hi, lo, ln, nh, *iv, merged=merge) is None


def test_length_above_128_rejected():
    with pytest.raises(pb.PlanbError):
        pb.intervals(np.zeros(1, np.uint64), np.zeros(1, np.uint64), np.array([129], np.uint8),
                     np.ones(1, np.uint16))


# ---------------------------------------------------------------- Section 3.2 layout arithmetic

def test_level_start_closed_form_and_listing_recurrence():
    for k in (2, 4, 8, 16):
        b = k + 1
        info = pb.layout_info(k, 10, depth=7)
        for d in range(7):
            assert info["level_start"][d] == k * (b ** d - 1) // (b - 1)
            assert info["level_start"][d] == b ** d - 1 if k == b - 1 else True
        # Listing 1's recurrence i' = (k+1) i + (c+1) k gives child_start(d, j, c)
        for d in range(5):
            for j in (0, 1, b ** d - 1):
                i = info["level_start"][d] + j * k
                for c in range(b):
                    assert (k + 1) * i + (c + 1) * k == pb.child_index(k, d, j, c)
                    assert pb.child_index(k, d, j, c) == info["level_start"][d + 1] + (j * b + c) * k


def test_capacity_figures_of_section_3_2():
    five = pb.layout_info(8, 1, depth=6)        # 5 internal levels + the leaf level
    assert five["leaf_capacity"] == 59_049
    assert five["key_capacity"] == 472_392
    # the paper prints 6,560 internal nodes; the sum 9^0 + .. + 9^4 is 7,381 (6,560 = 9^4 - 1)
    assert five["internal_nodes"] == 7_381
    assert 9 ** 4 - 1 == 6_560
    # with 64-byte nodes of 8-byte keys: 0.47 MB internal ("0.45 MB"), 3.6 MiB of leaves
    assert abs(five["internal_nodes"] * 64 / 1e6 - 0.47) < 0.01
    assert abs(five["leaf_capacity"] * 64 / 2 ** 20 - 3.6) < 0.01
    six = pb.layout_info(8, 1, depth=7)
    assert six["key_capacity"] == 4_251_528 > 4_200_000
    # automatic depth: smallest D with k * b^(D-1) >= keys
    assert pb.layout_info(8, 472_392)["depth"] == 6
    assert pb.layout_info(8, 472_393)["depth"] == 7
    assert pb.layout_info(8, 8)["depth"] == 1 and pb.layout_info(8, 9)["depth"] == 2
    assert pb.layout_info(16, 16 * 17 ** 3)["depth"] == 4
