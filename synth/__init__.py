"""Seeded synthetic inputs for batched IPv6 longest-prefix-match: prefix tables and lookup traces.

This module is shared by the CPU oracle tests and the CUDA path. It draws random numbers and places
prefixes; it contains none of the lookup method's arithmetic (no interval building, no tree, no
longest-match logic).

Randomness is counter-based: draw ``i`` of stream ``s`` under seed ``seed`` is the SplitMix64 output
function (Steele, Lea and Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014) applied
to ``key(seed, s) + (i + 1) * GAMMA``. Any sub-range of a stream can be regenerated independently, so a
trace can be produced in parallel chunks and a sample of it can be rebuilt by index.

Workload recipe (the paper's real FIBs and traces, Table 1 and Section 4, are not available, so these
stand in for them):

* prefix lengths: 45 % /48, 20 % /32, 10 % /40, 10 % /44, 1 % /128 host routes, the remaining 14 %
  uniform over /16../64 (the mix of Table 1, Section 2.1);
* placement: about 70 % of prefixes are roots whose top bits are uniform inside 2000::/3; about 30 %
  are nested uniformly inside an already placed shorter prefix; /128 routes are always nested;
  (prefix, length) duplicates are redrawn;
* next hops uniform in [1, nh_max]; the table ends with a ::/0 default route whose next hop is 0;
* traffic: a fraction ``covered`` of addresses is uniform inside a uniformly chosen prefix (Section 4,
  "Datasets"), the rest uniform over the whole 128-bit space; a locality variant draws the top 64 bits
  from a Zipf(s) law over a set of hot /64 blocks.

Addresses are 128-bit numbers held as two u64 halves: ``hi`` is the first 8 bytes of the address in
network order read big-endian, ``lo`` the last 8 (Section 3.1's example: 2001:db8:: has
hi = 0x20010db800000000, lo = 0).
"""
from __future__ import annotations

import os
from concurrent.futures import ThreadPoolExecutor
from dataclasses import dataclass

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
ALL = np.uint64(0xFFFFFFFFFFFFFFFF)

# stream tags (distinct streams for distinct purposes)
S_LEN, S_NEST, S_PARENT, S_HI, S_LO, S_NH, S_REDRAW = 1, 2, 3, 4, 5, 6, 7
T_KIND, T_PICK, T_HI, T_LO, T_HOT, T_ZIPF = 11, 12, 13, 14, 15, 16
U_KIND, U_HI, U_LO, U_LEN, U_NH, U_PICK = 21, 22, 23, 24, 25, 26


def _mix64(z: np.ndarray) -> np.ndarray:
    """SplitMix64 output function on a uint64 array (wrapping arithmetic)."""
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def _key(seed: int, stream: int) -> np.uint64:
    z = np.array([(seed * 0x9E3779B97F4A7C15 + stream * 0xD1B54A32D192ED03) & 0xFFFFFFFFFFFFFFFF],
                 dtype=np.uint64)
    return _mix64(z)[0]


def u64(seed: int, stream: int, start: int, count: int) -> np.ndarray:
    """Draws ``start .. start+count-1`` of a counter-based stream, as uint64."""
    idx = np.arange(start + 1, start + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return _mix64(_key(seed, stream) + idx * GAMMA)


def unit(u: np.ndarray) -> np.ndarray:
    """uint64 draws -> float64 uniform in [0, 1) (top 53 bits)."""
    return (u >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def below(u: np.ndarray, n) -> np.ndarray:
    """uint64 draws -> integers uniform in [0, n) (n may be an array)."""
    r = np.floor(unit(u) * np.asarray(n, dtype=np.float64)).astype(np.int64)
    return np.minimum(r, np.asarray(n, dtype=np.int64) - 1)


def top_mask(length: np.ndarray):
    """(mask_hi, mask_lo) with the top ``length`` bits of a 128-bit value set, for length in [0, 128]."""
    L = np.asarray(length, dtype=np.int64)
    sh_hi = np.clip(64 - L, 0, 63).astype(np.uint64)
    sh_lo = np.clip(128 - L, 0, 63).astype(np.uint64)
    mhi = np.where(L >= 64, ALL, np.where(L <= 0, np.uint64(0), ALL << sh_hi))
    mlo = np.where(L >= 128, ALL, np.where(L <= 64, np.uint64(0), ALL << sh_lo))
    return mhi.astype(np.uint64), mlo.astype(np.uint64)


def bit_range_mask(a: np.ndarray, b: np.ndarray):
    """(mask_hi, mask_lo) with bit positions [a, b) set, counting from the most significant bit."""
    ah, al = top_mask(a)
    bh, bl = top_mask(b)
    return bh & ~ah, bl & ~al


# -------------------------------------------------------------------------------------------- FIBs

LENGTH_MIX = ((48, 0.45), (32, 0.20), (40, 0.10), (44, 0.10), (128, 0.01))  # rest: uniform /16../64


@dataclass
class Fib:
    """A prefix table: arrays of equal length n (the last entry is ::/0 when ``default`` was asked)."""
    hi: np.ndarray   # uint64
    lo: np.ndarray   # uint64
    len: np.ndarray  # uint8
    nh: np.ndarray   # uint16
    seed: int

    @property
    def n(self) -> int:
        return int(self.hi.shape[0])


def sample_lengths(seed: int, n: int, start: int = 0, stream: int = S_LEN) -> np.ndarray:
    u = unit(u64(seed, stream, 2 * start, 2 * n)).reshape(n, 2)
    f = u[:, 0]
    out = np.empty(n, dtype=np.int64)
    lo = 0.0
    assigned = np.zeros(n, dtype=bool)
    for L, p in LENGTH_MIX:
        sel = (f >= lo) & (f < lo + p)
        out[sel] = L
        assigned |= sel
        lo += p
    rest = ~assigned
    out[rest] = 16 + np.minimum((u[rest, 1] * 49).astype(np.int64), 48)
    return out


def gen_fib(n: int, seed: int, nh_max: int = 255, nested_frac: float = 0.30,
            default: bool = True, root_prefix_bits: int = 3, root_prefix_value: int = 0x1) -> Fib:
    """``n`` distinct synthetic prefixes (plus ::/0 -> 0 when ``default``), seeded.

    Roots get their top ``root_prefix_bits`` bits equal to ``root_prefix_value`` (2000::/3 by default);
    a root too short to leave 12 free bits inside that region is placed in 2000::/3 instead.
    """
    lens = sample_lengths(seed, n)
    nested = unit(u64(seed, S_NEST, 0, n)) < nested_frac
    nested |= lens == 128
    hi = np.zeros(n, dtype=np.uint64)
    lo = np.zeros(n, dtype=np.uint64)
    placed = np.zeros(n, dtype=bool)
    seen: set = set()
    order_lens = np.unique(lens)
    rhi_all = u64(seed, S_HI, 0, n)
    rlo_all = u64(seed, S_LO, 0, n)
    rpar_all = u64(seed, S_PARENT, 0, n)
    redraw_ctr = 0
    rp_hi = np.uint64((root_prefix_value << (64 - root_prefix_bits)) & 0xFFFFFFFFFFFFFFFF)
    g_bits, g_hi = 3, np.uint64(0x2000000000000000)       # 2000::/3, for roots shorter than the region
    for L in order_lens:
        idx = np.nonzero(lens == L)[0]
        cand = np.nonzero(placed & (lens < L))[0]
        want_nest = nested[idx] & (cand.size > 0)
        pend = idx
        rhi, rlo, rpar = rhi_all[idx], rlo_all[idx], rpar_all[idx]
        nest = want_nest
        for attempt in range(64):
            k = pend.size
            Lk = np.full(k, L, dtype=np.int64)
            # roots: fixed top bits, random bits in [root_prefix_bits, L)
            rb, rh = (root_prefix_bits, rp_hi) if L >= root_prefix_bits + 12 else (g_bits, g_hi)
            mh, ml = bit_range_mask(np.full(k, rb), Lk)
            ahi = (rhi & mh) | rh
            alo = rlo & ml
            if cand.size:
                par = cand[below(rpar, cand.size)]
                plen = lens[par]
                nmh, nml = bit_range_mask(plen, Lk)
                nhi = hi[par] | (rhi & nmh)
                nlo = lo[par] | (rlo & nml)
                ahi = np.where(nest, nhi, ahi)
                alo = np.where(nest, nlo, alo)
            tm_h, tm_l = top_mask(Lk)
            ahi &= tm_h
            alo &= tm_l
            ok = np.ones(k, dtype=bool)
            for j in range(k):
                key = (int(ahi[j]), int(alo[j]), int(L))
                if key in seen:
                    ok[j] = False
                else:
                    seen.add(key)
            hi[pend[ok]] = ahi[ok]
            lo[pend[ok]] = alo[ok]
            placed[pend[ok]] = True
            if ok.all():
                break
            bad = ~ok
            pend, nest = pend[bad], nest[bad]
            kk = pend.size
            d = u64(seed, S_REDRAW, redraw_ctr, 3 * kk).reshape(kk, 3)
            redraw_ctr += 3 * kk
            rhi, rlo, rpar = d[:, 0], d[:, 1], d[:, 2]
        else:
            raise RuntimeError(f"could not place {pend.size} distinct /{L} prefixes")
    nh = (1 + below(u64(seed, S_NH, 0, n), nh_max)).astype(np.uint16)
    ln = lens.astype(np.uint8)
    if default:
        hi = np.concatenate([hi, np.zeros(1, np.uint64)])
        lo = np.concatenate([lo, np.zeros(1, np.uint64)])
        ln = np.concatenate([ln, np.zeros(1, np.uint8)])
        nh = np.concatenate([nh, np.zeros(1, np.uint16)])
    return Fib(hi=hi, lo=lo, len=ln, nh=nh, seed=seed)


# ------------------------------------------------------------------------------------------ traces

def _trace_chunk(fib_hi, fib_lo, fib_len, n_pick, seed, start, count, covered):
    kind = unit(u64(seed, T_KIND, start, count)) < covered
    rhi = u64(seed, T_HI, start, count)
    rlo = u64(seed, T_LO, start, count)
    if n_pick > 0:
        p = below(u64(seed, T_PICK, start, count), n_pick)
        mh, ml = top_mask(fib_len[p].astype(np.int64))
        chi = (fib_hi[p] & mh) | (rhi & ~mh)
        clo = (fib_lo[p] & ml) | (rlo & ~ml)
        rhi = np.where(kind, chi, rhi)
        rlo = np.where(kind, clo, rlo)
    return rhi, rlo


def gen_trace(fib: Fib, n: int, seed: int, covered: float = 0.70, out_hi: np.ndarray | None = None,
              out_lo: np.ndarray | None = None, start: int = 0, threads: int | None = None,
              chunk: int = 1 << 21):
    """``n`` lookup addresses (hi, lo uint64), drawn ``start .. start+n-1`` of the trace stream.

    A fraction ``covered`` is uniform inside a uniformly chosen non-default prefix, the rest uniform over
    all 2^128 addresses. Deterministic for a given (fib, seed) whatever the chunking or ``start``.
    """
    pick = fib.len > 0
    fh, fl, fn = fib.hi[pick], fib.lo[pick], fib.len[pick]
    if out_hi is None:
        out_hi = np.empty(n, dtype=np.uint64)
    if out_lo is None:
        out_lo = np.empty(n, dtype=np.uint64)
    threads = threads or min(16, os.cpu_count() or 1)

    def work(c0):
        c = min(chunk, n - c0)
        h, l = _trace_chunk(fh, fl, fn, fh.size, seed, start + c0, c, covered)
        out_hi[c0:c0 + c] = h
        out_lo[c0:c0 + c] = l

    starts = range(0, n, chunk)
    if threads > 1 and n > chunk:
        with ThreadPoolExecutor(threads) as ex:
            list(ex.map(work, starts))
    else:
        for c0 in starts:
            work(c0)
    return out_hi, out_lo


def gen_trace_zipf(fib: Fib, n: int, seed: int, hot: int = 100_000, s: float = 1.1,
                   out_hi: np.ndarray | None = None, out_lo: np.ndarray | None = None,
                   threads: int | None = None, chunk: int = 1 << 21):
    """Locality-skewed trace: top 64 bits from ``hot`` hot /64 blocks ranked by Zipf(s); low 64 uniform.

    The hot blocks are the top halves of ``hot`` covered addresses (uniform inside random prefixes).
    Ranks are sampled by inverse CDF over the Zipf probabilities.
    """
    hot_hi, _ = gen_trace(fib, hot, seed ^ 0x5A5A5A5A, covered=1.0, threads=1)
    w = 1.0 / np.power(np.arange(1, hot + 1, dtype=np.float64), s)
    cdf = np.cumsum(w)
    cdf /= cdf[-1]
    if out_hi is None:
        out_hi = np.empty(n, dtype=np.uint64)
    if out_lo is None:
        out_lo = np.empty(n, dtype=np.uint64)
    threads = threads or min(16, os.cpu_count() or 1)

    def work(c0):
        c = min(chunk, n - c0)
        r = np.searchsorted(cdf, unit(u64(seed, T_ZIPF, c0, c)), side="right")
        r = np.minimum(r, hot - 1)
        out_hi[c0:c0 + c] = hot_hi[r]
        out_lo[c0:c0 + c] = u64(seed, T_LO, c0, c)

    starts = range(0, n, chunk)
    if threads > 1 and n > chunk:
        with ThreadPoolExecutor(threads) as ex:
            list(ex.map(work, starts))
    else:
        for c0 in starts:
            work(c0)
    return out_hi, out_lo


# ------------------------------------------------------------------------------- route updates

def gen_updates(fib: Fib, n: int, seed: int, withdraw_frac: float = 0.5, nh_max: int = 4095,
                start: int = 0):
    """A batch of ``n`` route changes against ``fib``: withdraws of existing prefixes and inserts of new
    (or modified) ones, lengths from the same mix. Returns (ins_hi, ins_lo, ins_len, ins_nh, wd_hi,
    wd_lo, wd_len)."""
    kind = unit(u64(seed, U_KIND, start, n)) < withdraw_frac
    nw = int(kind.sum())
    ni = n - nw
    pick = fib.len > 0
    cand = np.nonzero(pick)[0]
    w = cand[below(u64(seed, U_PICK, start, nw), max(cand.size, 1))] if nw and cand.size else \
        np.zeros(0, dtype=np.int64)
    lens = sample_lengths(seed, ni, start=start, stream=U_LEN)
    rhi = u64(seed, U_HI, start, ni)
    rlo = u64(seed, U_LO, start, ni)
    # inserts are nested inside a random existing prefix when one is shorter, else placed in 2000::/3
    par = cand[below(u64(seed, U_PICK, start + n, ni), max(cand.size, 1))] if cand.size else None
    if par is not None:
        plen = fib.len[par].astype(np.int64)
        inside = plen < lens
        mh, ml = bit_range_mask(np.where(inside, plen, 3), lens)
        base_hi = np.where(inside, fib.hi[par], np.uint64(0x2000000000000000))
        base_lo = np.where(inside, fib.lo[par], np.uint64(0))
    else:
        mh, ml = bit_range_mask(np.full(ni, 3), lens)
        base_hi = np.full(ni, np.uint64(0x2000000000000000))
        base_lo = np.zeros(ni, dtype=np.uint64)
    tm_h, tm_l = top_mask(lens)
    ihi = (base_hi | (rhi & mh)) & tm_h
    ilo = (base_lo | (rlo & ml)) & tm_l
    inh = (1 + below(u64(seed, U_NH, start, ni), nh_max)).astype(np.uint16)
    return (ihi, ilo, lens.astype(np.uint8), inh,
            fib.hi[w].copy(), fib.lo[w].copy(), fib.len[w].copy())


# ---------------------------------------------------------------------------- multi-table (VRF)

def gen_vrf_workload(n_tables: int, n: int, seed: int, min_prefixes: int = 1000,
                     max_prefixes: int = 300_000, nh_max: int = 4095):
    """``n_tables`` tables whose sizes are log-uniform over [min_prefixes, max_prefixes] (each built
    like ``gen_fib``, with its own seed) and a trace of ``n`` addresses, each tagged with a u8 table
    id drawn proportional to table size; every address follows its table's traffic mix.

    Returns (sizes, fibs, tid, hi, lo). Sizes and ids come from numpy's seeded PCG64 stream (no
    lookup arithmetic here either)."""
    rng = np.random.default_rng(seed)
    sizes = np.exp(rng.uniform(np.log(min_prefixes), np.log(max_prefixes), n_tables)).astype(int)
    fibs = [gen_fib(int(sz), seed=seed + 1000 + t, nh_max=nh_max) for t, sz in enumerate(sizes)]
    p = sizes / sizes.sum()
    tid = rng.choice(n_tables, size=n, p=p).astype(np.uint8)
    hi = np.empty(n, np.uint64)
    lo = np.empty(n, np.uint64)
    for t, f in enumerate(fibs):
        idx = np.nonzero(tid == t)[0]
        h, l = gen_trace(f, idx.size, seed=seed + 2000 + t)
        hi[idx], lo[idx] = h, l
    return sizes, fibs, tid, hi, lo
