"""Autotuner for the lookup configuration of a table.

For a table, it builds the table under each candidate configuration and times ``planb_lookup`` on a
sample batch with CUDA events. A candidate is a node format and fanout (F8X128: 9-ary with 128-bit
keys; F8V7: 9-ary with next hops packed in the leaf lines; F16HI: 17-ary with 64-bit key halves),
a kernel (hybrid / coop), a shared-memory depth, threads per CTA, and a CTA-per-SM cap (together
these set the lookups in flight per SM). Every candidate gives the same results; only speed
differs. The winner is cached in a JSON file keyed by the GPU's name and the table's size class (half
octaves of the interval count), so tables of similar size share one tuning run.
"""
from __future__ import annotations

import json
import math
import os

import numpy as np

from .binding import Fib

DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "planb_gb300_autotune.json")


def size_class(n_intervals: int) -> float:
    return round(math.log2(max(int(n_intervals), 2)) * 2) / 2


# Index (+ directory) bytes a multi-table group's persistent launch stages per CTA; a larger index
# is searched in place there, which is slower than staging a shallower one.
PERSISTENT_STAGE_BYTES = 96 * 1024


def candidates(depth: int, auto_levels: int, persistent: bool = False,
               auto16: int | None = None) -> list[dict]:
    """Candidate option sets around the library's automatic choice (depth and auto_levels of the
    F8X128 layout; auto16 the F16HI layout's automatic index depth, when known). persistent=True
    keeps to the configurations a multi-table group can run in its single persistent launch (the
    hybrid kernel in any format; that launch fixes threads and CTAs per SM, so only the format and
    the index depth vary)."""
    out = []
    if persistent:
        for fmt in ("f8x128", "f8v7"):
            for s in sorted({auto_levels, max(auto_levels - 1, 0)}):
                out.append(dict(format=fmt, kernel="hybrid", smem_levels=s))
        if auto16 is None:
            out.append(dict(format="f16hi", kernel="hybrid", smem_levels=-1))
        else:
            for s in sorted({auto16, max(auto16 - 1, 0)}):
                out.append(dict(format="f16hi", kernel="hybrid", smem_levels=s))
        return out
    for fmt in ("f8x128", "f8v7"):
        for s in sorted({auto_levels, max(auto_levels - 1, 0)}):
            for threads, ctas in ((512, 0), (256, 0), (512, 1)):
                out.append(dict(format=fmt, kernel="hybrid", smem_levels=s, block_threads=threads,
                                ctas_per_sm=ctas))
    out.append(dict(format="f16hi", kernel="hybrid", smem_levels=-1, block_threads=0,
                    ctas_per_sm=0))
    out.append(dict(format="f8x128", kernel="coop", smem_levels=-1, block_threads=256,
                    ctas_per_sm=0))
    out.append(dict(format="f16hi", kernel="coop", smem_levels=-1, block_threads=256,
                    ctas_per_sm=0))
    return out


class Autotuner:
    def __init__(self, cache_path: str | None = DEFAULT_CACHE, warmup: int = 2, reps: int = 5,
                 persistent: bool = False):
        self.persistent = persistent
        self.cache_path = cache_path
        self.warmup = warmup
        self.reps = reps
        self.cache = {}
        if cache_path and os.path.exists(cache_path):
            try:
                with open(cache_path) as f:
                    self.cache = json.load(f)
            except (OSError, ValueError):
                self.cache = {}

    def _key(self, n_intervals: int) -> str:
        import torch
        mode = "|persistent" if self.persistent else ""
        return f"{torch.cuda.get_device_name()}|{size_class(n_intervals)}{mode}"

    def _time(self, fib: Fib, hi, lo, out) -> float:
        import torch
        n = hi.numel()
        s = torch.cuda.current_stream()
        for _ in range(self.warmup):
            fib.lookup_ptr(hi.data_ptr(), lo.data_ptr(), n, out.data_ptr(), s)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(s)
        for _ in range(self.reps):
            fib.lookup_ptr(hi.data_ptr(), lo.data_ptr(), n, out.data_ptr(), s)
        b.record(s)
        b.synchronize()
        return a.elapsed_time(b) / self.reps / 1e3

    def tune(self, hi, lo, ln, nh, sample_hi, sample_lo, device: int | None = None):
        """Times every candidate on the sample (CUDA int64 tensors); returns (best options,
        [(options, lookups/s)]) and records the winner in the cache."""
        import torch
        out = torch.empty(sample_hi.numel(), dtype=torch.int16, device=sample_hi.device)
        with Fib(hi, lo, ln, nh, device=device) as probe:
            st = probe.stats()
        auto16 = None
        if self.persistent:
            with Fib(hi, lo, ln, nh, format="f16hi", kernel="hybrid", device=device) as p16:
                auto16 = p16.stats()["smem_levels"]
        results = []
        for opts in candidates(st["depth"], st["smem_levels"], self.persistent, auto16):
            try:
                with Fib(hi, lo, ln, nh, device=device, **opts) as fib:
                    # the persistent launch would search a larger index in place: leave it out
                    if self.persistent and fib.stats()["smem_bytes"] > PERSISTENT_STAGE_BYTES:
                        continue
                    t = self._time(fib, sample_hi, sample_lo, out)
            except Exception:           # a configuration the table cannot take (e.g. no room)
                continue
            results.append((opts, sample_hi.numel() / t))
        results.sort(key=lambda r: -r[1])
        best = results[0][0]
        self.cache[self._key(st["n_intervals"])] = {"opts": best, "lookups_per_s": results[0][1]}
        self.save()
        return best, results

    def best(self, hi, lo, ln, nh, sample_hi, sample_lo, device: int | None = None) -> dict:
        """The cached choice for this table's size class, tuning on a miss."""
        with Fib(hi, lo, ln, nh, device=device) as probe:
            key = self._key(probe.stats()["n_intervals"])
        hit = self.cache.get(key)
        if hit:
            return dict(hit["opts"])
        return self.tune(hi, lo, ln, nh, sample_hi, sample_lo, device=device)[0]

    def save(self):
        if not self.cache_path:
            return
        try:
            os.makedirs(os.path.dirname(self.cache_path), exist_ok=True)
            tmp = self.cache_path + f".tmp{os.getpid()}"
            with open(tmp, "w") as f:
                json.dump(self.cache, f, indent=1, sort_keys=True)
            os.replace(tmp, self.cache_path)
        except OSError:
            pass
