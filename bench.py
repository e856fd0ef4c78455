#!/usr/bin/env python3
"""Benchmark of batched IPv6 longest-prefix-match on GB300 (PlanB linearized B+-tree).

Workload (default): a 200,000-prefix synthetic backbone FIB (BGP-like length mix, ~30 % nested,
1 % /128, next hops in [1, 4095], ::/0 -> 0) and 2^28 lookup addresses per GPU (70 % uniform inside
a random prefix, 30 % uniform over the 128-bit space). One step = one planb_lookup over all 2^28
device-resident addresses: key ingest, tree descent, next-hop gather and result store (hot-path
steps a5-a10). The 4 GiB key stream is larger than L2, so no flush is needed between steps. The
table is built as F16HI with the hybrid kernel (the fastest form at this size; ``--format``
chooses another); the ablation block times every other form on the same table and addresses.

Prints ONE JSON line on rank 0. ``--impl reference`` times the CPU oracle (binary trie) instead.
Multi-GPU (torchrun, one rank per GPU): each rank looks up its own 2^28 addresses against a replica
of the table (weak scaling; no collective on the data path).
"""
from __future__ import annotations

import argparse
import csv
import hashlib
import io
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "B lookups/s on 200k-prefix FIB, learned vs plain tree; p99 batch latency"
UNIT = "B lookups/s"
HBM_BYTES_PER_LOOKUP = 18          # 16-byte address in, 2-byte next hop out


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="planb", choices=["planb", "reference"])
    ap.add_argument("--prefixes", type=int, default=200_000)
    ap.add_argument("--lookups", type=int, default=1 << 28)
    # the headline configuration: 16-key leaves with the index over them (fastest at 200k prefixes)
    ap.add_argument("--format", default="f16hi", choices=["f8x128", "f8v7", "f16hi"])
    ap.add_argument("--kernel", default="auto", choices=["auto", "hybrid", "coop", "flat"])
    ap.add_argument("--ablation-steps", type=int, default=5,
                    help="timed steps per kernel variant in the ablation block (0 = skip)")
    ap.add_argument("--smem-levels", type=int, default=-1)
    ap.add_argument("--traffic", default="uniform", choices=["uniform", "zipf"])
    ap.add_argument("--seed", type=int, default=2604)
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--latency-batches", type=int, default=1000)
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--workload", default="backbone",
                    choices=["backbone", "vrf64", "learned1m", "small", "serve", "build"],
                    help="backbone: 200k prefixes, 2^28 lookups (the headline); vrf64: 64 VRF "
                         "tables of 1k-300k prefixes, 2^27 tagged lookups, one graph per batch; "
                         "learned1m: 1M prefixes, 2^28 lookups, learned vs plain tree; small: "
                         "1k prefixes, 10^6 lookups; serve: the serving engine under Poisson "
                         "arrivals and route updates; build: build and rebuild times, host "
                         "builder against the device builder")
    ap.add_argument("--serve-warmup", type=float, default=1.0,
                    help="serve: seconds of the same load before the measured phase")
    ap.add_argument("--per-table", action="store_true",
                    help="serve: one lookup launch per table instead of the single persistent one")
    ap.add_argument("--bucketed", action="store_true",
                    help="serve: group each batch by table even where the direct form applies")
    ap.add_argument("--builder", default="host", choices=["host", "device"],
                    help="where tables are built (and rebuilt by updates) in serve")
    ap.add_argument("--tables", type=int, default=64)
    ap.add_argument("--rate", type=float, default=20000.0, help="serve: requests per second")
    ap.add_argument("--duration", type=float, default=5.0, help="serve: seconds of arrivals")
    ap.add_argument("--update-rate", type=float, default=1000.0, help="serve: route changes/s")
    ap.add_argument("--no-tune", action="store_true")
    ap.add_argument("--no-extra", action="store_true",
                    help="default run: skip the learned1m, vrf64 and zipf blocks")
    ap.add_argument("--extra-steps", type=int, default=5,
                    help="timed steps of each extra block (after 3 warm-up steps)")
    return ap.parse_args()


# ----------------------------------------------------------------------------- distributed

def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def dist_init(world, use_cuda):
    if world <= 1:
        return None
    import torch.distributed as dist
    dist.init_process_group(backend="nccl" if use_cuda else "gloo")
    return dist


def barrier(dist, device=None):
    if dist is not None:
        if device is not None:
            dist.barrier(device_ids=[device])
        else:
            dist.barrier()


def max_over_ranks(dist, value, use_cuda):
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device="cuda" if use_cuda else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ----------------------------------------------------------------------------- clocks

class Clocks:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid: str | None):
        self.proc = None
        self.uuid = uuid

    def start(self):
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
               "-lms", "200"]
        if self.uuid:
            cmd[1:1] = ["-i", self.uuid]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                                         text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=10)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for row in csv.reader(io.StringIO(out)):
            if len(row) < 9:
                continue
            try:
                sm.append(float(row[1]))
                mx.append(float(row[2]))
            except ValueError:
                continue
            for name, v in zip(names, row[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d.get("hbm_gbs"), "measured"
    return 6800.0, "fallback"


def measured_peaks_mhz() -> float:
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            return float(json.load(f).get("sm_max_mhz", 2070.0))
    except (OSError, ValueError):
        return 2070.0


def f16_kernel_name(st) -> str:
    """The name ncu prints for an F16HI hybrid table's single-table lookup kernel: the in-place
    search of the index over the leaves (one level below it, four 256-thread CTAs per SM), or the
    staged form when the index holds every key."""
    return ("lookup_hybrid16<1, 0, 4>" if st["depth"] > st["smem_levels"]
            else "lookup_hybrid16<0, 0, 0>")


def recorded_counters(kernel: str):
    """Per-lookup counters of a kernel from the ncu capture summarised in profiles/traffic.json,
    if the kernel's source has not changed since the capture (else None)."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        rec = json.load(f)
    e = rec.get(kernel)
    if not e or not isinstance(e.get("sources"), list):
        return None
    h = hashlib.sha256()
    for src in e["sources"]:
        path = os.path.join(ROOT, src)
        if not os.path.exists(path):
            return None
        with open(path, "rb") as f:
            h.update(f.read())
    return e if e.get("sources_sha256") == h.hexdigest() else None


# ----------------------------------------------------------------------------- workload

def rank_shard(fib, n, seed, rank, traffic="uniform"):
    """Rank r looks up draws r*n .. (r+1)*n - 1 of one seeded trace stream (weak scaling: every rank
    has its own n addresses; the table is replicated)."""
    import synth
    if traffic == "zipf":
        return synth.gen_trace_zipf(fib, n, seed=seed + 1 + rank)
    return synth.gen_trace(fib, n, seed=seed + 1, start=rank * n)


def workload(args, rank):
    import synth
    fib = synth.gen_fib(args.prefixes, seed=args.seed, nh_max=255 if args.prefixes <= 1000 else 4095)
    xh, xl = rank_shard(fib, args.lookups, args.seed, rank, args.traffic)
    return fib, xh, xl


def workload_name(args):
    t = "70% covered / 30% uniform" if args.traffic == "uniform" else "Zipf(1.1) over 1e5 hot /64s"
    return (f"{args.prefixes}-prefix synthetic BGP-like IPv6 FIB, {args.lookups} lookups per GPU "
            f"({t})")


def cpu_oracle_rate(fib, xh, xl, seconds, threads=None, runs=5):
    """The oracle (O2 binary trie, as it stands) on the host cores (all of them by default): the
    median rate of `runs` timed passes over one bounded sample, sized so that all passes take
    about `seconds`. Returns (rate, threads used, sample, seconds per pass, every pass's rate)."""
    import oracle
    trie = oracle.Trie(fib.hi, fib.lo, fib.len, fib.nh)
    threads = threads or os.cpu_count() or 1
    probe = min(xh.size, 1 << 20)
    t0 = time.perf_counter()
    trie.lookup(xh[:probe], xl[:probe], threads=threads)
    dt = max(time.perf_counter() - t0, 1e-6)
    sample = int(min(xh.size, max(probe, probe * seconds / runs / dt)))
    out = np.empty(sample, np.uint16)
    rates = []
    for _ in range(runs):
        t0 = time.perf_counter()
        trie.lookup(xh[:sample], xl[:sample], threads=threads, out=out)
        rates.append(sample / (time.perf_counter() - t0))
    rate = statistics.median(rates)
    return rate, trie.last_threads, sample, sample / rate, rates


def host_info():
    """ISA, CPU model and core count of the host (lscpu's model name where it has one: on Arm
    hosts /proc/cpuinfo names only the implementer and part numbers)."""
    import platform
    model, vendor = None, None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            k, _, v = line.partition(":")
            if k.strip() == "Model name" and not model:
                model = v.strip()
            elif k.strip() == "Vendor ID" and not vendor:
                vendor = v.strip()
    except (OSError, subprocess.SubprocessError):
        pass
    if not model:
        try:
            with open("/proc/cpuinfo") as f:
                for line in f:
                    if line.lower().startswith(("model name", "cpu model")):
                        model = line.split(":", 1)[1].strip()
                        break
        except OSError:
            pass
    model = model or platform.processor() or platform.machine()
    if vendor and vendor not in model:
        model = f"{vendor} {model}"
    return {"arch": platform.machine(), "model": model, "nproc": os.cpu_count()}


def low_half_fraction(pb, fib_in, xh):
    """Share of addresses whose F16HI lookup reads the address's low half: those whose high-half
    count lands on an interval whose key (its inclusive end) shares the address's high half and
    has a low half other than all-ones (the next-hop word's flag). Counted on the host from the
    library's own interval list, for stating the bytes that cross the host link."""
    sh, sl, _ = pb.intervals(fib_in.hi, fib_in.lo, fib_in.len, fib_in.nh)
    if sh.size < 2:
        return 0.0
    nxt_h, nxt_l = sh[1:], sl[1:]
    key_hi = np.where(nxt_l == 0, nxt_h - np.uint64(1), nxt_h)     # high half of start[i+1] - 1
    flag = nxt_l != 0
    r = np.searchsorted(key_hi, xh, side="left")
    inside = r < key_hi.size
    rr = np.minimum(r, key_hi.size - 1)
    return float(np.mean(inside & flag[rr] & (key_hi[rr] == xh)))


# ----------------------------------------------------------------------------- reference arm

def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import oracle
    import synth
    fib = synth.gen_fib(args.prefixes, seed=args.seed, nh_max=4095)
    sample = min(1 << 22, args.lookups)   # a bounded sample of the workload's trace per step
    xh, xl = synth.gen_trace(fib, sample, seed=args.seed + 1)
    trie = oracle.Trie(fib.hi, fib.lo, fib.len, fib.nh)
    threads = os.cpu_count() or 1
    out = np.empty(sample, np.uint16)
    for _ in range(args.warmup):
        trie.lookup(xh, xl, threads=threads, out=out)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        trie.lookup(xh, xl, threads=threads, out=out)
        times.append(time.perf_counter() - t0)
    total = sum(times)
    value = sample * args.steps / total / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
        "data": "synthetic (seeded)",
        "config": {"workload": workload_name(args), "sample_per_step": sample,
                   "prefixes": args.prefixes, "lookups": args.lookups},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": trie.last_threads,
                         "kind": "oracle",
                         "sample": f"{sample} addresses of the same trace per step, binary trie",
                         "host": host_info()},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------------------- GPU arm

def run_planb(args):
    import torch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dist = dist_init(world, True)
    import paper_2604_14650_gb300 as pb
    fib_in, xh, xl = workload(args, rank)
    fib = pb.Fib(fib_in.hi, fib_in.lo, fib_in.len, fib_in.nh, format=args.format,
                 smem_levels=args.smem_levels, device=local, kernel=args.kernel)
    st = fib.stats()
    n = xh.size
    d_hi = torch.from_numpy(xh.view(np.int64)).cuda()
    d_lo = torch.from_numpy(xl.view(np.int64)).cuda()
    d_out = torch.empty(n, dtype=torch.int16, device="cuda")
    stream = torch.cuda.Stream()
    hp, lp, op = d_hi.data_ptr(), d_lo.data_ptr(), d_out.data_ptr()

    # parity spot check of this very launch configuration against the oracle (sampled)
    with torch.cuda.stream(stream):
        fib.lookup_ptr(hp, lp, n, op, stream)
    stream.synchronize()
    import oracle
    idx = np.random.default_rng(args.seed).integers(0, n, 1 << 16)
    want = oracle.Trie(fib_in.hi, fib_in.lo, fib_in.len, fib_in.nh).lookup(xh[idx], xl[idx])
    got = d_out.cpu().numpy().view(np.uint16)[idx]
    if not np.array_equal(got, want):
        raise SystemExit(f"parity failure: {int(np.count_nonzero(got != want))} of {idx.size}")

    for _ in range(args.warmup):
        fib.lookup_ptr(hp, lp, n, op, stream)
    stream.synchronize()
    uuid = None
    try:
        uuid = "GPU-" + str(torch.cuda.get_device_properties(local).uuid)
    except Exception:
        pass
    clocks = Clocks(uuid)
    clocks.start()
    time.sleep(0.3)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    barrier(dist, local)
    torch.cuda.synchronize()
    ev[0].record(stream)
    for i in range(args.steps):
        fib.lookup_ptr(hp, lp, n, op, stream)
        ev[i + 1].record(stream)
    stream.synchronize()
    torch.cuda.synchronize()
    barrier(dist, local)
    clk = clocks.stop()
    per_launch = [ev[i].elapsed_time(ev[i + 1]) for i in range(args.steps)]
    total_ms = ev[0].elapsed_time(ev[-1])
    total_ms = max_over_ranks(dist, total_ms, True)
    value = n * world * args.steps / (total_ms / 1e3) / 1e9
    avg_launch_s = statistics.mean(per_launch) / 1e3

    # e2e through the public API with host buffers (pinned), copies inside the timed region
    e2e = None
    if not args.no_e2e:
        ph = torch.from_numpy(xh.view(np.int64)).pin_memory()
        pl = torch.from_numpy(xl.view(np.int64)).pin_memory()
        po = torch.empty(n, dtype=torch.int16).pin_memory()
        fib.lookup_host(ph, pl, out=po)
        barrier(dist, local)
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            fib.lookup_host(ph, pl, out=po)
        torch.cuda.synchronize()
        barrier(dist, local)
        dt = max_over_ranks(dist, time.perf_counter() - t0, True)
        # bytes that cross the host link per step: every address's 8-byte high half, the 8-byte
        # low half only where an F16HI count needs settling (other formats read both halves), and
        # the 2-byte next hop back
        if args.format == "f16hi":
            frac_lo = low_half_fraction(pb, fib_in, xh[idx])
            h2d = int(round(8 * n + 8 * frac_lo * n))
        else:
            frac_lo, h2d = 1.0, 16 * n
        e2e = {"value": n * world * args.e2e_steps / dt / 1e9, "unit": UNIT,
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": 2 * n,
               "h2d_bytes_interface": 16 * n,
               "low_halves_read_fraction": frac_lo,
               "bytes_note": "h2d counts the bytes the zero-copy kernel reads over the host link "
                             "(8 B high half per address, plus the low half of the sampled share "
                             "of addresses whose count needs it); the interface holds 16 B per "
                             "address",
               "api": "planb_lookup_host (pinned host buffers: the lookup kernel reads the "
                      "addresses and writes the next hops over the host link)"}
        if not np.array_equal(po.numpy().view(np.uint16)[idx], want):
            raise SystemExit("e2e parity failure")
        # the same through planb_lookup_mapped: the kernel reads the pinned addresses and writes
        # the next hops over the host link itself, no copy engine in between
        po.fill_(-1)
        fib.lookup_mapped(ph, pl, po, stream)
        stream.synchronize()
        if not np.array_equal(po.numpy().view(np.uint16)[idx], want):
            raise SystemExit("mapped e2e parity failure")
        barrier(dist, local)
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            fib.lookup_mapped(ph, pl, po, stream)
        stream.synchronize()
        barrier(dist, local)
        dt = max_over_ranks(dist, time.perf_counter() - t0, True)
        e2e["mapped"] = {"value": n * world * args.e2e_steps / dt / 1e9, "unit": UNIT,
                         "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": 2 * n,
                         "api": "planb_lookup_mapped (pinned host buffers read and written by "
                                "the lookup kernel over the host link)"}
        # the host link's own rate for a plain pinned-to-device copy of the high halves: the
        # ceiling of a lookup path that must move at least 8 + 2 bytes per address across it
        dbuf = torch.empty(n, dtype=torch.int64, device=f"cuda:{local}")
        dbuf.copy_(ph, non_blocking=True)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(2):
            dbuf.copy_(ph, non_blocking=True)
        b.record()
        b.synchronize()
        link = 2 * 8 * n / (a.elapsed_time(b) / 1e3) / 1e9
        e2e["host_link"] = {"h2d_copy_gbs": link, "bytes_per_lookup_crossing": 10,
                            "ceiling_B_lookups_per_s": link / 10,
                            "frac": e2e["value"] * 10 / link}
        del ph, pl, po, dbuf

    # p50/p99 latency of 2^16-address batches, each launch event-timed
    lat = None
    if args.latency_batches > 0:
        bs = 1 << 16
        nb = args.latency_batches
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(nb)]
        for i in range(nb):
            off = (i * bs) % max(n - bs, 1)
            a, b = evs[i]
            a.record(stream)
            fib.lookup_ptr(hp + 8 * off, lp + 8 * off, bs, op + 2 * off, stream)
            b.record(stream)
        stream.synchronize()
        us = sorted(1e3 * a.elapsed_time(b) for a, b in evs)
        lat = {"batch": bs, "batches": nb, "p50_us": us[len(us) // 2],
               "p99_us": us[min(len(us) - 1, int(0.99 * len(us)))], "max_us": us[-1],
               "what": "each launch event-timed as the host submits it: the interval holds the "
                       "host's submission of the launch (the GPU waits for it) and the kernel"}
        # the same batches queued behind ~36 ms of earlier lookups, so that the GPU runs them back
        # to back and each interval holds the kernel alone
        for _ in range(10):
            fib.lookup_ptr(hp, lp, n, op, stream)
        for i in range(nb):
            off = (i * bs) % max(n - bs, 1)
            a, b = evs[i]
            a.record(stream)
            fib.lookup_ptr(hp + 8 * off, lp + 8 * off, bs, op + 2 * off, stream)
            b.record(stream)
        stream.synchronize()
        qs = sorted(1e3 * a.elapsed_time(b) for a, b in evs)
        lat["queued"] = {"p50_us": qs[len(qs) // 2],
                         "p99_us": qs[min(len(qs) - 1, int(0.99 * len(qs)))], "max_us": qs[-1]}

    # ablation (the GPU analogue of the paper's Section 4.5 study): every lookup kernel on the same
    # device-resident addresses
    ablation = None
    if args.ablation_steps > 0:
        ablation = {}
        fib.lookup_ptr(hp, lp, n, op, stream)
        stream.synchronize()
        ref_out = d_out.clone()
        for name, fmt, kern in (("flat binary search (std::lower_bound analogue)", "f8x128", "flat"),
                                ("linearized tree, coop 8-lane, 128-bit keys", "f8x128", "coop"),
                                ("linearized tree, coop 16-lane, 64-bit key halves", "f16hi", "coop"),
                                ("linearized tree, hybrid smem index + coop L2", "f8x128", "hybrid"),
                                ("hybrid + next hops packed in the leaf line", "f8v7", "hybrid"),
                                ("hybrid on 16-key leaves (index over the leaves, one L2 line)",
                                 "f16hi", "hybrid"),
                                ("learned position model (RMI, MLP root) + tree, 128-bit keys",
                                 "f8x128", "learned"),
                                ("learned position model (RMI, MLP root) + tree, packed leaves",
                                 "f8v7", "learned")):
            with pb.Fib(fib_in.hi, fib_in.lo, fib_in.len, fib_in.nh, format=fmt, kernel=kern,
                        device=local) as v:
                for _ in range(2):
                    v.lookup_ptr(hp, lp, n, op, stream)
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                for _ in range(args.ablation_steps):
                    v.lookup_ptr(hp, lp, n, op, stream)
                b.record(stream)
                stream.synchronize()
                vs = v.stats()
                ablation[f"{fmt}/{kern}"] = {
                    "what": name, "B_lookups_per_s": n * args.ablation_steps / a.elapsed_time(b) / 1e6,
                    "depth": vs["depth"], "smem_levels": vs["smem_levels"],
                    "smem_bytes": vs["smem_bytes"], "threads": vs["threads"], "ctas": vs["ctas"]}
                if kern == "learned":
                    ablation[f"{fmt}/{kern}"]["model"] = {
                        k[6:]: vs[k] for k in ("model_leaves", "model_iters", "model_max_err",
                                               "model_loss0", "model_loss", "model_covered",
                                               "model_mean_err", "model_train_ms")}
                # results of every variant equal the headline launch's (exactness across kernels)
                same = torch.equal(d_out.view(torch.int16), ref_out)
                ablation[f"{fmt}/{kern}"]["same_results_as_headline"] = bool(same)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        rate, cores, sample, secs, rates = cpu_oracle_rate(fib_in, xh, xl, args.cpu_seconds)
        rate1, _, sample1, secs1, rates1 = cpu_oracle_rate(fib_in, xh, xl, args.cpu_seconds / 4,
                                                           threads=1)
        cpu = {"value": rate / 1e9, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"first {sample} addresses of the same trace, binary trie, median of "
                         f"{len(rates)} passes of {secs:.2f} s",
               "runs_B_lookups_per_s": [r / 1e9 for r in rates],
               "host": host_info(),
               "one_core": {"value": rate1 / 1e9, "unit": UNIT, "cores": 1,
                            "sample": f"first {sample1} addresses, median of {len(rates1)} "
                                      f"passes of {secs1:.2f} s",
                            "runs_B_lookups_per_s": [r / 1e9 for r in rates1]}}

    peak, peak_kind = measured_peaks()
    kname = {1: "coop", 2: "hybrid", 3: "flat"}[st["kernel"]]
    # the kernel's name as ncu prints it
    if kname == "hybrid" and args.format == "f16hi":
        kernel = f16_kernel_name(st)
    elif kname == "hybrid":
        kernel = (f"lookup_hybrid<{st['depth'] - st['smem_levels']}, "
                  f"{1 if args.format == 'f8v7' else 0}, 0, 0, 0>")
    elif kname == "flat":
        kernel = "lookup_flat"
    else:
        kernel = f"lookup_coop_{'f16' if args.format == 'f16hi' else 'f8'}<{st['depth']}>"
    achieved = HBM_BYTES_PER_LOOKUP * n / avg_launch_s / 1e9
    rec = recorded_counters(kernel)
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak,
                "traffic": rec["dram_bytes_per_lookup"] * n if rec else None,
                "kernel": kernel, "peak_source": peak_kind,
                "algorithmic_bytes_per_launch": HBM_BYTES_PER_LOOKUP * n}
    # the other roofs of the descent: L2 -> SM bytes and the L1/LSU data pipe, per lookup from the
    # ncu capture in profiles/ (same kernel source), at this run's lookup rate
    roofs = None
    if rec:
        rate = n / avg_launch_s
        l2 = rec["l2_bytes_per_lookup"] * rate / 1e9
        roofs = {"l2": {"achieved": l2, "peak": rec["l2_peak_gbs"], "unit": "GB/s",
                        "frac": l2 / rec["l2_peak_gbs"] if rec["l2_peak_gbs"] else None,
                        "bytes_per_lookup": rec["l2_bytes_per_lookup"]},
                 "l1_lsu_pipe": {"frac_at_capture": rec["l1_lsu_wavefronts_pct_of_peak"] / 100,
                                 "smem_wavefronts_per_lookup": rec["smem_wavefronts_per_lookup"]},
                 # instruction issue: warp-instructions per lookup (capture) at this run's rate
                 # against 4 schedulers x SMs x the SM clock sampled under load
                 "issue": None,
                 "source": "profiles/traffic.json (ncu --set full capture of this kernel)"}
    # the grown workloads, each with its own value, roofline and sampled parity (rank 0, N = 1)
    extra = None
    if rank == 0 and world == 1 and not args.no_extra and args.workload == "backbone":
        del d_hi, d_lo, d_out
        torch.cuda.empty_cache()
        es, ew = args.extra_steps, 3
        extra = {"learned1m": block_learned1m(args, stream, es, ew),
                 "vrf64": block_vrf64(args, stream, es, ew),
                 "zipf": block_zipf(args, stream, es, ew, fib_in=fib_in),
                 "serve": block_serve(args)}
        torch.cuda.empty_cache()
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic (seeded)",
        "config": {"workload": workload_name(args), "prefixes": args.prefixes,
                   "lookups_per_gpu": n, "traffic": args.traffic, "format": args.format,
                   "kernel": kname, "depth": st["depth"], "smem_levels": st["smem_levels"],
                   "threads": st["threads"], "ctas": st["ctas"], "smem_bytes": st["smem_bytes"],
                   "intervals": st["n_intervals"], "table_bytes": st["node_bytes"] + st["value_bytes"],
                   "build_ms": st["build_ms"], "upload_ms": st["upload_ms"],
                   "l2": "inputs (16 B x lookups) larger than L2; no flush", "seed": args.seed,
                   "parallelism": f"dp{world} (table replicated, addresses sharded)"},
        "roofline": roofline,
        "roofs": roofs,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "latency": lat,
        "ablation": ablation,
        "learned_vs_plain": ({"learned_B_lookups_per_s": ablation["f8x128/learned"]["B_lookups_per_s"],
                              "plain_tree_same_format_B_lookups_per_s":
                                  ablation["f8x128/hybrid"]["B_lookups_per_s"],
                              "plain_tree_best_B_lookups_per_s": value,
                              "paper_plain_tree_coop_B_lookups_per_s":
                                  ablation["f8x128/coop"]["B_lookups_per_s"]}
                             if ablation else None),
        "workloads": extra,
        "clocks": clk,
        "gpu_launches": args.steps,
    }
    if extra and line["learned_vs_plain"] is not None:
        L1 = extra["learned1m"]
        line["learned_vs_plain"]["grown_1m_prefixes"] = {
            "learned_B_lookups_per_s": L1["value"],
            "plain_tree_best": L1["best_plain"],
            "plain_tree_best_B_lookups_per_s": L1["best_plain_B_lookups_per_s"],
            "model_max_err": L1["variants"]["learned_f8x128"]["model"]["max_err"]}
    if roofs is not None and rec.get("warp_inst_per_lookup"):
        sms = torch.cuda.get_device_properties(local).multi_processor_count
        mhz = (clk or {}).get("sm_mhz") or measured_peaks_mhz()
        peak_ginst = 4 * sms * mhz / 1e3
        ach = rec["warp_inst_per_lookup"] * (n / avg_launch_s) / 1e9
        roofs["issue"] = {"achieved": ach, "peak": peak_ginst, "unit": "G warp-instructions/s",
                          "frac": ach / peak_ginst,
                          "warp_inst_per_lookup": rec["warp_inst_per_lookup"],
                          "issue_active_at_capture": rec.get("issue_active_pct", 0) / 100}
    if rank == 0:
        print(json.dumps(line), flush=True)
    fib.close()
    if dist is not None:
        dist.destroy_process_group()
    return 0


def vrf_tables(args):
    """64 table sizes log-uniform over [1e3, 3e5] (seeded), the tables, and a tagged trace whose
    table ids are drawn proportional to table size."""
    import synth
    return synth.gen_vrf_workload(args.tables, args.lookups, args.seed)


def run_vrf64(args):
    import torch
    import paper_2604_14650_gb300 as pb
    from paper_2604_14650_gb300.autotune import Autotuner
    torch.cuda.set_device(0)
    if args.lookups == 1 << 28:
        args.lookups = 1 << 27
    sizes, fibs_in, tid, xh, xl = vrf_tables(args)
    n = xh.size
    d_hi = torch.from_numpy(xh.view(np.int64)).cuda()
    d_lo = torch.from_numpy(xl.view(np.int64)).cuda()
    d_t = torch.from_numpy(tid).cuda()
    d_out = torch.empty(n, dtype=torch.int16, device="cuda")
    # tuned within the configurations the single persistent launch runs
    tuner = Autotuner(persistent=True)   # cache: the library's default location
    choices, fibs = [], []
    t0 = time.perf_counter()
    for t, f in enumerate(fibs_in):
        opts = dict(format=args.format)
        if not args.no_tune:
            idx = np.nonzero(tid == t)[0][: 1 << 21]
            sh = torch.from_numpy(xh[idx].view(np.int64)).cuda()
            sl = torch.from_numpy(xl[idx].view(np.int64)).cuda()
            opts = tuner.best(f.hi, f.lo, f.len, f.nh, sh, sl)
        fibs.append(pb.Fib(f.hi, f.lo, f.len, f.nh, **opts))
        choices.append(opts)
    build_s = time.perf_counter() - t0
    stream = torch.cuda.Stream()
    args_ptr = (d_hi.data_ptr(), d_lo.data_ptr(), d_t.data_ptr(), n, d_out.data_ptr())
    import oracle
    rng = np.random.default_rng(1)
    sample = rng.integers(0, n, 1 << 16)

    def timed(per_table, bucketed=False, direct=False):
        mt = pb.MultiFib(fibs, max_batch=n, per_table=per_table, bucketed=bucketed,
                         direct=direct)
        d_out.fill_(-1)
        mt.lookup_ptr(*args_ptr, stream)
        stream.synchronize()
        got = d_out.cpu().numpy().view(np.uint16)[sample]
        for t, f in enumerate(fibs_in):
            sel = tid[sample] == t
            want = oracle.Trie(f.hi, f.lo, f.len, f.nh).lookup(xh[sample][sel], xl[sample][sel])
            if not np.array_equal(got[sel], want):
                raise SystemExit(f"parity failure in table {t}")
        for _ in range(args.warmup):
            mt.lookup_ptr(*args_ptr, stream)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        stream.synchronize()
        a.record(stream)
        for _ in range(args.steps):
            mt.lookup_ptr(*args_ptr, stream)
        b.record(stream)
        stream.synchronize()
        mode = mt.mode
        mt.close()
        if ((mode == "per_table") != per_table or (bucketed and mode != "bucketed") or
                (direct and mode != "direct" and args.format == "f16hi" and args.no_tune)):
            raise SystemExit(f"multi-table launch mode {mode} is not the one asked for")
        timed.modes.append(mode)
        return a.elapsed_time(b) / args.steps

    timed.modes = []
    ms = timed(False)
    form = timed.modes[-1]
    ms_direct = timed(False, direct=True)
    ms_bucketed = timed(False, bucketed=True)
    ms_per_table = timed(True)
    kinds = {}
    for c in choices:
        k = f"{c.get('format', 'f8x128')}/{c.get('kernel', 'auto')}"
        kinds[k] = kinds.get(k, 0) + 1
    line = {"metric": "B lookups/s, 64 VRF tables (multi-table graph)", "value": n / ms / 1e6,
            "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms, "higher_is_better": True, "dtype": "u64",
            "data": "synthetic (seeded)",
            "config": {"workload": f"{args.tables} VRF tables, sizes log-uniform 1e3..3e5 prefixes "
                                   f"(total {int(sizes.sum())}), {n} lookups tagged with a u8 table "
                                   "id drawn proportional to table size",
                       "tables": args.tables, "prefixes_total": int(sizes.sum()),
                       "autotuned": not args.no_tune, "chosen": kinds,
                       "build_s": build_s,
                       "form": form,
                       "graph": ("one persistent launch in input order (no bucketing), captured "
                                 "once, replayed per step" if form == "direct" else
                                 "bucketing (hist, scan, scatter) + one persistent lookup launch "
                                 "over all tables + gather, captured once, replayed per step"),
                       "direct_B_lookups_per_s": n / ms_direct / 1e6,
                       "direct_ms_per_step": ms_direct,
                       "bucketed_B_lookups_per_s": n / ms_bucketed / 1e6,
                       "bucketed_ms_per_step": ms_bucketed,
                       "per_table_launches_B_lookups_per_s": n / ms_per_table / 1e6,
                       "per_table_launches_ms_per_step": ms_per_table},
            "roofline": {"bound": "hbm", "achieved": 19 * n / (ms / 1e3) / 1e9,
                         "peak": measured_peaks()[0], "unit": "GB/s",
                         "frac": 19 * n / (ms / 1e3) / 1e9 / measured_peaks()[0],
                         "note": "19 B per lookup (16 B address + 1 B id + 2 B result) against the "
                                 "measured copy bandwidth"},
            "gpu_launches": args.steps * (1 if form == "direct" else 5)}
    print(json.dumps(line), flush=True)
    for f in fibs:
        f.close()
    return 0


def _timed_ms(launch, stream, steps, warmup):
    """Mean ms per launch of `launch()` over `steps` launches after `warmup`, CUDA events on
    `stream`."""
    import torch
    for _ in range(warmup):
        launch()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    stream.synchronize()
    a.record(stream)
    for _ in range(steps):
        launch()
    b.record(stream)
    stream.synchronize()
    return a.elapsed_time(b) / steps


def _hbm_roofline(bytes_per_lookup, n, ms, kernel):
    peak, kind = measured_peaks()
    ach = bytes_per_lookup * n / (ms / 1e3) / 1e9
    return {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
            "traffic": None, "kernel": kernel, "peak_source": kind,
            "algorithmic_bytes_per_launch": bytes_per_lookup * n}


def block_learned1m(args, stream, steps, warmup, lookups=1 << 28):
    """1,000,000 prefixes (1 % /128) and 2^28 device-resident addresses: the learned position
    model against the plain tree on the same table and addresses, each timed by CUDA events,
    every variant's results equal, a 2^16 sample equal to the oracle."""
    import torch
    import paper_2604_14650_gb300 as pb
    import synth
    import oracle
    f = synth.gen_fib(1_000_000, seed=args.seed, nh_max=4095)
    n = lookups
    xh, xl = synth.gen_trace(f, n, seed=args.seed + 1)
    d_hi = torch.from_numpy(xh.view(np.int64)).cuda()
    d_lo = torch.from_numpy(xl.view(np.int64)).cuda()
    d_out = torch.empty(n, dtype=torch.int16, device="cuda")
    res, ref = {}, None
    for name, kw in (("learned_f8x128", dict(kernel="learned")),
                     ("plain_f8x128_hybrid", dict(kernel="hybrid")),
                     ("plain_f16hi_hybrid", dict(format="f16hi", kernel="hybrid")),
                     ("plain_f8x128_coop", dict(kernel="coop"))):
        with pb.Fib(f.hi, f.lo, f.len, f.nh, **kw) as fib:
            ms = _timed_ms(lambda: fib.lookup_ptr(d_hi.data_ptr(), d_lo.data_ptr(), n,
                                                  d_out.data_ptr(), stream), stream, steps, warmup)
            st = fib.stats()
            # an F16HI table's launch searches its leaf-level index in place (one level below)
            below = st["depth"] - st["smem_levels"]
            res[name] = {"B_lookups_per_s": n / ms / 1e6, "ms_per_launch": ms,
                         "depth": st["depth"], "smem_levels": st["smem_levels"],
                         "levels_from_l2": min(1, below) if kw.get("format") == "f16hi" else below}
            if kw.get("kernel") == "learned":
                res[name]["model"] = {k[6:]: st[k] for k in st if k.startswith("model_")}
            if ref is None:
                ref = d_out.clone()
            res[name]["same_results_as_learned"] = bool(torch.equal(ref, d_out))
    idx = np.random.default_rng(2).integers(0, n, 1 << 16)
    want = oracle.Trie(f.hi, f.lo, f.len, f.nh).lookup(xh[idx], xl[idx])
    parity = bool(np.array_equal(ref.cpu().numpy().view(np.uint16)[idx], want))
    lv = res["learned_f8x128"]
    best_plain = max((k for k in res if k.startswith("plain")),
                     key=lambda k: res[k]["B_lookups_per_s"])
    del d_hi, d_lo, d_out, ref
    return {"workload": f"1,000,000-prefix synthetic FIB (1 % /128), {n} device-resident lookups",
            "value": lv["B_lookups_per_s"], "unit": UNIT, "steps": steps, "warmup": warmup,
            "what": "learned position model (F8X128) beside the plain tree forms",
            "best_plain": best_plain,
            "best_plain_B_lookups_per_s": res[best_plain]["B_lookups_per_s"],
            "roofline": _hbm_roofline(HBM_BYTES_PER_LOOKUP, n, lv["ms_per_launch"],
                                      f"lookup_hybrid<{lv['levels_from_l2']}, 0, 1, 0, 0>"),
            "variants": res, "sampled_parity_vs_oracle": parity,
            "all_variants_equal": all(v["same_results_as_learned"] for v in res.values())}


def block_zipf(args, stream, steps, warmup, fib_in=None, lookups=1 << 28):
    """The 200,000-prefix table under the locality-skewed trace (Zipf(1.1) over 10^5 hot /64
    blocks), 2^28 addresses, the headline kernel (F16HI hybrid)."""
    import torch
    import paper_2604_14650_gb300 as pb
    import synth
    import oracle
    f = fib_in if fib_in is not None else synth.gen_fib(200_000, seed=args.seed, nh_max=4095)
    n = lookups
    xh, xl = synth.gen_trace_zipf(f, n, seed=args.seed + 1)
    d_hi = torch.from_numpy(xh.view(np.int64)).cuda()
    d_lo = torch.from_numpy(xl.view(np.int64)).cuda()
    d_out = torch.empty(n, dtype=torch.int16, device="cuda")
    with pb.Fib(f.hi, f.lo, f.len, f.nh, format="f16hi", kernel="hybrid") as fib:
        ms = _timed_ms(lambda: fib.lookup_ptr(d_hi.data_ptr(), d_lo.data_ptr(), n,
                                              d_out.data_ptr(), stream), stream, steps, warmup)
        st = fib.stats()
    idx = np.random.default_rng(3).integers(0, n, 1 << 16)
    want = oracle.Trie(f.hi, f.lo, f.len, f.nh).lookup(xh[idx], xl[idx])
    parity = bool(np.array_equal(d_out.cpu().numpy().view(np.uint16)[idx], want))
    del d_hi, d_lo, d_out
    kernel = f16_kernel_name(st)
    return {"workload": f"200,000-prefix FIB, {n} lookups, Zipf(1.1) over 1e5 hot /64 blocks",
            "value": n / ms / 1e6, "unit": UNIT, "steps": steps, "warmup": warmup,
            "ms_per_launch": ms, "roofline": _hbm_roofline(HBM_BYTES_PER_LOOKUP, n, ms, kernel),
            "sampled_parity_vs_oracle": parity}


def block_vrf64(args, stream, steps, warmup, lookups=1 << 27, fmt="f16hi"):
    """64 VRF tables (sizes log-uniform over 1e3..3e5 prefixes) and 2^27 addresses tagged with a
    table id drawn proportional to table size: one captured graph per step, in each form of the
    multi-table lookup — the library's own choice (auto), direct (one launch in input order),
    bucketed (grouped by table, one persistent launch, gathered back) and one launch per
    table."""
    import torch
    import paper_2604_14650_gb300 as pb
    import synth
    import oracle
    sizes, fibs_in, tid, xh, xl = synth.gen_vrf_workload(64, lookups, args.seed)
    n = xh.size
    d_hi = torch.from_numpy(xh.view(np.int64)).cuda()
    d_lo = torch.from_numpy(xl.view(np.int64)).cuda()
    d_t = torch.from_numpy(tid).cuda()
    d_out = torch.empty(n, dtype=torch.int16, device="cuda")
    fibs = [pb.Fib(f.hi, f.lo, f.len, f.nh, format=fmt) for f in fibs_in]
    ptrs = (d_hi.data_ptr(), d_lo.data_ptr(), d_t.data_ptr(), n, d_out.data_ptr())
    sample = np.random.default_rng(1).integers(0, n, 1 << 16)
    want = np.zeros(sample.size, np.uint16)
    for t, f in enumerate(fibs_in):
        sel = tid[sample] == t
        want[sel] = oracle.Trie(f.hi, f.lo, f.len, f.nh).lookup(xh[sample][sel], xl[sample][sel])
    res = {}
    try:
        for mode in ("auto", "direct", "bucketed", "per_table"):
            with pb.MultiFib(fibs, max_batch=n, per_table=mode == "per_table",
                             bucketed=mode == "bucketed", direct=mode == "direct") as mt:
                d_out.fill_(-1)
                mt.lookup_ptr(*ptrs, stream)
                stream.synchronize()
                got = d_out.cpu().numpy().view(np.uint16)[sample]
                ms = _timed_ms(lambda: mt.lookup_ptr(*ptrs, stream), stream, steps, warmup)
                res[mode] = {"B_lookups_per_s": n / ms / 1e6, "ms_per_step": ms,
                             "sampled_parity_vs_oracle": bool(np.array_equal(got, want)),
                             "single_launch": bool(mt.persistent), "form": mt.mode}
    finally:
        for f in fibs:
            f.close()
    del d_hi, d_lo, d_t, d_out
    p = res["auto"]
    return {"workload": f"64 VRF tables, {int(sizes.sum())} prefixes in all, {n} lookups "
                        "tagged with a u8 table id drawn proportional to table size",
            "value": p["B_lookups_per_s"], "unit": UNIT, "steps": steps, "warmup": warmup,
            "format": fmt,
            "form": p["form"],
            "roofline": dict(_hbm_roofline(19, n, p["ms_per_step"],
                                           f"multi-table lookup, {p['form']} form (whole step)"),
                             note="19 B per lookup (16 B address + 1 B table id + 2 B result) over "
                                  "the whole captured step"),
            "modes": res,
            "sampled_parity_vs_oracle": all(r["sampled_parity_vs_oracle"] for r in res.values())}


def run_learned1m(args):
    """Config L: 1M prefixes (1 % /128), 2^28 lookups; the learned kernel against the plain tree
    forms on the same table and addresses (the block the default line carries, as its own line)."""
    import torch
    torch.cuda.set_device(0)
    stream = torch.cuda.Stream()
    b = block_learned1m(args, stream, args.steps, args.warmup, lookups=args.lookups)
    print(json.dumps({"metric": "B lookups/s, 1M-prefix FIB, learned vs plain tree",
                      "value": b["value"], "unit": UNIT, "n_gpus": 1, "steps": args.steps,
                      "warmup": args.warmup, "higher_is_better": True, "dtype": "u64",
                      "data": "synthetic (seeded)", "config": {"workload": b["workload"]},
                      **{k: v for k, v in b.items() if k not in ("workload", "value", "unit",
                                                                 "steps", "warmup")}}),
          flush=True)
    return 0


def serve_line(args):
    """Serving: Poisson arrivals of requests (32..65,536 addresses, log-uniform) over the 64 VRF
    tables (table drawn proportional to size), route updates at --update-rate changes per second
    applied while serving, latency from submit to results in place."""
    import torch
    import paper_2604_14650_gb300 as pb
    import synth
    torch.cuda.set_device(0)
    rng = np.random.default_rng(args.seed)
    sizes = np.exp(rng.uniform(np.log(1e3), np.log(3e5), args.tables)).astype(int)
    fibs_in = [synth.gen_fib(int(sz), seed=args.seed + 1000 + t, nh_max=4095)
               for t, sz in enumerate(sizes)]
    fibs = [pb.Fib(f.hi, f.lo, f.len, f.nh, format=args.format, builder=args.builder)
            for f in fibs_in]
    pool = 1 << 17
    pools = [synth.gen_trace(f, pool, seed=args.seed + 3000 + t) for t, f in enumerate(fibs_in)]
    nreq = int(args.rate * args.duration)
    p = sizes / sizes.sum()
    tabs = rng.choice(args.tables, size=nreq, p=p)
    lens = np.exp(rng.uniform(np.log(32), np.log(65536), nreq)).astype(int)
    offs = rng.integers(0, pool - 65536, nreq)
    gaps = rng.exponential(1.0 / args.rate, nreq)
    budget = int(sum(f.stats()["node_bytes"] + f.stats()["value_bytes"] for f in fibs) * 1.05)
    srv = pb.Server(slots=4, max_batch=1 << 18, mem_budget=budget, per_table=args.per_table,
                    bucketed=args.bucketed)
    try:
        line = _serve_loop(args, srv, fibs, fibs_in, pools, nreq, tabs, lens, offs, gaps, rng,
                           budget)
    finally:
        srv.close()
        for f in fibs:
            f.close()
    return line


def block_serve(args, rate=20000.0, duration=2.0, warmup=0.5):
    """The serving loop on the 64 VRF tables (device builder for the rebuilds), Poisson arrivals at
    `rate` requests per second for `duration` seconds after `warmup` seconds of the same load,
    1,000 route changes per second applied while serving."""
    import copy
    a = copy.copy(args)
    a.rate, a.duration, a.serve_warmup, a.update_rate = rate, duration, warmup, 1000.0
    a.builder, a.per_table, a.format, a.tables = "device", False, "f16hi", 64
    a.bucketed = False
    line = serve_line(a)
    return {"workload": line["config"]["workload"], "value": line["value"], "unit": UNIT,
            "latency_us": line["latency_us"], "batch_us": line["batch_us"],
            "requests_per_s": line["requests_per_s"], "mean_batch": line["mean_batch"],
            "updates_applied": line["updates_applied"], "rebuilds": line["rebuilds"],
            "rebuild_ms_mean": line["rebuild_ms_mean"], "graph_captures": line["graph_captures"],
            "requests_not_completed": line["requests_not_completed"],
            "last_error": line["last_error"],
            "parity": "each result equal alone, in the mix and to the oracle: "
                      "tests/test_gpu_server.py"}


def run_serve(args):
    print(json.dumps(serve_line(args)), flush=True)
    return 0


def _serve_loop(args, srv, fibs, fibs_in, pools, nreq, tabs, lens, offs, gaps, rng, budget):
    import threading
    import paper_2604_14650_gb300 as pb
    import synth
    out_pool = np.empty(1 << 26, np.uint16)
    for f in fibs:
        srv.add_table(f)
    tickets = []
    done = threading.Event()

    def updater():
        per = 10                                  # changes per 10 ms
        k = 0
        while not done.is_set():
            t = int(rng.integers(args.tables))
            upd = synth.gen_updates(fibs_in[t], per, seed=args.seed + 9, start=k * per)
            srv.update(t, *upd)
            k += 1
            time.sleep(per / args.update_rate)

    ut = threading.Thread(target=updater, daemon=True)
    ut.start()

    def phase(count):
        """Submits `count` requests on the Poisson schedule, then waits for them; returns
        (wall seconds, requests not completed)."""
        tickets.clear()
        t0 = time.perf_counter()
        nxt = t0
        pos = 0
        for i in range(count):
            nxt += gaps[i]
            while time.perf_counter() < nxt:
                pass
            n = int(lens[i])
            if pos + n > out_pool.size:
                pos = 0
            h, l = pools[tabs[i]]
            o = int(offs[i])
            tickets.append((srv.submit(int(tabs[i]), h[o:o + n], l[o:o + n],
                                       out_pool[pos:pos + n]), i))
            pos += n
        deadline = t0 + count / args.rate + 60.0    # never waits more than a minute past
        failed = 0
        for tk, _ in tickets:
            left = max(0.0, deadline - time.perf_counter())
            try:
                srv.wait(tk, int(left * 1e6))
            except pb.PlanbError:
                failed += 1
                if time.perf_counter() >= deadline:
                    break
        return time.perf_counter() - t0, failed

    # warm-up under the same load (first launches, graph captures, memory pools), then the
    # measured phase from zeroed statistics
    phase(min(nreq, int(args.rate * args.serve_warmup)))
    srv.reset_stats()
    wall, failed = phase(nreq)
    done.set()
    ut.join()
    st = srv.stats()
    detail = srv.error_detail()
    line = {"metric": "serving: lookups/s and p50/p99 request latency, 64 VRF tables",
            "value": st["lookups"] / wall / 1e9, "unit": UNIT, "n_gpus": 1,
            "higher_is_better": True, "dtype": "u64", "data": "synthetic (seeded)",
            "config": {"workload": f"Poisson arrivals at {args.rate:.0f} requests/s for "
                                   f"{args.duration:.1f} s, 32..65,536 addresses per request "
                                   f"(log-uniform), {args.tables} VRF tables, route updates at "
                                   f"{args.update_rate:.0f}/s, after {args.serve_warmup:.1f} s "
                                   "of the same load", "slots": 4,
                       "builder": args.builder,
                       "lookup_launch": "per table" if args.per_table else "single persistent",
                       "max_batch": 1 << 18, "mem_budget_bytes": budget},
            "latency_us": {"p50": st["p50_us"], "p99": st["p99_us"], "max": st["max_us"]},
            "batch_us": {"p50": st["batch_p50_us"], "p99": st["batch_p99_us"],
                         "max": st["batch_max_us"]},
            "graph_captures": st["recaptures"],
            "requests": st["requests"], "requests_per_s": st["requests"] / wall,
            "batches": st["batches"], "mean_batch": st["mean_batch"],
            "updates_applied": st["updates"], "rebuilds": st["update_batches"],
            "rebuild_ms_mean": st["rebuild_ms_mean"], "last_error": st["last_error"],
            "last_error_detail": detail, "requests_not_completed": failed}
    return line


def run_build(args):
    """Build and rebuild latency (Section 3.6 rebuild-and-swap; the paper quotes a full rebuild of
    a 1M-prefix table): planb_build, then planb_update with 1,000-change batches, by the host
    builder and by the device builder, on 200k- and 1M-prefix FIBs. Both builders' tables are
    checked to be identical."""
    import torch
    import paper_2604_14650_gb300 as pb
    import synth
    torch.cuda.set_device(0)
    res = {}
    for n in (200_000, 1_000_000):
        f = synth.gen_fib(n, seed=args.seed, nh_max=4095)
        row = {}
        images = {}
        for builder in ("host", "device"):
            walls = []
            for rep in range(3):
                t0 = time.perf_counter()
                fib = pb.Fib(f.hi, f.lo, f.len, f.nh, format=args.format, builder=builder)
                walls.append((time.perf_counter() - t0) * 1e3)
                if rep < 2:
                    fib.close()
            rebuild = []
            for k in range(max(3, args.steps)):
                upd = synth.gen_updates(f, 1000, seed=args.seed + 7, start=k * 1000)
                t0 = time.perf_counter()
                fib.update(*upd)
                rebuild.append((time.perf_counter() - t0) * 1e3)
            images[builder] = fib.table_dump()
            st = fib.stats()
            row[builder] = {"build_ms_median": float(np.median(walls)),
                            "rebuild_ms_median": float(np.median(rebuild)),
                            "rebuild_ms_p90": float(np.percentile(rebuild, 90)),
                            "stats_build_ms": st["build_ms"], "n_intervals": st["n_intervals"]}
            fib.close()
        row["identical_tables"] = bool(np.array_equal(images["host"], images["device"]))
        res[str(n)] = row
    v = res["1000000"]["device"]["rebuild_ms_median"]
    print(json.dumps({"metric": "rebuild latency, 1M-prefix FIB, 1,000-change batch",
                      "value": v, "unit": "ms", "n_gpus": 1, "steps": max(3, args.steps),
                      "warmup": 0, "higher_is_better": False, "dtype": "u64",
                      "data": "synthetic (seeded)",
                      "config": {"workload": "planb_build and planb_update (1,000 changes, half "
                                             "withdraws) on 200k- and 1M-prefix FIBs"},
                      "builders": res}), flush=True)
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "vrf64":
        return run_vrf64(args)
    if args.workload == "learned1m":
        return run_learned1m(args)
    if args.workload == "serve":
        return run_serve(args)
    if args.workload == "build":
        return run_build(args)
    if args.workload == "small":
        args.prefixes, args.lookups = 1000, 1_000_000
    return run_planb(args)


if __name__ == "__main__":
    sys.exit(main())
