"""Free Join on GB300: throughput of the star-join workload.

Workload (one step = the whole hot path, from the base tables): fact table F
with 10,000,000 rows of 4 int32 foreign keys, each Zipf(s=1.1) over its
dimension's keys; dimensions D1..D4 of 100K / 250K / 500K / 1M rows (int32
key, int32 attribute) with the selection attribute < 1e8 (10%).  The
left-deep plan [F, D1, D2, D3, D4] is converted by binary2fj and factored;
every step builds the COLT levels it needs from scratch and returns COUNT(*)
and MIN of each dimension attribute.

Metric: input + output tuples per second (inputs = rows of every atom,
outputs = COUNT), with the inputs resident in HBM; `e2e` repeats it through
the public API from pinned host buffers.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl fj|reference]
                    [--workload star|rmat-triangle|batched|chooser|ablation]

`--workload rmat-triangle` times the triangle count on the R-MAT graph of
2^20 vertices and 2^24 edges instead (a second JSON line format, same keys).
"""

from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2301_10841_gb300 import datagen as G  # noqa: E402

METRIC = "tuples/sec (in+out), star join, plain converted-binary Free Join plan"
UNIT = "tuples/s"
DIMS = G.STAR_DIMS
N_FACT = 10_000_000
THETA = G.STAR_THETA
MIN_VARS = [4, 5, 6, 7]
L2_FLUSH_BYTES = 256 << 20
L2_NOTE = ("flushed between steps: a 256 MB buffer written, then a second 256 MB buffer read, "
           "so the step starts with a cold L2 holding no dirty lines")
RESULT_D2H_BYTES = 8 + 4 * 32 + 8 + 4 + 4 + 8 * 16  # the library's result block


def workload_config(n_fact=N_FACT):
    return {
        "workload": f"star join: F {n_fact} rows x 4 int32 FK Zipf(1.1) via seeded permutation; "
                    f"D1..D4 = {'/'.join(str(d) for d in DIMS)} rows (int32 key, int32 attr "
                    f"uniform [0,1e9)), selection attr < 1e8; COUNT(*) + MIN(a1..a4)",
        "plan": "factor(binary2fj([F,D1,D2,D3,D4])), static cover, batch 1024",
        "launch": "one CUDA graph launch per step (the execution captured once)",
        "seed": 2,
        "l2": L2_NOTE,
        "in_tuples": n_fact + sum(DIMS),
    }


class L2Flush:
    """Evicts the L2 between timed steps: writes a buffer larger than the L2,
    then reads a second one, so the dirty lines of the write are written back
    before the next timed region instead of during it."""

    def __init__(self, dev):
        import torch
        self.w = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
        self.r = torch.ones(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)

    def zero_(self):
        self.w.zero_()
        self.r.max()


# ---------------------------------------------------------------------------
# Clock sampling during the timed region.
# ---------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index=0):
        self.dev = device_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.dev}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (FileNotFoundError, OSError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
# Algorithmic bytes of the probe phase (the dominant kernel).
# ---------------------------------------------------------------------------

def probe_phase_bytes(fact, dims, theta):
    """Compulsory HBM bytes of node 0 of the factored star plan: every 32-byte
    sector of a fact column that holds a row the plan must read (k1 for all
    rows; k_i only for rows that survived the probes of D1..D(i-1)), 16 bytes
    per distinct dimension key probed (one hash slot each), and the 4-byte
    per-survivor reads of the tail (vector length, offset and attribute).
    Computed from the data by a host pass."""
    n = len(fact["cols"][0])
    alive = np.ones(n, dtype=bool)
    total = 0
    for i, (fk, d) in enumerate(zip(fact["cols"], dims)):
        rows = np.nonzero(alive)[0]
        total += 32 * len(np.unique(rows >> 3))  # sectors of column k_i read
        keys = fk[rows]
        total += 16 * len(np.unique(keys))       # hash slots probed
        key, attr = d["cols"]
        passing = np.zeros(len(key) + 1, dtype=bool)
        passing[key[attr < theta]] = True
        hit = passing[np.clip(keys, 0, len(key))]
        alive[rows[~hit]] = False
    survivors = int(alive.sum())
    total += survivors * 4 * 4 * 3  # per tail atom: count, begin, perm -> attr
    return total, survivors


def build_bytes(dims, theta):
    """Compulsory bytes of the root build of the star plan's four dimension
    roots: 4 B per row for each column read (key and selection attribute),
    and per passing row (every key has one row) 16 B for clearing the slot
    the previous build used, 12 B of staging (row, slot, rank) and 48 B of
    entry (slot entry word, key word, count, first offset, fill cursor,
    child state, child first, child key count, slot list, the row's offset,
    the tail MIN)."""
    total = 0
    for d in dims:
        key, attr = d["cols"]
        total += 8 * len(key)
        total += (16 + 12 + 48) * int((attr < theta).sum())
    return total


def source_hash():
    h = hashlib.sha256()
    for f in ("fj_kernels.cuh", "fj_exec.cuh", "fj_scan.cuh", "fj_internal.h"):
        with open(os.path.join(ROOT, "paper_2301_10841_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def profiled_traffic(kernel_hash):
    """DRAM bytes per launch of the dominant kernel from the committed ncu
    summary, if it was taken on the current kernel source."""
    import re
    path = os.path.join(ROOT, "profiles", "scan_fused_star_F10M.md")
    try:
        with open(path) as f:
            text = f.read()
    except OSError:
        return None
    src = re.search(r"kernel_source:\s*([0-9a-f]+)", text)
    tr = re.search(r"traffic_bytes_per_launch:\s*([0-9]+)", text)
    if src and tr and src.group(1) == kernel_hash:
        return int(tr.group(1))
    return None


# ---------------------------------------------------------------------------
# CPU baseline (the oracle) -- the only place bench.py runs oracle/.
# ---------------------------------------------------------------------------

def _oracle_join_parallel(fact, dims, n, cores):
    """The oracle's binary join with its outer loop (the fact rows) split
    into `cores` contiguous parts run on as many host threads (ctypes drops
    the GIL during each call); counts add up and MINs take the least."""
    import oracle
    from concurrent.futures import ThreadPoolExecutor
    bounds = [n * i // cores for i in range(cores + 1)]
    parts = [G.star_query({"name": "F", "cols": [c[a:b] for c in fact["cols"]]}, dims,
                          theta=THETA) for a, b in zip(bounds, bounds[1:]) if b > a]
    with ThreadPoolExecutor(max_workers=len(parts)) as ex:
        res = list(ex.map(lambda q: oracle.binary_join(q, min_vars=MIN_VARS), parts))
    cnt = sum(r[0] for r in res)
    mins = []
    for i in range(len(MIN_VARS)):
        vals = [r[1][i] for r in res if r[1][i] is not None]
        mins.append(min(vals) if vals else None)
    return cnt, mins


def cpu_baseline_leg(fact, dims, budget_s=12.0, start_rows=250_000):
    """The oracle on the host cores -- the only part of the star workload
    that runs oracle/.

    (i) single thread: the oracle's left-deep hash join on a prefix of F
    (full dimensions), the prefix grown until one run takes a few seconds
    (the whole of F when that is quicker), repeated for about `budget_s`;
    (ii) the same join with F split over every host core.
    Also returns the exact result on the whole of F, computed twice:
    by the oracle's hash join and by the direct-address semi-join of
    `oracle.closed`, for the parity check of the GPU result."""
    import oracle
    from oracle import closed
    oracle.build()
    n = start_rows
    n_all = len(fact["cols"][0])
    while True:
        q = G.star_query({"name": "F", "cols": [c[:n] for c in fact["cols"]]}, dims, theta=THETA)
        t0 = time.perf_counter()
        cnt, mins, _ = oracle.binary_join(q, min_vars=MIN_VARS)
        dt = time.perf_counter() - t0
        if dt > 2.0 or n >= n_all:
            break
        n = min(n_all, n * 4)
    reps = max(1, int(budget_s / max(dt, 1e-3)))
    times = [dt]
    for _ in range(reps - 1):
        t0 = time.perf_counter()
        oracle.binary_join(q, min_vars=MIN_VARS)
        times.append(time.perf_counter() - t0)
    tin = n + sum(len(d["cols"][0]) for d in dims)
    tps = (tin + cnt) / statistics.median(times)
    cores = os.cpu_count() or 1
    ptimes = []
    for _ in range(3):
        t0 = time.perf_counter()
        pcnt, pmins = _oracle_join_parallel(fact, dims, n, cores)
        ptimes.append(time.perf_counter() - t0)
    if (pcnt, pmins) != (cnt, mins):
        raise SystemExit(f"oracle: split join {(pcnt, pmins)} differs from {(cnt, mins)}")
    ptps = (tin + cnt) / statistics.median(ptimes)
    cpu = {"value": tps, "unit": UNIT, "cores": 1, "kind": "oracle",
           "sample": f"hash binary join (oracle O1, single thread) on the first {n} fact rows "
                     f"with full dimensions, median of {len(times)} runs",
           "seconds": sum(times),
           "all_cores": {"value": ptps, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"the same join with the {n} fact rows split into {cores} "
                                   f"parts on {cores} host threads (nproc), median of "
                                   f"{len(ptimes)} runs", "seconds": sum(ptimes)}}
    # The exact result over the whole of F.
    if n < n_all:
        qa = G.star_query(fact, dims, theta=THETA)
        cnt, mins, _ = oracle.binary_join(qa, min_vars=MIN_VARS)
    dcnt, dmins = closed.star_join_direct(fact["cols"], [d["cols"] for d in dims],
                                          [THETA] * len(dims))
    exact = {"oracle_binary_join": {"count": cnt, "mins": mins},
             "direct_address": {"count": dcnt, "mins": dmins}, "fact_rows": n_all}
    return cpu, exact


def run_reference(args, rank, world):
    """Reference arm: the oracle on the host cores, a bounded sample per step."""
    if rank != 0:
        return
    import oracle
    oracle.build()
    fact, dims = G.star_schema(n_fact=N_FACT, dims=DIMS, s=1.1, seed=2)
    # A bounded prefix of F per step, so K steps stay within a few minutes.
    n = 1_000_000 if args.steps <= 100 else max(100_000, 100_000_000 // args.steps)
    q = G.star_query({"name": "F", "cols": [c[:n] for c in fact["cols"]]}, dims, theta=THETA)
    tin = n + sum(DIMS)
    for _ in range(args.warmup):
        oracle.binary_join(q, min_vars=MIN_VARS)
    times, cnt = [], 0
    for _ in range(args.steps):
        t0 = time.perf_counter()
        cnt, _, _ = oracle.binary_join(q, min_vars=MIN_VARS)
        times.append(time.perf_counter() - t0)
    ms = 1000 * statistics.mean(times)
    value = (tin + cnt) / (ms / 1000)
    sample = (f"hash binary join (oracle O1, single thread) on the first {n} of {N_FACT} fact "
              f"rows with full dimensions, per step")
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "i32",
            "data": "synthetic", "config": workload_config(), "impl": "reference",
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# The CUDA path.
# ---------------------------------------------------------------------------

def run_fj(args, rank, world):
    import torch

    from paper_2301_10841_gb300 import fj

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    fact, dims = G.star_schema(n_fact=args.n_fact, dims=DIMS, s=1.1, seed=2)
    rel_np = [fact] + dims
    ctx = fj.Context(local)
    dcols = {r["name"]: [torch.from_numpy(c).to(dev) for c in r["cols"]] for r in rel_np}
    rels = {name: ctx.relation(cols, name) for name, cols in dcols.items()}
    q = G.star_query(fact, dims, theta=THETA)
    atoms = [{"rel": rels[a["rel"]["name"]], "vars": a["vars"], "preds": a["preds"]} for a in q]
    plan = fj.binary_to_free_plan(atoms, [0, 1, 2, 3, 4], factor=True)
    prep = fj.Prepared(ctx, atoms, plan, out_mode="count_min", min_vars=MIN_VARS,
                       batch_size=args.batch, flags=fj.FLAG_TIMING)
    # One step = one launch of a CUDA graph holding the whole execution from
    # the base tables (COLT state reset, root build, node 0), captured once.
    batch = fj.Batch(ctx, [prep], graph=True)
    flush = L2Flush(dev)
    stream = torch.cuda.current_stream()

    for _ in range(args.warmup):
        batch.launch()
        ref = batch.results()[0]
    expect = (ref.count, ref.mins)

    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    times, expand_ns, expand_n, kernels, build_ns = [], 0, 0, 0, 0
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        batch.launch()
        e1.record(stream)
        res = batch.results()[0]
        torch.cuda.synchronize()
        if (res.count, res.mins) != expect:
            raise SystemExit(f"result changed between steps: {(res.count, res.mins)} vs {expect}")
        times.append(e0.elapsed_time(e1))
        expand_ns += res.counters["expand_ns"]
        expand_n += res.counters["expand_launches"]
        build_ns += res.counters["build_ns"]
        kernels += res.counters["kernels"]
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = sum(times) / len(times)
    if world > 1:
        t = torch.tensor([ms], device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms = float(t.item())
    in_tuples = args.n_fact + sum(DIMS)
    per_rank = in_tuples + expect[0]
    value = per_rank * world / (ms / 1000)

    # End to end through the public API from pinned host buffers.
    e2e = None
    if not args.no_e2e:
        pinned = {name: [torch.from_numpy(c).pin_memory() for c in r["cols"]]
                  for name, r in ((r["name"], r) for r in rel_np)}
        h2d = sum(c.numel() * 4 for cols in pinned.values() for c in cols)

        def e2e_step():
            hr = {name: ctx.relation_host(cols, name) for name, cols in pinned.items()}
            at = [{"rel": hr[a["rel"]["name"]], "vars": a["vars"], "preds": a["preds"]} for a in q]
            r = fj.execute(ctx, at, plan, out_mode="count_min", min_vars=MIN_VARS,
                           batch_size=args.batch)
            for h in hr.values():
                h.release()
            return r

        for _ in range(max(1, args.warmup // 2)):
            e2e_step()
        torch.cuda.synchronize()
        wall = []
        for _ in range(args.steps):
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            r = e2e_step()
            wall.append(time.perf_counter() - t0)
            if (r.count, r.mins) != expect:
                raise SystemExit("e2e result differs from the device-resident run")
        e2e = {"value": per_rank * world / statistics.mean(wall), "unit": UNIT,
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": RESULT_D2H_BYTES,
               "ms_per_step": 1000 * statistics.mean(wall)}

    if rank != 0:
        return
    peak, peak_kind = measured_peaks()
    alg, survivors = probe_phase_bytes(fact, dims, THETA)
    launch_s = expand_ns / max(1, expand_n) / 1e9
    achieved = alg / launch_s / 1e9 if launch_s > 0 else None
    khash = source_hash()
    roofline = {"bound": "hbm", "kernel": "k_scan_fused (node 0: cover stream, all probes, aggregate)",
                "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak if achieved else None, "peak_kind": peak_kind,
                "traffic": profiled_traffic(khash), "algorithmic_bytes": alg,
                "launch_us": launch_s * 1e6, "kernel_source": khash}
    # The root build (k_force_roots, one launch per step) against the same
    # peak, and the whole step: every algorithmic byte of the step over the
    # step's time.
    b_alg = build_bytes(dims, THETA)
    b_s = build_ns / max(1, args.steps) / 1e9
    b_ach = b_alg / b_s / 1e9 if b_s > 0 else None
    roofline_build = {"bound": "hbm", "kernel": "k_force_roots (the four dimension roots)",
                      "achieved": b_ach, "peak": peak, "unit": "GB/s",
                      "frac": b_ach / peak if b_ach else None, "peak_kind": peak_kind,
                      "algorithmic_bytes": b_alg, "launch_us": b_s * 1e6}
    step_s = statistics.mean(times) / 1000
    roofline_step = {"bound": "hbm", "algorithmic_bytes": alg + b_alg,
                     "achieved": (alg + b_alg) / step_s / 1e9, "peak": peak, "unit": "GB/s",
                     "frac": (alg + b_alg) / step_s / 1e9 / peak, "step_us": step_s * 1e6}
    cpu, parity = None, None
    if not args.no_cpu_baseline and world == 1:
        cpu, exact = cpu_baseline_leg(fact, dims)
        got = {"count": expect[0], "mins": list(expect[1])}
        ok = all(got == e for e in (exact["oracle_binary_join"], exact["direct_address"]))
        parity = {"exact": ok, "gpu": got, **exact}
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "i32",
            "data": "synthetic", "config": workload_config(args.n_fact),
            "result": {"count": expect[0], "mins": expect[1], "survivors": survivors},
            "parity": parity,
            "roofline": roofline, "roofline_build": roofline_build,
            "roofline_step": roofline_step, "cpu_baseline": cpu, "e2e": e2e, "clocks": clk,
            "counters": res.counters,
            "gpu_launches": kernels, "impl": "fj"}
    print(json.dumps(line), flush=True)
    if parity is not None and not parity["exact"]:
        raise SystemExit("the GPU result differs from the oracle's on the full workload")


# ---------------------------------------------------------------------------
# Second workload (--workload rmat-triangle): triangle count on the R-MAT
# graph with 2^20 vertices and 2^24 distinct directed edges.
# ---------------------------------------------------------------------------

RMAT_SCALE = 20
RMAT_METRIC = "tuples/sec (in+out), R-MAT triangle count, Free Join triangle plan"
# The triangle plan of Section 3.3 over E1(x,y), E2(y,z), E3(z,x).
TRI_PLAN = [[(0, (0, 1)), (1, (1,)), (2, (0,))], [(1, (2,)), (2, (2,))]]


def run_rmat(args, rank, world):
    import torch

    from paper_2301_10841_gb300 import fj

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    n_edges = 16 << RMAT_SCALE
    e = G.rmat(RMAT_SCALE, n_edges, seed=3)
    ctx = fj.Context(local)
    rel = ctx.relation([torch.from_numpy(c).to(dev) for c in e["cols"]], "E")
    q = G.triangle_query(e)
    atoms = [{"rel": rel, "vars": a["vars"], "rel_cols": a["rel_cols"]} for a in q]
    prep = fj.Prepared(ctx, atoms, TRI_PLAN, out_mode="count", cover="fewest",
                       flags=fj.FLAG_TIMING)
    flush = L2Flush(dev)
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        prep.reset()
        prep.execute_async()
        expect = prep.result().count
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    times, kernels = [], 0
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        prep.reset()
        prep.execute_async()
        e1.record(stream)
        res = prep.result()
        torch.cuda.synchronize()
        if res.count != expect:
            raise SystemExit(f"triangle count changed between steps: {res.count} vs {expect}")
        times.append(e0.elapsed_time(e1))
        kernels += res.counters["kernels"]
    clk = clocks.stop()
    ms = sum(times) / len(times)
    if world > 1:
        t = torch.tensor([ms], device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms = float(t.item())
    per_rank = 3 * n_edges + expect
    value = per_rank * world / (ms / 1000)
    e2e = None
    if not args.no_e2e:
        pinned = [torch.from_numpy(c).pin_memory() for c in e["cols"]]

        def e2e_step():
            hr = ctx.relation_host(pinned, "E")
            at = [{"rel": hr, "vars": a["vars"], "rel_cols": a["rel_cols"]} for a in q]
            r = fj.execute(ctx, at, TRI_PLAN, out_mode="count", cover="fewest")
            hr.release()
            return r

        e2e_step()
        wall = []
        for _ in range(max(3, min(args.steps, 10))):
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            r = e2e_step()
            wall.append(time.perf_counter() - t0)
            if r.count != expect:
                raise SystemExit("e2e triangle count differs from the device-resident run")
        e2e = {"value": per_rank * world / statistics.mean(wall), "unit": UNIT,
               "h2d_bytes_per_step": 2 * 4 * n_edges, "d2h_bytes_per_step": RESULT_D2H_BYTES,
               "ms_per_step": 1000 * statistics.mean(wall)}
    if rank != 0:
        return
    peak, peak_kind = measured_peaks()
    # Compulsory bytes: both columns of each of the three atoms read once.
    alg = 3 * 2 * 4 * n_edges
    achieved = alg / (ms / 1000) / 1e9
    cpu = None
    if not args.no_cpu_baseline and world == 1:
        import oracle
        oracle.build()
        small = G.rmat(16, 16 << 16, seed=3)
        t0 = time.perf_counter()
        c_small = oracle.generic_join(G.triangle_query(small))[0]
        dt = time.perf_counter() - t0
        cpu = {"value": (3 * (16 << 16) + c_small) / dt, "unit": UNIT, "cores": 1,
               "kind": "oracle",
               "sample": f"Generic Join (oracle O2, single thread) triangle count on the R-MAT "
                         f"graph of scale 16 (2^20 edges, {c_small} triangles), one run",
               "seconds": dt}
    line = {"metric": RMAT_METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "i32",
            "data": "synthetic",
            "config": {"workload": f"R-MAT (0.57, 0.19, 0.19), 2^{RMAT_SCALE} vertices, "
                                   f"{n_edges} distinct directed edges without self-loops, "
                                   f"seed 3; triangle count Q(x,y,z) :- E(x,y),E(y,z),E(z,x)",
                       "plan": "[[E1(x,y),E2(y),E3(x)],[E2(z),E3(z)]], fewest-keys cover",
                       "l2": L2_NOTE,
                       "in_tuples": 3 * n_edges},
            "result": {"count": expect},
            "roofline": {"bound": "hbm", "kernel": "whole step (every launch)",
                         "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "peak_kind": peak_kind, "traffic": None,
                         "algorithmic_bytes": alg, "launch_us": ms * 1000},
            "cpu_baseline": cpu, "e2e": e2e, "clocks": clk, "counters": res.counters,
            "gpu_launches": kernels, "impl": "fj"}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# Third workload (--workload batched): 256 independent PK-FK chain and star
# queries; the queries that run without a host decision form one batch
# captured into a CUDA graph (one launch per execution), the others run one
# by one; compared with all 256 run one by one with a synchronization each.
# ---------------------------------------------------------------------------

BATCH_METRIC = "tuples/sec (in+out), 256 batched PK-FK chain/star queries"


def run_batched(args, rank, world):
    import torch

    from paper_2301_10841_gb300 import fj

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    ctx = fj.Context(local)
    t_gen = time.perf_counter()
    queries = []
    in_tuples = 0
    alg = 0  # compulsory bytes: every column of every atom read once
    for q in range(args.n_queries):
        atoms, order, mins = G.batch_query(q, max_rows=args.max_rows)
        rels = {}
        dq = []
        for a in atoms:
            key = id(a["rel"])
            if key not in rels:
                rels[key] = ctx.relation([torch.from_numpy(c).to(dev) for c in a["rel"]["cols"]])
            dq.append({"rel": rels[key], "vars": a["vars"], "rel_cols": a["rel_cols"],
                       "preds": a["preds"]})
            in_tuples += len(a["cols"][0])
            alg += sum(4 * len(c) for c in a["cols"])
        plan = fj.binary_to_free_plan(dq, order, factor=True)
        queries.append((dq, plan, mins))
    t_gen = time.perf_counter() - t_gen
    # Autotune each query (cover-batch size x load factor), untimed.
    t_tune = time.perf_counter()
    tuned, choice = [], []
    for dq, plan, mins in queries:
        p, cfg, _ = fj.autotune(ctx, dq, plan, out_mode="count_min", min_vars=mins,
                                batch_sizes=(1024, 8192), load_factors=(0.25, 0.5), reps=1)
        tuned.append(p)
        choice.append(cfg)
    t_tune = time.perf_counter() - t_tune
    graphed, single = [], []
    for i, p in enumerate(tuned):
        try:
            fj.Batch(ctx, [p]).free()
            graphed.append(i)
        except fj.FJError:
            single.append(i)
    batch = fj.Batch(ctx, [tuned[i] for i in graphed], graph=True, concurrent=True)
    flush = L2Flush(dev)
    stream = torch.cuda.current_stream()

    def step_batched():
        res = dict(zip(graphed, batch.execute()))
        for i in single:
            tuned[i].reset()
            res[i] = tuned[i].execute()
        return [(res[i].count, res[i].mins) for i in range(len(tuned))]

    def step_plain():
        out = []
        for p in tuned:
            p.reset()
            r = p.execute()
            out.append((r.count, r.mins))
        return out

    for _ in range(args.warmup):
        expect = step_batched()
        if step_plain() != expect:
            raise SystemExit("plain and batched results differ")
    out_tuples = sum(c for c, _ in expect)
    launches = sum(r.counters["kernels"] for r in batch.execute())
    for i in single:
        tuned[i].reset()
        launches += tuned[i].execute().counters["kernels"]

    def timed(step):
        times = []
        for _ in range(args.steps):
            flush.zero_()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            got = step()
            e1.record(stream)
            torch.cuda.synchronize()
            if got != expect:
                raise SystemExit("result changed between steps")
            times.append(e0.elapsed_time(e1))
        return sum(times) / len(times)

    if world > 1:
        torch.distributed.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    ms = timed(step_batched)
    clk = clocks.stop()
    ms_plain = timed(step_plain)
    if world > 1:
        t = torch.tensor([ms], device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms = float(t.item())
    per_rank = in_tuples + out_tuples
    value = per_rank * world / (ms / 1000)
    if rank != 0:
        return
    peak, peak_kind = measured_peaks()
    achieved = alg / (ms / 1000) / 1e9
    line = {"metric": BATCH_METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "i32",
            "data": "synthetic",
            "config": {"workload": f"{args.n_queries} PK-FK queries (datagen.batch_query, seeds "
                                   f"4..{3 + args.n_queries}): chains and stars of 2-6 relations, "
                                   f"rows log-uniform in [1e3, {args.max_rows:.0e}], Zipf FKs "
                                   f"s in [0.5, 1.5], selection p2 < 5e8; COUNT + MIN(p1) each",
                       "plan": "factor(binary2fj(order)) per query, autotuned cover-batch "
                               "size and load factor; one CUDA graph with eight concurrent "
                               "branches",
                       "graphed_queries": len(graphed), "single_queries": len(single),
                       "l2": L2_NOTE, "in_tuples": in_tuples},
            "result": {"out_tuples": out_tuples},
            "plain": {"ms_per_step": ms_plain,
                      "value": per_rank * world / (ms_plain / 1000),
                      "note": "every query reset and executed one by one, one sync each"},
            "autotune": {"seconds": t_tune, "choices": {f"{b}/{l}": choice.count((b, l))
                                                        for b, l in sorted(set(choice))}},
            "generate_seconds": t_gen,
            "roofline": {"bound": "hbm", "kernel": "whole batch (every launch)",
                         "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "peak_kind": peak_kind, "traffic": None,
                         "algorithmic_bytes": alg, "launch_us": ms * 1000},
            "cpu_baseline": None, "e2e": None, "clocks": clk,
            "gpu_launches": launches * args.steps, "impl": "fj"}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# Fourth workload (--workload chooser): held-out 5-relation snowflake and
# cycle queries run with the plain converted binary plan, the same plan with
# the fewest-keys cover, and the order the learned chooser picks (its
# network trained first, untimed, on work the engine reports for smaller
# generated queries).
# ---------------------------------------------------------------------------

CHOOSER_METRIC = "tuples/sec (in+out), held-out snowflake/cycle queries, learned plan chooser"


def run_chooser(args, rank, world):
    import torch

    from paper_2301_10841_gb300 import chooser as C
    from paper_2301_10841_gb300 import fj

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    ctx = fj.Context(local)

    def device(atoms):
        return [{"rel": ctx.relation([torch.from_numpy(c).to(dev) for c in a["cols"]]),
                 "vars": a["vars"]} for a in atoms]

    # Pretraining: small engine-generated queries, four orders x two cover
    # policies each, labelled with the engine's work (untimed).
    t_train = time.perf_counter()
    rng = np.random.default_rng(0)
    xs, ys = [], []
    for q in range(args.train_queries):
        atoms, _ = G.chooser_query(q, args.train_min_rows, args.train_max_rows)
        d = device(atoms)
        cands = C.training_candidates([a["vars"] for a in atoms], 4, rng)
        for f, w, _ in C.samples(fj, ctx, d, cands, label=args.label):
            xs.append(f)
            ys.append(w)
        for a in d:
            a["rel"].release()
    # Fine-tuning: queries composed from a pool of relations at the held-out
    # scale (their own seeds and relations), six orders x two policies each,
    # labelled with the device time.
    xt, yt = [], []
    t_pool = 0.0
    if args.tune_queries:
        t0 = time.perf_counter()
        pool = G.chooser_pool(args.pool_size, args.pool_min_rows, args.pool_max_rows)
        dpool = {r["name"]: ctx.relation([torch.from_numpy(c).to(dev) for c in r["cols"]])
                 for r in pool}
        t_pool = time.perf_counter() - t0
        for q in range(args.tune_queries):
            atoms, _ = G.pool_query(pool, q)
            d = [{"rel": dpool[a["rel"]["name"]], "vars": a["vars"], "rel_cols": a["rel_cols"]}
                 for a in atoms]
            cands = C.training_candidates([a["vars"] for a in atoms], 6, rng)
            for f, t, _ in C.samples(fj, ctx, d, cands, label="time"):
                xt.append(f)
                yt.append(t)
        for r in dpool.values():
            r.release()
    if xs:
        model, losses = C.fit(fj, ctx, np.stack(xs), np.asarray(ys, dtype=np.float32),
                              scaler_rows=np.stack(xs + xt))
        if xt:
            losses += C.finetune(model, np.stack(xt), np.asarray(yt, dtype=np.float32))
    else:
        model, losses = C.fit(fj, ctx, np.stack(xt), np.asarray(yt, dtype=np.float32))
    t_train = time.perf_counter() - t_train

    # Held-out queries: the plain converted binary plan, the same plan with
    # the fewest-keys cover, and the chooser's plan and policy.  One query at
    # a time (its three prepared plans, then freed: the large ones do not
    # all fit at once); a step is one pass over every query, so each
    # policy's time per step is the sum over queries of its mean time per
    # execution (from scratch, L2 flushed before each, CUDA events).
    names = ("plain", "fewest", "learned")
    in_tuples, out_tuples = 0, 0
    choices = []
    flush = L2Flush(dev)
    stream = torch.cuda.current_stream()
    ms = {k: 0.0 for k in names}
    per_query = {k: [] for k in names}
    clocks = ClockSampler(local)
    clocks.start()
    for q in range(2000, 2000 + args.n_queries):
        atoms, kind = G.chooser_query(q, args.min_rows, args.max_rows)
        d = device(atoms)
        in_tuples += sum(len(a["cols"][0]) for a in atoms)
        declared = fj.binary_to_free_plan(d, list(range(len(atoms))), factor=True)
        plan, pol, order = fj.choose_plan(ctx, d, model)
        choices.append({"kind": kind, "order": order, "cover": pol})
        preps = {"plain": fj.Prepared(ctx, d, declared, out_mode="count"),
                 "fewest": fj.Prepared(ctx, d, declared, out_mode="count", cover="fewest"),
                 "learned": fj.Prepared(ctx, d, plan, out_mode="count", cover=pol)}
        counts = {k: p.execute().count for k, p in preps.items()}
        if len(set(counts.values())) != 1:
            raise SystemExit(f"query {q}: results differ between policies: {counts}")
        out_tuples += counts["plain"]
        for k, p in preps.items():
            times = []
            for i in range(args.warmup + args.steps):
                flush.zero_()
                torch.cuda.synchronize()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                p.reset()
                p.execute_async()
                e1.record(stream)
                r = p.result()
                torch.cuda.synchronize()
                if r.count != counts[k]:
                    raise SystemExit("result changed between steps")
                if i >= args.warmup:
                    times.append(e0.elapsed_time(e1))
            ms[k] += sum(times) / len(times)
            per_query[k].append(round(min(times), 3))
            p.free()
        for a in d:
            a["rel"].release()
    clk = clocks.stop()
    if rank != 0:
        return
    tot = in_tuples + out_tuples
    line = {"metric": CHOOSER_METRIC, "value": tot / (ms["learned"] / 1000), "unit": UNIT,
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms["learned"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "i32", "data": "synthetic",
            "config": {"workload": f"{args.n_queries} held-out queries (datagen.chooser_query, "
                                   f"seeds 2005..): 5-relation snowflakes and 5-cycles, rows "
                                   f"log-uniform in [{args.min_rows}, {args.max_rows}], Zipf "
                                   f"keys s in [0.8, 1.6]; COUNT(*)",
                       "training": f"pretraining: {args.train_queries} generated queries of "
                                   f"{args.train_min_rows}-{args.train_max_rows} rows, the "
                                   "declared order and three other connected orders each, both "
                                   f"cover policies, label log2 engine {args.label}, 60 epochs; "
                                   f"fine-tuning: {args.tune_queries} snowflakes and 5-cycles "
                                   f"over a pool of {args.pool_size} relations of "
                                   f"{args.pool_min_rows}-{args.pool_max_rows} rows "
                                   "(datagen.chooser_pool/pool_query, other seeds than the "
                                   "held-out queries), the declared order and five others, both "
                                   "policies, label log2 device time, 40 epochs; all on the "
                                   "library's kernels",
                       "l2": L2_NOTE, "in_tuples": in_tuples},
            "result": {"out_tuples": out_tuples},
            "policies": {k: {"ms_per_step": v, "value": tot / (v / 1000)} for k, v in ms.items()},
            "speedup_vs_plain": ms["plain"] / ms["learned"],
            "speedup_vs_fewest": ms["fewest"] / ms["learned"],
            "choices": choices,
            "per_query_ms": per_query,
            "train": {"seconds": t_train, "pool_seconds": t_pool, "samples": len(ys),
                      "tune_samples": len(yt), "loss_first": losses[0],
                      "loss_last": losses[-1]},
            "roofline": None, "cpu_baseline": None, "e2e": None, "clocks": clk,
            "gpu_launches": None, "impl": "fj"}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# Sixth workload (--workload rmat-4cycle): the 4-cycle count on the full-size
# R-MAT graph (config 3's cyclic query), one execution of minutes, checked
# against the oracle's 2-path count stored in tests/golden/rmat_counts.json
# (written by tests/golden/make_rmat_counts.py --full-size, oracle only).
# ---------------------------------------------------------------------------

RMAT4_METRIC = "tuples/sec (in+out), R-MAT 4-cycle count, Generic Join plan, fewest-keys cover"


def run_rmat4(args, rank, world):
    import torch

    from paper_2301_10841_gb300 import fj

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    scale = args.rmat_scale or RMAT_SCALE
    n_edges = 16 << scale
    e = G.rmat(scale, n_edges, seed=3)
    ctx = fj.Context(local)
    rel = ctx.relation([torch.from_numpy(c).to(dev) for c in e["cols"]], "E")
    q = G.four_cycle_query(e)
    atoms = [{"rel": rel, "vars": a["vars"], "rel_cols": a["rel_cols"]} for a in q]
    plan = fj.generic_join_plan(atoms, [0, 1, 2, 3])
    prep = fj.Prepared(ctx, atoms, plan, out_mode="count", cover="fewest")
    stream = torch.cuda.current_stream()
    clocks = ClockSampler(local)
    clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    prep.execute_async()
    e1.record(stream)
    res = prep.result()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    clk = clocks.stop()
    want = None
    try:
        with open(os.path.join(ROOT, "tests", "golden", "rmat_counts.json")) as f:
            gold = json.load(f)
        recs = gold["graphs"] + ([gold["full_size"]] if "full_size" in gold else [])
        for r in recs:
            if r["scale"] == scale and "four_cycles_two_paths" in r:
                want = r["four_cycles_two_paths"]
    except (OSError, KeyError, ValueError):
        pass
    if want is not None and want != res.count:
        raise SystemExit(f"4-cycle count {res.count} differs from the oracle's {want}")
    if rank != 0:
        return
    line = {"metric": RMAT4_METRIC, "value": (4 * n_edges + res.count) / (ms / 1000),
            "unit": UNIT, "n_gpus": world, "steps": 1, "warmup": 0, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "i32",
            "data": "synthetic",
            "config": {"workload": f"R-MAT scale {scale} (2^{scale} vertices, {n_edges} edges "
                                   "drawn, a,b,c = 0.57,0.19,0.19, seed 3), Q_4(w,x,y,z) :- "
                                   "E(w,x),E(x,y),E(y,z),E(z,w), COUNT(*)",
                       "plan": "Generic Join plan of the order w,x,y,z, fewest-keys cover",
                       "timing": "one execution from scratch between CUDA events (it takes "
                                 "minutes at full size: no warm-up and no repeats)"},
            "result": {"count": res.count},
            "parity": {"exact": want is not None, "oracle_two_paths": want},
            "counters": res.counters, "clocks": clk, "roofline": None, "cpu_baseline": None,
            "e2e": None, "gpu_launches": res.counters["kernels"], "impl": "fj"}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# Fifth workload (--workload ablation): the paper's COLT and vectorization
# ablations (Section 5.3) and its Generic Join baseline (Section 5.1), on the
# same GPU.  Tries: COLT (lazy), simple lazy trie (every root built eagerly)
# and simple trie (every level built eagerly); batch sizes of the general
# node kernel (cover elements per block round: 256 is one per thread, the
# tuple-at-a-time end; 4096 is sixteen per thread with their loads in flight
# together); Generic Join: one node per variable, every trie built eagerly,
# the smallest batch, no one-launch node-0 scan.
# ---------------------------------------------------------------------------

ABL_METRIC = "ms per query (lower is better), COLT and vectorization ablations, FJ vs GJ"


def _time_prepared(prep, flush, stream, steps, warmup):
    import torch
    out = None
    for _ in range(warmup):
        prep.reset()
        out = prep.execute()
    times = []
    for _ in range(steps):
        flush.zero_()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        prep.reset()
        prep.execute_async()
        e1.record(stream)
        r = prep.result()
        torch.cuda.synchronize()
        if (r.count, r.mins) != (out.count, out.mins):
            raise SystemExit("ablation: result changed between steps")
        times.append(e0.elapsed_time(e1))
    return statistics.mean(times), out


def run_ablation(args, rank, world):
    args.rmat_scale = args.rmat_scale or 18
    import torch

    from paper_2301_10841_gb300 import fj

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    ctx = fj.Context(local)
    flush = L2Flush(dev)
    stream = torch.cuda.current_stream()
    steps, warmup = max(2, min(args.steps, 10)), 3
    rows = []

    def sweep(name, atoms, fj_plan, gj_plan, out_mode, min_vars, cover):
        base = None
        cfgs = [("colt", "default", fj_plan, 0, 0, cover),
                ("colt", 256, fj_plan, 256, fj.FLAG_NO_FUSED_SCAN, cover),
                ("colt", 1024, fj_plan, 1024, fj.FLAG_NO_FUSED_SCAN, cover),
                ("colt", 4096, fj_plan, 4096, fj.FLAG_NO_FUSED_SCAN, cover),
                ("simple_lazy_trie", "default", fj_plan, 0, fj.FLAG_EAGER_ROOT, cover),
                ("simple_trie", "default", fj_plan, 0, fj.FLAG_EAGER_ALL, cover),
                ("generic_join", 256, gj_plan, 256,
                 fj.FLAG_EAGER_ALL | fj.FLAG_NO_FUSED_SCAN, "fewest")]
        for trie, batch, plan, bs, flags, cov in cfgs:
            prep = fj.Prepared(ctx, atoms, plan, out_mode=out_mode, min_vars=min_vars,
                               batch_size=bs, cover=cov, flags=flags)
            ms, r = _time_prepared(prep, flush, stream, steps, warmup)
            prep.free()
            if base is None:
                base = (r.count, r.mins)
            elif (r.count, r.mins) != base:
                raise SystemExit(f"ablation {name}: {trie}/{batch} differs from COLT")
            rows.append({"workload": name, "trie": trie, "batch": batch, "cover": cov,
                         "plan": "generic join" if plan is gj_plan else "free join",
                         "ms": ms, "count": r.count})

    fact, dims = G.star_schema(n_fact=args.n_fact, dims=DIMS, s=1.1, seed=2)
    rels = {r["name"]: ctx.relation([torch.from_numpy(c).to(dev) for c in r["cols"]], r["name"])
            for r in [fact] + dims}
    q = G.star_query(fact, dims, theta=THETA)
    atoms = [{"rel": rels[a["rel"]["name"]], "vars": a["vars"], "preds": a["preds"]} for a in q]
    sweep("star", atoms, fj.binary_to_free_plan(atoms, [0, 1, 2, 3, 4], factor=True),
          fj.generic_join_plan(atoms, [0, 1, 2, 3, 4, 5, 6, 7]), "count_min", MIN_VARS, "static")
    del rels, atoms
    e = G.rmat(args.rmat_scale, 16 << args.rmat_scale, seed=3)
    rel = ctx.relation([torch.from_numpy(c).to(dev) for c in e["cols"]], "E")
    tq = G.triangle_query(e)
    tatoms = [{"rel": rel, "vars": a["vars"], "rel_cols": a["rel_cols"]} for a in tq]
    sweep(f"rmat{args.rmat_scale}-triangle", tatoms, TRI_PLAN,
          fj.generic_join_plan(tatoms, [0, 1, 2]), "count", [], "fewest")
    if rank != 0:
        return

    def ms_of(w, trie, batch, plan="free join"):
        for r in rows:
            if r["workload"] == w and r["trie"] == trie and r["batch"] == batch and r["plan"] == plan:
                return r["ms"]
        return None

    summary = {}
    for w in sorted({r["workload"] for r in rows}):
        colt = ms_of(w, "colt", "default")
        summary[w] = {
            "colt_vs_simple_lazy_trie": ms_of(w, "simple_lazy_trie", "default") / colt,
            "colt_vs_simple_trie": ms_of(w, "simple_trie", "default") / colt,
            "batch4096_vs_batch256": ms_of(w, "colt", 256) / ms_of(w, "colt", 4096),
            "fj_vs_gj": ms_of(w, "generic_join", 256, "generic join") / colt}
    line = {"metric": ABL_METRIC, "value": ms_of("star", "colt", "default"), "unit": "ms",
            "n_gpus": world, "steps": steps, "warmup": warmup, "ms_per_step": None,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "i32",
            "data": "synthetic",
            "config": {"workload": f"star join (F {args.n_fact} rows, as the default workload) and "
                                   f"triangle count on R-MAT scale {args.rmat_scale} "
                                   f"({16 << args.rmat_scale} edges, seed 3)",
                       "l2": L2_NOTE},
            "rows": rows, "speedups": summary, "impl": "fj"}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=500)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="fj", choices=["fj", "reference"])
    ap.add_argument("--batch", type=int, default=1024)
    ap.add_argument("--n-fact", type=int, default=N_FACT)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default="star",
                    choices=["star", "rmat-triangle", "rmat-4cycle", "batched", "chooser",
                             "ablation"])
    ap.add_argument("--rmat-scale", type=int, default=None,
                    help="R-MAT scale of the ablation (default 18) and 4-cycle (default 20) "
                         "workloads")
    ap.add_argument("--train-queries", type=int, default=10_000)
    ap.add_argument("--train-min-rows", type=int, default=2_000)
    ap.add_argument("--train-max-rows", type=int, default=20_000)
    ap.add_argument("--label", default="work", choices=["work", "time"])
    ap.add_argument("--tune-queries", type=int, default=400)
    ap.add_argument("--pool-size", type=int, default=48)
    ap.add_argument("--pool-min-rows", type=int, default=1_000_000)
    ap.add_argument("--pool-max-rows", type=int, default=16_000_000)
    ap.add_argument("--min-rows", type=int, default=50_000)
    ap.add_argument("--n-queries", type=int, default=256)
    ap.add_argument("--max-rows", type=int, default=2_000_000)
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "gloo" if args.impl == "reference" else "nccl"
        if backend == "nccl":
            import torch
            torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        dist.init_process_group(backend=backend)
    try:
        if args.impl == "reference":
            run_reference(args, rank, world)
        elif args.workload == "rmat-triangle":
            run_rmat(args, rank, world)
        elif args.workload == "rmat-4cycle":
            run_rmat4(args, rank, world)
        elif args.workload == "batched":
            run_batched(args, rank, world)
        elif args.workload == "chooser":
            run_chooser(args, rank, world)
        elif args.workload == "ablation":
            run_ablation(args, rank, world)
        else:
            run_fj(args, rank, world)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
