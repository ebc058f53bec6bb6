"""Benchmark of the sparse COO tensor contraction on GB300.

One step = one full contraction (Y grouping, X survey, product count, expansion and
accumulation, compaction to COO) of one synthetic workload held in HBM. Default workload:
two order-4 256^4 COO tensors with 5e6 uniform entries each, X modes (2,3) paired with Y
modes (0,1) (about 3.8e8 products, 3.65e8 output entries).

Prints one JSON line (rank 0). ``--impl reference`` times the CPU oracle instead, on a
bounded sample of the same workload. Under torchrun each rank runs an independent
replica on its own GPU (the contraction needs no exchange); value = all ranks' products
divided by the slowest rank's time.
"""
from __future__ import annotations

import argparse
import datetime
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

def plain_large_slice(seed):
    """plain_large with X cut to its first 16 values of mode 0 (same per-group work, 1/16 of
    the groups): a profiling-sized case of the same kernels."""
    rng = W.rng_for(seed)
    X = W.uniform_coo(rng, (16, 256, 256, 256), 312_500)
    Y = W.uniform_coo(rng, (256,) * 4, 5_000_000)
    return W.Problem(X, Y, (2, 3), (0, 1), name="plain_large_slice")


WORKLOADS = {
    "batched": lambda seed: W.batched(seed=seed),
    "plain_large": lambda seed: W.plain_large(seed=seed),
    "plain_large_slice": plain_large_slice,
    "imbalanced": lambda seed: W.imbalanced(seed=seed),
    "imbalanced_both": lambda seed: W.imbalanced(seed=seed, both_zipf=True),
    "imbalanced_small_first": lambda seed: (lambda p: W.Problem(p.Y, p.X, p.cy, p.cx, out_order=(1, 0)))(
        W.imbalanced(seed=seed)),
    "plain_small": lambda seed: W.plain_small(seed=seed),
    "wide_keys": lambda seed: W.wide_keys(seed=seed),
}
SEEDS = {"batched": W.SEED_BASE + 4, "plain_large": W.SEED_BASE + 2, "plain_large_slice": W.SEED_BASE + 2, "imbalanced": W.SEED_BASE + 3, "imbalanced_both": W.SEED_BASE + 3,
         "imbalanced_small_first": W.SEED_BASE + 3,
         "plain_small": W.SEED_BASE + 1, "wide_keys": W.SEED_BASE + 6}
DESCRIPTIONS = {
    "batched": "2,048 order-3 pairs, lengths 16..512, one paired mode, nnz log-uniform 1e2..1e5 each, one batch call",
    "plain_large_slice": "X 16x256^3 3.125e5 nnz, Y 256^4 5e6 nnz, X modes (2,3) x Y modes (0,1) (profiling slice)",
    "plain_large": "X,Y order-4 256^4 COO, 5e6 uniform nnz each, X modes (2,3) x Y modes (0,1), FP64",
    "imbalanced": "X 4096x512x512 2e7 nnz, Y 512x512x64 2e4 nnz with Zipf(1.2) contract keys, X (1,2) x Y (0,1)",
    "imbalanced_both": "as imbalanced, X contract keys also Zipf(1.2)",
    "imbalanced_small_first": "as imbalanced with the operands given the other way round (Y (x) X, output modes "
                              "permuted back)",
    "plain_small": "X,Y order-3 64^3 COO, 5e3 distinct nnz each, X mode 2 x Y mode 0",
    "wide_keys": "X 256x256x65536x65536, Y 65536x65536x256x256, 5e6 nnz each, X modes (2,3) x Y modes (0,1) "
                 "(2^32 contract keys, renumbered to dense ids); paired cells from one pool of 65,536",
}


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons. Started before the warm-up (the tool
    takes a moment to start); only samples that arrive inside the marked timed window count."""

    FIELDS = ["timestamp", "clocks.sm", "clocks.max.sm", "power.draw", "clocks_event_reasons.hw_slowdown",
              "clocks_event_reasons.hw_thermal_slowdown", "clocks_event_reasons.sw_thermal_slowdown",
              "clocks_event_reasons.sw_power_cap"]

    def __init__(self, device: int, period_ms: int = 50):
        self.device = device
        self.period_ms = period_ms
        self.proc = None
        self.lines = []  # (sample time, line)
        self.window = None
        self.error = None
        self.raw = []

    def start(self, wait_s: float = 5.0):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), "--query-gpu=" + ",".join(self.FIELDS),
                 "--format=csv,noheader,nounits", "-lms", str(self.period_ms)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            time.sleep(min(wait_s, 1.0))  # let the tool start before the warm-up
        except Exception as e:  # no sampler: reported in the summary
            self.proc = None
            self.error = repr(e)
        return self

    def _read(self):
        # The pipe is block-buffered: each sample's own timestamp (local time) places it.
        for ln in self.proc.stdout:
            if len(self.raw) < 2:
                self.raw.append(ln.strip())
            try:
                stamp = datetime.datetime.strptime(ln.split(",")[0].strip(), "%Y/%m/%d %H:%M:%S.%f").timestamp()
            except ValueError:
                continue
            self.lines.append((stamp, ln.strip()))

    def mark(self, t0, t1):
        self.window = (t0, t1)

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.t.join(timeout=2)
            self.proc = None

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        lo, hi = self.window if self.window else (float("-inf"), float("inf"))
        inside = [ln for t, ln in self.lines if lo <= t <= hi]
        where = "timed window"
        if not inside and self.lines:
            # A timed region shorter than the sampling period: the samples nearest to it
            # (the warm-up just before and the stage pass just after run the same work).
            near = sorted(self.lines, key=lambda tl: min(abs(tl[0] - lo), abs(tl[0] - hi)))[:4]
            inside = [ln for _, ln in near]
            where = "nearest samples (timed region shorter than the sampling period)"
        for ln in inside:
            parts = [p.strip() for p in ln.split(",")][1:]
            if len(parts) != len(self.FIELDS) - 1:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for n, v in zip(names, parts[3:]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0,
                    "note": "no nvidia-smi sample inside the timed window",
                    "samples_total": len(self.lines), "error": self.error, "raw": self.raw,
                    "first": self.lines[0][0] if self.lines else None,
                    "last": self.lines[-1][0] if self.lines else None, "window": self.window}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm), "period_ms": self.period_ms, "from": where}


def replica_seed(workload: str, rank: int) -> int:
    """Every rank runs an independent replica: the same shapes with its own seed."""
    return SEEDS[workload] + 1000 * rank


def reduce_over_ranks(ms: float, products: float, world: int, device: str):
    """Whole-job timing across replicas: the slowest rank's time and the products of all
    ranks (rank 0 reports value = products / time)."""
    if world <= 1:
        return ms, products
    import torch
    import torch.distributed as dist

    t = torch.tensor([ms], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    pt = torch.tensor([products], device=device, dtype=torch.float64)
    dist.all_reduce(pt)
    return float(t.item()), float(pt.item())


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one launch of the dominant
# kernel, from ncu captures summarised in profiles/ncu_traffic.json. Each entry names the
# sources that define the kernel and their SHA-256 at capture time: a kernel changed since its
# capture reports null.
KERNEL_SOURCES = {"group_stream_kernel": ["grouped.cu", "common.cuh", "launch.h"],
                  "x_survey_bulk_kernel": ["prep.cu", "common.cuh", "launch.h"],
                  "x_survey_kernel": ["prep.cu", "common.cuh", "launch.h"]}


def source_sha(kernel):
    """Hash of the code (comments and blank lines left out) of the sources that define `kernel`."""
    import hashlib
    import re

    h = hashlib.sha256()
    for f in KERNEL_SOURCES.get(kernel, []):
        with open(os.path.join(ROOT, "paper_2410_10094_gb300", "csrc", f)) as fh:
            text = fh.read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        h.update("\n".join(ln.rstrip() for ln in text.splitlines() if ln.strip()).encode())
    return h.hexdigest()


TRAFFIC_FILE = os.path.join(ROOT, "profiles", "ncu_traffic.json")


def ncu_traffic(workload, path=None):
    """(kernel, bytes per launch) of the workload's capture when it matches today's sources."""
    try:
        with open(path or TRAFFIC_FILE) as f:
            entry = json.load(f).get(workload)
    except (OSError, ValueError):
        return None
    if not entry or entry.get("source_sha") != source_sha(entry["kernel"]):
        return None
    return entry["kernel"], float(entry["bytes_per_launch"])


def record_traffic(workload, kernel, csv_path, path=None):
    """Adds one capture to profiles/ncu_traffic.json (or `path`): the mean dram__bytes_read.sum +
    dram__bytes_write.sum per launch of `kernel` in an ncu --csv log, with today's source hash."""
    import csv

    per = {}
    with open(csv_path) as f:
        rows = [r for r in csv.reader(ln for ln in f if ln.startswith('"'))]
    head = rows[0]
    ki, mi, vi, ii = head.index("Kernel Name"), head.index("Metric Name"), head.index("Metric Value"), head.index("ID")
    for r in rows[1:]:
        if kernel in r[ki] and r[mi] in ("dram__bytes_read.sum", "dram__bytes_write.sum"):
            unit = r[head.index("Metric Unit")] if "Metric Unit" in head else "byte"
            scale = {"byte": 1, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9}.get(unit, 1)
            per[r[ii]] = per.get(r[ii], 0.0) + float(r[vi].replace(",", "")) * scale
    if not per:
        raise SystemExit(f"no DRAM counters of {kernel} in {csv_path}")
    path = path or TRAFFIC_FILE
    try:
        with open(path) as f:
            data = json.load(f)
    except (OSError, ValueError):
        data = {}
    data[workload] = {"kernel": kernel, "bytes_per_launch": sum(per.values()) / len(per), "launches": len(per),
                      "source_sha": source_sha(kernel), "capture": os.path.basename(csv_path)}
    with open(path, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    print(json.dumps(data[workload]))
    return 0


def l2_note(bytes_in, bytes_out, l2=129e6):
    """How the timed steps relate to the L2 (no flush between steps)."""
    fits = "working set exceeds" if bytes_in + bytes_out > l2 else "working set fits"
    return f"inputs {bytes_in / 1e6:.0f} MB, output {bytes_out / 1e6:.0f} MB: {fits} the 129 MB L2; no flush"


def alg_bytes(p, nz, oz):
    """Bytes the contraction must move: read both inputs once, write the output once."""
    return (4 * p.X.order + 8) * p.X.nnz + (4 * p.Y.order + 8) * p.Y.nnz + (4 * oz + 8) * nz


def key_sample(p, m):
    """The sub-contraction over the paired cells whose cell number is a multiple of m: every
    entry of X and Y on those cells, so every product of the sample is one of the workload's
    and each cell keeps all its work."""
    if m <= 1:
        return p, "the whole workload"

    def cell(t, modes):
        c = np.zeros(t.nnz, dtype=np.int64)
        for j in modes:
            c = (c * 1_000_003 + t.coords[:, j]) % (1 << 40)
        return c

    xi = np.flatnonzero(cell(p.X, p.cx) % m == 0)
    yi = np.flatnonzero(cell(p.Y, p.cy) % m == 0)
    return W.Problem(p.X.take(xi), p.Y.take(yi), p.cx, p.cy, p.out_order), \
        f"the paired cells with cell number = 0 mod {m}: {xi.size} of {p.X.nnz} X and {yi.size} of {p.Y.nnz} Y entries"


def run_oracle_sample(p, workload, m=1):
    """One timed oracle call on key_sample(p, m) (batches: the first 48 // m pairs)."""
    import oracle

    if workload == "batched":
        n = max(1, 48 // max(m, 1))
        t0 = time.perf_counter()
        prods = 0
        for q in p[:n]:
            prods += oracle.contract(q.X, q.Y, q.cx, q.cy).products
        return prods, time.perf_counter() - t0, f"the first {n} of the 2,048 pairs, one after another"
    sp, desc = key_sample(p, m)
    t0 = time.perf_counter()
    r = oracle.contract(sp.X, sp.Y, sp.cx, sp.cy, sp.out_order)
    dt = time.perf_counter() - t0
    return r.products, dt, desc


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def run_oracle_parallel(p, workload, m, threads):
    """The unchanged oracle on key_sample(p, m) split into `threads` independent parts that run
    at once on the host's cores (threads: ctypes releases the GIL during each call). X is split
    by ranges of its first free coordinate: outputs of different X free tuples never collide, so
    the parts are sub-contractions of their own (each part indexes all of the sample's Y).
    Batches: the first 48 // m pairs, one per task."""
    from concurrent.futures import ThreadPoolExecutor

    import oracle

    if workload == "batched":
        n = max(1, 48 // max(m, 1))
        t0 = time.perf_counter()
        with ThreadPoolExecutor(threads) as ex:
            prods = sum(ex.map(lambda q: oracle.contract(q.X, q.Y, q.cx, q.cy).products, p[:n]))
        return prods, time.perf_counter() - t0, f"the first {n} of the 2,048 pairs, {threads} at a time"
    sp, desc = key_sample(p, m)
    xfree = [j for j in range(sp.X.order) if j not in set(sp.cx)]
    if xfree and sp.out_order is None and threads > 1:
        first = sp.X.coords[:, xfree[0]]
        order = np.argsort(first, kind="stable")
        cuts = np.searchsorted(first[order], np.quantile(first, np.linspace(0, 1, threads + 1)[1:-1]), side="left")
        parts = [np.sort(c) for c in np.split(order, cuts) if c.size]
    else:
        parts = [np.arange(sp.X.nnz)]
    t0 = time.perf_counter()
    with ThreadPoolExecutor(len(parts)) as ex:
        prods = sum(ex.map(lambda rows: oracle.contract(sp.X.take(rows), sp.Y, sp.cx, sp.cy, sp.out_order).products,
                           parts))
    dt = time.perf_counter() - t0
    return prods, dt, desc + f", X split by its first free coordinate into {len(parts)} parts run at once"


REF_SECONDS = 120.0  # the reference arm's whole run (warm-up and timed steps) on the host
CPU_SECONDS = 15.0   # the one timed oracle call of cpu_baseline


def sample_fraction(p, workload, seconds):
    """m such that key_sample(p, m) takes about `seconds` in the oracle, estimated from one
    untimed call on 1/4096 of the paired cells. The oracle's ordered maps make its time grow
    about as size^1.1 (measured between 1/4096 and 1/16 of plain_large)."""
    if workload == "batched":  # m selects the first 48 // m pairs: count how many fit
        import oracle

        t, n = 0.0, 0
        while n < 48 and t < seconds:
            q = p[n]
            t0 = time.perf_counter()
            oracle.contract(q.X, q.Y, q.cx, q.cy)
            t += time.perf_counter() - t0
            n += 1
        return max(1, -(-48 // max(1, n - 1)))  # at most the n - 1 pairs that fitted
    probe = 4096
    _, t_probe, _ = run_oracle_sample(p, workload, probe)
    grow = (seconds / max(t_probe, 1e-6)) ** (1 / 1.1)
    return max(1, int(np.ceil(probe / grow)))


def reference_arm(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return 0
    import oracle

    oracle.build()
    if args.workload not in WORKLOADS:
        ap_err = f"--impl reference times single contractions; '{args.workload}' is reported by our arm only"
        print(json.dumps({"impl": "reference", "unavailable": ap_err}), flush=True)
        return 0
    p = WORKLOADS[args.workload](SEEDS[args.workload])
    # Each step is the sub-contraction over 1/m of the paired cells, m chosen so that warm-up
    # and timed steps together take about REF_SECONDS.
    # On all the host's cores: each step the oracle on T independent parts of the sample one
    # core would finish in REF_SECONDS / (steps + warm-up).
    T = host_cores()
    m = sample_fraction(p, args.workload, REF_SECONDS / max(1, args.steps + args.warmup))
    for _ in range(args.warmup):
        run_oracle_parallel(p, args.workload, m, T)
    prods, times, desc = 0, [], ""
    for _ in range(args.steps):
        pr, dt, desc = run_oracle_parallel(p, args.workload, m, T)
        prods += pr
        times.append(dt)
    total = sum(times)
    value = prods / total
    line = {
        "impl": "reference", "metric": "products/s", "value": value, "unit": "products/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"{args.workload}: {DESCRIPTIONS[args.workload]}", "sample": desc},
        "cpu_baseline": {"value": value, "unit": "products/s", "cores": T, "kind": "oracle", "sample": desc},
        "e2e": {"value": value, "unit": "products/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def serve_bench(args):
    """Requests with Poisson arrivals through the server: one-at-a-time launches against
    continuous batching on the same arrival trace (p50/p99 latency and throughput)."""
    import torch

    import paper_2410_10094_gb300 as stc

    clk = ClockSampler(0).start()
    torch.cuda.set_device(0)
    stc.load()
    ctx = stc.default_context(0)
    small, large, rng = W.served_pools()
    dev = lambda t: (t.shape, torch.from_numpy(t.coords).cuda(), torch.from_numpy(t.vals).cuda())
    dsmall = [(dev(q.X), dev(q.Y), q.cx, q.cy) for q in small]
    dlarge = [(dev(q.X), dev(q.Y), q.cx, q.cy) for q in large]
    R = args.requests
    pick = [(dlarge if kind == "large" else dsmall)[i] for kind, i in W.served_trace(rng, R, len(small), len(large))]
    prod = {}

    def run(trace, plain):
        srv = stc.Server(plain=plain, mem_budget_bytes=int(150e9), ctx=ctx)
        tickets = [None] * len(trace)
        ready = threading.Semaphore(0)
        t0 = time.perf_counter()

        def submitter():
            for i, at in enumerate(trace):
                delay = at - (time.perf_counter() - t0)
                if delay > 0:
                    time.sleep(delay)
                tickets[i] = srv.submit(*pick[i])
                ready.release()

        th = threading.Thread(target=submitter)
        th.start()
        lat, first, last, products = [], None, 0.0, 0
        for i in range(len(trace)):
            ready.acquire()
            r, (ts, tst, td) = srv.wait(tickets[i])
            lat.append(td - ts)
            first = ts if first is None else min(first, ts)
            last = max(last, td)
            products += r.stats.products
            del r
        th.join()
        srv.close()
        lat = np.asarray(lat)
        span = last - first
        return {"p50_ms": 1e3 * float(np.percentile(lat, 50)), "p99_ms": 1e3 * float(np.percentile(lat, 99)),
                "requests_per_s": len(trace) / span, "products_per_s": products / span, "span_s": span}

    warm = run(np.zeros(min(40, R)), plain=False)
    tw0 = time.time()
    base = run(np.zeros(min(200, R)), plain=True)
    mu_plain = base["requests_per_s"]
    rows = []
    for f in args.rates:
        lam = f * mu_plain
        trace = np.cumsum(rng.exponential(1.0 / lam, size=R))
        plain_r = run(trace, plain=True)
        batch_r = run(trace, plain=False)
        rows.append({"rate_over_mu_plain": f, "lambda_per_s": lam, "plain": plain_r, "served": batch_r})
    clk.mark(tw0, time.time())
    clk.stop()
    best = rows[-1]["served"]
    line = {
        "metric": "p50/p99 latency served vs plain", "value": best["p99_ms"], "unit": "ms (p99, highest rate)",
        "n_gpus": 1, "steps": R, "warmup": len(warm) if isinstance(warm, list) else 40,
        "ms_per_step": 1e3 / best["requests_per_s"], "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"served: {R} requests, 80% batched-mix pairs, 20% order-4 128^4 pairs with 1e6 nnz "
                               "each contracting 2 modes; Poisson arrivals; 150 GB admission budget",
                   "mu_plain_requests_per_s": mu_plain, "pools": "96 small and 12 large distinct problems"},
        "rates": rows, "clocks": clk.summary(),
    }
    print(json.dumps(line), flush=True)
    return 0


SWEEP_NNZ = (50_000, 100_000, 200_000, 300_000, 500_000)


def sweep_problems():
    """Table 1's Set 1 and Set 2 (A: order 5, B: order 4; A with A, B with B, A with B) at
    each entry count, then Table 2's shapes as random self-contractions."""
    probs = [W.set_sweep(s, pair, n) for s in (1, 2) for pair in ("AA", "BB", "AB") for n in SWEEP_NNZ]
    return probs + [W.table2(name) for name in W.TABLE2]


def sweep_bench(args):
    """Every sweep problem timed alone (CUDA events over --steps calls after --warmup), then
    the oracle on the 50K cases of Set 1 and Set 2 as the CPU baseline."""
    import torch

    import paper_2410_10094_gb300 as stc

    clk = ClockSampler(0).start()
    torch.cuda.set_device(0)
    stc.load()
    ctx = stc.default_context(0)
    stream = torch.cuda.current_stream()
    dev = lambda t: (t.shape, torch.from_numpy(t.coords).cuda(), torch.from_numpy(t.vals).cuda())
    rows, tot_p, tot_ms = [], 0, 0.0
    tw0 = time.time()
    for p in sweep_problems():
        X = dev(p.X)
        Y = X if p.Y is p.X else dev(p.Y)
        step = lambda: stc.contract(X, Y, p.cx, p.cy, p.out_order, stream=stream, ctx=ctx)
        for _ in range(args.warmup):
            r = step()
            P, nz, cids = r.stats.products, r.nnz, r.stats.contract_ids
            del r
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        ev0.record(stream)
        for _ in range(args.steps):
            r = step()
            del r
        ev1.record(stream)
        torch.cuda.synchronize()
        ms = ev0.elapsed_time(ev1) / args.steps
        rows.append({"name": p.name, "shape_x": list(p.X.shape), "shape_y": list(p.Y.shape), "nnz_x": p.X.nnz,
                     "nnz_y": p.Y.nnz, "products": int(P), "nnz_out": int(nz), "contract_ids": int(cids),
                     "ms": ms, "products_per_s": P / (ms / 1e3)})
        tot_p += P
        tot_ms += ms
        del X, Y
    clk.mark(tw0, time.time())
    clk.stop()
    cpu = None
    if not args.no_cpu_baseline:
        import oracle

        oracle.build()
        cases = [W.set_sweep(s, pair, SWEEP_NNZ[0]) for s in (1, 2) for pair in ("AA", "BB", "AB")]
        t0 = time.perf_counter()
        prods = sum(oracle.contract(q.X, q.Y, q.cx, q.cy).products for q in cases)
        dt = time.perf_counter() - t0
        cpu = {"value": prods / dt, "unit": "products/s", "cores": 1, "kind": "oracle",
               "sample": "the six 50K cases of Set 1 and Set 2", "seconds": dt}
    line = {
        "metric": "products/s", "value": tot_p / (tot_ms / 1e3), "unit": "products/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": tot_ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "sweep: Table 1 Sets 1-2 (A 5-order, B 4-order; AA, BB, AB; 50K-500K entries) and "
                               "Table 2 shapes as random self-contractions; second and third modes paired",
                   "problems": len(rows), "l2": "no flush; each problem's inputs stay resident"},
        "sweep": rows, "cpu_baseline": cpu, "clocks": clk.summary(),
    }
    print(json.dumps(line), flush=True)
    return 0


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="plain_large", choices=sorted(WORKLOADS) + ["served", "sweep"])
    ap.add_argument("--strategy", type=int, default=0, help="0 auto, 1 global table, 2 grouped")
    ap.add_argument("--group-load-factor", type=float, default=0.0, help="0 = library default")
    ap.add_argument("--accumulator", type=int, default=0, help="0 auto, 1 hash tables, 2 dense rows")
    ap.add_argument("--contract-ids", type=int, default=0, help="0 auto, 1 direct contract keys, 2 dense ids")
    ap.add_argument("--operands", type=int, default=0, help="0 auto, 1 as given, 2 swapped")
    ap.add_argument("--probe", type=int, default=0, help="one global table: lanes probing together (0 auto, 1, 4, 8)")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-secondary", action="store_true",
                    help="the default workload's line leaves out the other configurations' measurements")
    ap.add_argument("--requests", type=int, default=1000, help="served workload: requests per arrival rate")
    ap.add_argument("--rates", type=float, nargs="+", default=[0.5, 0.9, 1.2],
                    help="served workload: arrival rates as multiples of the one-at-a-time service rate")
    ap.add_argument("--record-traffic", nargs=2, metavar=("KERNEL", "NCU_CSV"),
                    help="store the DRAM bytes per launch of KERNEL from an ncu --csv log for --workload")
    args = ap.parse_args(argv)
    if args.record_traffic:
        return record_traffic(args.workload, *args.record_traffic)
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        return reference_arm(args)
    if args.workload == "served":
        return serve_bench(args)
    if args.workload == "sweep":
        return sweep_bench(args)

    import torch

    import paper_2410_10094_gb300 as stc

    world, rank, local = dist_env()
    # Sample clocks from before the first CUDA call in this process.
    clk = ClockSampler(local).start()
    if world > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    dev = torch.cuda.current_device()
    stc.load()
    ctx = stc.default_context(dev)

    seed = replica_seed(args.workload, rank)
    p = WORKLOADS[args.workload](seed)
    workload_problem = p
    stream = torch.cuda.current_stream()
    dev = lambda t: (t.shape, torch.from_numpy(t.coords).cuda(), torch.from_numpy(t.vals).cuda())
    if args.workload == "batched":
        batch = [(dev(q.X), dev(q.Y), q.cx, q.cy, q.out_order) for q in p]
        prepared = stc.BatchProblems(batch)  # descriptors built once: inputs stay resident

        class _Agg:  # one step's results seen as one
            def __init__(self, rs):
                self.rs = rs
                self.nnz = sum(r.nnz for r in rs)
                self.order = rs[0].order
                st = rs[0].stats
                self.stats = type(st)(sum(r.stats.products for r in rs), sum(r.stats.survivors for r in rs),
                                      sum(r.stats.out_capacity for r in rs),
                                      0, 0, st.strategy, st.launches, st.accumulator, st.stage_ms)

        # The timed steps replay one captured graph per step (a prepared batch whose first runs
        # tune the load factor and capture); the per-stage pass runs ordinary batches.
        plan = stc.BatchPlan(prepared, group_load_factor=args.group_load_factor, ctx=ctx)

        def step(record=False):
            if record:
                return _Agg(stc.contract_batch(prepared, group_load_factor=args.group_load_factor, record_times=True,
                                               stream=stream, ctx=ctx))
            return _Agg(plan.run(stream=stream))
    else:
        X, Y = dev(p.X), dev(p.Y)

        def step(record=False):
            return stc.contract(X, Y, p.cx, p.cy, p.out_order, strategy=args.strategy, record_times=record,
                                group_load_factor=args.group_load_factor, accumulator=args.accumulator,
                                contract_ids=args.contract_ids, operands=args.operands, probe=args.probe,
                                stream=stream, ctx=ctx)

    for _ in range(max(args.warmup, 4) if args.workload == "batched" else args.warmup):
        r = step()
        nz, oz, P, launches, ns = r.nnz, r.order, r.stats.products, r.stats.launches, r.stats.survivors
        cids, swp = r.stats.contract_ids, r.stats.swapped
        del r
    torch.cuda.synchronize()

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    # ---- timed region: K device-resident steps
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    torch.cuda.synchronize()
    tw0 = time.time()
    ev0.record(stream)
    for _ in range(args.steps):
        r = step()
        del r
    ev1.record(stream)
    torch.cuda.synchronize()
    clk.mark(tw0, time.time())
    barrier()
    ms, total_products = reduce_over_ranks(ev0.elapsed_time(ev1), float(P), world, "cuda")
    plan_stats = plan.stats() if args.workload == "batched" else None
    value = total_products * args.steps / (ms / 1e3)

    # ---- per-stage times: K more steps with the library's stage events on (they wait for
    # the last event of each call, so they run outside the timed region above)
    stage = np.zeros(8)
    acc_used = None
    for _ in range(args.steps):
        r = step(record=True)
        stage[: len(r.stats.stage_ms)] += np.asarray(r.stats.stage_ms)
        acc_used = getattr(r.stats, "accumulator", None)
        del r
    torch.cuda.synchronize()
    clk.stop()

    # ---- e2e: the public API call with host buffers, copies inside the timed region
    e2e = None
    sequential = None
    if args.workload == "batched":
        # The same 2,048 problems as 2,048 separate stc_contract calls (one at a time).
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for (Xq, Yq, cxq, cyq, ooq) in batch:
            rq = stc.contract(Xq, Yq, cxq, cyq, ooq, stream=stream, ctx=ctx)
            del rq
        torch.cuda.synchronize()
        seq_s = time.perf_counter() - t0
        sequential = {"ms": 1e3 * seq_s, "value": total_products / seq_s, "unit": "products/s",
                      "speedup_of_batch": (total_products / seq_s) and value / (total_products / seq_s)}
    if not args.no_e2e and args.workload != "batched":
        hx = [torch.from_numpy(p.X.coords).pin_memory(), torch.from_numpy(p.X.vals).pin_memory()]
        hy = [torch.from_numpy(p.Y.coords).pin_memory(), torch.from_numpy(p.Y.vals).pin_memory()]
        hc = torch.empty((nz, oz), dtype=torch.int32).pin_memory()
        hv = torch.empty((nz,), dtype=torch.float64).pin_memory()
        h2d = sum(t.numel() * t.element_size() for t in hx + hy)
        d2h = hc.numel() * 4 + hv.numel() * 8
        barrier()
        torch.cuda.synchronize()
        t0 = None
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        parts = np.zeros(3)
        for it in range(args.e2e_steps + 1):  # the first step warms the copies and is not timed
            if it == 1:
                torch.cuda.synchronize()
                t0 = time.perf_counter()
            evs[0].record(stream)
            Xd = (p.X.shape, hx[0].to("cuda", non_blocking=True), hx[1].to("cuda", non_blocking=True))
            Yd = (p.Y.shape, hy[0].to("cuda", non_blocking=True), hy[1].to("cuda", non_blocking=True))
            evs[1].record(stream)
            r = stc.contract(Xd, Yd, p.cx, p.cy, p.out_order, strategy=args.strategy,
                             group_load_factor=args.group_load_factor, accumulator=args.accumulator,
                             contract_ids=args.contract_ids, operands=args.operands, probe=args.probe,
                             stream=stream, ctx=ctx)
            evs[2].record(stream)
            hc[: r.nnz].copy_(r.coords, non_blocking=True)
            hv[: r.nnz].copy_(r.vals, non_blocking=True)
            evs[3].record(stream)
            torch.cuda.synchronize()
            if it >= 1:
                parts += [evs[i].elapsed_time(evs[i + 1]) for i in range(3)]
            del r, Xd, Yd
        dt = time.perf_counter() - t0
        parts /= args.e2e_steps
        barrier()
        if world > 1:
            t = torch.tensor([dt], device="cuda", dtype=torch.float64)
            torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
            dt = float(t.item())
        e2e = {"value": total_products * args.e2e_steps / dt, "unit": "products/s", "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "steps": args.e2e_steps, "ms_per_step": 1e3 * dt / args.e2e_steps,
               "parts_ms": {"h2d": parts[0], "contract": parts[1], "d2h": parts[2]},
               "d2h_gbs": d2h / (parts[2] * 1e-3) / 1e9 if parts[2] > 0 else None}
        del hc, hv

    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return 0

    # ---- roofline of the dominant kernel from the library's per-stage CUDA events
    hbm, peak_kind = peaks()
    stage_names = ["group_y", "survey_x", "group_x", "plan", "accumulate", "compact"]
    per_step = stage / args.steps
    dom = int(np.argmax(per_step[:6]))
    if args.workload == "batched":
        class _P:
            pass
        agg = _P()
        agg.X = _P(); agg.Y = _P()
        agg.X.order, agg.Y.order = 3, 3
        agg.X.nnz = sum(q.X.nnz for q in p)
        agg.Y.nnz = sum(q.Y.nnz for q in p)
        p = agg
    bytes_in = (4 * p.X.order + 8) * p.X.nnz + (4 * p.Y.order + 8) * p.Y.nnz
    kernel_bytes = {
        0: (4 * p.Y.order + 8) * p.Y.nnz + 16 * p.Y.nnz,            # read Y, write grouped Y
        1: 4 * p.X.order * p.X.nnz + 32 * ns,                        # X coordinates in; survivors' values in, records out
        4: 12 * p.X.nnz + 12 * p.Y.nnz + (4 * oz + 8) * nz,         # grouped X and Y runs in, COO output out
        5: (4 * oz + 8) * nz,                                        # write the COO output
    }.get(dom, bytes_in)
    dom_ms = per_step[dom]
    achieved = kernel_bytes / (dom_ms / 1e3) / 1e9 if dom_ms > 0 else None
    step_ms = ms / args.steps
    default_opts = args.strategy == 0 and args.accumulator == 0 and args.contract_ids == 0 and args.operands == 0
    traffic = ncu_traffic(args.workload) if default_opts else None
    roofline = {"bound": "hbm", "kernel": stage_names[dom], "achieved": achieved, "peak": hbm, "unit": "GB/s",
                "frac": (achieved / hbm) if achieved else None, "traffic": traffic[1] if traffic else None,
                "traffic_kernel": traffic[0] if traffic else None, "peak_kind": peak_kind,
                "kernel_ms": dom_ms, "alg_bytes": kernel_bytes}
    if args.workload == "imbalanced_both":
        # Products fall on at most 262,144 outputs, so the bounds are not HBM bandwidth but the
        # rates measured here (stc_measure_peaks): the one-global-table expansion issues one FP64
        # multiply and one FP64 atomic add in L2 per product; the lane-private rows (accumulator
        # ROWS, which AUTO takes once the shape is known to be rows-heavy) one FP64 multiply and
        # one FP64 add, so half the FP64 multiply rate bounds them.
        dmul, atom = stc.measure_peaks(torch.cuda.current_device())
        acc_ms = float(per_step[4])
        rate = P / (acc_ms / 1e3) if acc_ms > 0 else None
        if acc_used == stc.ACC_ROWS:
            roofline = {"bound": "fp64", "kernel": "accumulate", "achieved": rate and rate / 1e9,
                        "peak": dmul / 2e9, "unit": "G products/s (one FP64 multiply and one FP64 add each)",
                        "frac": rate and rate / (dmul / 2), "traffic": None, "peak_kind": "measured in this run",
                        "kernel_ms": acc_ms, "l2_atomic_peak": atom / 1e9, "accumulator": "rows", "hbm": roofline}
        else:
            roofline = {"bound": "l2_atomic", "kernel": "accumulate", "achieved": rate and rate / 1e9,
                        "peak": atom / 1e9, "unit": "G products/s (one L2 FP64 atomic add each)",
                        "frac": rate and rate / atom, "traffic": None, "peak_kind": "measured in this run",
                        "kernel_ms": acc_ms, "dmul_peak": dmul / 1e9, "dmul_frac": rate and rate / dmul,
                        "hbm": roofline}
    step_alg = alg_bytes(p, nz, oz)

    cpu = None
    if not args.no_cpu_baseline:
        # The oracle as it stands on all the host's cores (independent parts at once), beside
        # one core, on the same sample (sized for about CPU_SECONDS on one core).
        m = sample_fraction(workload_problem, args.workload, CPU_SECONDS) if args.workload != "batched" else 1
        prods, dt, desc = run_oracle_sample(workload_problem, args.workload, m)
        T = host_cores()
        pprods, pdt, pdesc = run_oracle_parallel(workload_problem, args.workload, m, T)
        cpu = {"value": pprods / pdt, "unit": "products/s", "cores": T, "kind": "oracle", "sample": pdesc,
               "seconds": pdt,
               "single_core": {"value": prods / dt, "cores": 1, "sample": desc, "seconds": dt}}

    line = {
        "metric": "products/s", "value": value, "unit": "products/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": step_ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"{args.workload}: {DESCRIPTIONS[args.workload]}", "seed": seed,
                   "products_per_step": P, "nnz_out": nz, "parallelism": f"replicas x{world}",
                   "l2": l2_note(bytes_in, (4 * oz + 8) * nz), "strategy": args.strategy,
                   "group_load_factor": args.group_load_factor, "accumulator": args.accumulator,
                   "contract_ids_mode": args.contract_ids, "contract_ids": int(cids),
                   "operands_mode": args.operands, "swapped": int(swp), "probe": args.probe},
        "step_hbm": {"alg_bytes": step_alg, "gbs": step_alg / (step_ms / 1e3) / 1e9,
                     "frac": step_alg / (step_ms / 1e3) / 1e9 / hbm},
        "stage_ms": {n: float(per_step[i]) for i, n in enumerate(stage_names)},
        "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(launches) * args.steps,
        "sequential_calls": sequential,
        "batch_plan": ({"runs": plan_stats[0], "graph_replays": plan_stats[1], "group_load_factor": plan_stats[2],
                        "warp_table_max": plan_stats[3], "expansion_depth": plan_stats[4]} if plan_stats else None),
        "clocks": clk.summary(),
    }
    if args.workload == "plain_large" and world == 1 and default_opts and not args.no_secondary:
        line["secondary"] = secondary_workloads()
    print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def secondary_workloads():
    """The other configurations' lines, measured in this run (each in a process of its own):
    the imbalanced contraction (config 3), the batched workload replayed as one captured graph
    per step with the 2,048 sequential calls beside it (config 4), and a short served trace
    (config 5: 2,000 requests at the plain server's own rate; the full 20,000-request sweep over
    six rates is `--workload served --requests 20000`)."""
    out = {}
    for wl, steps in (("imbalanced", 20), ("batched", 10), ("served", 0)):
        cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--workload", wl, "--steps", str(steps), "--warmup", "4",
               "--no-e2e", "--no-cpu-baseline", "--no-secondary"]
        if wl == "served":
            cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--workload", "served", "--requests", "2000",
                   "--rates", "1.0", "--warmup", "3", "--no-secondary"]
        try:
            r = subprocess.run(cmd, capture_output=True, text=True, timeout=900)
            ln = [x for x in r.stdout.splitlines() if x.startswith("{")]
            d = json.loads(ln[-1]) if ln else {"error": (r.stderr or "")[-300:]}
        except Exception as e:  # reported, never fatal to the main line
            d = {"error": repr(e)}
        keep = ("metric", "value", "unit", "ms_per_step", "stage_ms", "roofline", "sequential_calls", "batch_plan",
                "rates", "clocks", "config", "error")
        out[wl] = {k: d.get(k) for k in keep if k in d}
    return out


if __name__ == "__main__":
    sys.exit(main())
