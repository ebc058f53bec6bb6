"""Full-size parity: the unchanged oracle run on independent parts of a problem across the
host's cores, every output of the library compared with it element by element.

Outputs of different X free tuples never collide (Section 2.4.2: each X free group
accumulates into its own part of the output), so splitting X by ranges of its first free
mode splits the contraction into independent sub-contractions whose outputs occupy disjoint,
contiguous ranges of the output's lexicographic order. Each part is one ordinary
``oracle.contract`` call on a subset of X's rows and the Y entries that can meet them; the
oracle itself is not changed. ctypes releases the GIL during the call, so a thread pool runs
the parts on all cores.

The library's result is sorted by its row-major output key on the device once, and each
part's slice is compared there with the oracle's part: coordinates and nnz bit-exact,
values within REL_TOL * sum|x*y|, outputs of at most two products bit-exact.

Test infrastructure only: nothing here is used by the library.
"""
from __future__ import annotations

import os
import time
from collections import deque
from concurrent.futures import ThreadPoolExecutor
from dataclasses import dataclass
from typing import List, Optional

import numpy as np

from helpers import REL_TOL


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:  # pragma: no cover
        return os.cpu_count() or 1


def mem_available_bytes() -> int:
    try:
        with open("/proc/meminfo") as f:
            for ln in f:
                if ln.startswith("MemAvailable:"):
                    return int(ln.split()[1]) * 1024
    except OSError:
        pass
    return 16 << 30


def _cells(t, modes) -> np.ndarray:
    """Row-major number of each entry's cell over ``modes`` (test-side bookkeeping, used only
    to size and filter the parts)."""
    c = np.zeros(t.nnz, dtype=np.int64)
    for j in modes:
        c = c * int(t.shape[j]) + t.coords[:, j].astype(np.int64)
    return c


@dataclass
class Part:
    lo: int                 # first output coordinate range [lo, hi) of this part
    hi: int
    xrows: np.ndarray       # X rows of the part
    yrows: Optional[np.ndarray]  # Y rows that can meet them (None: all of Y)
    products: int


def plan_parts(p, max_products: float = 4e6) -> List[Part]:
    """Parts of at most about ``max_products`` products (one range of the first output
    coordinate cannot be split further). A problem with a permuted output order or without X
    free modes is one part."""
    xfree = [j for j in range(p.X.order) if j not in set(p.cx)]
    cx_cell = _cells(p.X, p.cx)
    cy_cell = _cells(p.Y, p.cy)
    K = int(np.prod([p.X.shape[j] for j in p.cx], dtype=np.float64)) if p.cx else 1
    if p.X.nnz == 0 or p.Y.nnz == 0:
        return [Part(0, 1 << 62, np.arange(p.X.nnz), None, 0)]
    # Work per X row: the number of Y entries on its contract cell (Section 4.3).
    if K <= (1 << 26):
        ny = np.bincount(cy_cell, minlength=K) if p.cy else np.array([p.Y.nnz])
        w = ny[cx_cell] if p.cx else np.full(p.X.nnz, p.Y.nnz)
    else:
        uy, cnt = np.unique(cy_cell, return_counts=True)
        pos = np.searchsorted(uy, cx_cell)
        pos = np.minimum(pos, uy.size - 1)
        w = np.where(uy[pos] == cx_cell, cnt[pos], 0)
    total = int(w.sum())
    if p.out_order is not None or not xfree or total <= max_products:
        return [Part(0, 1 << 62, np.arange(p.X.nnz), None, total)]
    first = p.X.coords[:, xfree[0]].astype(np.int64)
    n0 = int(p.X.shape[xfree[0]])
    per = np.bincount(first, weights=w, minlength=n0)
    parts, lo, acc = [], 0, 0.0
    for v in range(n0):
        if acc > 0 and acc + per[v] > max_products:
            parts.append((lo, v, acc))
            lo, acc = v, 0.0
        acc += per[v]
    parts.append((lo, n0, acc))
    order = np.argsort(first, kind="stable")
    bounds = np.searchsorted(first[order], [a for a, _, _ in parts] + [n0])
    out = []
    for i, (a, b, acc) in enumerate(parts):
        rows = np.sort(order[bounds[i]:bounds[i + 1]])
        # Y entries whose contract cell some X row of the part has: the others meet nothing.
        ycells = np.unique(cx_cell[rows])
        yrows = np.flatnonzero(np.isin(cy_cell, ycells)) if ycells.size < 0.5 * K else None
        out.append(Part(a, b, rows, yrows, int(acc)))
    return out


def device_sorted(res):
    """The result's output keys (row-major over its shape) sorted on the device, with the
    coordinates and values in the same order."""
    import torch

    if res.nnz == 0:
        e = torch.empty(0, dtype=torch.int64, device="cuda")
        return e, torch.empty((0, res.order), dtype=torch.int32, device="cuda"), e.double()
    key = torch.zeros(res.nnz, dtype=torch.int64, device="cuda")
    for q, n in enumerate(res.shape):
        key.mul_(int(n)).add_(res.coords[:, q].to(torch.int64))
    key, order = torch.sort(key)
    return key, res.coords[order], res.vals[order]


def compare_part_on_device(coords_d, vals_d, ref, rel: float = REL_TOL) -> None:
    """One part: the library's sorted slice against the oracle's part (lexicographic order)."""
    import torch

    n = int(ref.vals.shape[0])
    assert coords_d.shape[0] == n, f"nnz {coords_d.shape[0]} != oracle {n}"
    if n == 0:
        return
    rc = torch.from_numpy(np.ascontiguousarray(ref.coords)).cuda()
    if not torch.equal(coords_d.reshape(n, -1), rc.reshape(n, -1)):
        bad = torch.nonzero((coords_d.reshape(n, -1) != rc.reshape(n, -1)).any(dim=1))[:3, 0].tolist()
        raise AssertionError(f"coordinates differ at rows {bad}")
    rv = torch.from_numpy(ref.vals).cuda()
    ra = torch.from_numpy(ref.abs).cuda()
    ok = (vals_d - rv).abs() <= rel * ra
    if not bool(ok.all()):
        bad = torch.nonzero(~ok)[:5, 0].tolist()
        raise AssertionError(f"{int((~ok).sum())} values outside tolerance, e.g. rows {bad}: gpu "
                             f"{vals_d[bad].tolist()} oracle {ref.vals[bad]} abs {ref.abs[bad]} cnt {ref.cnt[bad]}")
    few = torch.from_numpy(ref.cnt <= 2).cuda()
    if not torch.equal(vals_d[few], rv[few]):
        raise AssertionError("an output of at most two products is not bit-exact")


@dataclass
class FullCheck:
    parts: int
    products: int
    outputs: int
    seconds: float
    threads: int


def check_full_many(items, threads: Optional[int] = None, max_products: float = 4e6,
                    bytes_per_product: float = 300.0) -> FullCheck:
    """Every output of every (problem, library result) pair in ``items`` against the oracle.
    The parts of all problems share one thread pool (the host's cores, capped so that the
    parts in flight fit in half the available memory); each problem's result is sorted on the
    device when its first part is compared and dropped after its last."""
    import torch

    import oracle

    t0 = time.perf_counter()
    plans = [plan_parts(p, max_products) for p, _ in items]
    tasks = [(k, part) for k, pl in enumerate(plans) for part in pl]
    biggest_y = max((p.Y.nnz for p, _ in items), default=0)
    per_task = bytes_per_product * max_products + 200.0 * biggest_y
    mem_cap = max(1, int(mem_available_bytes() * 0.5 // max(1.0, per_task)))
    nthreads = max(1, min(threads or host_cores(), mem_cap, len(tasks)))

    def run(task):
        k, part = task
        p = items[k][0]
        X = p.X.take(part.xrows)
        Y = p.Y if part.yrows is None else p.Y.take(part.yrows)
        return oracle.contract(X, Y, p.cx, p.cy, p.out_order)

    nprod = nout = 0
    cur_k, cur = -1, None
    seen_out = [0] * len(items)
    seen_prod = [0] * len(items)
    # A window of tasks in flight (twice the threads): parts finished ahead of the one being
    # compared wait in memory, so the window bounds the memory they hold.
    window = deque()
    nxt = 0
    with ThreadPoolExecutor(max_workers=nthreads) as ex:
        while nxt < len(tasks) or window:
            while nxt < len(tasks) and len(window) < 2 * nthreads:
                window.append((tasks[nxt], ex.submit(run, tasks[nxt])))
                nxt += 1
            (k, part), f = window.popleft()
            ref = f.result()
            res = items[k][1]
            if k != cur_k:
                cur_k, cur = k, None
                cur = device_sorted(res)
            key, coords, vals = cur
            if len(plans[k]) == 1:
                a, b = 0, res.nnz
            else:
                stride = int(np.prod(res.shape[1:], dtype=np.float64)) if res.order > 1 else 1
                lim = torch.tensor([part.lo * stride, part.hi * stride], dtype=torch.int64, device="cuda")
                a, b = (int(v) for v in torch.searchsorted(key, lim).tolist())
            try:
                compare_part_on_device(coords[a:b], vals[a:b], ref)
            except AssertionError as e:
                raise AssertionError(f"problem {k} ({items[k][0].name}), part [{part.lo}, {part.hi}): {e}") from None
            seen_out[k] += ref.nnz
            seen_prod[k] += ref.products
            nprod += ref.products
            nout += ref.nnz
            del ref, f
    for k, (p, res) in enumerate(items):
        assert seen_out[k] == res.nnz, f"problem {k}: nnz {res.nnz} != oracle {seen_out[k]}"
        assert seen_prod[k] == res.stats.products, f"problem {k}: products {res.stats.products} != oracle {seen_prod[k]}"
    return FullCheck(len(tasks), nprod, nout, time.perf_counter() - t0, nthreads)


def check_full(p, res, **kw) -> FullCheck:
    """Every output of one library result against the oracle (see check_full_many)."""
    return check_full_many([(p, res)], **kw)
