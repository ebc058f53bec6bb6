"""The served workload at its full size: a trace of 20,000 requests (80% pairs of the batched
mix, 20% order-4 128^4 pairs with 1e6 entries each contracting two modes) through the
contraction server with continuous batching, every result checked.

* Each distinct problem the trace draws from is contracted alone and that result is checked
  against the oracle output by output (the oracle run in independent parts on the host's
  cores).
* Each of the 20,000 results taken from the server, where requests overlap on the device
  and share batched launches, is checked against the same problem's result alone:
  coordinates and nnz identical, values within 1e-12 * sum|x*y| per output, sum|x*y| taken
  from the library's contraction of |X| and |Y|.
"""
import numpy as np
import pytest

import workloads as W
from gpu_util import to_dev
from helpers import REL_TOL

pytestmark = pytest.mark.gpu

N_REQUESTS = 20_000
BURST = 64  # requests submitted together (bounds the results held)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2410_10094_gb300 import build

    build.build()
    import paper_2410_10094_gb300 as stc

    stc.load()


def _keys(res):
    import torch

    key = torch.zeros(res.nnz, dtype=torch.int64, device="cuda")
    for q, n in enumerate(res.shape):
        key.mul_(int(n)).add_(res.coords[:, q].to(torch.int64))
    return key


class Reference:
    """A problem's result alone, sorted by key, with sum|x*y| per output. Problems whose
    output key space is at most 2^29 also get a dense key -> position map, so a result from
    the server is compared by one gather instead of a sort."""

    def __init__(self, alone, scale):
        import torch

        key = _keys(alone)
        order = torch.argsort(key)
        self.key = key[order]
        self.vals = alone.vals[order]
        ks = _keys(scale)
        so = torch.argsort(ks)
        assert torch.equal(ks[so], self.key), "|X| (x) |Y| has other output keys"
        self.scale = scale.vals[so]
        self.nnz = alone.nnz
        self.products = alone.stats.products
        F = int(np.prod(alone.shape, dtype=np.float64)) if alone.order else 1
        self.pos = None
        if F <= (1 << 29) and self.nnz > 100_000:
            self.pos = torch.full((F,), -1, dtype=torch.int32, device="cuda")
            self.pos[self.key] = torch.arange(self.nnz, dtype=torch.int32, device="cuda")

    def check(self, r):
        import torch

        assert r.nnz == self.nnz and r.stats.products == self.products
        if self.nnz == 0:
            return
        key = _keys(r)
        if self.pos is not None:
            idx = self.pos[key].to(torch.int64)
            assert bool((idx >= 0).all()), "an output coordinate the alone result lacks"
            seen = torch.zeros(self.nnz, dtype=torch.int32, device="cuda")
            seen.index_add_(0, idx, torch.ones_like(idx, dtype=torch.int32))
            assert bool((seen == 1).all()), "an output coordinate twice"
            ref, sc, v = self.vals[idx], self.scale[idx], r.vals
        else:
            order = torch.argsort(key)
            assert torch.equal(key[order], self.key)
            ref, sc, v = self.vals, self.scale, r.vals[order]
        assert bool(((v - ref).abs() <= REL_TOL * sc).all()), "a value differs from the alone result"


def test_served_trace_20000_every_result_checked():
    import torch

    import paper_2410_10094_gb300 as stc
    from fullsize import check_full_many

    small, large, rng = W.served_pools()
    trace = W.served_trace(rng, N_REQUESTS, len(small), len(large))
    pools = {"small": small, "large": large}
    dev = {kind: [(to_dev(p.X), to_dev(p.Y), p.cx, p.cy) for p in probs] for kind, probs in pools.items()}
    # Every distinct problem alone, pinned against the oracle.
    alone = {kind: [stc.contract(*d) for d in dev[kind]] for kind in pools}
    items = [(p, r) for kind in pools for p, r in zip(pools[kind], alone[kind])]
    info = check_full_many(items)
    print(f"served pools: {len(items)} distinct problems, {info.outputs} outputs against the oracle in "
          f"{info.parts} parts on {info.threads} threads, {info.seconds:.1f} s")
    refs = {}
    for kind, probs in pools.items():
        refs[kind] = []
        for (X, Y, cx, cy), a in zip(dev[kind], alone[kind]):
            sx = (X[0], X[1], X[2].abs())
            sy = (Y[0], Y[1], Y[2].abs())
            refs[kind].append(Reference(a, stc.contract(sx, sy, cx, cy)))
    del alone
    torch.cuda.synchronize()

    srv = stc.Server(mem_budget_bytes=int(150e9))
    # Requests arrive in bursts of BURST (each burst submitted at once, then taken back and
    # checked), so that every burst's requests queue up together and share the device.
    times = np.zeros((len(trace), 3))
    try:
        for b0 in range(0, len(trace), BURST):
            burst = list(range(b0, min(b0 + BURST, len(trace))))
            tickets = [srv.submit(*dev[trace[i][0]][trace[i][1]]) for i in burst]
            for i, t in zip(burst, tickets):
                kind, j = trace[i]
                r, tt = srv.wait(t)
                times[i] = tt
                try:
                    refs[kind][j].check(r)
                except AssertionError as e:
                    raise AssertionError(f"request {i} ({kind} problem {j}): {e}") from None
                del r
    finally:
        srv.close()
    # A request is in the mix when another request ran on the device between its arrival and
    # its completion (start_j < done_i and done_j > submit_i for some j != i).
    ts, tst, td = times[:, 0], times[:, 1], times[:, 2]
    order = np.argsort(tst)
    st_sorted, td_sorted = tst[order], td[order]
    k = np.searchsorted(st_sorted, td, side="left")  # requests that started before i finished
    rank = np.empty(len(trace), dtype=np.int64)
    rank[order] = np.arange(len(trace))
    # the latest finish among those requests, other than i itself
    run_max = np.empty(len(trace))
    run_second = np.empty(len(trace))
    b1 = b2 = -np.inf
    for q, v in enumerate(td_sorted):
        if v >= b1:
            b1, b2 = v, b1
        elif v > b2:
            b2 = v
        run_max[q], run_second[q] = b1, b2
    mixed = 0
    for i in range(len(trace)):
        if k[i] == 0:
            continue
        q = k[i] - 1
        other = run_second[q] if (rank[i] <= q and td[i] == run_max[q]) else run_max[q]
        mixed += bool(other > ts[i])
    print(f"served trace: {len(trace)} results equal to their problems alone; {mixed} ran while another "
          f"request was on the device")
    assert mixed > len(trace) // 2
