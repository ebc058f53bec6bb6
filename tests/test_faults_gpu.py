"""Failure paths, each made on the host (nothing faults, traps or hangs the GPU):

* an accumulation table sized too small on purpose (stc_opts.table_shrink): the kernel's
  bounded probe flags the overflow, the call retries at full capacity and the result still
  matches the oracle;
* a context budget smaller than one call's bound: STC_ERR_OUT_OF_MEMORY, nothing left held,
  and the context still serves smaller calls;
* a request cancelled while it waits in the server's queue: its wait reports
  STC_ERR_CANCELLED, every other request finishes with its correct product count, and the
  server keeps serving.
"""
import pytest

import oracle
import workloads as W
from gpu_util import assert_matches_oracle, gpu_contract, result_host, to_dev

pytestmark = pytest.mark.gpu

STATUS_OUT_OF_MEMORY = 4
STATUS_CANCELLED = 10


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2410_10094_gb300 import build

    build.build()
    import paper_2410_10094_gb300 as stc

    stc.load()


@pytest.mark.parametrize("probe", [1, 4, 8])
@pytest.mark.parametrize("shrink", [0, 8])
def test_undersized_global_table_is_retried(shrink, probe):
    rng = W.rng_for(9500)
    X = W.uniform_coo(rng, (30, 20, 40), 60_000)
    Y = W.uniform_coo(rng, (40, 25), 3_000)
    p = W.Problem(X, Y, (2,), (0,))
    ref = oracle.contract(p.X, p.Y, p.cx, p.cy)
    res = gpu_contract(p, strategy=1, table_shrink=shrink, probe=probe)
    c, v = result_host(res)
    assert_matches_oracle(c, v, ref)
    # A table with fewer slots than distinct output keys must overflow and be retried once (a
    # small one: every product whose key is missing probes the whole table before it gives up).
    first = max(64, res.stats.table_slots >> shrink)
    assert res.stats.retries == (1 if first < ref.nnz else 0)
    assert res.stats.retries == (1 if shrink else 0)


def test_budget_smaller_than_one_call():
    import paper_2410_10094_gb300 as stc

    rng = W.rng_for(9510)
    p = W.Problem(W.uniform_coo(rng, (64, 64, 64), 200_000), W.uniform_coo(rng, (64, 64, 64), 200_000), (2,), (0,))
    _, need = stc.count(to_dev(p.X), to_dev(p.Y), p.cx, p.cy)
    ctx = stc.Context(0, mem_budget_bytes=need // 4)
    try:
        with pytest.raises(stc.StcError) as e:
            stc.contract(to_dev(p.X), to_dev(p.Y), p.cx, p.cy, ctx=ctx)
        assert e.value.status == STATUS_OUT_OF_MEMORY
        assert ctx.stats() == (0, 0)  # the failed call released what it had taken
        small = W.Problem(W.uniform_coo(rng, (16, 8), 300), W.uniform_coo(rng, (8, 16), 300), (1,), (0,))
        r = stc.contract(to_dev(small.X), to_dev(small.Y), small.cx, small.cy, ctx=ctx)
        c, v = result_host(r)
        assert_matches_oracle(c, v, oracle.contract(small.X, small.Y, small.cx, small.cy))
        del r
    finally:
        import gc

        gc.collect()
        ctx.close()


def test_server_cancel_queued_request():
    import paper_2410_10094_gb300 as stc

    rng = W.rng_for(9520)
    probs = [W.served_large(rng, nnz=300_000, n=128) for _ in range(12)]
    dev = [(to_dev(p.X), to_dev(p.Y), p.cx, p.cy) for p in probs]
    # A budget of one byte admits one request at a time, so the later ones wait in the queue.
    srv = stc.Server(mem_budget_bytes=1)
    try:
        tickets = [srv.submit(*d) for d in dev]
        cancelled = {t for t in reversed(tickets[-4:]) if srv.cancel(t)}
        assert cancelled, "no queued request to cancel"
        for t, p in zip(tickets, probs):
            if t in cancelled:
                with pytest.raises(stc.StcError) as e:
                    srv.wait(t)
                assert e.value.status == STATUS_CANCELLED
            else:
                r, _ = srv.wait(t, timeout_ms=600_000)
                assert r.stats.products == oracle.group_bounds(p.X, p.Y, p.cx, p.cy).total
                del r
        t = srv.submit(*dev[1])  # the server keeps serving after the cancellations
        r, _ = srv.wait(t, timeout_ms=600_000)
        assert r.stats.products == oracle.group_bounds(probs[1].X, probs[1].Y, probs[1].cx, probs[1].cy).total
    finally:
        srv.close()
