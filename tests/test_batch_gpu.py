"""GPU parity of stc_contract_batch: every problem of a batch against the CPU oracle (small
batches, and a seeded sample of the 2,048-pair batched workload), and every problem of the
full batched workload against the same problem contracted alone."""
import numpy as np
import pytest

import oracle
import workloads as W
from gpu_util import assert_matches_oracle, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2410_10094_gb300 import build

    build.build()
    import paper_2410_10094_gb300 as stc

    stc.load()


def run_batch(probs, **kw):
    import paper_2410_10094_gb300 as stc

    return stc.contract_batch([(to_dev(p.X), to_dev(p.Y), p.cx, p.cy, p.out_order) for p in probs], **kw)


def host(res):
    return res.coords.cpu().numpy().reshape(res.nnz, res.order), res.vals.cpu().numpy()


def test_batch_random_mixed():
    """Mixed orders, paired-mode counts, output orders, empty tensors, outer products and
    order-0 outputs in one batch."""
    rng = W.rng_for(8000)
    probs = [W.random_case(rng, max_order=4, max_size=7, max_nnz=150) for _ in range(60)]
    probs.append(W.Problem(W.uniform_coo(rng, (5, 6), 0), W.uniform_coo(rng, (6, 7), 20), (1,), (0,)))
    probs.append(W.Problem(W.uniform_coo(rng, (3, 4), 9), W.uniform_coo(rng, (5,), 4), (), ()))
    res = run_batch(probs)
    assert len(res) == len(probs)
    for p, r in zip(probs, res):
        ref = oracle.contract(p.X, p.Y, p.cx, p.cy, p.out_order)
        c, v = host(r)
        assert_matches_oracle(c, v, ref)
        assert r.stats.products == ref.products and r.shape == ref.shape


@pytest.mark.parametrize("ga", [0.5, 0.75])
def test_batch_small_pairs_against_oracle(ga):
    """128 pairs of the batched mix (order 3, lengths 16..512, one paired mode), nnz
    log-uniform in 1e2..3e3: every problem against the oracle."""
    rng = W.rng_for(8100)
    probs = [W.small_pair(rng, nnz_hi=3e3) for _ in range(128)]
    res = run_batch(probs, group_load_factor=ga)
    for p, r in zip(probs, res):
        ref = oracle.contract(p.X, p.Y, p.cx, p.cy)
        c, v = host(r)
        assert_matches_oracle(c, v, ref)


def test_batch_heavy_groups():
    """Problems whose groups land in every class, including the global overflow table."""
    rng = W.rng_for(8200)
    probs = [
        W.Problem(W.uniform_coo(rng, (3, 50), 3_000), W.uniform_coo(rng, (50, 100_000), 40_000), (1,), (0,)),
        W.Problem(W.uniform_coo(rng, (40, 30), 4_000), W.uniform_coo(rng, (30, 5_000), 9_000), (1,), (0,)),
        W.Problem(W.uniform_coo(rng, (4, 6, 5), 20_000), W.uniform_coo(rng, (5, 3), 5_000), (2,), (0,)),
        W.Problem(W.uniform_coo(rng, (300, 7), 20_000), W.uniform_coo(rng, (7, 70_000, 70_000), 30_000), (1,), (0,)),
    ]
    res = run_batch(probs)
    for p, r in zip(probs, res):
        ref = oracle.contract(p.X, p.Y, p.cx, p.cy)
        c, v = host(r)
        assert_matches_oracle(c, v, ref)


def abs_problem(p):
    """The same problem on |X| and |Y|: its values are sum|x*y| per output, the scale of the
    value tolerance, computed by the library where the oracle would be slow."""
    return W.Problem(W.COO(p.X.shape, p.X.coords, np.abs(p.X.vals)), W.COO(p.Y.shape, p.Y.coords, np.abs(p.Y.vals)),
                     p.cx, p.cy, p.out_order)


def assert_same_result(alone, mixed, scale):
    """Keys and nnz identical; values within REL_TOL * sum|x*y| (``scale``: the sorted values
    of the |X| (x) |Y| contraction); outputs' keys compared on the device."""
    import torch

    from fullsize import device_sorted
    from helpers import REL_TOL

    assert alone.nnz == mixed.nnz and alone.stats.products == mixed.stats.products
    ka, _, va = device_sorted(alone)
    kb, _, vb = device_sorted(mixed)
    ks, _, vs = device_sorted(scale)
    assert torch.equal(ka, kb) and torch.equal(ka, ks)
    assert bool(((va - vb).abs() <= REL_TOL * vs).all())


def test_batched_workload_full():
    """The 2,048-pair batched workload: every output of every problem against the oracle (run
    in independent parts across the host's cores), and the larger problems against the same
    problem contracted alone, within 1e-12 * sum|x*y|."""
    import paper_2410_10094_gb300 as stc
    from fullsize import check_full_many

    probs = W.batched()
    res = run_batch(probs)
    assert len(res) == 2048
    info = check_full_many(list(zip(probs, res)))
    print(f"batched: all 2048 problems, {info.outputs} outputs and {info.products} products against the oracle "
          f"in {info.parts} parts on {info.threads} threads, {info.seconds:.1f} s")
    rng = W.rng_for(8300)
    big = np.argsort([-r.stats.products for r in res])
    for i in list(big[:4]) + list(rng.choice(big[4:], size=12, replace=False)):
        p = probs[i]
        alone = stc.contract(to_dev(p.X), to_dev(p.Y), p.cx, p.cy)
        q = abs_problem(p)
        scale = stc.contract(to_dev(q.X), to_dev(q.Y), q.cx, q.cy)
        assert_same_result(alone, res[i], scale)
        del alone, scale


def test_batch_autotuned_calls_agree():
    """Repeated calls on one size bucket: the autotuner tries each of its five candidates once
    (load factor, largest warp table, expansion split) and then keeps the fastest; every call's
    results match the oracle."""
    rng = W.rng_for(8400)
    probs = [W.small_pair(rng, nnz_hi=2e3) for _ in range(48)]
    refs = [oracle.contract(p.X, p.Y, p.cx, p.cy) for p in probs]
    import paper_2410_10094_gb300 as stc

    ctx = stc.Context(0)
    bp = stc.BatchProblems([(to_dev(p.X), to_dev(p.Y), p.cx, p.cy, p.out_order) for p in probs])
    for _ in range(8):
        res = stc.contract_batch(bp, ctx=ctx)
        for ref, r in zip(refs, res):
            c, v = host(r)
            assert_matches_oracle(c, v, ref)
        del res


def test_batch_overflow_groups_twice_in_a_row():
    """A batch whose groups overflow every shared-memory class, run twice on one context: the
    second run reuses the pool's memory of the first, so its overflow table must start cleared
    (keys and values)."""
    import paper_2410_10094_gb300 as stc

    rng = W.rng_for(8250)
    probs = [W.Problem(W.uniform_coo(rng, (3, 50), 3_000), W.uniform_coo(rng, (50, 100_000), 40_000), (1,), (0,)),
             W.Problem(W.uniform_coo(rng, (4, 30), 2_000), W.uniform_coo(rng, (30, 80_000), 30_000), (1,), (0,))]
    refs = [oracle.contract(p.X, p.Y, p.cx, p.cy) for p in probs]
    ctx = stc.Context(0)
    try:
        for _ in range(2):
            res = stc.contract_batch([(to_dev(p.X), to_dev(p.Y), p.cx, p.cy) for p in probs], ctx=ctx)
            for ref, r in zip(refs, res):
                c, v = host(r)
                assert_matches_oracle(c, v, ref)
            del res, r
    finally:
        import gc

        gc.collect()
        ctx.close()


def test_batch_single_entry_groups_and_repeated_y_keys():
    """Groups of one X entry (most X free keys hold a single entry here) over Y runs with and
    without repeated free keys: runs whose free keys are all different take the scaled-copy
    path, runs with a repeated (contract, free) coordinate must still sum the repeats. Both
    against the oracle, in an ordinary batch and in a replayed plan."""
    import numpy as np

    import paper_2410_10094_gb300 as stc

    rng = W.rng_for(8500)
    probs = []
    for i in range(12):
        X = W.uniform_coo(rng, (400, 300, 24), 2_500)
        Y = W.uniform_coo(rng, (24, 40, 30), 3_000)
        if i % 2:  # repeat some of Y's coordinates with new values
            k = 200
            Y = W.COO(Y.shape, np.concatenate([Y.coords, Y.coords[:k]]), np.concatenate([Y.vals, W.nonzero_values(rng, k)]))
        probs.append(W.Problem(X, Y, (2,), (0,)))
    refs = [oracle.contract(p.X, p.Y, p.cx, p.cy) for p in probs]
    dev = [(to_dev(p.X), to_dev(p.Y), p.cx, p.cy) for p in probs]
    for ref, r in zip(refs, stc.contract_batch(dev)):
        c, v = host(r)
        assert_matches_oracle(c, v, ref)
    plan = stc.BatchPlan(dev, group_load_factor=0.75)
    try:
        for _ in range(3):
            res = plan.run()
            for ref, r in zip(refs, res):
                c, v = host(r)
                assert_matches_oracle(c, v, ref)
            del res
        assert plan.stats()[1] >= 2
    finally:
        plan.close()


def test_batch_single_entry_groups_over_long_runs():
    """One-entry groups over Y runs of 1,500 entries (the CTA table classes, and the per-run
    uniqueness check for long runs): runs with all-different free keys are written as scaled
    copies, runs with a repeated coordinate keep the table path. Against the oracle."""
    import numpy as np

    import paper_2410_10094_gb300 as stc

    rng = W.rng_for(8510)
    probs = []
    for i in range(4):
        X = W.uniform_coo(rng, (500, 400, 8), 3_000)
        cells = [rng.choice(60 * 60, size=1_500, replace=False) for _ in range(8)]
        yc = np.concatenate([np.stack([np.full(1_500, k), c // 60, c % 60], axis=1) for k, c in enumerate(cells)])
        yv = W.nonzero_values(rng, yc.shape[0])
        if i % 2:  # a repeated coordinate in some runs
            yc = np.concatenate([yc, yc[::997]])
            yv = np.concatenate([yv, W.nonzero_values(rng, yc.shape[0] - yv.shape[0])])
        probs.append(W.Problem(X, W.COO((8, 60, 60), yc, yv), (2,), (0,)))
    refs = [oracle.contract(p.X, p.Y, p.cx, p.cy) for p in probs]
    dev = [(to_dev(p.X), to_dev(p.Y), p.cx, p.cy) for p in probs]
    for ref, r in zip(refs, stc.contract_batch(dev)):
        c, v = host(r)
        assert_matches_oracle(c, v, ref)
