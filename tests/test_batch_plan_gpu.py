"""GPU parity of prepared batches (stc_batch_plan_*): the first runs go through the host, then
every run replays one captured CUDA graph. Every run's results are checked against the CPU
oracle; a run whose inputs changed so that its outputs outgrow the captured layout is run
again the ordinary way and is still exact."""
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


def host(res):
    return res.coords.cpu().numpy().reshape(res.nnz, res.order), res.vals.cpu().numpy()


def mixed_problems(seed, n=60):
    rng = W.rng_for(seed)
    probs = [W.random_case(rng, max_order=4, max_size=7, max_nnz=150) for _ in range(n)]
    probs += [W.small_pair(rng, nnz_hi=3e3) for _ in range(24)]
    probs.append(W.Problem(W.uniform_coo(rng, (5, 6), 0), W.uniform_coo(rng, (6, 7), 20), (1,), (0,)))
    probs.append(W.Problem(W.uniform_coo(rng, (3, 50), 3_000), W.uniform_coo(rng, (50, 100_000), 40_000), (1,), (0,)))
    return probs


def run_and_check(plan, probs, refs, runs):
    for _ in range(runs):
        res = plan.run()
        for p, ref, r in zip(probs, refs, res):
            c, v = host(r)
            assert_matches_oracle(c, v, ref)
            assert r.stats.products == ref.products and r.shape == ref.shape


@pytest.mark.parametrize("ga", [0.75, 0.0])
def test_plan_runs_replay_and_match_oracle(ga):
    """Given load factor: the first run captures; tuned (0): the first five runs time the
    candidates (load factor, warp-table size, expansion split), then the graph is captured. Every run of either plan matches the oracle."""
    import gc

    import paper_2410_10094_gb300 as stc

    probs = mixed_problems(8600 if ga else 8601)
    refs = [oracle.contract(p.X, p.Y, p.cx, p.cy, p.out_order) for p in probs]
    ctx = stc.Context(0)  # a fresh context: its autotuner starts with this batch's size bucket
    plan = stc.BatchPlan([(to_dev(p.X), to_dev(p.Y), p.cx, p.cy, p.out_order) for p in probs],
                         group_load_factor=ga, ctx=ctx)
    try:
        runs = 7
        run_and_check(plan, probs, refs, runs)
        n_runs, graph_runs, ga_used, warp_max, depth = plan.stats()
        assert n_runs == runs
        # tuned: one ordinary run per candidate (five), then the capture
        assert graph_runs >= (runs - 1 if ga else runs - 5)
        assert ga_used > 0 and warp_max in (256, 1024) and depth in (0, 1)
    finally:
        plan.close()
        gc.collect()
        ctx.close()


def test_plan_inputs_change_between_runs():
    """The device arrays keep their place but their contents change: values only (the
    captured layout still fits), then coordinates that make far more products (the run is
    redone through the host and captured anew). Each run matches the oracle of what the
    arrays then hold."""
    import torch

    import paper_2410_10094_gb300 as stc

    rng = W.rng_for(8700)
    probs = [W.small_pair(rng, nnz_lo=200, nnz_hi=2e3) for _ in range(32)]
    dev = [(to_dev(p.X), to_dev(p.Y), p.cx, p.cy) for p in probs]
    plan = stc.BatchPlan(dev, group_load_factor=0.75)
    try:
        for step in range(4):
            if step == 2:  # new values, same coordinates
                for p, d in zip(probs, dev):
                    p.X.vals[:] = W.nonzero_values(rng, p.X.nnz)
                    d[0][2].copy_(torch.from_numpy(p.X.vals))
            if step == 3:  # every X entry of problem 0 moved onto its Y's most common contract coordinate
                p, d = probs[0], dev[0]
                cy = p.Y.coords[:, p.cy[0]]
                top = int(np.bincount(cy).argmax())
                p.X.coords[:, p.cx[0]] = top
                d[0][1].copy_(torch.from_numpy(p.X.coords))
            res = plan.run()
            for p, r in zip(probs, res):
                ref = oracle.contract(p.X, p.Y, p.cx, p.cy)
                c, v = host(r)
                assert_matches_oracle(c, v, ref)
            del res
        assert plan.stats()[1] >= 1
    finally:
        plan.close()


def test_plan_batched_workload():
    """The 2,048-pair batched workload through a plan: after the tuning runs every run
    replays the graph; a replayed run's products and nnz equal an ordinary batch's for every
    problem, and a seeded sample of 256 problems matches the oracle output by output."""
    import paper_2410_10094_gb300 as stc
    from fullsize import check_full_many

    probs = W.batched()
    bp = stc.BatchProblems([(to_dev(p.X), to_dev(p.Y), p.cx, p.cy, p.out_order) for p in probs])
    plan = stc.BatchPlan(bp)
    try:
        for _ in range(6):  # five tuning runs (one per candidate), then replays
            res = plan.run()
            del res
        res = plan.run()
        assert plan.stats()[1] >= 2
        ref = stc.contract_batch(bp)
        for r, q in zip(res, ref):
            assert r.stats.products == q.stats.products and r.nnz == q.nnz
        del ref
        rng = W.rng_for(8800)
        pick = rng.choice(len(probs), size=256, replace=False)
        info = check_full_many([(probs[i], res[i]) for i in pick])
        print(f"plan replay: 256 sampled problems, {info.outputs} outputs against the oracle")
    finally:
        plan.close()
