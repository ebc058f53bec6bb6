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


def device_sorted(res):
    """Output entries of a result sorted by their linear key, on the device."""
    import torch

    if res.nnz == 0:
        return torch.empty(0, dtype=torch.int64, device="cuda"), torch.empty(0, dtype=torch.float64, device="cuda")
    key = torch.zeros(res.nnz, dtype=torch.int64, device="cuda")
    for q, n in enumerate(res.shape):
        key = key * int(n) + res.coords[:, q].to(torch.int64)
    key, order = torch.sort(key)
    return key, res.vals[order]


def test_batched_workload_full():
    """The 2,048-pair batched workload: every problem's product count against the counting
    entry point, a seeded sample against the oracle, and a seeded sample of the larger
    problems against the same problem contracted alone."""
    import torch

    import paper_2410_10094_gb300 as stc

    probs = W.batched()
    res = run_batch(probs)
    assert len(res) == 2048
    for p, r in zip(probs, res):
        P, _ = stc.count(to_dev(p.X), to_dev(p.Y), p.cx, p.cy)
        assert r.stats.products == P
        assert 0 <= r.nnz <= r.stats.out_capacity
    rng = W.rng_for(8300)
    small = [i for i, p in enumerate(probs) if p.X.nnz * p.Y.nnz <= 4e7]
    for i in rng.choice(small, size=16, replace=False):
        p = probs[i]
        ref = oracle.contract(p.X, p.Y, p.cx, p.cy)
        c, v = host(res[i])
        assert_matches_oracle(c, v, ref)
    big = np.argsort([-r.stats.products for r in res])
    for i in list(big[:4]) + list(rng.choice(big[4:], size=12, replace=False)):
        p = probs[i]
        alone = stc.contract(to_dev(p.X), to_dev(p.Y), p.cx, p.cy)
        assert alone.stats.products == res[i].stats.products and alone.nnz == res[i].nnz
        ka, va = device_sorted(alone)
        kb, vb = device_sorted(res[i])
        assert torch.equal(ka, kb)
        assert torch.allclose(vb, va, rtol=1e-9, atol=1e-12)
        del alone, ka, va, kb, vb


def test_batch_autotuned_calls_agree():
    """Repeated calls on one size bucket: the autotuner tries each load factor once and then
    keeps the fastest; every call's results match the oracle."""
    rng = W.rng_for(8400)
    probs = [W.small_pair(rng, nnz_hi=2e3) for _ in range(48)]
    refs = [oracle.contract(p.X, p.Y, p.cx, p.cy) for p in probs]
    import paper_2410_10094_gb300 as stc

    ctx = stc.Context(0)
    bp = stc.BatchProblems([(to_dev(p.X), to_dev(p.Y), p.cx, p.cy, p.out_order) for p in probs])
    for _ in range(5):
        res = stc.contract_batch(bp, ctx=ctx)
        for ref, r in zip(refs, res):
            c, v = host(r)
            assert_matches_oracle(c, v, ref)
        del res
