"""GPU tests of the contraction server: every request's result in a mixed, overlapping
stream equals the same request contracted alone (and the oracle, for the small ones), in
both the batching and the one-at-a-time modes; admission under a small budget; timeouts."""
import threading

import numpy as np
import pytest

import oracle
import workloads as W
from gpu_util import assert_matches_oracle, to_dev
from helpers import within_tol

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


def requests(seed, n_small, n_large):
    rng = W.rng_for(seed)
    probs = [W.small_pair(rng, nnz_hi=5e3) for _ in range(n_small)]
    probs += [W.served_large(rng, nnz=100_000, n=64) for _ in range(n_large)]
    order = rng.permutation(len(probs))
    return [probs[i] for i in order]


@pytest.mark.parametrize("plain", [False, True])
def test_server_mix_equals_alone(plain):
    import paper_2410_10094_gb300 as stc

    probs = requests(9000, 48, 6)
    dev = [(to_dev(p.X), to_dev(p.Y), p.cx, p.cy) for p in probs]
    srv = stc.Server(plain=plain, max_batch=16)
    tickets = []

    def submitter():
        for d in dev:
            tickets.append(srv.submit(*d))

    th = threading.Thread(target=submitter)
    th.start()
    th.join()
    got = {}
    for t, p in zip(tickets, probs):
        r, times = srv.wait(t)
        assert times[0] <= times[1] <= times[2]
        got[t] = host(r)
    srv.close()
    for t, p, d in zip(tickets, probs, dev):
        c, v = got[t]
        # Every request against the oracle (sum|x*y| per output is the tolerance's scale), and
        # against the same request contracted alone, within the same tolerance.
        ref = oracle.contract(p.X, p.Y, p.cx, p.cy)
        assert_matches_oracle(c, v, ref)
        alone = stc.contract(*d)
        ac, av = host(alone)
        oa, ob = np.lexsort(ac.T[::-1]), np.lexsort(c.T[::-1])
        np.testing.assert_array_equal(ac[oa], c[ob])
        np.testing.assert_array_equal(ac[oa], ref.coords)
        assert within_tol(v[ob], av[oa], ref.abs).all()


def test_server_small_budget_admits_one_at_a_time():
    """A budget smaller than any two requests still finishes everything (one by one)."""
    import paper_2410_10094_gb300 as stc

    probs = requests(9100, 6, 2)
    dev = [(to_dev(p.X), to_dev(p.Y), p.cx, p.cy) for p in probs]
    srv = stc.Server(mem_budget_bytes=1)
    tickets = [srv.submit(*d) for d in dev]
    for t, p in zip(tickets, probs):
        r, _ = srv.wait(t, timeout_ms=120_000)
        assert r.stats.products == oracle.group_bounds(p.X, p.Y, p.cx, p.cy).total
    srv.close()


def test_server_wait_timeout_keeps_ticket():
    import paper_2410_10094_gb300 as stc

    rng = W.rng_for(9200)
    p = W.served_large(rng, nnz=1_000_000, n=128)
    srv = stc.Server()
    t = srv.submit(to_dev(p.X), to_dev(p.Y), p.cx, p.cy)
    try:
        r, _ = srv.wait(t, timeout_ms=0)
    except stc.StcError as e:
        assert e.status == 6
        r, _ = srv.wait(t, timeout_ms=600_000)
    assert r.stats.products > 0
    with pytest.raises(stc.StcError):
        srv.poll(t)  # consumed
    srv.close()
