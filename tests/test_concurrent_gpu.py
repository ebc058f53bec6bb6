"""Contractions launched at once from several host threads, each on its own stream, with
contract key spaces of different sizes (so that the survey's shared-memory bitmap differs
from call to call): every result matches the oracle. Kernel attributes are shared by all the
threads that launch a kernel, so a limit set for one call's size must hold for every other
call's launch (a server's workers launch this way)."""
import threading

import pytest

import oracle
import workloads as W
from gpu_util import assert_matches_oracle, result_host, to_dev

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


def test_threads_with_different_key_spaces():
    import torch

    import paper_2410_10094_gb300 as stc

    rng = W.rng_for(9800)
    probs = []
    for i in range(24):
        k = [24, 300, 2_000, 9_000][i % 4]  # contract key spaces from 24 to 9,000 keys
        probs.append(W.Problem(W.uniform_coo(rng, (40, 30, k), 6_000), W.uniform_coo(rng, (k, 50), 4_000), (2,), (0,)))
    refs = [oracle.contract(p.X, p.Y, p.cx, p.cy) for p in probs]
    dev = [(to_dev(p.X), to_dev(p.Y)) for p in probs]
    errors, results = [], {}
    start = threading.Barrier(4)

    def worker(t):
        try:
            s = torch.cuda.Stream()
            start.wait()
            for rep in range(6):
                for i in range(t, len(probs), 4):
                    X, Y = dev[i]
                    r = stc.contract(X, Y, probs[i].cx, probs[i].cy, strategy=1, stream=s)
                    s.synchronize()
                    results[(i, rep)] = result_host(r)
                    del r
        except Exception as e:  # reported by the main thread
            errors.append(repr(e))

    threads = [threading.Thread(target=worker, args=(t,)) for t in range(4)]
    for th in threads:
        th.start()
    for th in threads:
        th.join()
    assert not errors, errors[:3]
    for (i, _), (c, v) in results.items():
        assert_matches_oracle(c, v, refs[i])
