"""GPU parity of the operand-order choice and of chained contractions: X (x) Y computed as
Y (x) X with the output modes permuted back (Eq. 2 is symmetric; Section 5.4 swaps the
operands of imbalanced pairs), and a result fed straight into the next contraction."""
import numpy as np
import pytest

import oracle
import workloads as W
from gpu_util import assert_matches_oracle, gpu_contract, result_host, to_dev

pytestmark = pytest.mark.gpu

MODES = [dict(strategy=1), dict(strategy=2, accumulator=1), dict(strategy=2, accumulator=0)]
MODE_IDS = ["global", "grouped-hash", "grouped-auto"]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2410_10094_gb300 import build

    build.build()
    import paper_2410_10094_gb300 as stc

    stc.load()
    return stc


def check(p, **kw):
    ref = oracle.contract(p.X, p.Y, p.cx, p.cy, p.out_order)
    res = gpu_contract(p, **kw)
    c, v = result_host(res)
    assert_matches_oracle(c, v, ref)
    assert res.stats.products == ref.products
    assert res.shape == ref.shape
    return res, ref


@pytest.mark.parametrize("mode", MODES, ids=MODE_IDS)
@pytest.mark.parametrize("seed", range(30))
def test_random_cases_swapped(seed, mode):
    """Forced swap on tiny random problems (any paired modes, output permutations)."""
    import paper_2410_10094_gb300 as stc

    p = W.random_case(W.rng_for(7300 + seed), max_order=5, max_size=6, max_nnz=120)
    res, _ = check(p, operands=stc.OPERANDS_SWAPPED, **mode)
    assert res.stats.swapped == 1


def test_auto_swaps_when_y_is_larger():
    import paper_2410_10094_gb300 as stc

    rng = W.rng_for(7400)
    small = W.uniform_coo(rng, (30, 40, 9), 2_000)
    large = W.uniform_coo(rng, (40, 9, 500), 20_000)
    res, _ = check(W.Problem(small, large, (1, 2), (0, 1), out_order=(1, 0)), operands=stc.OPERANDS_AUTO)
    assert res.stats.swapped == 1
    res, _ = check(W.Problem(large, small, (0, 1), (1, 2)), operands=stc.OPERANDS_AUTO)
    assert res.stats.swapped == 0


def test_imbalanced_given_small_first():
    """The imbalanced pair (Y 512x512x64 with 2e4 entries, X 4096x512x512 with 2e7) written
    small-first: AUTO swaps it back."""
    import paper_2410_10094_gb300 as stc

    p = W.imbalanced()
    ref = oracle.contract(p.X, p.Y, p.cx, p.cy)
    # q's output modes are (Y's free mode, X's free mode); out_order (1, 0) restores p's order,
    # so the oracle runs in p's cheap orientation (grouping the small tensor).
    q = W.Problem(p.Y, p.X, p.cy, p.cx, out_order=(1, 0))
    res = gpu_contract(q, operands=stc.OPERANDS_AUTO)
    c, v = result_host(res)
    assert_matches_oracle(c, v, ref)
    assert res.stats.swapped == 1 and res.stats.products == ref.products


def test_chained_contractions():
    """((A (x) B) (x) C) with the first result passed on as a device tensor. The second stage's
    tolerance comes from the oracle run on absolute values through both stages."""
    import paper_2410_10094_gb300 as stc

    rng = W.rng_for(7500)
    A = W.uniform_coo(rng, (20, 30, 40), 4_000)
    B = W.uniform_coo(rng, (40, 25), 600)
    C = W.uniform_coo(rng, (25, 30, 7), 900)
    z1 = stc.contract(to_dev(A), to_dev(B), (2,), (0,))  # (20, 30, 25)
    z2 = stc.contract(z1.tensor, to_dev(C), (1, 2), (1, 0))  # (20, 7)
    r1 = oracle.contract(A, B, (2,), (0,))
    Z1 = W.COO(r1.shape, r1.coords, r1.vals)
    r2 = oracle.contract(Z1, C, (1, 2), (1, 0))
    absA = W.COO(A.shape, A.coords, np.abs(A.vals))
    absB = W.COO(B.shape, B.coords, np.abs(B.vals))
    absC = W.COO(C.shape, C.coords, np.abs(C.vals))
    a1 = oracle.contract(absA, absB, (2,), (0,))
    a2 = oracle.contract(W.COO(a1.shape, a1.coords, a1.vals), absC, (1, 2), (1, 0))
    c, v = result_host(z2)
    order = np.lexsort(c.T[::-1])
    c, v = c[order], v[order]
    np.testing.assert_array_equal(c, r2.coords)
    np.testing.assert_array_equal(c, a2.coords)
    assert np.all(np.abs(v - r2.vals) <= 4e-12 * a2.vals)
    assert z2.shape == r2.shape
