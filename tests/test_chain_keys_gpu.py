"""GPU parity of chains of contractions handed over in key form (the chains of Section 5.4):
each result is kept as its output keys (row-major indices over its shape) and passed to the
next contraction without being turned into coordinates; only the last result is decoded. The
chain is checked against the oracle's chain in coordinate form, with the tolerance carried
through the steps by the oracle run on absolute values."""
import numpy as np
import pytest

import oracle
import workloads as W
from gpu_util import result_host, to_dev

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


def coo_of(r):
    return W.COO(r.shape, r.coords, r.vals)


def abs_coo(t):
    return W.COO(t.shape, t.coords, np.abs(t.vals))


def decode(keys, shape):
    """Coordinates of row-major keys (test-side check of the key form)."""
    return np.stack(np.unravel_index(keys.astype(np.uint64).astype(np.int64), tuple(shape)), axis=1).astype(np.int32)


@pytest.mark.parametrize("mode", MODES, ids=MODE_IDS)
def test_three_step_chain_in_key_form(mode):
    """Z1 = X (x) Y (keys out); Z2 = Z1 (x) W contracting Z1's last two modes (keys in, keys
    out); Z3 = Z2 (x) V contracting Z2's first mode (keys in, coordinates out)."""
    import paper_2410_10094_gb300 as stc

    rng = W.rng_for(9700)
    X = W.uniform_coo(rng, (12, 10, 30), 3_000)
    Y = W.uniform_coo(rng, (30, 9, 11), 2_000)
    Wt = W.uniform_coo(rng, (9, 11, 13), 700)
    V = W.uniform_coo(rng, (8, 12), 60)
    z1 = stc.contract(to_dev(X), to_dev(Y), (2,), (0,), output_keys=True, operands=stc.OPERANDS_AS_GIVEN, **mode)
    assert z1.keys_form and z1.coords is None and z1.shape == (12, 10, 9, 11)
    z2 = stc.contract_keyed(z1.tensor, to_dev(Wt), (2, 3), (0, 1), output_keys=True, **mode)  # (12, 10, 13)
    z3 = stc.contract_keyed(z2.tensor, to_dev(V), (0,), (1,), **mode)  # (10, 13, 8)
    r1 = oracle.contract(X, Y, (2,), (0,))
    r2 = oracle.contract(coo_of(r1), Wt, (2, 3), (0, 1))
    r3 = oracle.contract(coo_of(r2), V, (0,), (1,))
    a1 = oracle.contract(abs_coo(X), abs_coo(Y), (2,), (0,))
    a2 = oracle.contract(W.COO(a1.shape, a1.coords, a1.vals), abs_coo(Wt), (2, 3), (0, 1))
    a3 = oracle.contract(W.COO(a2.shape, a2.coords, a2.vals), abs_coo(V), (0,), (1,))
    # The intermediate keys decode to the oracle's coordinates.
    k1 = np.sort(z1.keys.cpu().numpy().view(np.uint64))
    np.testing.assert_array_equal(decode(k1, z1.shape), r1.coords)
    k2 = np.sort(z2.keys.cpu().numpy().view(np.uint64))
    np.testing.assert_array_equal(decode(k2, z2.shape), r2.coords)
    c, v = result_host(z3)
    order = np.lexsort(c.T[::-1])
    c, v = c[order], v[order]
    assert z3.shape == r3.shape
    np.testing.assert_array_equal(c, r3.coords)
    np.testing.assert_array_equal(c, a3.coords)
    # Each step adds at most 1e-12 of its absolute sum; three steps.
    assert np.all(np.abs(v - r3.vals) <= 4e-12 * a3.vals)


def test_key_form_edges():
    """Keys in range checks, a contract block that is not at an end of X, every mode of X
    contracted, and an empty operand."""
    import torch

    import paper_2410_10094_gb300 as stc

    rng = W.rng_for(9710)
    X = W.uniform_coo(rng, (6, 7, 5), 300)
    Y = W.uniform_coo(rng, (7, 4), 50)
    keys = torch.from_numpy(np.ravel_multi_index(tuple(X.coords.T.astype(np.int64)), X.shape).astype(np.int64)).cuda()
    xv = torch.from_numpy(X.vals).cuda()
    with pytest.raises(stc.StcError):  # mode 1 is neither the first nor the last block
        stc.contract_keyed((X.shape, keys, xv), to_dev(Y), (1,), (0,))
    bad = keys.clone()
    bad[3] = 6 * 7 * 5  # outside prod(shape)
    with pytest.raises(stc.StcError):
        stc.contract_keyed((X.shape, bad, xv), to_dev(W.uniform_coo(rng, (5, 3), 40)), (2,), (0,))
    # every mode contracted: an order-0 output
    Z = W.uniform_coo(rng, (6, 7, 5), 200)
    r = stc.contract_keyed((X.shape, keys, xv), to_dev(Z), (0, 1, 2), (0, 1, 2))
    ref = oracle.contract(X, Z, (0, 1, 2), (0, 1, 2))
    assert r.nnz == ref.nnz and r.stats.products == ref.products
    if ref.nnz:
        assert abs(float(r.vals.cpu()[0]) - ref.vals[0]) <= 1e-12 * ref.abs[0]
    # an empty operand
    e = stc.contract_keyed((X.shape, keys[:0], xv[:0]), to_dev(W.uniform_coo(rng, (5, 3), 40)), (2,), (0,))
    assert e.nnz == 0


@pytest.mark.parametrize("mode", MODES, ids=MODE_IDS)
def test_key_form_above_2_32(mode):
    """Output keys above 2^32 (a 3000 x 2000 x 1000 x 900 output, 5.4e12 keys), written as two
    32-bit halves, then handed to a contraction over the last two modes (a contract block of
    9e5 keys split off by one division)."""
    import paper_2410_10094_gb300 as stc

    rng = W.rng_for(9720)
    X = W.uniform_coo(rng, (3000, 2000, 40), 6_000)
    Y = W.uniform_coo(rng, (40, 1000, 900), 5_000)
    Wt = W.uniform_coo(rng, (1000, 900, 7), 200_000)
    z1 = stc.contract(to_dev(X), to_dev(Y), (2,), (0,), output_keys=True, operands=stc.OPERANDS_AS_GIVEN, **mode)
    assert z1.shape == (3000, 2000, 1000, 900)
    r1 = oracle.contract(X, Y, (2,), (0,))
    k1 = np.sort(z1.keys.cpu().numpy().view(np.uint64))
    assert int(k1[-1]) >= 1 << 32
    np.testing.assert_array_equal(decode(k1, z1.shape), r1.coords)
    z2 = stc.contract_keyed(z1.tensor, to_dev(Wt), (2, 3), (0, 1), **mode)  # (3000, 2000, 7)
    r2 = oracle.contract(coo_of(r1), Wt, (2, 3), (0, 1))
    a1 = oracle.contract(abs_coo(X), abs_coo(Y), (2,), (0,))
    a2 = oracle.contract(W.COO(a1.shape, a1.coords, a1.vals), abs_coo(Wt), (2, 3), (0, 1))
    c, v = result_host(z2)
    order = np.lexsort(c.T[::-1])
    c, v = c[order], v[order]
    assert z2.shape == r2.shape and r2.nnz > 100
    np.testing.assert_array_equal(c, r2.coords)
    assert np.all(np.abs(v - r2.vals) <= 3e-12 * a2.vals)
