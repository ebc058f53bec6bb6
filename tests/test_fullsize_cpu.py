"""CPU checks of the full-size parity helper: the oracle run in independent parts (X split by
ranges of its first free coordinate, Y cut to the entries those parts can meet) gives exactly
the oracle run whole, output by output. Section 2.4.2 is what makes the parts independent:
outputs of different X free tuples never collide."""
import numpy as np
import pytest

import oracle
import workloads as W
from fullsize import plan_parts


def run_parts(p, max_products):
    parts = plan_parts(p, max_products)
    got = []
    for part in parts:
        X = p.X.take(part.xrows)
        Y = p.Y if part.yrows is None else p.Y.take(part.yrows)
        got.append((part, oracle.contract(X, Y, p.cx, p.cy, p.out_order)))
    return parts, got


@pytest.mark.parametrize("seed", range(6))
def test_parts_reassemble_the_whole(oracle_lib, seed):
    rng = W.rng_for(7700 + seed)
    if seed < 3:
        p = W.small_pair(rng, nnz_lo=2e3, nnz_hi=2e4, size_lo=8, size_hi=40)
    else:
        X = W.uniform_coo(rng, (12, 9, 7, 5), 4_000)
        Y = W.uniform_coo(rng, (7, 5, 6), 3_000)
        p = W.Problem(X, Y, (2, 3), (0, 1))
    whole = oracle.contract(p.X, p.Y, p.cx, p.cy)
    parts, got = run_parts(p, max_products=max(1.0, whole.products / 7))
    assert len(parts) > 1
    # every X row in exactly one part, parts in increasing order of their coordinate range
    rows = np.concatenate([pt.xrows for pt in parts])
    np.testing.assert_array_equal(np.sort(rows), np.arange(p.X.nnz))
    assert all(a.hi <= b.lo for a, b in zip(parts, parts[1:]))
    coords = np.concatenate([r.coords for _, r in got])
    np.testing.assert_array_equal(coords, whole.coords)
    # same summation order (x, then y, in input order), so the values are bit-identical
    np.testing.assert_array_equal(np.concatenate([r.vals for _, r in got]), whole.vals)
    np.testing.assert_array_equal(np.concatenate([r.abs for _, r in got]), whole.abs)
    np.testing.assert_array_equal(np.concatenate([r.cnt for _, r in got]), whole.cnt)
    assert sum(r.products for _, r in got) == whole.products
    assert sum(pt.products for pt in parts) == whole.products
    for pt, r in got:  # each part's outputs lie in its own range of the first coordinate
        if r.nnz:
            assert pt.lo <= r.coords[:, 0].min() and r.coords[:, 0].max() < pt.hi


def test_permuted_or_small_problems_are_one_part(oracle_lib):
    rng = W.rng_for(7790)
    X = W.uniform_coo(rng, (6, 5, 4), 500)
    Y = W.uniform_coo(rng, (4, 3), 200)
    assert len(plan_parts(W.Problem(X, Y, (2,), (0,), out_order=(2, 0, 1)), max_products=10)) == 1
    assert len(plan_parts(W.Problem(X, Y, (2,), (0,)), max_products=1e9)) == 1
    Z = W.uniform_coo(rng, (6, 5, 4), 0)
    assert len(plan_parts(W.Problem(Z, Y, (2,), (0,)), max_products=10)) == 1
