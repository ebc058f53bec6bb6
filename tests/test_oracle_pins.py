"""Pins for the CPU oracle against things other than itself: the paper's worked examples
(tests/golden), dense brute force via numpy.einsum, the matrix-multiply special case,
closed forms (mode sums, the global checksum, the product count) and invariants (swap,
linearity). A dropped term, a wrong sign, a swapped index or a transposed operand in the
oracle fails at least one of these."""
import itertools

import numpy as np
import pytest

import oracle
from helpers import (REL_TOL, canonical, coo_from_json, coo_to_dense, contract_groups_py, dense_contract,
                     golden, within_tol)
from workloads import COO, Problem, nonzero_values, random_case, rng_for, uniform_coo


def oracle_dense(p: Problem, res) -> np.ndarray:
    """Scatter the oracle's COO output into a dense array of the output shape."""
    out = np.zeros(res.shape, dtype=np.float64)
    if res.nnz:
        out[tuple(res.coords.T.astype(np.int64))] = res.vals
    return out


def check_against_dense(p: Problem):
    res = oracle.contract(p.X, p.Y, p.cx, p.cy, p.out_order)
    count = dense_contract(p, "count")
    # Coordinates: exactly the outputs that received >= 1 product, with the right count.
    want = np.argwhere(count > 0)
    got, cnt = canonical(res.coords, res.cnt)
    if count.ndim == 0:
        assert res.nnz == (1 if count > 0 else 0)
        if res.nnz:
            assert res.cnt[0] == int(count)
    else:
        assert got.shape[0] == want.shape[0]
        np.testing.assert_array_equal(got, want)
        np.testing.assert_array_equal(cnt, count[tuple(want.T)].astype(np.int64))
    # Values against einsum, with the sum-of-|terms| scale.
    vals = dense_contract(p, "vals")
    absd = dense_contract(p, "abs")
    dz = oracle_dense(p, res) if count.ndim else np.float64(res.vals.sum())
    assert np.all(np.abs(dz - vals) <= REL_TOL * absd + 0.0)
    # abs column equals sum |x||y|
    if res.nnz and count.ndim:
        np.testing.assert_allclose(res.abs, absd[tuple(res.coords.T.astype(np.int64))], rtol=1e-13, atol=0)
    assert res.products == int(count.sum())


# ---------------------------------------------------------------------- worked examples

def test_golden_accumulate_example():
    g = golden("accumulate_eq34.json")
    X, Y = coo_from_json(g["X"]), coo_from_json(g["Y"])
    res = oracle.contract(X, Y, g["cx"], g["cy"])
    np.testing.assert_array_equal(res.coords, np.asarray(g["expect_coords"], dtype=np.int32))
    assert res.cnt.tolist() == [2]
    assert abs(res.vals[0] - g["expect_vals"][0]) <= 4 * np.spacing(g["expect_vals"][0])
    assert abs(res.abs[0] - sum(g["expect_products"])) <= 4 * np.spacing(0.21)
    assert res.shape == (8, 8, 8, 8)


def test_golden_ln_key():
    g = golden("ln_key_fig3.json")
    keys = oracle.ln_key(g["shape"], np.asarray(g["coords"]), g["modes"])
    assert keys.tolist() == g["expect"]


def test_golden_counting_sort():
    g = golden("counting_sort_fig6.json")
    keys = np.asarray(g["keys"], dtype=np.uint64)
    off, perm = oracle.counting_sort(keys, g["k"])
    assert off.tolist() == g["expect_offsets"]
    for v, c in g["expect_counts"].items():
        assert off[int(v) + 1] - off[int(v)] == c
    for v, last in g["expect_last_slot_1based"].items():
        assert off[int(v) + 1] == last
    assert keys[perm].tolist() == sorted(g["keys"])


def test_golden_first_seen():
    g = golden("first_seen_fig7.json")
    ids, nd = oracle.first_seen_ids(np.asarray(g["keys"], dtype=np.uint64))
    assert ids.tolist() == g["expect_ids"]
    assert nd == g["expect_distinct"]


def test_golden_group_bound():
    g = golden("group_bound_sec43.json")
    X, Y = coo_from_json(g["X"]), coo_from_json(g["Y"])
    gb = oracle.group_bounds(X, Y, g["cx"], g["cy"])
    assert gb.coords.tolist() == [[0]]
    assert int(gb.bound[0]) == g["expect_bound"]
    assert gb.total == g["expect_bound"]
    assert oracle.table_slots(int(gb.bound[0])) == g["expect_slots"]
    # The bound is exact here: every product lands on a distinct Y free coordinate or not;
    # the contraction produces 7 products.
    assert oracle.contract(X, Y, g["cx"], g["cy"]).products == g["expect_bound"]


# ---------------------------------------------------------------------- dense brute force

@pytest.mark.parametrize("seed", range(60))
def test_dense_bruteforce_random(seed):
    rng = rng_for(1000 + seed)
    p = random_case(rng, max_order=5 if seed % 3 == 0 else 4, max_size=5, max_nnz=60)
    check_against_dense(p)


@pytest.mark.parametrize("ox,oy", [(1, 1), (2, 3), (3, 3), (4, 2), (5, 4)])
def test_dense_every_contract_subset(ox, oy):
    """Every choice of paired modes (as ordered lists) for a pair of orders."""
    rng = rng_for(77 + 10 * ox + oy)
    done = 0
    for m in range(0, min(ox, oy) + 1):
        for cx in itertools.permutations(range(ox), m):
            for cy in itertools.combinations(range(oy), m):
                xs = [int(v) for v in rng.integers(1, 4, size=ox)]
                ys = [int(v) for v in rng.integers(1, 4, size=oy)]
                for a, b in zip(cx, cy):
                    ys[b] = xs[a]
                X = uniform_coo(rng, xs, int(rng.integers(0, 25)))
                Y = uniform_coo(rng, ys, int(rng.integers(0, 25)))
                check_against_dense(Problem(X, Y, tuple(cx), tuple(cy)))
                done += 1
                if done > 80:
                    return


def test_matmul_special_case():
    """Order 2, X mode 1 paired with Y mode 0 is the matrix product (Fig. 2)."""
    rng = rng_for(5)
    A = rng.uniform(-1, 1, size=(7, 9)) * (rng.random((7, 9)) < 0.4)
    B = rng.uniform(-1, 1, size=(9, 5)) * (rng.random((9, 5)) < 0.4)
    ia = np.argwhere(A != 0)
    ib = np.argwhere(B != 0)
    X = COO((7, 9), ia, A[tuple(ia.T)])
    Y = COO((9, 5), ib, B[tuple(ib.T)])
    res = oracle.contract(X, Y, (1,), (0,))
    Z = np.zeros((7, 5))
    Z[tuple(res.coords.T.astype(np.int64))] = res.vals
    ref = A @ B
    absref = np.abs(A) @ np.abs(B)
    assert np.all(np.abs(Z - ref) <= REL_TOL * absref)
    # Structural nonzeros: (i, j) appears iff some k has A[i,k] != 0 and B[k,j] != 0.
    struct = ((A != 0).astype(int) @ (B != 0).astype(int)) > 0
    assert sorted(map(tuple, res.coords.tolist())) == sorted(map(tuple, np.argwhere(struct).tolist()))
    # Transposed operands give the transposed product, not the same one.
    rest = oracle.contract(Y, X, (0,), (1,))
    Zt = np.zeros((5, 7))
    Zt[tuple(rest.coords.T.astype(np.int64))] = rest.vals
    assert np.all(np.abs(Zt - ref.T) <= REL_TOL * absref.T)


def test_mode_sums_all_ones():
    """Y all ones over the contracted modes with one free mode of length 1: z = sum_c x[fX, c]."""
    rng = rng_for(9)
    X = uniform_coo(rng, (5, 4, 6), 150)
    cells = np.argwhere(np.ones((4, 6, 1)))
    Y = COO((4, 6, 1), cells, np.ones(cells.shape[0]))
    res = oracle.contract(X, Y, (1, 2), (0, 1))
    ref = coo_to_dense(X).sum(axis=(1, 2))
    got = np.zeros(5)
    got[res.coords[:, 0]] = res.vals
    assert res.coords[:, 1].max() == 0
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-13)


def test_global_checksum_closed_form():
    """sum_Z z = sum_c (sum_{x: c_x=c} x)(sum_{y: c_y=c} y)."""
    rng = rng_for(11)
    X = uniform_coo(rng, (6, 7, 8), 400)
    Y = uniform_coo(rng, (8, 7, 5), 300)
    cx, cy = (1, 2), (1, 0)
    res = oracle.contract(X, Y, cx, cy)
    sx, sy = {}, {}
    for i in range(X.nnz):
        c = (X.coords[i, 1], X.coords[i, 2])
        sx[c] = sx.get(c, 0.0) + X.vals[i]
    for j in range(Y.nnz):
        c = (Y.coords[j, 1], Y.coords[j, 0])
        sy[c] = sy.get(c, 0.0) + Y.vals[j]
    closed = sum(v * sy.get(c, 0.0) for c, v in sx.items())
    assert abs(res.vals.sum() - closed) <= 1e-12 * res.abs.sum()


def test_product_count_and_bounds():
    rng = rng_for(12)
    X = uniform_coo(rng, (5, 6, 7), 500)
    Y = uniform_coo(rng, (7, 6, 4), 500)
    cx, cy = (2,), (0,)
    res = oracle.contract(X, Y, cx, cy)
    nxc = np.bincount(X.coords[:, 2], minlength=7)
    nyc = np.bincount(Y.coords[:, 0], minlength=7)
    P = int((nxc * nyc).sum())
    assert res.products == P
    assert int(res.cnt.sum()) == P
    assert res.nnz <= P
    assert res.nnz <= 5 * 6 * 6 * 4
    gb = oracle.group_bounds(X, Y, cx, cy)
    assert gb.total == P
    py = contract_groups_py(X, Y, cx, cy)
    assert {tuple(k): int(v) for k, v in zip(gb.coords.tolist(), gb.bound)} == py
    # Each group's outputs fit its bound (Section 4.3).
    rows = {}
    for c in res.coords:
        rows[(c[0], c[1])] = rows.get((c[0], c[1]), 0) + 1
    for k, v in rows.items():
        assert v <= py[k]


def test_swap_symmetry():
    """Y (x) X equals X (x) Y up to the output mode order (Section 5.4)."""
    rng = rng_for(13)
    X = uniform_coo(rng, (5, 6, 7, 3), 600)
    Y = uniform_coo(rng, (7, 4, 5), 500)
    cx, cy = (2, 0), (0, 2)
    a = oracle.contract(X, Y, cx, cy)               # (x1, x3, y1)
    b = oracle.contract(Y, X, cy, cx, out_order=(1, 2, 0))  # Y free (y1) then X free (x1, x3) -> reorder
    np.testing.assert_array_equal(a.coords, b.coords)
    assert np.all(within_tol(b.vals, a.vals, a.abs))
    np.testing.assert_array_equal(a.cnt, b.cnt)


def test_chain_associativity():
    """(A (x) B) (x) C equals A (x) (B (x) C) when the pairings do not overlap (Eq. 2 summed in
    either order): the same structural entries, values within the propagated bound. Pins the
    oracle for chains, where one call's output is the next call's input."""
    rng = rng_for(16)
    A = uniform_coo(rng, (3, 4, 5), 50)
    B = uniform_coo(rng, (5, 6, 2), 60)
    C = uniform_coo(rng, (6, 7), 30)
    ab = oracle.contract(A, B, (2,), (0,))                               # (a0, a1, b1, b2)
    left = oracle.contract(COO(ab.shape, ab.coords, ab.vals), C, (2,), (0,))  # (a0, a1, b2, c1)
    bc = oracle.contract(B, C, (1,), (0,))                               # (b0, b2, c1)
    right = oracle.contract(A, COO(bc.shape, bc.coords, bc.vals), (2,), (0,))  # (a0, a1, b2, c1)
    np.testing.assert_array_equal(left.coords, right.coords)
    absd = lambda t: COO(t.shape, t.coords, np.abs(t.vals))
    ab_abs = oracle.contract(absd(A), absd(B), (2,), (0,))
    bound = oracle.contract(COO(ab_abs.shape, ab_abs.coords, ab_abs.vals), absd(C), (2,), (0,))
    np.testing.assert_array_equal(bound.coords, left.coords)
    assert np.all(np.abs(left.vals - right.vals) <= 4 * REL_TOL * bound.vals)
    # against the dense definition
    dense = np.einsum("ijk,klm,ln->ijmn", coo_to_dense(A), coo_to_dense(B), coo_to_dense(C))
    got = np.zeros_like(dense)
    got[tuple(left.coords.T)] = left.vals
    assert np.allclose(got, dense, rtol=0, atol=1e-12 * (1 + np.abs(dense).max()))


def test_linearity_split_x():
    rng = rng_for(14)
    X = uniform_coo(rng, (6, 6, 6), 700)
    Y = uniform_coo(rng, (6, 6), 200)
    cx, cy = (1,), (0,)
    z = oracle.contract(X, Y, cx, cy)
    half = X.nnz // 2
    z1 = oracle.contract(X.take(slice(0, half)), Y, cx, cy)
    z2 = oracle.contract(X.take(slice(half, None)), Y, cx, cy)
    acc = {}
    for r in (z1, z2):
        for c, v in zip(map(tuple, r.coords.tolist()), r.vals):
            acc[c] = acc.get(c, 0.0) + v
    assert sorted(acc) == sorted(map(tuple, z.coords.tolist()))
    got = np.array([acc[tuple(c)] for c in z.coords.tolist()])
    assert np.all(within_tol(got, z.vals, z.abs))


def test_out_order_permutes_columns():
    rng = rng_for(15)
    X = uniform_coo(rng, (3, 4, 5), 40)
    Y = uniform_coo(rng, (5, 2), 10)
    a = oracle.contract(X, Y, (2,), (0,))
    b = oracle.contract(X, Y, (2,), (0,), out_order=(2, 0, 1))
    assert b.shape == (2, 3, 4)
    ca, va = canonical(a.coords[:, [2, 0, 1]], a.vals)
    np.testing.assert_array_equal(ca, b.coords)
    np.testing.assert_array_equal(va, b.vals)


# ---------------------------------------------------------------------- edge cases

def test_empty_inputs():
    rng = rng_for(16)
    X = uniform_coo(rng, (4, 4), 0)
    Y = uniform_coo(rng, (4, 4), 10)
    r = oracle.contract(X, Y, (1,), (0,))
    assert r.nnz == 0 and r.products == 0
    r = oracle.contract(Y, X, (1,), (0,))
    assert r.nnz == 0


def test_outer_product_no_contracted_modes():
    rng = rng_for(17)
    X = uniform_coo(rng, (3, 2), 4, distinct=True)
    Y = uniform_coo(rng, (2,), 2, distinct=True)
    r = oracle.contract(X, Y, (), ())
    assert r.nnz == 8 and r.products == 8
    check_against_dense(Problem(X, Y, (), ()))


def test_full_contraction_is_order_zero():
    rng = rng_for(18)
    X = uniform_coo(rng, (4, 5), 12)
    Y = uniform_coo(rng, (5, 4), 12)
    r = oracle.contract(X, Y, (0, 1), (1, 0))
    dx, dy = coo_to_dense(X), coo_to_dense(Y)
    ref = float((dx * dy.T).sum())
    if r.products:
        assert r.nnz == 1 and r.coords.shape == (1, 0)
        assert abs(r.vals[0] - ref) <= 1e-12 * float((np.abs(dx) * np.abs(dy.T)).sum())
    else:
        assert r.nnz == 0


def test_cancellation_keeps_structural_zero():
    X = COO((1, 2), [[0, 0], [0, 1]], [1.0, 1.0])
    Y = COO((2, 1), [[0, 0], [1, 0]], [1.0, -1.0])
    r = oracle.contract(X, Y, (1,), (0,))
    assert r.nnz == 1 and r.vals[0] == 0.0 and r.cnt[0] == 2 and r.abs[0] == 2.0


@pytest.mark.parametrize("bad,code", [
    ("shape", 2), ("coord", 3), ("mode", 1), ("dupmode", 1), ("outorder", 1)])
def test_errors(bad, code):
    X = COO((3, 4), [[0, 1], [2, 3]], [1.0, 2.0])
    Y = COO((4, 5), [[1, 1], [3, 4]], [1.0, 2.0])
    cx, cy, oo = (1,), (0,), None
    if bad == "shape":
        Y = COO((5, 5), [[1, 1]], [1.0])
    elif bad == "coord":
        X = COO((3, 4), [[0, 4]], [1.0])
    elif bad == "mode":
        cx = (2,)
    elif bad == "dupmode":
        cx, cy = (1, 1), (0, 1)
    elif bad == "outorder":
        oo = (0, 0)
    with pytest.raises(oracle.OracleError) as e:
        oracle.contract(X, Y, cx, cy, oo)
    assert e.value.code == code


# ---------------------------------------------------------------------- helper functions

def test_ln_key_matches_ravel_multi_index():
    rng = rng_for(19)
    shape = (7, 3, 11, 5)
    co = np.stack([rng.integers(0, s, 500) for s in shape], axis=1).astype(np.int32)
    for modes in [(0,), (2, 1), (3, 0, 2), (0, 1, 2, 3), (1, 3)]:
        got = oracle.ln_key(shape, co, modes)
        ref = np.ravel_multi_index(tuple(co[:, m] for m in modes), tuple(shape[m] for m in modes))
        np.testing.assert_array_equal(got, ref.astype(np.uint64))
    with pytest.raises(oracle.OracleError):
        oracle.ln_key((2 ** 40, 2 ** 40), np.zeros((1, 2), dtype=np.int32), (0, 1))


def test_counting_sort_matches_stable_argsort():
    rng = rng_for(20)
    keys = rng.integers(0, 37, 2000).astype(np.uint64)
    off, perm = oracle.counting_sort(keys, 40)
    np.testing.assert_array_equal(perm, np.argsort(keys, kind="stable"))
    np.testing.assert_array_equal(np.diff(off), np.bincount(keys.astype(np.int64), minlength=40))
    assert off[0] == 0 and off[-1] == 2000


def test_first_seen_matches_unique():
    rng = rng_for(21)
    keys = rng.integers(0, 10 ** 12, 50).astype(np.uint64)
    keys = keys[rng.integers(0, 50, 400)]
    ids, nd = oracle.first_seen_ids(keys)
    uniq, first, inv = np.unique(keys, return_index=True, return_inverse=True)
    rank = np.argsort(np.argsort(first))
    np.testing.assert_array_equal(ids, rank[inv])
    assert nd == uniq.size
