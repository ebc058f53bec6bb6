"""GPU parity: the CUDA path, called through the C ABI, against the CPU oracle on the same
seeded inputs. Coordinates and nnz must match bit-exactly, values within
1e-12 * sum|x*y| per output (bit-exactly where at most two products meet)."""
import numpy as np
import pytest

import oracle
import workloads as W
from gpu_util import assert_matches_oracle, gpu_contract, result_host, to_dev
from helpers import REL_TOL

pytestmark = pytest.mark.gpu

# per-X-free-group hash tables (direct output, table scan); bitmap rows for
# every group; AUTO (bitmap rows for the large groups, hash tables for the small ones)
# one global table probed lane by lane, and by tiles of 4 and 8 lanes over buckets;
MODES = [dict(strategy=1, probe=1), dict(strategy=1, probe=4), dict(strategy=1, probe=8),
         dict(strategy=2, accumulator=1), dict(strategy=2, accumulator=3),
         dict(strategy=2, accumulator=2), dict(strategy=2, accumulator=0)]
MODE_IDS = ["global", "global-coop4", "global-coop8", "grouped-hash", "grouped-hash-scan", "grouped-dense",
            "grouped-auto"]
STRATEGIES = [1, 2]


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


# ------------------------------------------------------------------ small and random cases

@pytest.mark.parametrize("mode", MODES, ids=MODE_IDS)
def test_plain_small_workload(mode):
    """64^3 tensors with 5,000 distinct entries each, X mode 2 with Y mode 0 (full parity)."""
    res, ref = check(W.plain_small(), **mode)
    assert ref.nnz > 300_000


@pytest.mark.parametrize("mode", MODES, ids=MODE_IDS)
@pytest.mark.parametrize("seed", range(40))
def test_random_cases(seed, mode):
    rng = W.rng_for(5000 + seed)
    p = W.random_case(rng, max_order=5, max_size=6, max_nnz=120)
    check(p, **mode)


@pytest.mark.parametrize("mode", MODES, ids=MODE_IDS)
def test_several_tiles_ragged_non_pow2(mode):
    """Non-power-of-two mode lengths (division decode path) and a product count that spans
    many 2048-product tiles with a ragged last tile."""
    rng = W.rng_for(6001)
    X = W.uniform_coo(rng, (37, 53, 29), 60_000)
    Y = W.uniform_coo(rng, (29, 41, 7), 9_000)
    res, ref = check(W.Problem(X, Y, (2,), (0,)), **mode)
    assert ref.products % 2048 != 0 and ref.products > 20 * 2048


@pytest.mark.parametrize("mode", MODES, ids=MODE_IDS)
def test_heavy_duplicates(mode):
    """Few cells, many repeated coordinates: many products per output (summation order matters)."""
    rng = W.rng_for(6002)
    X = W.uniform_coo(rng, (4, 6, 5), 20_000)
    Y = W.uniform_coo(rng, (5, 3), 5_000)
    res, ref = check(W.Problem(X, Y, (2,), (0,)), **mode)
    assert ref.cnt.max() > 1000


@pytest.mark.parametrize("mode", MODES, ids=MODE_IDS)
def test_out_order_and_two_mode_pairing(mode):
    rng = W.rng_for(6003)
    X = W.uniform_coo(rng, (9, 16, 8, 4), 8_000)
    Y = W.uniform_coo(rng, (4, 12, 16), 3_000)
    check(W.Problem(X, Y, (3, 1), (0, 2), out_order=(2, 0, 1)), **mode)


@pytest.mark.parametrize("fy", [5, 63, 64, 4096, 10_000, 65_536, 65_537, 100_000, 300_000, 1_048_576])
def test_dense_rows_segments(fy):
    """Bitmap-row accumulation over Y free key spaces that are below, at and above one
    segment (2^16 free keys), including a last segment that is only partly used."""
    rng = W.rng_for(7000 + fy)
    X = W.uniform_coo(rng, (40, 37), 6_000)
    Y = W.uniform_coo(rng, (37, fy), 30_000)
    res, ref = check(W.Problem(X, Y, (1,), (0,)), strategy=2, accumulator=2)
    assert res.stats.accumulator == 2


def test_dense_rows_multi_chunk_groups():
    """Groups with more X entries than one CTA stages at a time (several chunks per segment)."""
    rng = W.rng_for(7100)
    X = W.uniform_coo(rng, (3, 2_000), 5_000)
    Y = W.uniform_coo(rng, (2_000, 9_000), 20_000)
    res, ref = check(W.Problem(X, Y, (1,), (0,)), strategy=2, accumulator=2)
    assert res.stats.accumulator == 2


def test_dense_rows_rank_windows():
    """Segments holding more distinct keys than the value array: the accumulation pass is
    repeated per window of ranks (one chunk per group)."""
    rng = W.rng_for(7150)
    X = W.uniform_coo(rng, (4, 60), 200)
    Y = W.uniform_coo(rng, (60, 65_536), 60_000)
    res, ref = check(W.Problem(X, Y, (1,), (0,)), strategy=2, accumulator=2)
    assert res.stats.accumulator == 2 and res.nnz > 4 * 20_000


def test_dense_rows_rank_windows_multi_chunk():
    """Rank windows in groups of several chunks."""
    rng = W.rng_for(7160)
    X = W.uniform_coo(rng, (2, 1200), 2_000)
    Y = W.uniform_coo(rng, (1200, 30_000), 40_000)
    res, ref = check(W.Problem(X, Y, (1,), (0,)), strategy=2, accumulator=2)
    assert res.stats.accumulator == 2 and res.nnz > 2 * 10_000


def test_auto_mixes_hash_and_bitmap_groups():
    """AUTO on a row space where some groups fit the warp-sized hash tables and others do not:
    both accumulators run in one call and the result is the oracle's."""
    rng = W.rng_for(7170)
    Xa = W.uniform_coo(rng, (60, 40), 300)
    # a few long rows: every entry of X row 0..3 present
    xc = np.concatenate([Xa.coords.reshape(-1, 2), np.array([[r, c] for r in range(4) for c in range(40)], np.int32)])
    xc = np.unique(xc, axis=0)
    X = W.COO((60, 40), xc.astype(np.int32), rng.uniform(-1, 1, len(xc)))
    Y = W.uniform_coo(rng, (40, 5_000), 2_000)
    res, ref = check(W.Problem(X, Y, (1,), (0,)), strategy=2, accumulator=0)
    assert res.stats.accumulator == 0


def test_dense_rows_sparse_survey():
    """Dense rows when few X entries have a Y run (survivor list keeps contract keys)."""
    rng = W.rng_for(7200)
    X = W.uniform_coo(rng, (50, 3000), 40_000)
    Y = W.uniform_coo(rng, (3000, 700), 400)
    res, ref = check(W.Problem(X, Y, (1,), (0,)), strategy=2, accumulator=2)
    assert res.stats.accumulator == 2


def test_grouped_overflow_groups():
    """Groups whose bound exceeds every shared-memory class use the global overflow table."""
    rng = W.rng_for(6011)
    X = W.uniform_coo(rng, (3, 50), 3_000)
    Y = W.uniform_coo(rng, (50, 100_000), 40_000)
    res, ref = check(W.Problem(X, Y, (1,), (0,)), strategy=2, accumulator=1)
    assert res.stats.table_slots > 0 and res.stats.strategy == 2


def test_grouped_wide_local_keys():
    """Y free key space above 2^32: per-group tables keyed on 64-bit local keys."""
    rng = W.rng_for(6012)
    X = W.uniform_coo(rng, (300, 7), 20_000)
    Y = W.uniform_coo(rng, (7, 70_000, 70_000), 30_000)
    res, ref = check(W.Problem(X, Y, (1,), (0,)))
    assert res.stats.strategy == 2


_DENSE_TABLE = {}


@pytest.mark.parametrize("probe", [1, 4, 8])
@pytest.mark.parametrize("lf", [0.25, 0.9])
def test_global_probe_load_factors(probe, lf):
    """The one global table sized for load factor 0.25 and 0.9 of its bound P = 1.87e6, with
    1.37e6 distinct keys: at 0.9 the 2^21 slots end 65% full, so most keys meet
    occupied slots (or buckets) before their own. Probed lane by lane and by tiles of 4 and 8."""
    if not _DENSE_TABLE:
        rng = W.rng_for(6010)
        X = W.uniform_coo(rng, (2000, 32), 7_735)
        Y = W.uniform_coo(rng, (32, 2000), 7_735)
        p = W.Problem(X, Y, (1,), (0,))
        _DENSE_TABLE["p"] = p
        _DENSE_TABLE["ref"] = oracle.contract(p.X, p.Y, p.cx, p.cy)
    p, ref = _DENSE_TABLE["p"], _DENSE_TABLE["ref"]
    res = gpu_contract(p, strategy=1, probe=probe, load_factor=lf)
    c, v = result_host(res)
    assert_matches_oracle(c, v, ref)
    assert res.stats.strategy == 1 and res.stats.retries == 0
    assert res.stats.table_slots == (1 << 21 if lf == 0.9 else 1 << 23)
    assert ref.nnz > 0.6 * (1 << 21)


def test_grouped_load_factors_agree():
    """The table class thresholds change only memory and speed, never the result."""
    p = W.plain_small()
    ref = oracle.contract(p.X, p.Y, p.cx, p.cy)
    for ga in (0.25, 0.5, 0.75, 0.9):
        res = gpu_contract(p, strategy=2, accumulator=1, group_load_factor=ga)
        c, v = result_host(res)
        assert_matches_oracle(c, v, ref)


def test_empty_and_degenerate():
    rng = W.rng_for(6004)
    A = W.uniform_coo(rng, (5, 6), 0)
    B = W.uniform_coo(rng, (6, 7), 50)
    for p in [W.Problem(A, B, (1,), (0,)), W.Problem(B, W.uniform_coo(rng, (7, 3), 0), (1,), (0,))]:
        for strategy in STRATEGIES:
            res = gpu_contract(p, strategy=strategy)
            assert res.nnz == 0 and res.stats.products == 0
    # no common contract key at all
    X = W.COO((4, 8), [[0, 1], [1, 1]], [1.0, 2.0])
    Y = W.COO((8, 3), [[2, 0], [3, 1]], [1.0, 2.0])
    assert gpu_contract(W.Problem(X, Y, (1,), (0,))).nnz == 0
    # outer product (no paired modes)
    check(W.Problem(W.uniform_coo(rng, (3, 5), 9), W.uniform_coo(rng, (4,), 3), (), ()))
    # full contraction: order-0 output
    X = W.uniform_coo(rng, (6, 7), 30)
    Y = W.uniform_coo(rng, (7, 6), 30)
    res, ref = check(W.Problem(X, Y, (0, 1), (1, 0)))
    assert res.order == 0 and res.nnz == ref.nnz
    # cancellation keeps the structural zero
    X = W.COO((1, 2), [[0, 0], [0, 1]], [1.0, 1.0])
    Y = W.COO((2, 1), [[0, 0], [1, 0]], [1.0, -1.0])
    res, ref = check(W.Problem(X, Y, (1,), (0,)))
    assert res.nnz == 1 and float(res.vals[0]) == 0.0


def test_wide_keys_non_pow2():
    """Output keys above 2^32 with non-power-of-two lengths (64-bit division decode)."""
    rng = W.rng_for(6005)
    X = W.uniform_coo(rng, (1_000_003, 7, 999_983), 3_000)
    Y = W.uniform_coo(rng, (7, 65_537), 500)
    check(W.Problem(X, Y, (1,), (0,)))


def test_results_are_released():
    """Dropping a result (and the tensors viewing it) returns its memory to the context."""
    import gc

    import paper_2410_10094_gb300 as stc

    ctx = stc.default_context()
    p = W.plain_small()
    held0, live0 = stc.stc_ctx_stats(ctx.handle)
    for _ in range(3):
        res = gpu_contract(p)
        coords = res.coords
        del res
        assert stc.stc_ctx_stats(ctx.handle)[1] == live0 + 1  # the tensor keeps it alive
        del coords
        gc.collect()
        held, live = stc.stc_ctx_stats(ctx.handle)
        assert live == live0 and held == held0


def test_errors():
    import paper_2410_10094_gb300 as stc

    rng = W.rng_for(6006)
    X = W.uniform_coo(rng, (5, 6), 10)
    Y = W.uniform_coo(rng, (7, 3), 10)
    with pytest.raises(stc.StcError) as e:
        stc.contract(to_dev(X), to_dev(Y), (1,), (0,))
    assert e.value.status == 2
    bad = W.COO((5, 6), [[0, 6]], [1.0])
    Y2 = W.uniform_coo(rng, (6, 3), 10)
    with pytest.raises(stc.StcError) as e:
        stc.contract(to_dev(bad), to_dev(Y2), (1,), (0,))
    assert e.value.status == 8
    big = W.COO((2 ** 31, 2 ** 31, 4), [[0, 0, 0]], [1.0])
    Yb = W.COO((4, 2 ** 31), [[0, 0]], [1.0])
    with pytest.raises(stc.StcError) as e:
        stc.contract(to_dev(big), to_dev(Yb), (2,), (0,))
    assert e.value.status == 3
    with pytest.raises(stc.StcError) as e:
        stc.contract(to_dev(X), to_dev(W.uniform_coo(rng, (6, 3), 5)), (1,), (0,), out_order=(0, 0))
    assert e.value.status == 1


# ------------------------------------------------------------------ step-level entry points

def test_linearize_matches_oracle_ln_key():
    import paper_2410_10094_gb300 as stc

    rng = W.rng_for(6007)
    T = W.uniform_coo(rng, (7, 300, 11, 5000), 40_000)
    for modes in [(0,), (2, 1), (3, 0, 2), (0, 1, 2, 3), (1, 3)]:
        got = stc.linearize(to_dev(T), modes).cpu().numpy().view(np.uint64)
        ref = oracle.ln_key(T.shape, T.coords, modes)
        np.testing.assert_array_equal(got, ref)
    g = __import__("helpers").golden("ln_key_fig3.json")
    Tg = W.COO(tuple(g["shape"]), g["coords"], [1.0])
    assert stc.linearize(to_dev(Tg), g["modes"]).cpu().tolist() == g["expect"]


def test_group_keys_matches_oracle_counting_sort():
    import torch

    import paper_2410_10094_gb300 as stc

    rng = W.rng_for(6008)
    for n, k in [(0, 5), (1, 1), (5000, 7), (300_000, 65_536), (100_000, 1_000_003)]:
        keys = rng.integers(0, k, n).astype(np.uint64)
        off, perm = stc.group_keys(torch.from_numpy(keys.view(np.int64)).cuda(), k)
        off = off.cpu().numpy().astype(np.int64)
        perm = perm.cpu().numpy().astype(np.int64)
        ref_off, ref_perm = oracle.counting_sort(keys, k)
        np.testing.assert_array_equal(off, ref_off)
        np.testing.assert_array_equal(np.sort(perm), np.arange(n))
        np.testing.assert_array_equal(keys[perm], keys[ref_perm])
        # the same members in every run (order inside a run is unspecified)
        for v in np.unique(keys)[:50]:
            a, b = ref_off[v], ref_off[v + 1]
            assert sorted(perm[a:b]) == sorted(ref_perm[a:b])
    g = __import__("helpers").golden("counting_sort_fig6.json")
    off, _ = stc.group_keys(torch.tensor(g["keys"], dtype=torch.int64).cuda(), g["k"])
    assert off.cpu().tolist() == g["expect_offsets"]


def test_count_matches_oracle_products():
    import paper_2410_10094_gb300 as stc

    rng = W.rng_for(6009)
    X = W.uniform_coo(rng, (40, 30, 20), 50_000)
    Y = W.uniform_coo(rng, (20, 30, 9), 20_000)
    P, nbytes = stc.count(to_dev(X), to_dev(Y), (2, 1), (0, 1))
    assert P == oracle.group_bounds(X, Y, (2, 1), (0, 1)).total
    assert nbytes > 0
    g = __import__("helpers").golden("group_bound_sec43.json")
    Xg = W.COO(tuple(g["X"]["shape"]), g["X"]["coords"], g["X"]["vals"])
    Yg = W.COO(tuple(g["Y"]["shape"]), g["Y"]["coords"], g["Y"]["vals"])
    P, _ = stc.count(to_dev(Xg), to_dev(Yg), g["cx"], g["cy"])
    assert P == g["expect_bound"]


# ------------------------------------------------------------------ benchmark-sized workloads

@pytest.mark.parametrize("mode", MODES, ids=MODE_IDS)
def test_imbalanced_zipf_full(mode):
    """X 4096x512x512 with 2e7 entries, Y 512x512x64 with 2e4 Zipf(1.2) contract keys:
    full parity against the oracle."""
    p = W.imbalanced()
    check(p, **mode)


def test_plain_large_full():
    """256^4 tensors with 5e6 entries each, X modes (2,3) with Y modes (0,1), in the launch
    configuration the benchmark times: every one of the ~3.65e8 outputs against the oracle
    (run in independent parts by X's first free coordinate across the host's cores), nnz and
    P equal to the oracle's, plus the global checksum's closed form."""
    from fullsize import check_full

    p = W.plain_large()
    res = gpu_contract(p, operands=0)
    info = check_full(p, res)
    assert info.outputs == res.nnz and info.products == res.stats.products
    print(f"plain_large: {info.outputs} outputs, {info.products} products in {info.parts} oracle parts on "
          f"{info.threads} threads, {info.seconds:.1f} s")
    # closed form of the checksum: sum_Z z = sum_c (sum_{x: c_x=c} x) (sum_{y: c_y=c} y)
    cxk = p.X.coords[:, 2].astype(np.int64) * 256 + p.X.coords[:, 3]
    cyk = p.Y.coords[:, 0].astype(np.int64) * 256 + p.Y.coords[:, 1]
    sx = np.bincount(cxk, weights=p.X.vals, minlength=65536)
    sy = np.bincount(cyk, weights=p.Y.vals, minlength=65536)
    ax = np.bincount(cxk, weights=np.abs(p.X.vals), minlength=65536)
    ay = np.bincount(cyk, weights=np.abs(p.Y.vals), minlength=65536)
    total = float(res.vals.sum())
    # sum over 3.65e8 outputs in any order: within (n-1) u sum|z| of the exact sum
    assert abs(total - float(sx @ sy)) <= 4e8 * 2.0 ** -53 * float(ax @ ay) * 2


def test_imbalanced_both_zipf():
    """Both operands' contract cells Zipf(1.2) (the product-heavy variant of the imbalanced
    workload). Full size (2e10 products into at most 262,144 outputs): P equal to the count per
    cell, nnz bounded by the output space, and the checksum's closed form within the bound of
    a sum of P terms. Output by output against the oracle on a sub-problem of the same tensors:
    the paired cells at Zipf ranks 8, 12 and 20 (hundreds of terms per output) and every 97th
    cell, all of their entries."""
    from fullsize import check_full

    p = W.imbalanced(both_zipf=True)
    cx = p.X.coords[:, 1].astype(np.int64) * 512 + p.X.coords[:, 2]
    cy = p.Y.coords[:, 0].astype(np.int64) * 512 + p.Y.coords[:, 1]
    nxc = np.bincount(cx, minlength=512 * 512)
    nyc = np.bincount(cy, minlength=512 * 512)
    res = gpu_contract(p, operands=0)
    assert res.stats.products == int((nxc * nyc).sum())
    assert 0 < res.nnz <= 4096 * 64
    sx = np.bincount(cx, weights=p.X.vals, minlength=512 * 512)
    sy = np.bincount(cy, weights=p.Y.vals, minlength=512 * 512)
    ax = np.bincount(cx, weights=np.abs(p.X.vals), minlength=512 * 512)
    ay = np.bincount(cy, weights=np.abs(p.Y.vals), minlength=512 * 512)
    total = float(res.vals.sum())
    bound = 2 * (res.stats.products + res.nnz) * 2.0 ** -53 * float(ax @ ay)
    assert abs(total - float(sx @ sy)) <= bound
    del res
    by_rank = np.argsort(-nyc, kind="stable")
    cells = np.concatenate([by_rank[[7, 11, 19]], np.arange(0, 512 * 512, 97)])
    xi = np.flatnonzero(np.isin(cx, cells))
    yi = np.flatnonzero(np.isin(cy, cells))
    sub = W.Problem(p.X.take(xi), p.Y.take(yi), p.cx, p.cy)
    res = gpu_contract(sub, operands=0)
    info = check_full(sub, res)
    print(f"imbalanced_both sample: {info.products} products into {info.outputs} outputs "
          f"({info.products / max(info.outputs, 1):.0f} per output) against the oracle")
    assert info.products > 50 * info.outputs


# ------------------------------------------------------------------ lane-private dense rows

@pytest.mark.parametrize("shape", [((4, 6, 5), (5, 3)), ((40, 30, 7), (7, 64)), ((9, 7), (7, 1)), ((3, 50), (50, 8))])
def test_lane_rows_against_oracle(shape):
    """STC_ACC_ROWS (F_Y <= 64): heavy repeats per output, F_Y = 64 and F_Y = 1; outputs of one
    or two products bit-exact (the rows are summed in a fixed lane order)."""
    import paper_2410_10094_gb300 as stc

    rng = W.rng_for(6100 + shape[1][1])
    X = W.uniform_coo(rng, shape[0], 6_000)
    Y = W.uniform_coo(rng, shape[1], 3_000)
    res, ref = check(W.Problem(X, Y, (len(shape[0]) - 1,), (0,)), strategy=2, accumulator=stc.ACC_ROWS)
    assert res.stats.accumulator == stc.ACC_ROWS


def test_lane_rows_rejects_wide_rows():
    import paper_2410_10094_gb300 as stc

    rng = W.rng_for(6110)
    p = W.Problem(W.uniform_coo(rng, (10, 5), 100), W.uniform_coo(rng, (5, 65), 100), (1,), (0,))
    with pytest.raises(stc.StcError) as e:
        gpu_contract(p, strategy=2, accumulator=stc.ACC_ROWS)
    assert e.value.status == 1  # STC_ERR_INVALID_ARG


def test_auto_remembers_rows_heavy_shapes():
    """AUTO on a small output key space takes the one global table; once a run of a shape has
    averaged 64 or more products per output cell, the next AUTO call of that shape in the same
    context groups X and takes the lane-private rows, and a later run of the shape that is not
    rows-heavy sends it back. Every result against the oracle."""
    import gc

    import numpy as np

    import paper_2410_10094_gb300 as stc

    rng = W.rng_for(6120)
    X = W.uniform_coo(rng, (512, 8, 8), 50_000)
    X.coords[:, 1] = X.coords[:, 1] % 2  # X's contract cells on 16 of the 64
    X.coords[:, 2] = X.coords[:, 2] % 8
    Y = W.uniform_coo(rng, (8, 8, 16), 2_000)
    p = W.Problem(X, Y, (1, 2), (0, 1))
    ref = oracle.contract(p.X, p.Y, p.cx, p.cy)
    assert ref.products >= 64 * 512 * 16
    ctx = stc.Context(0)
    try:
        def run(prob):
            r = stc.contract(to_dev(prob.X), to_dev(prob.Y), prob.cx, prob.cy, ctx=ctx,
                             operands=stc.OPERANDS_AS_GIVEN)
            return r, (r.stats.strategy, r.stats.accumulator)

        r1, k1 = run(p)
        r2, k2 = run(p)
        assert k1[0] == stc.STRATEGY_GLOBAL and k2 == (stc.STRATEGY_GROUPED, stc.ACC_ROWS)
        for r in (r1, r2):
            c, v = result_host(r)
            assert_matches_oracle(c, v, ref)
        # Same shapes and entry counts, few products: grouped once more, then forgotten. Y's
        # entries move to contract cells (0..3, *), X's to (7, *) but for one in a hundred.
        Xs = W.COO(X.shape, X.coords.copy(), X.vals)
        Xs.coords[:, 1] = np.where(np.arange(X.nnz) % 100 == 0, 0, 7)
        Ys = W.COO(Y.shape, Y.coords.copy(), Y.vals)
        Ys.coords[:, 0] = Ys.coords[:, 0] % 4
        ps = W.Problem(Xs, Ys, (1, 2), (0, 1))
        refs = oracle.contract(ps.X, ps.Y, ps.cx, ps.cy)
        r3, k3 = run(ps)
        r4, k4 = run(ps)
        assert k3[0] == stc.STRATEGY_GROUPED and k3[1] != stc.ACC_ROWS and k4[0] == stc.STRATEGY_GLOBAL
        for r in (r3, r4):
            c, v = result_host(r)
            assert_matches_oracle(c, v, refs)
        del r, r1, r2, r3, r4
    finally:
        gc.collect()
        ctx.close()
