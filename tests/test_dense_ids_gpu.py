"""GPU parity of dense ids for large contract key spaces (Section 4.1.2, Fig. 7): the
stc_dense_ids entry point against the oracle's first-seen numbering, and contractions whose
contract key space exceeds 2^26 (renumbered before grouping) against the oracle."""
import numpy as np
import pytest

import oracle
import workloads as W
from gpu_util import assert_matches_oracle, gpu_contract, result_host, to_dev
from helpers import REL_TOL

pytestmark = pytest.mark.gpu

MODES = [dict(strategy=1), dict(strategy=2, accumulator=1), dict(strategy=2, accumulator=2),
         dict(strategy=2, accumulator=0)]
MODE_IDS = ["global", "grouped-hash", "grouped-dense", "grouped-auto"]


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


def assert_same_partition(ids_gpu, d_gpu, keys):
    """Ids are unique only up to renaming: the GPU ids must be dense in [0, D) and induce the
    same partition of the positions as the oracle's first-seen ids."""
    ref, d_ref = oracle.first_seen_ids(keys)
    assert d_gpu == d_ref
    g = np.asarray(ids_gpu, dtype=np.int64)
    assert g.shape == ref.shape
    if g.size == 0:
        return
    assert g.min() >= 0 and g.max() < d_gpu
    # one GPU id per oracle id and one oracle id per GPU id
    pairs = np.unique(np.stack([ref, g], axis=1), axis=0)
    assert pairs.shape[0] == d_ref
    assert np.unique(pairs[:, 1]).size == d_ref


def keys_dev(keys):
    import torch

    return torch.from_numpy(np.ascontiguousarray(keys).view(np.int64)).cuda()


@pytest.mark.parametrize("n,pool", [(0, 1), (1, 1), (1000, 37), (100_003, 5_000), (2_000_000, 600_000),
                                    (300_000, 300_000)])
def test_dense_ids_partition(n, pool):
    import paper_2410_10094_gb300 as stc

    rng = W.rng_for(7000 + n)
    cands = rng.integers(0, 2 ** 63, size=pool, dtype=np.int64).astype(np.uint64) * np.uint64(2) + \
        rng.integers(0, 2, size=pool).astype(np.uint64)
    keys = cands[rng.integers(0, pool, size=n)] if n else np.zeros(0, dtype=np.uint64)
    ids, d = stc.dense_ids(keys_dev(keys))
    assert_same_partition(ids.cpu().numpy(), d, keys)


def test_dense_ids_extreme_keys():
    """0, 2^64 - 1 (the value that marks empty table slots) and 2^64 - 2 are ordinary keys."""
    import paper_2410_10094_gb300 as stc

    top = np.uint64(2 ** 64 - 1)
    keys = np.array([top, 0, top, 5, 0, top - np.uint64(1), top], dtype=np.uint64)
    ids, d = stc.dense_ids(keys_dev(keys))
    assert d == 4
    assert_same_partition(ids.cpu().numpy(), d, keys)
    ids, d = stc.dense_ids(keys_dev(np.full(1000, top, dtype=np.uint64)))
    assert d == 1 and int(ids.max()) == 0


def distinct_y_cells(p):
    return np.unique(p.Y.coords[:, list(p.cy)], axis=0).shape[0]


def check(p, **kw):
    ref = oracle.contract(p.X, p.Y, p.cx, p.cy, p.out_order)
    res = gpu_contract(p, **kw)
    c, v = result_host(res)
    assert_matches_oracle(c, v, ref)
    assert res.stats.products == ref.products
    assert res.shape == ref.shape
    return res, ref


@pytest.mark.parametrize("mode", MODES, ids=MODE_IDS)
@pytest.mark.parametrize("pool,nx,ny", [(1, 3_001, 2_003), (97, 30_011, 20_003), (2_000, 30_011, 20_003)])
def test_wide_keys_parity(mode, pool, nx, ny):
    """A 2^32 contract key space (paired modes of length 65,536), several tiles and a ragged
    tail: full parity, and the number of dense ids equals Y's distinct paired cells."""
    p = W.wide_keys(nnz=nx, n=24, pool=pool, nnz_y=ny)
    res, ref = check(p, **mode)
    assert res.stats.contract_ids == distinct_y_cells(p)
    assert ref.nnz > 0


def test_wide_keys_boundary():
    """2^26 bins exactly can be counted directly (and are renumbered under AUTO, being sparse);
    2^26 + 2^14 are always renumbered. Non-power-of-two lengths, three paired modes, an output
    permutation."""
    import paper_2410_10094_gb300 as stc

    rng = W.rng_for(7101)
    for shape, renum in [((4096, 8192), False), ((4097, 8192), True)]:
        xs = (shape[0], 5, shape[1], 2)
        ys = (7, shape[1], shape[0], 2)
        X = W.uniform_coo(rng, xs, 4_000)
        Y = W.uniform_coo(rng, ys, 3_000)
        # put most entries on a few paired cells so that products exist
        cells = np.stack([rng.integers(0, shape[0], 40), rng.integers(0, shape[1], 40),
                          rng.integers(0, 2, 40)], axis=1)
        X.coords[:, [0, 2, 3]] = cells[rng.integers(0, 40, X.nnz)]
        Y.coords[:, [2, 1, 3]] = cells[rng.integers(0, 40, Y.nnz)]
        p = W.Problem(X, Y, (0, 2, 3), (2, 1, 3), out_order=(1, 0))
        res, ref = check(p, contract_ids=stc.IDS_DIRECT)
        assert (res.stats.contract_ids > 0) == renum
        res, ref = check(p)
        assert res.stats.contract_ids == distinct_y_cells(p)


def test_wide_keys_degenerate():
    """Empty X, empty Y, no common contract key, one shared key, order-0 output."""
    L = 1 << 20
    rng = W.rng_for(7102)
    A = W.uniform_coo(rng, (5, L, L), 0)
    B = W.uniform_coo(rng, (L, L, 7), 300)
    for p in [W.Problem(A, B, (1, 2), (0, 1)), W.Problem(W.uniform_coo(rng, (5, L, L), 300),
                                                         W.uniform_coo(rng, (L, L, 7), 0), (1, 2), (0, 1))]:
        for mode in MODES:
            res = gpu_contract(p, **mode)
            assert res.nnz == 0 and res.stats.products == 0
    # X and Y on disjoint paired cells: every X entry takes the spare id D
    X = W.COO((3, L, L), [[0, 1, 1], [2, 5, 9]], [1.0, 2.0])
    Y = W.COO((L, L, 4), [[1, 2, 0], [9, 5, 3]], [1.0, 2.0])
    res = gpu_contract(W.Problem(X, Y, (1, 2), (0, 1)))
    assert res.nnz == 0 and res.stats.contract_ids == 2
    # one shared key
    X = W.COO((3, L, L), [[0, L - 1, L - 1], [2, L - 1, L - 1], [1, 0, 0]], [1.5, 2.0, 3.0])
    Y = W.COO((L, L, 4), [[L - 1, L - 1, 0], [L - 1, L - 1, 3], [L - 1, L - 1, 3]], [1.0, 2.0, 4.0])
    res, ref = check(W.Problem(X, Y, (1, 2), (0, 1)))
    assert res.nnz == 4 and res.stats.contract_ids == 1
    # full contraction over a 2^40 key space: a scalar
    X = W.uniform_coo(rng, (L, L), 500)
    Y = W.COO((L, L), X.coords[rng.permutation(500)[:300]], W.nonzero_values(rng, 300))
    res, ref = check(W.Problem(X, Y, (0, 1), (0, 1)))
    assert res.order == 0 and res.nnz == 1


def test_wide_keys_count_and_errors():
    import paper_2410_10094_gb300 as stc

    p = W.wide_keys(nnz=40_000, n=16, pool=300)
    P, nbytes = stc.count(to_dev(p.X), to_dev(p.Y), p.cx, p.cy)
    assert P == oracle.group_bounds(p.X, p.Y, p.cx, p.cy).total
    assert nbytes > 0
    bad = W.COO(p.X.shape, p.X.coords.copy(), p.X.vals)
    bad.coords[17, 3] = 65536  # outside its mode
    with pytest.raises(stc.StcError) as e:
        stc.contract(to_dev(bad), to_dev(p.Y), p.cx, p.cy)
    assert e.value.status == 8


def test_wide_keys_full_size_sampled():
    """The benchmark's 2^32-key workload (5e6 entries each, 65,536 shared paired cells) in the
    launch configuration it times: 32 sampled output rows against the oracle, plus full-size
    properties (P exact, unique coordinates, the checksum's closed form)."""
    import torch

    p = W.wide_keys()
    res = gpu_contract(p)
    groups = oracle.group_bounds(p.X, p.Y, p.cx, p.cy)
    assert res.stats.products == groups.total
    assert res.stats.contract_ids == distinct_y_cells(p)
    assert res.nnz <= groups.total
    rng = W.rng_for(7103)
    rows = p.X.coords[rng.integers(0, p.X.nnz, 32)][:, :2].astype(np.int64)
    row_keys = np.unique(rows[:, 0] * 256 + rows[:, 1])
    xkey = p.X.coords[:, 0].astype(np.int64) * 256 + p.X.coords[:, 1]
    ref = oracle.contract(p.X.take(np.isin(xkey, row_keys)), p.Y, p.cx, p.cy)
    zc = res.coords
    zkey = zc[:, 0].to(torch.int64) * 256 + zc[:, 1].to(torch.int64)
    sel = torch.isin(zkey, torch.from_numpy(row_keys).cuda())
    assert_matches_oracle(zc[sel].cpu().numpy(), res.vals[sel].cpu().numpy(), ref)
    full = ((zc[:, 0].to(torch.int64) * 256 + zc[:, 1]) * 256 + zc[:, 2]) * 256 + zc[:, 3]
    assert torch.unique(full).numel() == res.nnz
    cxk = p.X.coords[:, 2].astype(np.int64) * 65536 + p.X.coords[:, 3]
    cyk = p.Y.coords[:, 0].astype(np.int64) * 65536 + p.Y.coords[:, 1]
    cells, inv = np.unique(np.concatenate([cxk, cyk]), return_inverse=True)
    ix, iy = inv[:p.X.nnz], inv[p.X.nnz:]
    sx = np.bincount(ix, weights=p.X.vals, minlength=cells.size)
    sy = np.bincount(iy, weights=p.Y.vals, minlength=cells.size)
    ax = np.bincount(ix, weights=np.abs(p.X.vals), minlength=cells.size)
    ay = np.bincount(iy, weights=np.abs(p.Y.vals), minlength=cells.size)
    total = float(res.vals.sum())
    assert abs(total - float(sx @ sy)) <= REL_TOL * float(ax @ ay) * 10


def test_server_routes_wide_keys_alone():
    """A request with a 2^32 contract key space among small ones: the server runs it as a
    plain contraction and its result matches the oracle, as do the others'."""
    import paper_2410_10094_gb300 as stc

    rng = W.rng_for(7104)
    probs = [W.small_pair(rng, nnz_hi=3e3) for _ in range(6)]
    probs.insert(3, W.wide_keys(nnz=20_000, n=16, pool=200))
    sv = stc.Server(max_batch=8, workers=1)
    tickets = [sv.submit(to_dev(p.X), to_dev(p.Y), p.cx, p.cy, p.out_order) for p in probs]
    got = [result_host(sv.wait(t)[0]) for t in tickets]
    sv.close()
    for p, (c, v) in zip(probs, got):
        assert_matches_oracle(c, v, oracle.contract(p.X, p.Y, p.cx, p.cy, p.out_order))


@pytest.mark.parametrize("seed", range(30))
def test_random_cases_renumbered(seed):
    """Tiny random problems (orders 1-5, repeated coordinates, any number of paired modes)
    with the contract keys renumbered even where direct counting applies."""
    import paper_2410_10094_gb300 as stc

    rng = W.rng_for(7200 + seed)
    p = W.random_case(rng, max_order=5, max_size=6, max_nnz=120)
    for mode in (dict(strategy=1), dict(strategy=2, accumulator=0)):
        res, ref = check(p, contract_ids=stc.IDS_DENSE, **mode)
        K = int(np.prod([p.X.shape[j] for j in p.cx], dtype=object))
        if K > 1 and p.Y.nnz:
            assert res.stats.contract_ids == distinct_y_cells(p)


def test_direct_request_above_limit_is_renumbered():
    import paper_2410_10094_gb300 as stc

    p = W.wide_keys(nnz=5_000, n=8, pool=50)
    res, _ = check(p, contract_ids=stc.IDS_DIRECT)
    assert res.stats.contract_ids == distinct_y_cells(p)
