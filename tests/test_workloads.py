"""The seeded generators (CPU): shapes, entry counts, structure and determinism of the
workloads that stand in for the paper's tensors, and the bench's reference arm on a workload
it does not time."""
import json
import subprocess
import sys
import os

import numpy as np

import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def same(a, b):
    return a.shape == b.shape and np.array_equal(a.coords, b.coords) and np.array_equal(a.vals, b.vals)


def test_wide_keys_structure():
    p = W.wide_keys(nnz=20_000, n=16, pool=300, nnz_y=7_000)
    assert p.X.shape == (16, 16, 65536, 65536) and p.Y.shape == (65536, 65536, 16, 16)
    assert p.X.nnz == 20_000 and p.Y.nnz == 7_000
    assert p.cx == (2, 3) and p.cy == (0, 1)
    xc = {tuple(r) for r in p.X.coords[:, 2:4]}
    yc = {tuple(r) for r in p.Y.coords[:, 0:2]}
    # one shared pool of paired cells, spread over the 2^32 space
    assert len(xc | yc) <= 300 and len(xc & yc) > 250
    assert p.X.coords[:, 2:].max() > 60_000
    assert p.X.coords[:, :2].max() < 16 and p.Y.coords[:, 2:].max() < 16
    assert np.all(p.X.vals != 0) and np.all(np.abs(p.Y.vals) <= 1)
    q = W.wide_keys(nnz=20_000, n=16, pool=300, nnz_y=7_000)
    assert same(p.X, q.X) and same(p.Y, q.Y)


def test_table2_shapes_and_counts():
    for name, (shape, nnz) in W.TABLE2.items():
        if nnz > 1_000_000:
            continue
        p = W.table2(name)
        assert p.X is p.Y, "Table 2 cases are self-contractions"
        assert p.X.shape == shape and p.X.nnz == nnz
        assert p.cx == (1, 2) and p.cy == (1, 2)
        assert p.X.coords.min() >= 0 and np.all(p.X.coords < np.asarray(shape))
    small = W.table2("nips", nnz=1000)
    assert small.X.shape == W.TABLE2["nips"][0] and small.X.nnz == 1000


def test_set_sweep_cases():
    for set_no, L in ((1, 50), (2, 100)):
        aa = W.set_sweep(set_no, "AA", 5_000)
        bb = W.set_sweep(set_no, "BB", 5_000)
        ab = W.set_sweep(set_no, "AB", 5_000)
        assert aa.X is aa.Y and aa.X.shape == (L,) * 5
        assert bb.X is bb.Y and bb.X.shape == (L,) * 4
        assert ab.X.shape == (L,) * 5 and ab.Y.shape == (L,) * 4
        for p in (aa, bb, ab):
            assert p.cx == (1, 2) and p.cy == (1, 2) and p.X.nnz == 5_000
        assert same(aa.X, W.set_sweep(set_no, "AA", 5_000).X)


def test_reference_arm_declines_multi_problem_workloads():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload", "sweep",
                          "--steps", "1", "--warmup", "3"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr
    line = json.loads(out.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and "unavailable" in line


def test_key_sample_is_a_sub_contraction():
    """bench.key_sample keeps whole paired cells: every X and Y entry on a kept cell, no other,
    so its products are exactly the workload's products on those cells."""
    import bench

    p = W.plain_large(seed=W.SEED_BASE + 2, nnz=40_000, n=16)
    sp, desc = bench.key_sample(p, 7)
    cell = lambda t, modes: [tuple(r) for r in t.coords[:, list(modes)]]
    kept = set(cell(sp.X, sp.cx)) | set(cell(sp.Y, sp.cy))
    xs, ys = cell(p.X, p.cx), cell(p.Y, p.cy)
    assert sp.X.nnz == sum(c in kept for c in xs) and sp.Y.nnz == sum(c in kept for c in ys)
    from collections import Counter

    cx, cy = Counter(xs), Counter(ys)
    cxs, cys = Counter(cell(sp.X, sp.cx)), Counter(cell(sp.Y, sp.cy))
    for c in kept:
        assert cxs[c] == cx[c] and cys[c] == cy[c]
    assert 0.05 < len(kept) / len(set(xs) | set(ys)) < 0.3
    assert bench.key_sample(p, 1)[0] is p
