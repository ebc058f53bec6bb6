"""Helpers for the GPU parity tests: move seeded inputs to the device, call the library
through its C ABI binding, and compare with the oracle element by element."""
from __future__ import annotations

import numpy as np

from helpers import REL_TOL, canonical, within_tol


def to_dev(t):
    import torch

    coords = torch.from_numpy(np.ascontiguousarray(t.coords)).cuda()
    vals = torch.from_numpy(np.ascontiguousarray(t.vals)).cuda()
    return (t.shape, coords, vals)


def gpu_contract(p, **kw):
    """The library on p's tensors. The operands keep their roles unless the caller passes
    operands=...: most tests aim at a kernel path chosen through Y's shape."""
    import paper_2410_10094_gb300 as stc

    kw.setdefault("operands", stc.OPERANDS_AS_GIVEN)
    return stc.contract(to_dev(p.X), to_dev(p.Y), p.cx, p.cy, p.out_order, **kw)


def result_host(res):
    return res.coords.cpu().numpy().reshape(res.nnz, res.order), res.vals.cpu().numpy()


def assert_matches_oracle(coords, vals, ref, rel: float = REL_TOL):
    """Coordinates and nnz bit-exact; values within rel * sum|x*y|; outputs made of at most
    two products bit-exact (their sum does not depend on order)."""
    vals = np.asarray(vals)
    coords = np.asarray(coords).reshape(vals.shape[0], ref.coords.shape[1] if ref.coords.ndim == 2 else 0)
    gc, gv = canonical(coords, vals)
    assert gc.shape[0] == ref.coords.shape[0], f"nnz {gc.shape[0]} != oracle {ref.coords.shape[0]}"
    np.testing.assert_array_equal(gc, ref.coords)
    ok = within_tol(gv, ref.vals, ref.abs, rel)
    if not ok.all():
        bad = np.flatnonzero(~ok)[:5]
        raise AssertionError(f"{(~ok).sum()} values outside tolerance, e.g. idx {bad}: gpu {gv[bad]} "
                             f"oracle {ref.vals[bad]} abs {ref.abs[bad]} cnt {ref.cnt[bad]}")
    few = ref.cnt <= 2
    np.testing.assert_array_equal(gv[few], ref.vals[few])
