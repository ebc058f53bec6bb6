"""Shared test helpers: dense brute force (numpy einsum), canonical ordering and the
value tolerance. Nothing here is used by the library or by the oracle."""
from __future__ import annotations

import json
import os
import string
from typing import Optional, Sequence

import numpy as np

from workloads import COO, Problem

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")

# Values: |z - z_ref| <= REL_TOL * sum|x*y| per output. Two summation orders of the same
# n terms differ by at most 2(n-1)u * sum|t| (u = 2^-53), which stays below 1e-12 * sum|t|
# for n up to about 4,500 terms per output.
REL_TOL = 1e-12


def golden(name: str) -> dict:
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def coo_from_json(d: dict) -> COO:
    return COO(tuple(d["shape"]), np.asarray(d["coords"], dtype=np.int32).reshape(-1, len(d["shape"])),
               np.asarray(d["vals"], dtype=np.float64))


def coo_to_dense(t: COO, absval: bool = False, ones: bool = False) -> np.ndarray:
    """Dense array with repeated coordinates summed (COO entries are additive)."""
    a = np.zeros(t.shape, dtype=np.float64)
    if t.nnz:
        v = np.ones(t.nnz) if ones else (np.abs(t.vals) if absval else t.vals)
        np.add.at(a, tuple(t.coords.T.astype(np.int64)), v)
    return a


def einsum_spec(ox: int, oy: int, cx: Sequence[int], cy: Sequence[int],
                out_order: Optional[Sequence[int]] = None) -> str:
    letters = iter(string.ascii_letters)
    xl = [next(letters) for _ in range(ox)]
    yl = [next(letters) for _ in range(oy)]
    for a, b in zip(cx, cy):
        yl[b] = xl[a]
    fx = [xl[j] for j in range(ox) if j not in set(cx)]
    fy = [yl[j] for j in range(oy) if j not in set(cy)]
    cat = fx + fy
    out = [cat[q] for q in out_order] if out_order is not None else cat
    return "".join(xl) + "," + "".join(yl) + "->" + "".join(out)


def dense_contract(p: Problem, kind: str = "vals") -> np.ndarray:
    """Brute-force dense contraction with numpy.einsum.

    kind="vals": the values; "abs": sum of |x||y| (the tolerance scale);
    "count": number of products per output (exact small integers)."""
    spec = einsum_spec(p.X.order, p.Y.order, p.cx, p.cy, p.out_order)
    if kind == "vals":
        a, b = coo_to_dense(p.X), coo_to_dense(p.Y)
    elif kind == "abs":
        a, b = coo_to_dense(p.X, absval=True), coo_to_dense(p.Y, absval=True)
    else:
        a, b = coo_to_dense(p.X, ones=True), coo_to_dense(p.Y, ones=True)
    return np.einsum(spec, a, b)


def canonical(coords: np.ndarray, *cols: np.ndarray):
    """Sort rows of ``coords`` lexicographically and apply the same order to ``cols``."""
    coords = np.asarray(coords)
    if coords.ndim != 2 or coords.shape[1] == 0 or coords.shape[0] <= 1:
        return (coords,) + tuple(np.asarray(c) for c in cols)
    order = np.lexsort(coords.T[::-1])
    return (coords[order],) + tuple(np.asarray(c)[order] for c in cols)


def within_tol(z: np.ndarray, z_ref: np.ndarray, abs_ref: np.ndarray, rel: float = REL_TOL) -> np.ndarray:
    return np.abs(z - z_ref) <= rel * abs_ref


def contract_groups_py(X: COO, Y: COO, cx, cy):
    """Pure-Python Section 4.3 bound per X free tuple (tiny inputs only)."""
    xfree = [j for j in range(X.order) if j not in set(cx)]
    cnt = {}
    for j in range(Y.nnz):
        c = tuple(int(Y.coords[j, k]) for k in cy)
        cnt[c] = cnt.get(c, 0) + 1
    b = {}
    for i in range(X.nnz):
        c = tuple(int(X.coords[i, k]) for k in cx)
        f = tuple(int(X.coords[i, k]) for k in xfree)
        b[f] = b.get(f, 0) + cnt.get(c, 0)
    return b
