"""TEST INFRASTRUCTURE: ctypes access to the plain CPU oracle in ``stc_oracle.cpp``.

Only the test suite, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg
may import this package. The library (``paper_2410_10094_gb300``) never imports it,
and the two share no code: the oracle works on coordinate tuples in ordered maps,
the library on linearised 64-bit keys in GPU hash tables.

Functions and the passages they follow (Swift, arXiv 2410.10094):

* :func:`contract`         Eq. 2, the contraction itself (Section 2.2)
* :func:`ln_key`           the LN key of a mode subset (Section 2.4.1, Fig. 3)
* :func:`counting_sort`    count / cumulative sum / place (Section 4.1.1, Fig. 6)
* :func:`first_seen_ids`   small numbers for keys (Section 4.1.2, Fig. 7)
* :func:`group_bounds`     exact per-group table bound (Section 4.3)
* :func:`table_slots`      the x1.3 probing-table rule (Section 2.3.1, Section 4.3)
"""
from __future__ import annotations

import ctypes as C
import os
import platform
import subprocess
from dataclasses import dataclass
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "stc_oracle.cpp")
_BUILD = os.path.join(_HERE, "_build")
_LIB = None

_ERRORS = {1: "invalid argument", 2: "paired mode lengths differ", 3: "coordinate out of range",
           4: "key does not fit in 64 bits"}


class OracleError(RuntimeError):
    def __init__(self, code: int):
        super().__init__(f"oracle error {code}: {_ERRORS.get(code, 'unknown')}")
        self.code = code


def compile_source(src: str, out: str) -> str:
    """Compile one oracle source file into a shared library at ``out``."""
    cmd = ["g++", "-std=c++17", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-o", out, src]
    subprocess.run(cmd, check=True)
    return out


def lib_path() -> str:
    return os.path.join(_BUILD, f"libstc_oracle_{platform.machine()}.so")


def build(force: bool = False) -> str:
    """Compile the oracle with g++ (-O2, -ffp-contract=off: products rounded before adds).

    ``STC_ORACLE_LIB`` names a prebuilt library to load instead; the mutation test uses it
    to run the pins against deliberately broken copies of the oracle."""
    override = os.environ.get("STC_ORACLE_LIB")
    if override:
        return override
    out = lib_path()
    if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(_SRC):
        return out
    os.makedirs(_BUILD, exist_ok=True)
    tmp = out + f".tmp{os.getpid()}"
    compile_source(_SRC, tmp)
    os.replace(tmp, out)
    return out


def _lib():
    global _LIB
    if _LIB is None:
        L = C.CDLL(build())
        p, i32, i64, u64, vp = C.c_void_p, C.c_int32, C.c_int64, C.c_uint64, C.c_void_p
        L.oracle_contract.argtypes = [i32, p, i64, p, p, i32, p, i64, p, p, i32, p, p, p, C.POINTER(vp)]
        L.oracle_contract.restype = C.c_int
        L.oracle_result_nnz.argtypes = [vp]
        L.oracle_result_nnz.restype = i64
        L.oracle_result_order.argtypes = [vp]
        L.oracle_result_order.restype = i32
        L.oracle_result_products.argtypes = [vp]
        L.oracle_result_products.restype = u64
        L.oracle_result_copy.argtypes = [vp, p, p, p, p]
        L.oracle_result_copy.restype = None
        L.oracle_result_free.argtypes = [vp]
        L.oracle_result_free.restype = None
        L.oracle_ln_key.argtypes = [i32, p, i64, p, i32, p, p]
        L.oracle_ln_key.restype = C.c_int
        L.oracle_counting_sort.argtypes = [i64, p, u64, p, p]
        L.oracle_counting_sort.restype = C.c_int
        L.oracle_first_seen_ids.argtypes = [i64, p, p, p]
        L.oracle_first_seen_ids.restype = C.c_int
        L.oracle_group_bounds.argtypes = [i32, p, i64, p, i32, p, i64, p, i32, p, p, C.POINTER(vp)]
        L.oracle_group_bounds.restype = C.c_int
        L.oracle_groups_count.argtypes = [vp]
        L.oracle_groups_count.restype = i64
        L.oracle_groups_order.argtypes = [vp]
        L.oracle_groups_order.restype = i32
        L.oracle_groups_total.argtypes = [vp]
        L.oracle_groups_total.restype = u64
        L.oracle_groups_copy.argtypes = [vp, p, p, p]
        L.oracle_groups_copy.restype = None
        L.oracle_groups_free.argtypes = [vp]
        L.oracle_groups_free.restype = None
        L.oracle_table_slots.argtypes = [u64]
        L.oracle_table_slots.restype = u64
        _LIB = L
    return _LIB


def _ptr(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _tensor_args(t):
    shape = np.ascontiguousarray(np.asarray(t.shape, dtype=np.int64))
    coords = np.ascontiguousarray(t.coords, dtype=np.int32)
    vals = np.ascontiguousarray(t.vals, dtype=np.float64)
    return shape, coords, vals


def _modes(v: Sequence[int]) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(list(v), dtype=np.int32))


@dataclass
class Result:
    """Output of :func:`contract`, in lexicographic coordinate order.

    ``abs`` is the sum of |x*y| over the products that landed on each entry and
    ``cnt`` their number; ``products`` is the total number of products P."""

    shape: tuple
    coords: np.ndarray
    vals: np.ndarray
    abs: np.ndarray
    cnt: np.ndarray
    products: int

    @property
    def nnz(self) -> int:
        return int(self.vals.shape[0])


def contract(X, Y, cx: Sequence[int], cy: Sequence[int], out_order: Optional[Sequence[int]] = None) -> Result:
    """Eq. 2 over COO lists: Z = X (x) Y, pairing X mode cx[i] with Y mode cy[i]."""
    L = _lib()
    xs, xc, xv = _tensor_args(X)
    ys, yc, yv = _tensor_args(Y)
    mcx, mcy = _modes(cx), _modes(cy)
    oo = None if out_order is None else _modes(out_order)
    h = C.c_void_p()
    rc = L.oracle_contract(len(X.shape), _ptr(xs), xv.shape[0], _ptr(xc), _ptr(xv),
                           len(Y.shape), _ptr(ys), yv.shape[0], _ptr(yc), _ptr(yv),
                           len(mcx), _ptr(mcx), _ptr(mcy), _ptr(oo), C.byref(h))
    if rc:
        raise OracleError(rc)
    try:
        n = L.oracle_result_nnz(h)
        o = L.oracle_result_order(h)
        coords = np.empty((n, o), dtype=np.int32)
        vals = np.empty(n, dtype=np.float64)
        ab = np.empty(n, dtype=np.float64)
        cnt = np.empty(n, dtype=np.int64)
        L.oracle_result_copy(h, _ptr(coords), _ptr(vals), _ptr(ab), _ptr(cnt))
        products = int(L.oracle_result_products(h))
    finally:
        L.oracle_result_free(h)
    free_x = [int(X.shape[j]) for j in range(len(X.shape)) if j not in set(cx)]
    free_y = [int(Y.shape[j]) for j in range(len(Y.shape)) if j not in set(cy)]
    cat = free_x + free_y
    shape = tuple(cat[q] for q in out_order) if out_order is not None else tuple(cat)
    return Result(shape, coords, vals, ab, cnt, products)


def ln_key(shape: Sequence[int], coords: np.ndarray, modes: Sequence[int]) -> np.ndarray:
    """LN keys (Fig. 3) of the listed modes of each coordinate row, first mode most significant."""
    L = _lib()
    sh = np.ascontiguousarray(np.asarray(shape, dtype=np.int64))
    co = np.ascontiguousarray(coords, dtype=np.int32).reshape(-1, len(shape))
    md = _modes(modes)
    out = np.empty(co.shape[0], dtype=np.uint64)
    rc = L.oracle_ln_key(len(shape), _ptr(sh), co.shape[0], _ptr(co), len(md), _ptr(md), _ptr(out))
    if rc:
        raise OracleError(rc)
    return out


def counting_sort(keys: np.ndarray, k: int):
    """Counting sort (Fig. 6): returns (offsets[k+1], perm[n]) with perm stable."""
    L = _lib()
    ks = np.ascontiguousarray(keys, dtype=np.uint64)
    off = np.empty(int(k) + 1, dtype=np.int64)
    perm = np.empty(ks.shape[0], dtype=np.int64)
    rc = L.oracle_counting_sort(ks.shape[0], _ptr(ks), int(k), _ptr(off), _ptr(perm))
    if rc:
        raise OracleError(rc)
    return off, perm


def first_seen_ids(keys: np.ndarray):
    """Small numbers (Fig. 7): returns (ids[n], number of distinct keys)."""
    L = _lib()
    ks = np.ascontiguousarray(keys, dtype=np.uint64)
    ids = np.empty(ks.shape[0], dtype=np.int64)
    nd = C.c_int64()
    rc = L.oracle_first_seen_ids(ks.shape[0], _ptr(ks), _ptr(ids), C.byref(nd))
    if rc:
        raise OracleError(rc)
    return ids, int(nd.value)


@dataclass
class Groups:
    coords: np.ndarray   # [G, number of X free modes], lexicographic order
    bound: np.ndarray    # [G] uint64, Section 4.3 bound per group
    entries: np.ndarray  # [G] X entries per group
    total: int           # sum of bounds = number of products P


def group_bounds(X, Y, cx: Sequence[int], cy: Sequence[int]) -> Groups:
    """Per X-free-group bound of Section 4.3 and the total product count P."""
    L = _lib()
    xs, xc, _ = _tensor_args(X)
    ys, yc, _ = _tensor_args(Y)
    mcx, mcy = _modes(cx), _modes(cy)
    h = C.c_void_p()
    rc = L.oracle_group_bounds(len(X.shape), _ptr(xs), xc.shape[0], _ptr(xc),
                               len(Y.shape), _ptr(ys), yc.shape[0], _ptr(yc),
                               len(mcx), _ptr(mcx), _ptr(mcy), C.byref(h))
    if rc:
        raise OracleError(rc)
    try:
        g = L.oracle_groups_count(h)
        o = L.oracle_groups_order(h)
        coords = np.empty((g, o), dtype=np.int32)
        bound = np.empty(g, dtype=np.uint64)
        entries = np.empty(g, dtype=np.int64)
        L.oracle_groups_copy(h, _ptr(coords), _ptr(bound), _ptr(entries))
        total = int(L.oracle_groups_total(h))
    finally:
        L.oracle_groups_free(h)
    return Groups(coords, bound, entries, total)


def table_slots(bound: int) -> int:
    """Slots of a probing table for ``bound`` entries under the x1.3 rule (Section 2.3.1)."""
    return int(_lib().oracle_table_slots(int(bound)))
