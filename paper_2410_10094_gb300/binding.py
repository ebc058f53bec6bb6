"""ctypes binding of ``libstc.so`` (include/stc.h). Argument marshalling only: every step of
the contraction runs in the library's CUDA kernels. PyTorch supplies device memory and
streams; there is no CPU path, and a missing library raises instead of falling back."""
from __future__ import annotations

import ctypes as C
import os
import threading
from dataclasses import dataclass
from typing import Optional, Sequence

from .build import LIB as LIB_PATH

STC_OK = 0
STATUS_NAMES = {
    0: "STC_OK", 1: "STC_ERR_INVALID_ARG", 2: "STC_ERR_SHAPE_MISMATCH", 3: "STC_ERR_KEY_OVERFLOW",
    4: "STC_ERR_OUT_OF_MEMORY", 5: "STC_ERR_TABLE_FULL", 6: "STC_ERR_TIMEOUT", 7: "STC_ERR_CUDA",
    8: "STC_ERR_COORD_OUT_OF_RANGE", 9: "STC_ERR_UNSUPPORTED", 10: "STC_ERR_CANCELLED",
}
STRATEGY_AUTO, STRATEGY_GLOBAL, STRATEGY_GROUPED = 0, 1, 2
ACC_AUTO, ACC_HASH, ACC_DENSE, ACC_HASH_SCAN, ACC_ROWS = 0, 1, 2, 3, 4
IDS_AUTO, IDS_DIRECT, IDS_DENSE = 0, 1, 2
OPERANDS_AUTO, OPERANDS_AS_GIVEN, OPERANDS_SWAPPED = 0, 1, 2
STC_MAX_ORDER = 8


class StcError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class stc_coo(C.Structure):
    _fields_ = [("order", C.c_int32), ("shape", C.POINTER(C.c_int64)), ("nnz", C.c_int64),
                ("coords", C.c_void_p), ("vals", C.c_void_p)]


class stc_keyed(C.Structure):
    _fields_ = [("order", C.c_int32), ("shape", C.POINTER(C.c_int64)), ("nnz", C.c_int64),
                ("keys", C.c_void_p), ("vals", C.c_void_p)]


class stc_problem(C.Structure):
    _fields_ = [("X", stc_coo), ("Y", stc_coo), ("ncontract", C.c_int32), ("cx", C.POINTER(C.c_int32)),
                ("cy", C.POINTER(C.c_int32)), ("out_order", C.POINTER(C.c_int32))]


class stc_server_opts(C.Structure):
    _fields_ = [("mem_budget_bytes", C.c_uint64), ("max_batch", C.c_int32), ("workers", C.c_int32),
                ("plain", C.c_int32), ("reserved_", C.c_int32)]


class stc_opts(C.Structure):
    _fields_ = [("strategy", C.c_int32), ("record_times", C.c_int32), ("load_factor", C.c_double),
                ("group_load_factor", C.c_double), ("accumulator", C.c_int32), ("contract_ids", C.c_int32),
                ("operands", C.c_int32), ("table_shrink", C.c_int32), ("output_keys", C.c_int32),
                ("probe", C.c_int32)]


class stc_stats(C.Structure):
    _fields_ = [("products", C.c_uint64), ("survivors", C.c_uint64), ("out_capacity", C.c_uint64),
                ("table_slots", C.c_uint64), ("groups", C.c_uint64), ("strategy", C.c_int32),
                ("nstages", C.c_int32), ("launches", C.c_uint32), ("accumulator", C.c_int32),
                ("stage_ms", C.c_float * 8), ("contract_ids", C.c_uint64), ("swapped", C.c_int32),
                ("retries", C.c_int32)]


EXPORTS = {
    "stc_status_string": ([C.c_int], C.c_char_p),
    "stc_last_error": ([], C.c_char_p),
    "stc_create": ([C.POINTER(C.c_void_p), C.c_int, C.c_size_t], C.c_int),
    "stc_destroy": ([C.c_void_p], C.c_int),
    "stc_ctx_stats": ([C.c_void_p, C.POINTER(C.c_uint64), C.POINTER(C.c_int64)], C.c_int),
    "stc_contract": ([C.c_void_p, C.POINTER(stc_coo), C.POINTER(stc_coo), C.c_int32, C.c_void_p, C.c_void_p,
                      C.c_void_p, C.POINTER(stc_opts), C.c_void_p, C.POINTER(C.c_void_p)], C.c_int),
    "stc_contract_batch": ([C.c_void_p, C.c_int32, C.POINTER(stc_problem), C.POINTER(stc_opts), C.c_void_p,
                            C.POINTER(C.c_void_p)], C.c_int),
    "stc_server_create": ([C.c_void_p, C.POINTER(stc_server_opts), C.POINTER(C.c_void_p)], C.c_int),
    "stc_server_submit": ([C.c_void_p, C.POINTER(stc_problem), C.POINTER(C.c_uint64)], C.c_int),
    "stc_server_poll": ([C.c_void_p, C.c_uint64, C.POINTER(C.c_int32)], C.c_int),
    "stc_server_wait": ([C.c_void_p, C.c_uint64, C.c_int64, C.POINTER(C.c_void_p), C.POINTER(C.c_double)], C.c_int),
    "stc_server_destroy": ([C.c_void_p], C.c_int),
    "stc_server_cancel": ([C.c_void_p, C.c_uint64, C.POINTER(C.c_int32)], C.c_int),
    "stc_batch_plan_create": ([C.c_void_p, C.c_int32, C.POINTER(stc_problem), C.POINTER(stc_opts),
                               C.POINTER(C.c_void_p)], C.c_int),
    "stc_batch_plan_run": ([C.c_void_p, C.c_void_p, C.POINTER(C.c_void_p)], C.c_int),
    "stc_batch_plan_stats": ([C.c_void_p, C.POINTER(C.c_int64), C.POINTER(C.c_int64), C.POINTER(C.c_double),
                              C.POINTER(C.c_int32), C.POINTER(C.c_int32)], C.c_int),
    "stc_batch_plan_destroy": ([C.c_void_p], C.c_int),
    "stc_measure_peaks": ([C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_double)], C.c_int),
    "stc_contract_keyed": ([C.c_void_p, C.POINTER(stc_keyed), C.POINTER(stc_coo), C.c_int32, C.c_void_p,
                            C.c_void_p, C.c_void_p, C.POINTER(stc_opts), C.c_void_p, C.POINTER(C.c_void_p)], C.c_int),
    "stc_result_keys": ([C.c_void_p, C.POINTER(C.c_void_p)], C.c_int),
    "stc_result_as_keyed": ([C.c_void_p, C.POINTER(stc_keyed)], C.c_int),
    "stc_count": ([C.c_void_p, C.POINTER(stc_coo), C.POINTER(stc_coo), C.c_int32, C.c_void_p, C.c_void_p,
                   C.c_void_p, C.POINTER(C.c_uint64), C.POINTER(C.c_uint64)], C.c_int),
    "stc_linearize": ([C.c_void_p, C.POINTER(stc_coo), C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p], C.c_int),
    "stc_group_keys": ([C.c_void_p, C.c_void_p, C.c_int64, C.c_uint64, C.c_void_p, C.c_void_p, C.c_void_p],
                       C.c_int),
    "stc_group_keys_static": ([C.c_void_p, C.c_int64, C.c_uint64, C.c_void_p, C.c_void_p, C.c_void_p], C.c_int),
    "stc_dense_ids": ([C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.POINTER(C.c_uint64), C.c_void_p], C.c_int),
    "stc_result_as_coo": ([C.c_void_p, C.POINTER(stc_coo)], C.c_int),
    "stc_result_info": ([C.c_void_p, C.POINTER(C.c_int64), C.POINTER(C.c_int32),
                         C.POINTER(C.POINTER(C.c_int64))], C.c_int),
    "stc_result_data": ([C.c_void_p, C.POINTER(C.c_void_p), C.POINTER(C.c_void_p)], C.c_int),
    "stc_result_stats": ([C.c_void_p, C.POINTER(stc_stats)], C.c_int),
    "stc_result_free": ([C.c_void_p], C.c_int),
}

_lib = None
_lib_lock = threading.Lock()


def load(path: Optional[str] = None):
    """Load libstc.so (built by ``paper_2410_10094_gb300.build``); raises if it is missing."""
    global _lib
    with _lib_lock:
        if _lib is None:
            p = path or LIB_PATH
            if not os.path.exists(p):
                raise ImportError(f"{p} is not built; run `python -m paper_2410_10094_gb300.build` "
                                  "(there is no CPU fallback)")
            L = C.CDLL(p)
            for name, (args, res) in EXPORTS.items():
                fn = getattr(L, name)
                fn.argtypes = args
                fn.restype = res
            _lib = L
        return _lib


def check(status: int):
    if status != STC_OK:
        msg = load().stc_last_error().decode(errors="replace")
        raise StcError(status, msg)


# ---------------------------------------------------------------- thin wrappers, same names

def stc_status_string(s: int) -> str:
    return load().stc_status_string(s).decode()


def stc_create(device: int = 0, mem_budget_bytes: int = 0) -> int:
    h = C.c_void_p()
    check(load().stc_create(C.byref(h), device, mem_budget_bytes))
    return h.value


def stc_destroy(ctx: int):
    check(load().stc_destroy(C.c_void_p(ctx)))


def stc_ctx_stats(ctx: int):
    """(device bytes held, live results) of a context."""
    held, live = C.c_uint64(), C.c_int64()
    check(load().stc_ctx_stats(C.c_void_p(ctx), C.byref(held), C.byref(live)))
    return int(held.value), int(live.value)


def _mode_array(v: Sequence[int]):
    n = len(v)
    arr = (C.c_int32 * max(n, 1))(*[int(x) for x in v])
    return arr


class _CooArg:
    """Keeps the ctypes views of one input alive for the duration of a call."""

    def __init__(self, shape, coords, vals):
        import torch

        self.shape_arr = (C.c_int64 * max(len(shape), 1))(*[int(s) for s in shape])
        order = len(shape)
        if coords is not None and coords.numel():
            if coords.device.type != "cuda" or coords.dtype != torch.int32 or not coords.is_contiguous():
                raise ValueError("coords must be a contiguous CUDA int32 tensor of shape [nnz, order]")
        if vals is not None and vals.numel():
            if vals.device.type != "cuda" or vals.dtype != torch.float64 or not vals.is_contiguous():
                raise ValueError("vals must be a contiguous CUDA float64 tensor of shape [nnz]")
        nnz = int(vals.shape[0]) if vals is not None else 0
        if coords is not None and coords.dim() == 2 and (coords.shape[0] != nnz or coords.shape[1] != order):
            raise ValueError("coords must have shape [nnz, order]")
        self.coo = stc_coo(order, C.cast(self.shape_arr, C.POINTER(C.c_int64)), nnz,
                           C.c_void_p(coords.data_ptr() if coords is not None and coords.numel() else 0),
                           C.c_void_p(vals.data_ptr() if vals is not None and vals.numel() else 0))


def _stream_handle(stream) -> int:
    import torch

    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream) if hasattr(stream, "cuda_stream") else int(stream)


def stc_contract(ctx: int, X, Y, cx: Sequence[int], cy: Sequence[int], out_order=None, opts: stc_opts = None,
                 stream=None) -> int:
    """Calls stc_contract; X and Y are (shape, coords, vals) with CUDA tensors. Returns the
    stc_result handle (free with stc_result_free)."""
    xa, ya = _CooArg(*X), _CooArg(*Y)
    if len(cx) != len(cy):
        raise ValueError("cx and cy must have the same length")
    acx, acy = _mode_array(cx), _mode_array(cy)
    oo = _mode_array(out_order) if out_order is not None else None
    r = C.c_void_p()
    check(load().stc_contract(C.c_void_p(ctx), C.byref(xa.coo), C.byref(ya.coo), len(cx), acx, acy, oo,
                              C.byref(opts) if opts is not None else None, C.c_void_p(_stream_handle(stream)),
                              C.byref(r)))
    return r.value


def stc_contract_keyed(ctx: int, X, Y, cx: Sequence[int], cy: Sequence[int], out_order=None,
                       opts: stc_opts = None, stream=None) -> int:
    """Calls stc_contract_keyed; X is (shape, keys, vals) with keys a CUDA int64 tensor holding
    the uint64 keys, Y is (shape, coords, vals). Returns the stc_result handle."""
    import torch

    shape, keys, vals = X
    if keys.numel() and (keys.device.type != "cuda" or keys.dtype not in (torch.int64, getattr(torch, "uint64", torch.int64))
                         or not keys.is_contiguous()):
        raise ValueError("keys must be a contiguous CUDA int64 (or uint64) tensor")
    xs = (C.c_int64 * max(len(shape), 1))(*[int(v) for v in shape])
    xk = stc_keyed(len(shape), C.cast(xs, C.POINTER(C.c_int64)), int(vals.shape[0]),
                   C.c_void_p(keys.data_ptr() if keys.numel() else 0), C.c_void_p(vals.data_ptr() if vals.numel() else 0))
    ya = _CooArg(*Y)
    if len(cx) != len(cy):
        raise ValueError("cx and cy must have the same length")
    acx, acy = _mode_array(cx), _mode_array(cy)
    oo = _mode_array(out_order) if out_order is not None else None
    r = C.c_void_p()
    check(load().stc_contract_keyed(C.c_void_p(ctx), C.byref(xk), C.byref(ya.coo), len(cx), acx, acy, oo,
                                    C.byref(opts) if opts is not None else None, C.c_void_p(_stream_handle(stream)),
                                    C.byref(r)))
    return r.value


class BatchProblems:
    """The stc_problem array of a batch, built once (the inputs' device memory must stay
    alive and unchanged while it is used). problems: sequence of (X, Y, cx, cy[, out_order])
    with X and Y as (shape, coords, vals) CUDA tensors."""

    def __init__(self, problems):
        probs = [tuple(p) + (None,) * (5 - len(p)) for p in problems]
        self.n = len(probs)
        self._keep = []
        self.arr = (stc_problem * max(self.n, 1))()
        for i, (X, Y, cx, cy, out_order) in enumerate(probs):
            xa, ya = _CooArg(*X), _CooArg(*Y)
            acx, acy = _mode_array(cx), _mode_array(cy)
            oo = _mode_array(out_order) if out_order is not None else None
            self._keep.extend([X, Y, xa, ya, acx, acy, oo])
            self.arr[i].X = xa.coo
            self.arr[i].Y = ya.coo
            self.arr[i].ncontract = len(cx)
            self.arr[i].cx = C.cast(acx, C.POINTER(C.c_int32))
            self.arr[i].cy = C.cast(acy, C.POINTER(C.c_int32))
            self.arr[i].out_order = C.cast(oo, C.POINTER(C.c_int32)) if oo is not None else None


def stc_contract_batch(ctx: int, problems, opts: stc_opts = None, stream=None):
    """Calls stc_contract_batch; problems is a BatchProblems or a sequence of (X, Y, cx, cy,
    out_order) with X and Y as (shape, coords, vals) CUDA tensors. Returns the list of
    stc_result handles."""
    bp = problems if isinstance(problems, BatchProblems) else BatchProblems(problems)
    n = bp.n
    outs = (C.c_void_p * max(n, 1))()
    check(load().stc_contract_batch(C.c_void_p(ctx), n, bp.arr, C.byref(opts) if opts is not None else None,
                                    C.c_void_p(_stream_handle(stream)), outs))
    return [outs[i] for i in range(n)]


def stc_count(ctx: int, X, Y, cx, cy, stream=None):
    xa, ya = _CooArg(*X), _CooArg(*Y)
    acx, acy = _mode_array(cx), _mode_array(cy)
    P, B = C.c_uint64(), C.c_uint64()
    check(load().stc_count(C.c_void_p(ctx), C.byref(xa.coo), C.byref(ya.coo), len(cx), acx, acy,
                           C.c_void_p(_stream_handle(stream)), C.byref(P), C.byref(B)))
    return int(P.value), int(B.value)


def stc_linearize(ctx: int, T, modes: Sequence[int], keys_out, stream=None):
    ta = _CooArg(*T)
    am = _mode_array(modes)
    check(load().stc_linearize(C.c_void_p(ctx), C.byref(ta.coo), len(modes), am,
                               C.c_void_p(keys_out.data_ptr() if keys_out.numel() else 0),
                               C.c_void_p(_stream_handle(stream))))


def stc_group_keys(ctx: int, keys, k: int, offsets_out, perm_out, stream=None):
    n = int(keys.numel())
    check(load().stc_group_keys(C.c_void_p(ctx), C.c_void_p(keys.data_ptr() if n else 0), n, int(k),
                                C.c_void_p(offsets_out.data_ptr()), C.c_void_p(perm_out.data_ptr() if n else 0),
                                C.c_void_p(_stream_handle(stream))))


def stc_dense_ids(ctx: int, keys, ids_out, stream=None) -> int:
    """Dense ids of device uint64/int64 keys into int32/uint32 ids_out; returns D."""
    n = int(keys.numel())
    d = C.c_uint64()
    check(load().stc_dense_ids(C.c_void_p(ctx), C.c_void_p(keys.data_ptr() if n else 0), n,
                               C.c_void_p(ids_out.data_ptr() if n else 0), C.byref(d),
                               C.c_void_p(_stream_handle(stream))))
    return d.value


def _check_static_group_args(keys, k: int, offsets_out, perm_out):
    """The C call cannot see the size, type or device of the arrays it is given: anything
    short or misplaced would be written past its end on the device. Checked here."""
    import torch

    for name, t in (("keys", keys), ("offsets_out", offsets_out), ("perm_out", perm_out)):
        if not isinstance(t, torch.Tensor):
            raise ValueError(f"{name} must be a torch tensor")
        if not t.is_cuda:
            raise ValueError(f"{name} must be a CUDA tensor, not on {t.device}")
        if t.device.index != torch.cuda.current_device():
            raise ValueError(f"{name} is on {t.device}, not the current device cuda:{torch.cuda.current_device()}")
        if not t.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
    if keys.dtype not in (torch.int64, getattr(torch, "uint64", torch.int64)):
        raise ValueError(f"keys must be int64 or uint64, not {keys.dtype}")
    for name, t in (("offsets_out", offsets_out), ("perm_out", perm_out)):
        if t.dtype not in (torch.int32, getattr(torch, "uint32", torch.int32)):
            raise ValueError(f"{name} must be int32 or uint32, not {t.dtype}")
    if int(k) < 0:
        raise ValueError("k must be >= 0")
    if offsets_out.numel() < int(k) + 1:
        raise ValueError(f"offsets_out holds {offsets_out.numel()} entries; k + 1 = {int(k) + 1} are written")
    if perm_out.numel() < keys.numel():
        raise ValueError(f"perm_out holds {perm_out.numel()} entries; n = {keys.numel()} are written")


def stc_group_keys_static(keys, k: int, offsets_out, perm_out, stream=None):
    """stc_group_keys without allocation (fixed device scratch; k <= 262144). Runs on the
    current device; calls that overlap on the GPU race on the shared scratch. The arrays'
    sizes, types, layout and device are checked before the call (ValueError)."""
    _check_static_group_args(keys, k, offsets_out, perm_out)
    n = int(keys.numel())
    check(load().stc_group_keys_static(C.c_void_p(keys.data_ptr() if n else 0), n, int(k),
                                       C.c_void_p(offsets_out.data_ptr()),
                                       C.c_void_p(perm_out.data_ptr() if n else 0),
                                       C.c_void_p(_stream_handle(stream))))


def stc_result_info(r: int):
    nnz, order = C.c_int64(), C.c_int32()
    shape = C.POINTER(C.c_int64)()
    check(load().stc_result_info(C.c_void_p(r), C.byref(nnz), C.byref(order), C.byref(shape)))
    return int(nnz.value), int(order.value), tuple(shape[i] for i in range(order.value))


def stc_result_data(r: int):
    co, va = C.c_void_p(), C.c_void_p()
    check(load().stc_result_data(C.c_void_p(r), C.byref(co), C.byref(va)))
    return co.value or 0, va.value or 0


def stc_result_stats(r: int) -> stc_stats:
    st = stc_stats()
    check(load().stc_result_stats(C.c_void_p(r), C.byref(st)))
    return st


def stc_result_free(r: int):
    check(load().stc_result_free(C.c_void_p(r)))


# ---------------------------------------------------------------- convenience layer

class _Handle:
    """Owns one stc_result; frees it when the last Result or tensor view lets go."""

    def __init__(self, handle: int):
        self.handle = handle

    def __del__(self):
        h = getattr(self, "handle", 0)
        if h and _lib is not None:
            stc_result_free(h)
            self.handle = 0


class _DeviceArray:
    """Exposes library-owned device memory through __cuda_array_interface__; keeps the
    owning handle alive while any tensor views it."""

    def __init__(self, owner: _Handle, ptr: int, shape, typestr: str):
        self._owner = owner
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": typestr, "data": (ptr, False),
                                         "version": 3, "strides": None}


class Context:
    """An stc_ctx on one device (its memory pool lives as long as the context)."""

    def __init__(self, device: int = 0, mem_budget_bytes: int = 0):
        self.device = device
        self.handle = stc_create(device, mem_budget_bytes)

    def stats(self):
        """(device bytes the context holds now, live results)."""
        return stc_ctx_stats(self.handle)

    def close(self):
        if self.handle:
            stc_destroy(self.handle)
            self.handle = 0


_default_ctx = {}


def default_context(device: Optional[int] = None) -> Context:
    import torch

    dev = torch.cuda.current_device() if device is None else device
    if dev not in _default_ctx:
        _default_ctx[dev] = Context(dev)
    return _default_ctx[dev]


@dataclass
class Stats:
    products: int
    survivors: int
    out_capacity: int
    table_slots: int
    groups: int
    strategy: int
    launches: int
    accumulator: int
    stage_ms: tuple
    contract_ids: int = 0
    swapped: int = 0
    retries: int = 0


class Result:
    """A finished contraction. ``coords`` (int32 [nnz, order]) and ``vals`` (float64 [nnz])
    are zero-copy CUDA tensors over the library's memory, made on first access; they keep it
    alive."""

    def __init__(self, handle: int):
        self._h = _Handle(handle)
        self.handle = handle
        self.nnz, self.order, self.shape = stc_result_info(handle)
        st = stc_result_stats(handle)
        self.stats = Stats(st.products, st.survivors, st.out_capacity, st.table_slots, st.groups, st.strategy,
                           st.launches, st.accumulator, tuple(st.stage_ms[i] for i in range(max(st.nstages, 0))),
                           st.contract_ids, st.swapped, st.retries)
        self._coords = self._vals = self._keys = None
        kp = C.c_void_p()
        check(load().stc_result_keys(C.c_void_p(handle), C.byref(kp)))
        self.keys_form = bool(kp.value)

    @property
    def keys(self):
        """Output keys (int64 [nnz], the uint64 row-major indices over ``shape``) of a result made
        with output_keys; None for a result in coordinate form."""
        if not self.keys_form:
            return None
        if self._keys is None:
            import torch

            if self.nnz:
                kp = C.c_void_p()
                check(load().stc_result_keys(C.c_void_p(self.handle), C.byref(kp)))
                self._keys = torch.as_tensor(_DeviceArray(self._h, kp.value, (self.nnz,), "<i8"), device="cuda")
            else:
                self._keys = torch.empty((0,), dtype=torch.int64, device="cuda")
        return self._keys

    @property
    def coords(self):
        if self.keys_form:
            return None
        if self._coords is None:
            import torch

            if self.nnz and self.order:
                cp, _ = stc_result_data(self.handle)
                self._coords = torch.as_tensor(_DeviceArray(self._h, cp, (self.nnz, self.order), "<i4"),
                                               device="cuda")
            else:
                self._coords = torch.empty((self.nnz, self.order), dtype=torch.int32, device="cuda")
        return self._coords

    @property
    def vals(self):
        if self._vals is None:
            import torch

            if self.nnz:
                _, vp = stc_result_data(self.handle)
                self._vals = torch.as_tensor(_DeviceArray(self._h, vp, (self.nnz,), "<f8"), device="cuda")
            else:
                self._vals = torch.empty((0,), dtype=torch.float64, device="cuda")
        return self._vals

    @property
    def tensor(self):
        """(shape, coords, vals), or (shape, keys, vals) for a result in key form: the result as
        the input of a further contraction (a chain; stc_contract_keyed takes the key form), with
        no copy; the tensors keep the result's memory alive."""
        return (tuple(self.shape), self.keys if self.keys_form else self.coords, self.vals)



def contract(X, Y, cx: Sequence[int], cy: Sequence[int], out_order=None, *, strategy: int = STRATEGY_AUTO,
             load_factor: float = 0.0, group_load_factor: float = 0.0, accumulator: int = ACC_AUTO,
             contract_ids: int = IDS_AUTO, operands: int = OPERANDS_AUTO, record_times: bool = False,
             table_shrink: int = 0, output_keys: bool = False, probe: int = 0, stream=None,
             ctx: Context = None) -> Result:
    """Z = X (x) Y (Eq. 2) on the GPU. X and Y are (shape, coords, vals) with coords a CUDA
    int32 [nnz, order] tensor and vals a CUDA float64 [nnz] tensor. ``table_shrink`` is the
    fault-injection knob of stc_opts (an undersized first table, retried inside the call);
    ``probe`` the lanes that probe the one global table together (0 auto, 1, 4 or 8)."""
    ctx = ctx or default_context()
    o = stc_opts(int(strategy), 1 if record_times else 0, float(load_factor), float(group_load_factor),
                 int(accumulator), int(contract_ids), int(operands), int(table_shrink), 1 if output_keys else 0,
                 int(probe))
    return Result(stc_contract(ctx.handle, X, Y, cx, cy, out_order, o, stream))


def contract_keyed(X, Y, cx: Sequence[int], cy: Sequence[int], out_order=None, *, strategy: int = STRATEGY_AUTO,
                   accumulator: int = ACC_AUTO, output_keys: bool = False, record_times: bool = False, stream=None,
                   ctx: Context = None) -> Result:
    """Z = X (x) Y with X in key form, (shape, keys, vals) as Result.tensor gives for a result made
    with output_keys; X's contracted modes must be its last (or first) len(cx) modes, in order."""
    ctx = ctx or default_context()
    o = stc_opts(int(strategy), 1 if record_times else 0, 0.0, 0.0, int(accumulator), IDS_DIRECT, OPERANDS_AS_GIVEN, 0,
                 1 if output_keys else 0, 0)
    return Result(stc_contract_keyed(ctx.handle, X, Y, cx, cy, out_order, o, stream))


def contract_batch(problems, *, group_load_factor: float = 0.0, record_times: bool = False, stream=None,
                   ctx: Context = None):
    """Many independent contractions in one batch (shared passes). problems: a BatchProblems
    or a sequence of (X, Y, cx, cy) or (X, Y, cx, cy, out_order). Returns one Result per
    problem."""
    ctx = ctx or default_context()
    bp = problems if isinstance(problems, BatchProblems) else BatchProblems(problems)
    o = stc_opts(STRATEGY_GROUPED, 1 if record_times else 0, 0.0, float(group_load_factor), ACC_HASH, 0, 0, 0)
    return [Result(h) for h in stc_contract_batch(ctx.handle, bp, o, stream)]


class BatchPlan:
    """A prepared batch (stc_batch_plan_*): the problems held by the library across runs; once
    the group load factor is settled each run replays one captured CUDA graph. problems: a
    BatchProblems or a sequence of (X, Y, cx, cy[, out_order]); their device tensors must stay
    alive (kept here) for the plan's lifetime."""

    def __init__(self, problems, *, group_load_factor: float = 0.0, record_times: bool = False,
                 ctx: Context = None):
        self.ctx = ctx or default_context()
        self.problems = problems if isinstance(problems, BatchProblems) else BatchProblems(problems)
        o = stc_opts(STRATEGY_GROUPED, 1 if record_times else 0, 0.0, float(group_load_factor), ACC_HASH, 0, 0, 0)
        h = C.c_void_p()
        check(load().stc_batch_plan_create(C.c_void_p(self.ctx.handle), self.problems.n, self.problems.arr,
                                           C.byref(o), C.byref(h)))
        self.handle = h.value
        self.n = self.problems.n

    def run(self, stream=None):
        """One run: one Result per problem."""
        outs = (C.c_void_p * max(self.n, 1))()
        check(load().stc_batch_plan_run(C.c_void_p(self.handle), C.c_void_p(_stream_handle(stream)), outs))
        return [Result(outs[i]) for i in range(self.n)]

    def stats(self):
        """(runs, runs that replayed the captured graph, load factor of the graph or 0, largest
        warp table, expansion split)."""
        r, g, a, w, d = C.c_int64(), C.c_int64(), C.c_double(), C.c_int32(), C.c_int32()
        check(load().stc_batch_plan_stats(C.c_void_p(self.handle), C.byref(r), C.byref(g), C.byref(a), C.byref(w),
                                          C.byref(d)))
        return int(r.value), int(g.value), float(a.value), int(w.value), int(d.value)

    def close(self):
        if self.handle:
            check(load().stc_batch_plan_destroy(C.c_void_p(self.handle)))
            self.handle = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """The contraction server (stc_server_*). submit() takes (X, Y, cx, cy[, out_order]) with
    CUDA tensors (kept alive here until the request finishes) and returns a ticket;
    wait(ticket) returns (Result, (t_submit, t_start, t_done))."""

    def __init__(self, *, mem_budget_bytes: int = 0, max_batch: int = 0, workers: int = 0, plain: bool = False,
                 ctx: Context = None):
        self.ctx = ctx or default_context()
        o = stc_server_opts(int(mem_budget_bytes), int(max_batch), int(workers), 1 if plain else 0, 0)
        h = C.c_void_p()
        check(load().stc_server_create(C.c_void_p(self.ctx.handle), C.byref(o), C.byref(h)))
        self.handle = h.value
        self._inputs = {}

    def submit(self, X, Y, cx, cy, out_order=None) -> int:
        xa, ya = _CooArg(*X), _CooArg(*Y)
        acx, acy = _mode_array(cx), _mode_array(cy)
        oo = _mode_array(out_order) if out_order is not None else None
        req = stc_problem(xa.coo, ya.coo, len(cx), C.cast(acx, C.POINTER(C.c_int32)),
                          C.cast(acy, C.POINTER(C.c_int32)),
                          C.cast(oo, C.POINTER(C.c_int32)) if oo is not None else None)
        t = C.c_uint64()
        check(load().stc_server_submit(C.c_void_p(self.handle), C.byref(req), C.byref(t)))
        self._inputs[t.value] = (X, Y)
        return t.value

    def cancel(self, ticket: int) -> bool:
        """Take a still-queued request off the queue (its wait then raises STC_ERR_CANCELLED);
        False when a worker had already taken it."""
        c = C.c_int32()
        check(load().stc_server_cancel(C.c_void_p(self.handle), ticket, C.byref(c)))
        return bool(c.value)

    def poll(self, ticket: int) -> bool:
        d = C.c_int32()
        check(load().stc_server_poll(C.c_void_p(self.handle), ticket, C.byref(d)))
        return bool(d.value)

    def wait(self, ticket: int, timeout_ms: int = -1):
        r = C.c_void_p()
        times = (C.c_double * 3)()
        st = load().stc_server_wait(C.c_void_p(self.handle), ticket, int(timeout_ms), C.byref(r), times)
        if st != 6:  # a timeout leaves the ticket (and its inputs) in place
            self._inputs.pop(ticket, None)
        check(st)
        return Result(r.value), (times[0], times[1], times[2])

    def close(self):
        if self.handle:
            check(load().stc_server_destroy(C.c_void_p(self.handle)))
            self.handle = 0
            self._inputs.clear()


def measure_peaks(device: int = 0):
    """(FP64 multiplies per second, L2 FP64 atomic adds per second) measured on the device."""
    d, a = C.c_double(), C.c_double()
    check(load().stc_measure_peaks(int(device), C.byref(d), C.byref(a)))
    return float(d.value), float(a.value)


def count(X, Y, cx, cy, *, stream=None, ctx: Context = None):
    """(P, peak device bytes) of the contraction: the exact product count of Section 4.3."""
    ctx = ctx or default_context()
    return stc_count(ctx.handle, X, Y, cx, cy, stream)


def linearize(T, modes, *, stream=None, ctx: Context = None):
    """LN keys (Fig. 3) of the listed modes of each entry of T, as a CUDA int64 tensor
    holding the unsigned 64-bit keys."""
    import torch

    ctx = ctx or default_context()
    n = int(T[2].shape[0]) if T[2] is not None else 0
    out = torch.empty(n, dtype=torch.int64, device="cuda")
    stc_linearize(ctx.handle, T, modes, out, stream)
    return out


def dense_ids(keys, *, stream=None, ctx: Context = None):
    """Small numbers for large keys (Section 4.1.2): returns (ids int32 [n], D)."""
    import torch

    ctx = ctx or default_context()
    ids = torch.empty(int(keys.numel()), dtype=torch.int32, device="cuda")
    d = stc_dense_ids(ctx.handle, keys, ids, stream)
    return ids, d


def group_keys(keys, k: int, *, stream=None, ctx: Context = None):
    """Counting-sort grouping (Fig. 6) of keys in [0, k): returns (offsets[k+1], perm[n])."""
    import torch

    ctx = ctx or default_context()
    off = torch.empty(int(k) + 1, dtype=torch.int32, device="cuda")
    perm = torch.empty(int(keys.numel()), dtype=torch.int32, device="cuda")
    stc_group_keys(ctx.handle, keys, k, off, perm, stream)
    return off, perm
