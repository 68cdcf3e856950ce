"""Python binding of libagg, the GB300 (sm_103a) in-memory aggregation library.

The binding only marshals arguments: every step of an aggregation runs in the
library's CUDA kernels behind the C ABI declared in ``include/agg.h``. PyTorch
provides device memory and streams. There is no CPU fallback: if the compiled
library is missing, loading it raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libagg.so")

AGG_I32, AGG_I64, AGG_U32, AGG_F32, AGG_F64 = range(5)
AGG_SUM, AGG_MIN, AGG_MAX, AGG_COUNT, AGG_AVG = 1, 2, 4, 8, 16
AGG_ALL = 31
AGG_FLAG_EXACT_SUM = 1  # options(flags=...): exactly rounded float sums, identical across strategies
AGG_FLAG_SUM_ERROR = 2  # options(flags=...): per-group |sum - exactly rounded sum| in Groups.to_host()["sum_err"]
AGG_OK, AGG_ERR_INVALID, AGG_ERR_OOM, AGG_ERR_CUDA, AGG_ERR_TABLE_FULL, AGG_ERR_TIMEOUT = 0, -1, -2, -3, -4, -5

DTYPE_NAMES = {AGG_I32: "i32", AGG_I64: "i64", AGG_U32: "u32", AGG_F32: "f32", AGG_F64: "f64"}
DTYPE_CODES = {v: k for k, v in DTYPE_NAMES.items()}
NP_DTYPES = {AGG_I32: np.int32, AGG_I64: np.int64, AGG_U32: np.uint32, AGG_F32: np.float32, AGG_F64: np.float64}


class AggError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"agg status {status}: {msg}")
        self.status = status


class AggScalar(ctypes.Structure):
    """Mirror of ``agg_scalar`` (80 bytes)."""
    _fields_ = [
        ("count", ctypes.c_int64),
        ("sum_i", ctypes.c_int64),
        ("sum_f", ctypes.c_double),
        ("avg", ctypes.c_double),
        ("min_i", ctypes.c_int64),
        ("max_i", ctypes.c_int64),
        ("min_f", ctypes.c_double),
        ("max_f", ctypes.c_double),
        ("dtype", ctypes.c_uint32),
        ("ops", ctypes.c_uint32),
        ("err_bound", ctypes.c_double),
    ]

    def as_dict(self) -> dict:
        fp = self.dtype in (AGG_F32, AGG_F64)
        return {
            "count": int(self.count),
            "sum": float(self.sum_f) if fp else int(self.sum_i),
            "min": float(self.min_f) if fp else int(self.min_i),
            "max": float(self.max_f) if fp else int(self.max_i),
            "avg": float(self.avg),
        }


SCALAR_BYTES = ctypes.sizeof(AggScalar)

AGG_STRAT_AUTO, AGG_STRAT_SMEM, AGG_STRAT_GLOBAL, AGG_STRAT_SORT, AGG_STRAT_LEARNED, AGG_STRAT_AUTOTUNE = range(6)
STRATEGY_NAMES = {AGG_STRAT_AUTO: "auto", AGG_STRAT_SMEM: "smem", AGG_STRAT_GLOBAL: "global",
                  AGG_STRAT_SORT: "sort", AGG_STRAT_LEARNED: "learned", AGG_STRAT_AUTOTUNE: "autotune"}
N_FEATURES = 16


class AggOptions(ctypes.Structure):
    """Mirror of ``agg_options``."""
    _fields_ = [
        ("strategy", ctypes.c_int32),
        ("block_threads", ctypes.c_int32),
        ("blocks_per_sm", ctypes.c_int32),
        ("smem_slots", ctypes.c_int32),
        ("table_slots", ctypes.c_int64),
        ("sample_offset", ctypes.c_uint64),
        ("items_per_thread", ctypes.c_int32),
        ("partition", ctypes.c_int32),
        ("flags", ctypes.c_int32),
        ("tile_rows", ctypes.c_int32),
    ]


AGG_TUNE_MAX = 8


class AggTuneResult(ctypes.Structure):
    """Mirror of ``agg_tune_result``."""
    _fields_ = [
        ("ncand", ctypes.c_int32),
        ("best", ctypes.c_int32),
        ("strategy", ctypes.c_int32 * AGG_TUNE_MAX),
        ("threads", ctypes.c_int32 * AGG_TUNE_MAX),
        ("smem_slots", ctypes.c_int32 * AGG_TUNE_MAX),
        ("items_per_thread", ctypes.c_int32 * AGG_TUNE_MAX),
        ("tile_rows", ctypes.c_int32 * AGG_TUNE_MAX),
        ("ms", ctypes.c_float * AGG_TUNE_MAX),
        ("best_ms_per_strategy", ctypes.c_float * 3),
        ("features", ctypes.c_float * 16),
    ]


class AggQuery(ctypes.Structure):
    """Mirror of ``agg_query``."""
    _fields_ = [
        ("keys", ctypes.c_void_p),
        ("vals", ctypes.c_void_p),
        ("n", ctypes.c_int64),
        ("dtype", ctypes.c_int32),
        ("ops", ctypes.c_uint32),
        ("strategy", ctypes.c_int32),
        ("reserved", ctypes.c_int32),
    ]


class AggGroups(ctypes.Structure):
    """Mirror of ``agg_groups``."""
    _fields_ = [
        ("num_groups", ctypes.c_int64),
        ("dtype", ctypes.c_int32),
        ("ops", ctypes.c_uint32),
        ("strategy", ctypes.c_int32),
        ("retries", ctypes.c_int32),
        ("table_slots", ctypes.c_int64),
        ("smem_slots", ctypes.c_int32),
        ("reserved", ctypes.c_int32),
        ("keys", ctypes.c_void_p),
        ("count", ctypes.c_void_p),
        ("sum", ctypes.c_void_p),
        ("min", ctypes.c_void_p),
        ("max", ctypes.c_void_p),
        ("avg", ctypes.c_void_p),
        ("sum_err", ctypes.c_void_p),
        ("features", ctypes.c_float * 16),
        ("priv", ctypes.c_void_p),
    ]

AGG_MAX_COLUMNS = 4


class AggColumn(ctypes.Structure):
    """Mirror of ``agg_column``."""
    _fields_ = [("data", ctypes.c_void_p), ("dtype", ctypes.c_int32), ("ops", ctypes.c_uint32)]


class AggRange(ctypes.Structure):
    """Mirror of ``agg_range``."""
    _fields_ = [("data", ctypes.c_void_p), ("dtype", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("lo_i", ctypes.c_int64), ("hi_i", ctypes.c_int64), ("lo_f", ctypes.c_double),
                ("hi_f", ctypes.c_double)]


class AggMulti(ctypes.Structure):
    """Mirror of ``agg_multi``."""
    _fields_ = [("num_groups", ctypes.c_int64), ("ncols", ctypes.c_int32), ("retries", ctypes.c_int32),
                ("table_slots", ctypes.c_int64), ("keys", ctypes.c_void_p), ("count", ctypes.c_void_p),
                ("sum", ctypes.c_void_p * AGG_MAX_COLUMNS), ("min", ctypes.c_void_p * AGG_MAX_COLUMNS),
                ("max", ctypes.c_void_p * AGG_MAX_COLUMNS), ("avg", ctypes.c_void_p * AGG_MAX_COLUMNS),
                ("priv", ctypes.c_void_p)]


AGG_PACK_FRAME = 1024


class AggPackedInfo(ctypes.Structure):
    """Mirror of ``agg_packed_info``."""
    _fields_ = [("n", ctypes.c_int64), ("dtype", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("nframes", ctypes.c_int64), ("nwords", ctypes.c_int64), ("bytes", ctypes.c_int64)]


_lib = None

# name -> (restype, argtypes) of every exported entry point
_vp, _i64, _i32, _u32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_uint32
SIGNATURES = {
    "agg_reduce": (_i32, [_vp, _i64, _i32, _u32, _vp, _vp]),
    "agg_reduce_host": (_i32, [_vp, _i64, _i32, _u32, _vp, _vp]),
    "agg_reduce_noalloc": (_i32, [_vp, _i64, _i32, _u32, _vp, _vp]),
    "agg_pack_for_bound": (ctypes.c_size_t, [_i64, _i32]),
    "agg_pack_for": (_i32, [_vp, _i64, _i32, _vp, ctypes.c_size_t, _vp]),
    "agg_reduce_packed": (_i32, [_vp, _vp, _u32, _vp, _vp]),
    "agg_reduce_packed_host": (_i32, [_vp, _vp, _u32, _vp, _vp]),
    "agg_groupby": (_i32, [_vp, _vp, _i64, _i32, _u32, _vp, _vp, _vp]),
    "agg_groupby_host": (_i32, [_vp, _vp, _i64, _i32, _u32, _vp, _vp, _vp]),
    "agg_groups_to_host": (_i32, [_vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "agg_groups_free": (None, [_vp]),
    "agg_sketch": (_i32, [_vp, _i64, _i32, _u32, ctypes.c_uint64, _vp, _vp]),
    "agg_groupby_multi": (_i32, [_vp, _vp, _i64, _vp, _i32, _vp, _vp, _vp]),
    "agg_distinct_estimate": (_i32, [_vp, _i64, _vp, _vp]),
    "agg_multi_to_host": (_i32, [_vp, _vp, _vp, _i32, _vp, _vp, _vp, _vp]),
    "agg_multi_free": (None, [_vp]),
    "agg_autotune": (_i32, [_vp, _vp, _i64, _i32, _u32, _i32, _vp, _vp]),
    "agg_autotune_cache_size": (ctypes.c_int64, []),
    "agg_autotune_clear": (None, []),
    "agg_autotune_save": (_i32, [ctypes.c_char_p]),
    "agg_autotune_load": (_i32, [ctypes.c_char_p]),
    "agg_mlp_param_count": (_i32, []),
    "agg_mlp_forward": (_i32, [_vp, _vp, _vp, _vp, _i32, _vp, _vp]),
    "agg_mlp_grad": (_i32, [_vp, _vp, _vp, _vp, _vp, _i32, _vp, _vp, _vp]),
    "agg_mlp_adam": (_i32, [_vp, _vp, _vp, _vp, _i64, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                            ctypes.c_float, _vp]),
    "agg_mlp_train": (_i32, [_vp, _vp, _vp, _vp, _vp, _vp, _vp, _i32, _i32, _i32, ctypes.c_float,
                             ctypes.c_uint64, _i64, _vp, _vp]),
    "agg_selector_set": (_i32, [_vp, _vp, _vp]),
    "agg_selector_clear": (None, []),
    "agg_selector_installed": (_i32, []),
    "agg_rule_strategy": (_i32, [_vp, _u32]),
    "agg_batch_plan_create": (_i32, [_vp, _i32, _vp, _vp]),
    "agg_batch_run": (_i32, [_vp, _vp]),
    "agg_batch_result": (_i32, [_vp, _i32, _vp]),
    "agg_batch_size": (_i32, [_vp]),
    "agg_batch_plan_free": (None, [_vp]),
    "agg_batch": (_i32, [_vp, _i32, _vp, _vp]),
    "agg_batch_tune": (_i32, [_vp, _i32, _vp, _vp]),
    "agg_launch_count": (ctypes.c_int64, []),
    "agg_stream_release": (_i32, [_vp]),
    "agg_debug_fail_alloc": (None, [_i64]),
    "agg_profile_enable": (None, [_i32]),
    "agg_profile_read": (_i32, [_vp, _vp]),
    "agg_energy_counter": (_i32, [_i32, _vp]),
    "agg_last_error": (ctypes.c_char_p, []),
    "agg_version": (_i32, []),
}


def build(force: bool = False) -> str:
    """Compile libagg.so for sm_103a (nvcc; cross-compiles without a GPU)."""
    return _build.build(force=force)


def lib():
    """Load libagg.so. Raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_2606_10030_gb300.build()")
        try:
            import torch  # noqa: F401  (load torch's CUDA runtime first so both share it)
        except Exception:
            pass
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def last_error() -> str:
    return lib().agg_last_error().decode()


def check(status: int) -> None:
    if status != AGG_OK:
        raise AggError(status, last_error())


def _stream_ptr(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def dtype_code(t) -> int:
    import torch
    m = {torch.int32: AGG_I32, torch.int64: AGG_I64, torch.uint32: AGG_U32,
         torch.float32: AGG_F32, torch.float64: AGG_F64}
    if t.dtype not in m:
        raise TypeError(f"unsupported column dtype {t.dtype}")
    return m[t.dtype]


def decode_scalar(buf) -> AggScalar:
    """Decode an agg_scalar from an 80-byte uint8 tensor or bytes."""
    if not isinstance(buf, (bytes, bytearray)):
        buf = bytes(buf.cpu().numpy().tobytes())
    return AggScalar.from_buffer_copy(buf[:SCALAR_BYTES])


# ---------------------------------------------------------------------------
# Entry points (same names as the C ABI)
# ---------------------------------------------------------------------------

def agg_reduce(col, ops: int = AGG_ALL, out=None, stream=None, n: int | None = None):
    """Ungrouped aggregation of a 1-D device tensor; returns the 80-byte device result.

    The result is written asynchronously on ``stream``; decode it with
    ``decode_scalar(out)`` (which synchronises by copying to the host).
    """
    import torch
    assert col.is_cuda and col.dim() == 1 and col.is_contiguous()
    if out is None:
        out = torch.empty(SCALAR_BYTES, dtype=torch.uint8, device=col.device)
    n = col.numel() if n is None else n
    check(lib().agg_reduce(ctypes.c_void_p(col.data_ptr()), n, dtype_code(col), ops,
                           ctypes.c_void_p(out.data_ptr()), _stream_ptr(stream)))
    return out


def agg_reduce_noalloc(col, ops: int = AGG_ALL, out=None, stream=None):
    """agg_reduce without device allocation (static scratch inside the library).

    For callers that cannot allocate device memory. Calls that overlap on the
    GPU share the static scratch and race; issue them on one stream.
    """
    import torch
    assert col.is_cuda and col.dim() == 1 and col.is_contiguous()
    if out is None:
        out = torch.empty(SCALAR_BYTES, dtype=torch.uint8, device=col.device)
    check(lib().agg_reduce_noalloc(ctypes.c_void_p(col.data_ptr()), col.numel(), dtype_code(col), ops,
                                   ctypes.c_void_p(out.data_ptr()), _stream_ptr(stream)))
    return out


class Packed:
    """A frame-of-reference bit-packed integer column in host memory (see agg_pack_for)."""

    def __init__(self, buf, info: AggPackedInfo):
        self.buf = buf
        self.info = info

    @property
    def nbytes(self) -> int:
        return int(self.info.bytes)

    def to(self, device):
        import torch
        return Packed(self.buf[: self.nbytes].to(device), self.info)


def agg_pack_for(col) -> Packed:
    """Encode a 1-D int32 / int64 / uint32 host tensor into a uint8 host tensor (pinned when a GPU is present)."""
    import torch
    assert not col.is_cuda and col.dim() == 1 and col.is_contiguous()
    dt = dtype_code(col)
    cap = int(lib().agg_pack_for_bound(col.numel(), dt))
    buf = torch.empty(cap + 16, dtype=torch.uint8)
    if torch.cuda.is_available():
        buf = buf.pin_memory()
    off = (-buf.data_ptr()) % 16
    view = buf[off: off + cap]
    info = AggPackedInfo()
    check(lib().agg_pack_for(ctypes.c_void_p(col.data_ptr()) if col.numel() else None, col.numel(), dt,
                             ctypes.c_void_p(view.data_ptr()), cap, ctypes.byref(info)))
    return Packed(view, info)


def agg_reduce_packed(p: Packed, ops: int = AGG_ALL, out=None, stream=None):
    """Ungrouped aggregation of a packed column held in device memory; returns the 80-byte device result."""
    import torch
    assert p.buf.is_cuda
    if out is None:
        out = torch.empty(SCALAR_BYTES, dtype=torch.uint8, device=p.buf.device)
    check(lib().agg_reduce_packed(ctypes.c_void_p(p.buf.data_ptr()), ctypes.byref(p.info), ops,
                                  ctypes.c_void_p(out.data_ptr()), _stream_ptr(stream)))
    return out


def agg_reduce_packed_host(p: Packed, ops: int = AGG_ALL, stream=None) -> AggScalar:
    """End-to-end aggregation of a packed column in (pinned) host memory; synchronous."""
    out = AggScalar()
    check(lib().agg_reduce_packed_host(ctypes.c_void_p(p.buf.data_ptr()), ctypes.byref(p.info), ops,
                                       ctypes.byref(out), _stream_ptr(stream)))
    return out


def agg_reduce_host(col, ops: int = AGG_ALL, stream=None) -> AggScalar:
    """End-to-end ungrouped aggregation of a (pinned) host tensor; synchronous."""
    assert not col.is_cuda and col.dim() == 1 and col.is_contiguous()
    out = AggScalar()
    check(lib().agg_reduce_host(ctypes.c_void_p(col.data_ptr()), col.numel(), dtype_code(col), ops,
                                ctypes.byref(out), _stream_ptr(stream)))
    return out


class Groups:
    """A GROUP BY result owned by the library; ``to_host()`` copies it to NumPy."""

    def __init__(self, ptr):
        self._ptr = ptr
        g = ctypes.cast(ptr, ctypes.POINTER(AggGroups)).contents
        self.num_groups = int(g.num_groups)
        self.dtype = int(g.dtype)
        self.ops = int(g.ops)
        self.strategy = int(g.strategy)
        self.retries = int(g.retries)
        self.table_slots = int(g.table_slots)
        self.smem_slots = int(g.smem_slots)
        self.has_sum_err = bool(g.sum_err)
        self.features = np.array(list(g.features), dtype=np.float32)

    def to_host(self) -> dict:
        d = self.num_groups
        fp = self.dtype in (AGG_F32, AGG_F64)
        keys = np.empty(d, np.uint32)
        count = np.empty(d, np.int64)
        s = np.empty(d, np.float64 if fp else np.int64)
        mn = np.empty(d, np.float64 if fp else np.int64)
        mx = np.empty(d, np.float64 if fp else np.int64)
        avg = np.empty(d, np.float64)
        err = np.empty(d, np.float64) if self.has_sum_err else None
        p = lambda a: a.ctypes.data_as(ctypes.c_void_p) if a is not None else None  # noqa: E731
        check(lib().agg_groups_to_host(self._ptr, p(keys), p(count), p(s), p(mn), p(mx), p(avg), p(err)))
        out = {"keys": keys, "count": count, "sum": s, "min": mn, "max": mx, "avg": avg}
        if err is not None:
            out["sum_err"] = err
        return out

    def free(self):
        if self._ptr:
            lib().agg_groups_free(self._ptr)
            self._ptr = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def options(strategy: int = AGG_STRAT_AUTO, **kw) -> AggOptions:
    o = AggOptions()
    o.strategy = strategy
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def agg_groupby(keys, vals, ops: int = AGG_ALL, opts: AggOptions | None = None, stream=None,
                n: int | None = None) -> Groups:
    """GROUP BY keys (uint32 device tensor) over vals (device tensor); synchronous."""
    assert keys.is_cuda and vals.is_cuda and keys.dim() == 1 and vals.dim() == 1
    assert keys.is_contiguous() and vals.is_contiguous()
    n = keys.numel() if n is None else n
    out = ctypes.c_void_p()
    check(lib().agg_groupby(ctypes.c_void_p(keys.data_ptr()), ctypes.c_void_p(vals.data_ptr()), n,
                            dtype_code(vals), ops, ctypes.byref(opts) if opts is not None else None,
                            ctypes.byref(out), _stream_ptr(stream)))
    return Groups(out.value)


def agg_groupby_host(keys, vals, ops: int = AGG_ALL, opts: AggOptions | None = None, stream=None) -> Groups:
    """End-to-end GROUP BY of (pinned) host tensors; synchronous."""
    assert not keys.is_cuda and not vals.is_cuda and keys.is_contiguous() and vals.is_contiguous()
    out = ctypes.c_void_p()
    check(lib().agg_groupby_host(ctypes.c_void_p(keys.data_ptr()), ctypes.c_void_p(vals.data_ptr()),
                                 keys.numel(), dtype_code(vals), ops,
                                 ctypes.byref(opts) if opts is not None else None, ctypes.byref(out),
                                 _stream_ptr(stream)))
    return Groups(out.value)


class Multi:
    """A multi-column GROUP BY result owned by the library; ``to_host()`` copies it to NumPy."""

    def __init__(self, ptr, dtypes):
        self._ptr = ptr
        m = ctypes.cast(ptr, ctypes.POINTER(AggMulti)).contents
        self.num_groups = int(m.num_groups)
        self.ncols = int(m.ncols)
        self.retries = int(m.retries)
        self.table_slots = int(m.table_slots)
        self.dtypes = dtypes

    def to_host(self) -> dict:
        d = self.num_groups
        keys = np.empty(d, np.uint64)
        count = np.empty(d, np.int64)
        p = lambda a: a.ctypes.data_as(ctypes.c_void_p)  # noqa: E731
        out = {"keys": keys, "count": count, "cols": []}
        for c in range(self.ncols):
            fp = self.dtypes[c] in (AGG_F32, AGG_F64)
            s = np.empty(d, np.float64 if fp else np.int64)
            mn = np.empty(d, np.float64 if fp else np.int64)
            mx = np.empty(d, np.float64 if fp else np.int64)
            avg = np.empty(d, np.float64)
            check(lib().agg_multi_to_host(self._ptr, p(keys) if c == 0 else None, p(count) if c == 0 else None, c,
                                          p(s), p(mn), p(mx), p(avg)))
            out["cols"].append({"sum": s, "min": mn, "max": mx, "avg": avg})
        return out

    def free(self):
        if self._ptr:
            lib().agg_multi_free(self._ptr)
            self._ptr = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def agg_groupby_multi(key_lo, key_hi, cols, filt=None, stream=None) -> Multi:
    """GROUP BY the 64-bit key (key_hi << 32) | key_lo over device tensors.

    cols: list of (values, ops); filt: None or (column, lo, hi), both bounds inclusive.
    """
    n = key_lo.numel()
    arr = (AggColumn * len(cols))()
    keep = [key_lo, key_hi]
    for i, (v, ops) in enumerate(cols):
        assert v.is_cuda and v.numel() == n and v.is_contiguous()
        arr[i].data = v.data_ptr() if n else None
        arr[i].dtype = dtype_code(v)
        arr[i].ops = ops
        keep.append(v)
    rng = None
    if filt is not None:
        f, lo, hi = filt
        assert f.is_cuda and f.numel() == n and f.is_contiguous()
        rng = AggRange()
        rng.data = f.data_ptr() if n else None
        rng.dtype = dtype_code(f)
        if rng.dtype in (AGG_F32, AGG_F64):
            rng.lo_f, rng.hi_f = float(lo), float(hi)
        else:
            rng.lo_i, rng.hi_i = int(lo), int(hi)
    out = ctypes.c_void_p()
    check(lib().agg_groupby_multi(ctypes.c_void_p(key_lo.data_ptr()) if n else None,
                                  ctypes.c_void_p(key_hi.data_ptr()) if key_hi is not None and n else None, n, arr,
                                  len(cols), ctypes.byref(rng) if rng is not None else None, ctypes.byref(out),
                                  _stream_ptr(stream)))
    return Multi(out.value, [dtype_code(v) for v, _ in cols])


def agg_distinct_estimate(keys, stream=None) -> float:
    """HyperLogLog estimate of the distinct keys of a uint32 device tensor (synchronous)."""
    est = ctypes.c_double(0.0)
    check(lib().agg_distinct_estimate(ctypes.c_void_p(keys.data_ptr()) if keys.numel() else None, keys.numel(),
                                      ctypes.byref(est), _stream_ptr(stream)))
    return float(est.value)


def agg_sketch(keys, vdtype: int, ops: int = AGG_ALL, sample_offset: int = 0, out=None, stream=None):
    """The 16 sketch features of a device key column (float32 device tensor)."""
    import torch
    if out is None:
        out = torch.empty(N_FEATURES, dtype=torch.float32, device=keys.device)
    check(lib().agg_sketch(ctypes.c_void_p(keys.data_ptr()), keys.numel(), vdtype, ops, sample_offset,
                           ctypes.c_void_p(out.data_ptr()), _stream_ptr(stream)))
    return out


PHASES = ["scan", "sketch", "build", "finalize", "sort", "segreduce", "batch", "mlp"]


def agg_stream_release(stream) -> None:
    """Free the library's cached scratch of a stream (call before the stream is destroyed)."""
    check(lib().agg_stream_release(_stream_ptr(stream)))


def agg_energy_counter(device: int = 0) -> int:
    """NVML's energy counter of a CUDA device in millijoules (read-only)."""
    mj = ctypes.c_uint64(0)
    check(lib().agg_energy_counter(device, ctypes.byref(mj)))
    return int(mj.value)


def launch_count() -> int:
    """Kernels launched by the library so far in this process."""
    return int(lib().agg_launch_count())


def profile_enable(on: bool = True) -> None:
    lib().agg_profile_enable(1 if on else 0)


def profile_read() -> dict:
    """Accumulated per-phase event time (ms) and call counts since the last read."""
    ms = (ctypes.c_double * len(PHASES))()
    calls = (ctypes.c_int64 * len(PHASES))()
    check(lib().agg_profile_read(ms, calls))
    return {p: (float(ms[i]), int(calls[i])) for i, p in enumerate(PHASES)}


def agg_autotune(keys, vals, ops: int = AGG_ALL, reps: int = 1, stream=None) -> AggTuneResult:
    """Time every GROUP BY candidate on the query; returns the timings (and fills the cache)."""
    r = AggTuneResult()
    check(lib().agg_autotune(ctypes.c_void_p(keys.data_ptr()), ctypes.c_void_p(vals.data_ptr()), keys.numel(),
                             dtype_code(vals), ops, reps, ctypes.byref(r), _stream_ptr(stream)))
    return r


def _p(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def agg_mlp_forward(params, x, mean=None, std=None, out=None, stream=None):
    import torch
    n = x.shape[0]
    out = torch.empty((n, 3), dtype=torch.float32, device=x.device) if out is None else out
    check(lib().agg_mlp_forward(_p(params), _p(mean), _p(std), _p(x), n, _p(out), _stream_ptr(stream)))
    return out


def agg_mlp_grad(params, x, y, mean=None, std=None, stream=None):
    import torch
    g = torch.empty(lib().agg_mlp_param_count(), dtype=torch.float32, device=x.device)
    loss = torch.empty(1, dtype=torch.float32, device=x.device)
    check(lib().agg_mlp_grad(_p(params), _p(mean), _p(std), _p(x), _p(y), x.shape[0], _p(g), _p(loss),
                             _stream_ptr(stream)))
    return g, loss


def agg_mlp_adam(params, grads, m, v, t: int, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
    check(lib().agg_mlp_adam(_p(params), _p(grads), _p(m), _p(v), t, lr, beta1, beta2, eps, _stream_ptr(stream)))


def agg_mlp_train(params, m, v, x, y, mean=None, std=None, epochs=30, batch=256, lr=1e-3, seed=0, t0=0,
                  stream=None):
    """Train in place on the device; returns the per-epoch mean loss."""
    losses = np.zeros(max(1, epochs), dtype=np.float32)
    check(lib().agg_mlp_train(_p(params), _p(m), _p(v), _p(mean), _p(std), _p(x), _p(y), x.shape[0], epochs, batch,
                              lr, seed, t0, losses.ctypes.data_as(ctypes.c_void_p), _stream_ptr(stream)))
    return losses[:epochs]


def agg_selector_set(params: np.ndarray, mean: np.ndarray, std: np.ndarray) -> None:
    params = np.ascontiguousarray(params, dtype=np.float32)
    mean = np.ascontiguousarray(mean, dtype=np.float32)
    std = np.ascontiguousarray(std, dtype=np.float32)
    check(lib().agg_selector_set(params.ctypes.data_as(ctypes.c_void_p), mean.ctypes.data_as(ctypes.c_void_p),
                                 std.ctypes.data_as(ctypes.c_void_p)))


def agg_rule_strategy(features, ops: int) -> int:
    f = np.ascontiguousarray(features, dtype=np.float32)
    return int(lib().agg_rule_strategy(f.ctypes.data_as(ctypes.c_void_p), ops))


class BatchPlan:
    """A planned batch of GROUP BY queries over device tensors (see agg_batch_plan_create)."""

    def __init__(self, queries, stream=None):
        """queries: list of (keys, vals, ops, strategy) with device tensors."""
        self._keep = [(k, v) for k, v, _, _ in queries]
        arr = (AggQuery * max(1, len(queries)))()
        for i, (k, v, ops, strat) in enumerate(queries):
            arr[i].keys = k.data_ptr() if k.numel() else None
            arr[i].vals = v.data_ptr() if v.numel() else None
            arr[i].n = k.numel()
            arr[i].dtype = dtype_code(v)
            arr[i].ops = ops
            arr[i].strategy = strat
        self._arr = arr
        self.nq = len(queries)
        h = ctypes.c_void_p()
        check(lib().agg_batch_plan_create(arr, self.nq, ctypes.byref(h), _stream_ptr(stream)))
        self._h = h

    def run(self, stream=None):
        check(lib().agg_batch_run(self._h, _stream_ptr(stream)))

    def tune(self, reps: int = 2, stream=None) -> int:
        """Pick the fastest work-item size (16, 32 or 64 Ki rows) by timing runs; returns it."""
        t = ctypes.c_int32(0)
        check(lib().agg_batch_tune(self._h, reps, ctypes.byref(t), _stream_ptr(stream)))
        return int(t.value)

    def result(self, i) -> Groups:
        out = ctypes.c_void_p()
        check(lib().agg_batch_result(self._h, i, ctypes.byref(out)))
        return Groups(out.value)

    def free(self):
        if self._h:
            lib().agg_batch_plan_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass
