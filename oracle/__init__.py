"""CPU oracle for in-memory aggregation (test infrastructure only).

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` import this package. The library under test never does, and the
two share no code: the oracle is a plain single-threaded C++ fold
(``oracle.cpp``) plus NumPy float64 restatements of the key sketch and of the
selector network (``sketch.py``, ``mlp.py``).

``build()`` compiles ``oracle.cpp`` with g++ into ``liboracle.so`` beside it.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

DT = {"i32": 0, "i64": 1, "u32": 2, "f32": 3, "f64": 4}
NP_DT = {"i32": np.int32, "i64": np.int64, "u32": np.uint32, "f32": np.float32, "f64": np.float64}


class OracleScalar(ctypes.Structure):
    _fields_ = [
        ("count", ctypes.c_int64),
        ("sum_i", ctypes.c_int64),
        ("sum_f", ctypes.c_double),
        ("avg", ctypes.c_double),
        ("min_i", ctypes.c_int64),
        ("max_i", ctypes.c_int64),
        ("min_f", ctypes.c_double),
        ("max_f", ctypes.c_double),
    ]


SCALAR_DTYPE = np.dtype([
    ("count", np.int64), ("sum_i", np.int64), ("sum_f", np.float64), ("avg", np.float64),
    ("min_i", np.int64), ("max_i", np.int64), ("min_f", np.float64), ("max_f", np.float64),
])


def build(force: bool = False) -> str:
    """Compile the oracle (plain -O2, no vectorisation flags beyond the default)."""
    with _lock:
        if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
            tmp = _LIB + f".tmp{os.getpid()}"
            subprocess.check_call(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-o", tmp, _SRC])
            os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        vp, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
        L.oracle_exact_sum_f64.argtypes = [vp, i64]
        L.oracle_exact_sum_f64.restype = ctypes.c_double
        L.oracle_exact_sum_f32.argtypes = [vp, i64]
        L.oracle_exact_sum_f32.restype = ctypes.c_double
        L.oracle_reduce.argtypes = [vp, i64, i32, ctypes.POINTER(OracleScalar)]
        L.oracle_reduce.restype = i32
        L.oracle_groupby.argtypes = [vp, vp, i64, i32, ctypes.POINTER(i64)]
        L.oracle_groupby.restype = vp
        L.oracle_groupby_selected.argtypes = [vp, vp, i64, i32, vp, i64, ctypes.POINTER(i64)]
        L.oracle_groupby_selected.restype = vp
        L.oracle_groups_fetch.argtypes = [vp, vp, vp]
        L.oracle_groups_fetch.restype = None
        L.oracle_groups_free.argtypes = [vp]
        L.oracle_groups_free.restype = None
        L.oracle_groupby_multi.argtypes = [vp, vp, i64, vp, vp, i32, vp, i32, i64, i64, ctypes.c_double,
                                           ctypes.c_double, ctypes.POINTER(i64)]
        L.oracle_groupby_multi.restype = vp
        L.oracle_multi_fetch.argtypes = [vp, vp, vp]
        L.oracle_multi_fetch.restype = None
        L.oracle_multi_free.argtypes = [vp]
        L.oracle_multi_free.restype = None
        _lib = L
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def exact_sum(x: np.ndarray) -> float:
    """Exact sum of a float32/float64 array, rounded once to float64."""
    x = np.ascontiguousarray(x)
    if x.dtype == np.float32:
        return lib().oracle_exact_sum_f32(_ptr(x), x.size)
    if x.dtype == np.float64:
        return lib().oracle_exact_sum_f64(_ptr(x), x.size)
    raise TypeError(x.dtype)


def dtype_name(a: np.ndarray) -> str:
    for k, v in NP_DT.items():
        if a.dtype == v:
            return k
    raise TypeError(a.dtype)


def reduce(col: np.ndarray) -> dict:
    """Ungrouped SUM/MIN/MAX/COUNT/AVG of a column (all computed)."""
    col = np.ascontiguousarray(col)
    dt = dtype_name(col)
    out = OracleScalar()
    rc = lib().oracle_reduce(_ptr(col), col.size, DT[dt], ctypes.byref(out))
    if rc != 0:
        raise ValueError("oracle_reduce rejected its arguments")
    return _scalar_dict(out, dt)


def _scalar_dict(o: OracleScalar, dt: str) -> dict:
    fp = dt in ("f32", "f64")
    return {
        "count": int(o.count),
        "sum": float(o.sum_f) if fp else int(o.sum_i),
        "min": float(o.min_f) if fp else int(o.min_i),
        "max": float(o.max_f) if fp else int(o.max_i),
        "avg": float(o.avg),
    }


class Groups:
    """GROUP BY result in ascending key order, as NumPy arrays."""

    def __init__(self, keys, rows, dt):
        fp = dt in ("f32", "f64")
        self.dtype = dt
        self.keys = keys
        self.count = rows["count"].copy()
        self.sum = rows["sum_f"].copy() if fp else rows["sum_i"].copy()
        self.min = rows["min_f"].copy() if fp else rows["min_i"].copy()
        self.max = rows["max_f"].copy() if fp else rows["max_i"].copy()
        self.avg = rows["avg"].copy()

    def __len__(self):
        return len(self.keys)


def _fetch(h, d: int, dt: str) -> Groups:
    keys = np.empty(d, dtype=np.uint32)
    rows = np.empty(d, dtype=SCALAR_DTYPE)
    lib().oracle_groups_fetch(h, _ptr(keys), _ptr(rows))
    lib().oracle_groups_free(h)
    return Groups(keys, rows, dt)


def groupby(keys: np.ndarray, vals: np.ndarray) -> Groups:
    """GROUP BY keys: SUM/MIN/MAX/COUNT/AVG of vals per distinct key."""
    keys = np.ascontiguousarray(keys, dtype=np.uint32)
    vals = np.ascontiguousarray(vals)
    assert keys.size == vals.size
    dt = dtype_name(vals)
    d = ctypes.c_int64(0)
    h = lib().oracle_groupby(_ptr(keys), _ptr(vals), keys.size, DT[dt], ctypes.byref(d))
    if not h:
        raise ValueError("oracle_groupby rejected its arguments")
    return _fetch(h, d.value, dt)


def groupby_selected(keys: np.ndarray, vals: np.ndarray, sel: np.ndarray) -> Groups:
    """GROUP BY restricted to the distinct keys in sel (ascending key order)."""
    keys = np.ascontiguousarray(keys, dtype=np.uint32)
    vals = np.ascontiguousarray(vals)
    sel = np.ascontiguousarray(np.unique(sel), dtype=np.uint32)
    dt = dtype_name(vals)
    d = ctypes.c_int64(0)
    h = lib().oracle_groupby_selected(_ptr(keys), _ptr(vals), keys.size, DT[dt], _ptr(sel), sel.size,
                                      ctypes.byref(d))
    if not h:
        raise ValueError("oracle_groupby_selected rejected its arguments")
    return _fetch(h, d.value, dt)


def groupby_multi(key_lo: np.ndarray, key_hi: np.ndarray | None, cols: list, filt=None) -> dict:
    """GROUP BY the 64-bit key (key_hi << 32) | key_lo over several value columns,
    counting only rows with lo <= f <= hi when filt = (f, lo, hi) is given.

    Returns {"keys": uint64[d] ascending, "count": int64[d], "cols": [{"sum", "min",
    "max", "avg"} per value column]}.
    """
    key_lo = np.ascontiguousarray(key_lo, dtype=np.uint32)
    n = key_lo.size
    if key_hi is not None:
        key_hi = np.ascontiguousarray(key_hi, dtype=np.uint32)
        assert key_hi.size == n
    cols = [np.ascontiguousarray(c) for c in cols]
    assert all(c.size == n for c in cols)
    dts = np.array([DT[dtype_name(c)] for c in cols], dtype=np.int32)
    ptrs = (ctypes.c_void_p * len(cols))(*[c.ctypes.data for c in cols])
    fp, fdt, lo_i, hi_i, lo_f, hi_f = None, 0, 0, 0, 0.0, 0.0
    if filt is not None:
        f, lo, hi = filt
        f = np.ascontiguousarray(f)
        assert f.size == n
        fdt = DT[dtype_name(f)]
        if f.dtype.kind == "f":
            lo_f, hi_f = float(lo), float(hi)
        else:
            lo_i, hi_i = int(lo), int(hi)
        fp = f
    d = ctypes.c_int64(0)
    h = lib().oracle_groupby_multi(_ptr(key_lo), _ptr(key_hi) if key_hi is not None else None, n, ptrs,
                                   _ptr(dts), len(cols), _ptr(fp) if fp is not None else None, fdt, lo_i, hi_i,
                                   lo_f, hi_f, ctypes.byref(d))
    if not h:
        raise ValueError("oracle_groupby_multi rejected its arguments")
    keys = np.empty(d.value, dtype=np.uint64)
    rows = np.empty(d.value * len(cols), dtype=SCALAR_DTYPE)
    lib().oracle_multi_fetch(h, _ptr(keys), _ptr(rows))
    lib().oracle_multi_free(h)
    rows = rows.reshape(d.value, len(cols)) if len(cols) else rows
    out = {"keys": keys, "count": rows[:, 0]["count"].copy() if d.value else np.zeros(0, np.int64), "cols": []}
    for c, col in enumerate(cols):
        fpc = col.dtype.kind == "f"
        r = rows[:, c]
        out["cols"].append({"sum": (r["sum_f"] if fpc else r["sum_i"]).copy(),
                            "min": (r["min_f"] if fpc else r["min_i"]).copy(),
                            "max": (r["max_f"] if fpc else r["max_i"]).copy(), "avg": r["avg"].copy()})
    return out
