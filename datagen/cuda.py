"""GPU generation of the seeded input columns (same draws as datagen/__init__.py).

Columns of hundreds of millions of rows are generated directly in device
memory by ``libdatagen.so`` (built from ``datagen.cu`` by ``build()``).
"""
from __future__ import annotations

import ctypes
import os
import shutil
import subprocess

import numpy as np

from . import DTYPE_CODE, zipf_thresholds

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "datagen.cu")
_LIB = os.path.join(_HERE, "libdatagen.so")
_lib = None


def build(force: bool = False) -> str:
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
        libdir = os.path.join(os.path.dirname(os.path.dirname(os.path.realpath(nvcc))), "lib64")
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17",
                               "-Xcompiler", "-fPIC", "-shared", "-cudart", "shared", "-o", tmp, _SRC,
                               "-Xlinker", f"-rpath,{libdir}", "-L", libdir])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(_LIB):
            build()
        import torch  # noqa: F401
        L = ctypes.CDLL(_LIB)
        vp, i64, u64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_uint64, ctypes.c_int
        L.dg_keys_uniform.argtypes = [vp, i64, u64, u64, i64, vp]
        L.dg_keys_zipf.argtypes = [vp, i64, u64, vp, i64, i64, vp]
        L.dg_values.argtypes = [vp, i32, i64, u64, i64, vp]
        for f in (L.dg_keys_uniform, L.dg_keys_zipf, L.dg_values):
            f.restype = i32
        _lib = L
    return _lib


def _s():
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ok(rc):
    if rc != 0:
        raise RuntimeError(f"datagen kernel launch failed with CUDA error {rc}")


_TORCH_DT = {}


def torch_dtype(name):
    import torch
    return {"i32": torch.int32, "i64": torch.int64, "u32": torch.uint32,
            "f32": torch.float32, "f64": torch.float64}[name]


def values(dtype: str, n: int, seed: int, start: int = 0, out=None):
    import torch
    out = torch.empty(n, dtype=torch_dtype(dtype), device="cuda") if out is None else out
    _ok(lib().dg_values(ctypes.c_void_p(out.data_ptr()), DTYPE_CODE[dtype], n, seed, start, _s()))
    return out


def keys_uniform(n: int, D: int, seed: int, start: int = 0, out=None):
    import torch
    out = torch.empty(n, dtype=torch.uint32, device="cuda") if out is None else out
    _ok(lib().dg_keys_uniform(ctypes.c_void_p(out.data_ptr()), n, seed, D, start, _s()))
    return out


def keys_zipf(n: int, D: int, s: float, seed: int, start: int = 0, out=None, thresholds=None):
    import torch
    t = zipf_thresholds(D, s) if thresholds is None else thresholds
    td = torch.from_numpy(t.view(np.int64)).to("cuda")
    out = torch.empty(n, dtype=torch.uint32, device="cuda") if out is None else out
    _ok(lib().dg_keys_zipf(ctypes.c_void_p(out.data_ptr()), n, seed, ctypes.c_void_p(td.data_ptr()), D, start,
                           _s()))
    torch.cuda.current_stream().synchronize()
    del td
    return out


def group_column(q, out_keys=None, out_vals=None):
    """Keys and values of a datagen.GroupQuery, generated on the GPU."""
    if q.zipf_s > 0:
        k = keys_zipf(q.n, q.D, q.zipf_s, q.seed, out=out_keys)
    else:
        k = keys_uniform(q.n, q.D, q.seed, out=out_keys)
    v = values(q.dtype, q.n, q.seed, out=out_vals)
    return k, v
