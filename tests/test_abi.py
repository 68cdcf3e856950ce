"""The C-ABI library loads, exports every entry point declared in include/*.h,
and rejects bad arguments before touching the GPU (no GPU needed)."""
import ctypes
import glob
import os
import re

import pytest

import paper_2606_10030_gb300 as agg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        names += re.findall(r"^[A-Za-z_][\w \*]*?\b(agg_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def L():
    agg.build()
    return agg.lib()


def test_header_declares_entry_points():
    names = declared_functions()
    assert "agg_reduce" in names and "agg_reduce_host" in names and "agg_last_error" in names


def test_every_declared_symbol_is_exported(L):
    for name in declared_functions():
        assert hasattr(L, name), name
        assert name in agg.SIGNATURES, f"binding lacks {name}"


def test_version(L):
    assert L.agg_version() == 100


def test_reduce_rejects_bad_arguments_without_launching(L):
    p = ctypes.c_void_p(0x1000)
    out = ctypes.c_void_p(0x2000)
    assert L.agg_reduce(p, 10, 9, agg.AGG_SUM, out, None) == agg.AGG_ERR_INVALID
    assert "dtype" in agg.last_error()
    assert L.agg_reduce(p, 10, agg.AGG_I32, 0, out, None) == agg.AGG_ERR_INVALID
    assert L.agg_reduce(p, 10, agg.AGG_I32, 64, out, None) == agg.AGG_ERR_INVALID
    assert L.agg_reduce(p, -1, agg.AGG_I32, agg.AGG_SUM, out, None) == agg.AGG_ERR_INVALID
    assert L.agg_reduce(None, 10, agg.AGG_I32, agg.AGG_SUM, out, None) == agg.AGG_ERR_INVALID
    assert L.agg_reduce(p, 10, agg.AGG_I32, agg.AGG_SUM, None, None) == agg.AGG_ERR_INVALID
    assert L.agg_reduce(ctypes.c_void_p(0x1002), 10, agg.AGG_I32, agg.AGG_SUM, out, None) == agg.AGG_ERR_INVALID
    assert "aligned" in agg.last_error()
    assert L.agg_reduce_host(p, 10, agg.AGG_F64, 0, out, None) == agg.AGG_ERR_INVALID


def test_scalar_struct_layout():
    assert agg.SCALAR_BYTES == 80
