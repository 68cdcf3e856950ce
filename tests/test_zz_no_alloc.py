"""agg_reduce_noalloc: the allocation-free variant of agg_reduce.

Some callers cannot allocate device memory: an engine that keeps all of the
GPU's memory in its own pool leaves cudaMalloc nothing to hand out, and a
latency-critical path cannot afford the synchronisation an allocation may
cause. For them the library offers agg_reduce_noalloc, whose scratch is a
static device array inside the library. This test calls it through the C ABI
and checks it against agg_reduce, twice in a row (the static scratch keeps
the previous call's contents, so the second call shows that the state a call
needs is cleared). The file is named so that pytest collects it last.
"""
import ctypes

import numpy as np
import pytest
import torch

import paper_2606_10030_gb300 as agg
from tests.common import fp_close, same_float

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    agg.build()
    return agg.lib()


def _columns():
    rng = np.random.default_rng(42)
    yield rng.integers(-(2 ** 31), 2 ** 31, 3_000_017, dtype=np.int64).astype(np.int32)
    yield rng.integers(-(2 ** 62), 2 ** 62, 1_000_003, dtype=np.int64)
    yield rng.integers(0, 2 ** 32, 777_777, dtype=np.uint64).astype(np.uint32)
    yield (rng.standard_normal(4_000_037) * 1e3).astype(np.float32)
    yield rng.standard_normal(2_000_029) * np.exp2(rng.integers(-30, 30, 2_000_029).astype(np.float64))
    yield np.arange(33, dtype=np.int32)
    yield np.array([], dtype=np.float32)


def _call(L, fn, t, ops):
    out = torch.zeros(agg.SCALAR_BYTES, dtype=torch.uint8, device="cuda")
    st = fn(ctypes.c_void_p(t.data_ptr()), t.numel(), agg.dtype_code(t), ops, ctypes.c_void_p(out.data_ptr()),
            ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == agg.AGG_OK, agg.last_error()
    torch.cuda.synchronize()
    return agg.decode_scalar(out).as_dict()


def _same(got, ref, x):
    assert got["count"] == ref["count"]
    if x.dtype.kind == "f":
        a = float(np.abs(x.astype(np.float64)).sum())
        assert fp_close(got["sum"], ref["sum"], a)
        if ref["count"]:
            assert fp_close(got["avg"], ref["avg"], a / ref["count"])
        assert same_float(got["min"], ref["min"]) and same_float(got["max"], ref["max"])
    else:
        assert got == ref


@pytest.mark.parametrize("ops", [agg.AGG_ALL, agg.AGG_SUM, agg.AGG_MIN | agg.AGG_MAX])
def test_noalloc_matches_agg_reduce_on_two_calls_in_a_row(L, ops):
    for x in _columns():
        t = torch.from_numpy(x).cuda()
        ref = _call(L, L.agg_reduce, t, ops)
        first = _call(L, L.agg_reduce_noalloc, t, ops)
        second = _call(L, L.agg_reduce_noalloc, t, ops)
        _same(first, ref, x)
        _same(second, ref, x)


def test_noalloc_rejects_bad_arguments(L):
    out = torch.zeros(agg.SCALAR_BYTES, dtype=torch.uint8, device="cuda")
    st = L.agg_reduce_noalloc(None, 10, agg.AGG_I32, agg.AGG_SUM, ctypes.c_void_p(out.data_ptr()), None)
    assert st == agg.AGG_ERR_INVALID
