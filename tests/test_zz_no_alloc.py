"""agg_reduce_noalloc: the allocation-free variant of agg_reduce.

Some callers cannot allocate device memory: an engine that keeps all of the
GPU's memory in its own pool leaves cudaMalloc nothing to hand out, and a
latency-critical path cannot afford the synchronisation an allocation may
cause. For them the library offers agg_reduce_noalloc, whose scratch is a
static device array inside the library. This test calls it through the C ABI
and checks it against the CPU oracle and against agg_reduce, twice in a row
(the static scratch keeps the previous call's contents, so the second call
shows that the state a call needs is cleared), and checks that a call makes
no device allocation. The file is named so that pytest collects it last.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
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


def _as_requested(ref, ops):
    """The oracle computes every function; keep those in ops (count is always set)."""
    out = {"count": ref["count"]}
    if ops & (agg.AGG_SUM | agg.AGG_AVG):
        out["sum"], out["avg"] = ref["sum"], ref["avg"]
    if ops & (agg.AGG_MIN | agg.AGG_MAX):
        out["min"], out["max"] = ref["min"], ref["max"]
    return out


def _same(got, ref, x):
    got = {k: got[k] for k in ref}
    assert got["count"] == ref["count"]
    if x.dtype.kind == "f":
        a = float(np.abs(x.astype(np.float64)).sum())
        if "sum" in ref:
            assert fp_close(got["sum"], ref["sum"], a)
            if ref["count"]:
                assert fp_close(got["avg"], ref["avg"], a / ref["count"])
        if "min" in ref:
            assert same_float(got["min"], ref["min"]) and same_float(got["max"], ref["max"])
    else:
        assert got == ref


@pytest.mark.parametrize("ops", [agg.AGG_ALL, agg.AGG_SUM, agg.AGG_MIN | agg.AGG_MAX])
def test_noalloc_matches_the_oracle_on_two_calls_in_a_row(L, ops):
    for x in _columns():
        t = torch.from_numpy(x).cuda()
        ref = _as_requested(oracle.reduce(x), ops)
        first = _call(L, L.agg_reduce_noalloc, t, ops)
        second = _call(L, L.agg_reduce_noalloc, t, ops)
        _same(first, ref, x)
        _same(second, ref, x)
        # and the same results as the allocating entry point
        _same(_call(L, L.agg_reduce, t, ops), ref, x)


def test_noalloc_makes_no_device_allocation(L):
    """On a fresh stream agg_reduce must allocate its scratch; with the next
    allocation set to fail, agg_reduce_noalloc still succeeds (twice), and the
    armed failure is still there for agg_reduce afterwards."""
    x = np.arange(-500_000, 700_001, dtype=np.int64).astype(np.int32)
    t = torch.from_numpy(x).cuda()
    ref = oracle.reduce(x)
    s = torch.cuda.Stream()
    torch.cuda.synchronize()
    agg.agg_stream_release(s)  # torch recycles stream handles: drop any scratch cached for this one
    try:
        L.agg_debug_fail_alloc(1)
        with torch.cuda.stream(s):
            for _ in range(2):
                got = _call(L, L.agg_reduce_noalloc, t, agg.AGG_ALL)
                assert got == ref
            out = torch.zeros(agg.SCALAR_BYTES, dtype=torch.uint8, device="cuda")
            st = L.agg_reduce(ctypes.c_void_p(t.data_ptr()), t.numel(), agg.AGG_I32, agg.AGG_ALL,
                              ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(s.cuda_stream))
            assert st == agg.AGG_ERR_OOM, agg.last_error()
    finally:
        L.agg_debug_fail_alloc(0)
    torch.cuda.synchronize()


def test_noalloc_rejects_bad_arguments(L):
    out = torch.zeros(agg.SCALAR_BYTES, dtype=torch.uint8, device="cuda")
    st = L.agg_reduce_noalloc(None, 10, agg.AGG_I32, agg.AGG_SUM, ctypes.c_void_p(out.data_ptr()), None)
    assert st == agg.AGG_ERR_INVALID
