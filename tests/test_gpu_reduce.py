"""Parity of the ungrouped scan (agg_reduce, agg_reduce_host) with the CPU oracle.

Integer SUM/MIN/MAX/COUNT/AVG and float MIN/MAX/COUNT must be bit-identical;
float SUM/AVG within the 1e-6 bar of tests/common.py.
"""
import math

import numpy as np
import pytest
import torch

import datagen as dg
import oracle
import paper_2606_10030_gb300 as agg
from tests.common import fp_close, same_float

pytestmark = pytest.mark.gpu

DTS = [np.int32, np.int64, np.uint32, np.float32, np.float64]
SIZES = [0, 1, 3, 31, 32, 33, 255, 1000, 4097, 65537, (1 << 20) + 7, 3_000_001]


@pytest.fixture(scope="module", autouse=True)
def _build():
    agg.build()
    agg.lib()


def make(dt, n, seed=0, kind="normal"):
    rng = np.random.default_rng(seed)
    if np.dtype(dt).kind == "f":
        if kind == "wide":
            x = rng.standard_normal(n) * np.exp2(rng.integers(-40, 40, n).astype(np.float64))
        else:
            x = rng.standard_normal(n) * 1e3
        return x.astype(dt)
    info = np.iinfo(dt)
    return rng.integers(info.min, info.max, n, dtype=np.int64 if dt != np.uint32 else np.uint64,
                        endpoint=True).astype(dt)


def check(got: dict, x: np.ndarray, ops=agg.AGG_ALL):
    ref = oracle.reduce(x)
    assert got["count"] == ref["count"]
    fp = x.dtype.kind == "f"
    if fp:
        a = float(np.abs(x.astype(np.float64)).sum())
        if ops & (agg.AGG_SUM | agg.AGG_AVG):
            assert fp_close(got["sum"], ref["sum"], a), (got["sum"], ref["sum"])
            if ref["count"]:
                assert fp_close(got["avg"], ref["avg"], a / ref["count"]), (got["avg"], ref["avg"])
            else:
                assert math.isnan(got["avg"])
        if ops & (agg.AGG_MIN | agg.AGG_MAX):
            assert same_float(got["min"], ref["min"]) and same_float(got["max"], ref["max"])
    else:
        if ops & (agg.AGG_SUM | agg.AGG_AVG):
            assert got["sum"] == ref["sum"]
            assert same_float(got["avg"], ref["avg"])
        if ops & (agg.AGG_MIN | agg.AGG_MAX):
            assert got["min"] == ref["min"] and got["max"] == ref["max"]


def run_dev(x: np.ndarray, ops=agg.AGG_ALL):
    t = torch.from_numpy(x).cuda()
    return agg.decode_scalar(agg.agg_reduce(t, ops)).as_dict()


@pytest.mark.parametrize("dt", DTS)
@pytest.mark.parametrize("n", SIZES)
def test_reduce_parity(dt, n):
    x = make(dt, n, seed=n)
    check(run_dev(x), x)


@pytest.mark.parametrize("dt", DTS)
def test_reduce_op_subsets(dt):
    x = make(dt, 123457, seed=5)
    for ops in [agg.AGG_SUM, agg.AGG_MIN, agg.AGG_MAX, agg.AGG_COUNT, agg.AGG_AVG,
                agg.AGG_MIN | agg.AGG_MAX, agg.AGG_SUM | agg.AGG_COUNT, agg.AGG_ALL]:
        got = run_dev(x, ops)
        check(got, x, ops)


@pytest.mark.parametrize("dt", DTS)
@pytest.mark.parametrize("off", [1, 2, 3])
def test_reduce_unaligned_start(dt, off):
    x = make(dt, 100000, seed=off)
    t = torch.from_numpy(x).cuda()
    sub = t[off:]
    got = agg.decode_scalar(agg.agg_reduce(sub, agg.AGG_ALL)).as_dict()
    check(got, x[off:])


def test_config_2p20_int32_uniform_bit_exact():
    """2^20-row int32 column, uniform in [-2^20, 2^20), seed 0: all five functions bit-exact."""
    x = dg.values("i32", 1 << 20, 0)
    got = run_dev(x)
    ref = oracle.reduce(x)
    assert got == ref


def test_integer_extremes_and_wrap():
    x = np.array([2 ** 63 - 1, 2 ** 63 - 1, -(2 ** 63), 5], dtype=np.int64)
    check(run_dev(x), x)
    x = np.full(1000, np.iinfo(np.int32).min, dtype=np.int32)
    check(run_dev(x), x)
    x = np.full(77777, 0xFFFFFFFF, dtype=np.uint32)
    check(run_dev(x), x)


def test_signed_zero_and_infinities():
    x = np.zeros(5000, dtype=np.float32)
    x[1234] = -0.0
    got = run_dev(x)
    assert same_float(got["min"], -0.0) and same_float(got["max"], 0.0)
    x = np.full(3000, -0.0, dtype=np.float64)
    got = run_dev(x)
    assert same_float(got["max"], -0.0)
    x = np.array([1.0, np.inf, -np.inf, 2.0], dtype=np.float32)
    got = run_dev(x, agg.AGG_MIN | agg.AGG_MAX)
    assert got["min"] == -np.inf and got["max"] == np.inf


@pytest.mark.parametrize("dt", [np.float32, np.float64])
def test_compensated_sum_wide_exponents(dt):
    x = make(dt, 2_000_003, seed=9, kind="wide")
    check(run_dev(x), x)
    # heavy cancellation: pairs x, -x plus a small residue
    y = np.concatenate([x, -x, np.array([0.25], dtype=dt)])
    got = run_dev(y)
    assert abs(got["sum"] - 0.25) <= 1e-6 * max(0.25, 2.0 ** -24 * float(np.abs(y.astype(np.float64)).sum()))


@pytest.mark.parametrize("case", ["subnormal", "extreme_exponents", "tiny_beside_huge", "near_max"])
def test_float64_sum_edge_cases(case):
    """The float64 sum is kept as a 128-bit fixed-point number at the scale of the
    largest exponent: subnormal rows, exponents across the whole range, rows far
    below the largest, and sums near the top of the range."""
    rng = np.random.default_rng(5)
    n = 100_003
    if case == "subnormal":
        x = rng.integers(1, 1000, n).astype(np.float64) * 5e-324 * rng.choice([-1.0, 1.0], n)
    elif case == "extreme_exponents":
        x = rng.standard_normal(n) * np.exp2(rng.integers(-1020, 1000, n).astype(np.float64))
    elif case == "tiny_beside_huge":
        x = np.concatenate([np.full(1000, 1e300), rng.standard_normal(5000), np.full(1000, -1e300)])
    else:
        x = np.full(4096, 1.7e308 / 8192) * rng.choice([0.5, 1.0], 4096)
    check(run_dev(x), x)


def test_float64_sum_of_a_column_with_an_infinity_is_not_finite():
    x = np.concatenate([np.ones(5000), [np.inf], np.ones(3000)])
    assert not math.isfinite(run_dev(x, agg.AGG_SUM)["sum"])


@pytest.mark.parametrize("dt", [np.float32, np.float64])
def test_fp_sum_is_deterministic(dt):
    t = torch.from_numpy(make(dt, 5_000_000, seed=1)).cuda()
    a = agg.decode_scalar(agg.agg_reduce(t, agg.AGG_SUM)).sum_f
    b = agg.decode_scalar(agg.agg_reduce(t, agg.AGG_SUM)).sum_f
    assert same_float(a, b)


@pytest.mark.parametrize("dt", DTS)
@pytest.mark.parametrize("n", [0, 1, 1000, (1 << 24) + 3, 50_000_017])
def test_reduce_host_parity(dt, n):
    x = make(dt, n, seed=n + 3)
    got = agg.agg_reduce_host(torch.from_numpy(x).pin_memory(), agg.AGG_ALL).as_dict()
    check(got, x)


def test_reduce_host_pageable_memory():
    x = make(np.int32, 3_000_000, seed=2)
    got = agg.agg_reduce_host(torch.from_numpy(x), agg.AGG_ALL).as_dict()
    check(got, x)


@pytest.mark.parametrize("dt", ["i32", "f32", "i64", "f64"])
def test_full_size_column_on_device(dt):
    """2^28 rows (i32/f32: 1 GiB; 64-bit: 2 GiB) in the launch shape the benchmark uses."""
    n = 1 << 28
    t = dg_cuda_values(dt, n)
    got = agg.decode_scalar(agg.agg_reduce(t, agg.AGG_ALL)).as_dict()
    x = t.cpu().numpy()
    check(got, x)


def dg_cuda_values(dt, n):
    from datagen import cuda as dgc
    return dgc.values(dt, n, 0)


def test_gpu_generator_matches_host_generator():
    from datagen import cuda as dgc
    n = 100003
    for dt in ["i32", "i64", "u32"]:
        assert np.array_equal(dgc.values(dt, n, 3, start=17).cpu().numpy(), dg.values(dt, n, 3, start=17))
    f = dgc.values("f64", n, 3).cpu().numpy()
    assert np.allclose(f, dg.values("f64", n, 3), rtol=1e-12, atol=1e-9)
    assert np.array_equal(dgc.keys_uniform(n, 1000, 4).cpu().numpy(), dg.keys_uniform(n, 1000, 4))
    assert np.array_equal(dgc.keys_zipf(n, 5000, 1.0, 4).cpu().numpy(), dg.keys_zipf(n, 5000, 1.0, 4))


def _scalar(x: np.ndarray, ops=agg.AGG_ALL, host=False):
    if host:
        return agg.agg_reduce_host(torch.from_numpy(x).pin_memory(), ops)
    return agg.decode_scalar(agg.agg_reduce(torch.from_numpy(x).cuda(), ops))


@pytest.mark.parametrize("dt", [np.float32, np.float64])
@pytest.mark.parametrize("kind", ["normal", "wide", "cancel", "tiny"])
@pytest.mark.parametrize("n", [1, 33, 65537, 3_000_001])
def test_float_sum_error_bound_holds(dt, kind, n):
    """err_bound, computed on the device with the sum, bounds |sum_f - oracle sum|."""
    rng = np.random.default_rng(n)
    if kind == "cancel":
        h = rng.standard_normal(n // 2 + 1) * 1e6
        x = np.concatenate([h, -h[::-1]])[:n]
        x[::97] += 1e-3
    elif kind == "tiny":  # subnormal float32 / float64 magnitudes beside normal ones
        tiny = np.finfo(dt).smallest_subnormal
        x = rng.integers(-1000, 1000, n).astype(np.float64) * float(tiny)
        x[::5] = rng.standard_normal(x[::5].size)
    else:
        x = make(dt, n, seed=n, kind=kind)
    x = np.asarray(x).astype(dt)
    ref = oracle.reduce(x)["sum"]
    for host in (False, True):
        r = _scalar(x, host=host)
        assert np.isfinite(r.err_bound) and r.err_bound >= 0
        assert abs(r.sum_f - ref) <= r.err_bound, (host, r.sum_f, ref, r.err_bound)
        a = float(np.abs(x.astype(np.float64)).sum())
        # the bound is itself far inside the 1e-6 bar on these columns
        assert r.err_bound <= 1e-6 * max(abs(ref), 2.0 ** -24 * a) or r.err_bound <= 2.0 ** -1000


def test_error_bound_of_integer_and_nonfinite_columns():
    x = make(np.int64, 100_000, seed=1)
    assert _scalar(x).err_bound == 0.0
    y = np.array([1.0, np.inf, 2.0], dtype=np.float32)
    assert _scalar(y).err_bound == np.inf
    z = np.arange(1000, dtype=np.float64)
    r = _scalar(z, agg.AGG_MIN | agg.AGG_MAX)
    assert r.err_bound == 0.0  # no SUM asked
