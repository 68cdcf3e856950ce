"""The exact-sum arithmetic of the exact float GROUP BY mode (csrc/exact.cuh),
built for the host and checked against exact rational sums.

Python's float(Fraction) rounds a rational to the nearest float64, ties to
even, so sum(Fraction(x)) rounded that way is the exactly rounded sum the mode
promises; the oracle's exact accumulator is checked beside it.
"""
import ctypes
import os
import shutil
import subprocess
import tempfile
from fractions import Fraction

import numpy as np
import pytest

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def lib():
    cxx = shutil.which("g++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    d = tempfile.mkdtemp()
    so = os.path.join(d, "exact_host.so")
    subprocess.run([cxx, "-O2", "-std=c++17", "-shared", "-fPIC", "-o", so, os.path.join(HERE, "exact_host.cpp")],
                   check=True)
    L = ctypes.CDLL(so)
    for name in ("exact_host_sum_f64", "exact_host_sum_f32"):
        f = getattr(L, name)
        f.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.POINTER(ctypes.c_int)]
        f.restype = ctypes.c_double
    yield L
    shutil.rmtree(d, ignore_errors=True)


def host_sum(L, x: np.ndarray):
    x = np.ascontiguousarray(x)
    digits = ctypes.c_int(0)
    f = L.exact_host_sum_f32 if x.dtype == np.float32 else L.exact_host_sum_f64
    return f(x.ctypes.data, x.size, ctypes.byref(digits)), digits.value


def exact(x: np.ndarray) -> float:
    return float(sum((Fraction(float(v)) for v in x), Fraction(0)))


def same(a: float, b: float) -> bool:
    return np.float64(a).tobytes() == np.float64(b).tobytes()


def cases():
    rng = np.random.default_rng(11)
    yield "normal", rng.standard_normal(20000) * 1e3
    yield "wide", rng.standard_normal(5000) * np.exp2(rng.integers(-300, 300, 5000).astype(np.float64))
    yield "extreme", rng.standard_normal(3000) * np.exp2(rng.integers(-1070, 1020, 3000).astype(np.float64))
    x = rng.standard_normal(4000)
    yield "cancel_to_zero", np.concatenate([x, -x[::-1]])
    yield "tie_to_even_down", np.array([1.0, 2.0 ** -53])
    yield "tie_to_even_up", np.array([1.0 + 2.0 ** -52, 2.0 ** -53])
    yield "above_tie", np.array([1.0, 2.0 ** -53, 2.0 ** -1000])
    yield "below_tie", np.array([1.0, 2.0 ** -53, -(2.0 ** -1000)])
    yield "subnormal", rng.integers(1, 1000, 5000).astype(np.float64) * 5e-324
    yield "near_max", np.full(64, 1.7e308 / 128)
    yield "overflow", np.full(4, 1.7e308)
    yield "one_row", np.array([-3.25])
    yield "zeros", np.array([0.0, -0.0, 0.0])
    yield "f32_normal", (rng.standard_normal(20000) * 1e3).astype(np.float32)
    yield "f32_wide", (rng.standard_normal(5000) * np.exp2(rng.integers(-120, 120, 5000))).astype(np.float32)
    yield "f32_subnormal", (rng.integers(1, 100, 1000) * np.float32(1.4e-45)).astype(np.float32)


@pytest.mark.parametrize("name,x", list(cases()), ids=[c[0] for c in cases()])
def test_exactly_rounded(lib, name, x):
    got, digits = host_sum(lib, x)
    if name == "overflow":
        assert got == np.inf
        return
    ref = exact(x)
    assert same(got, ref), (got, ref)
    assert same(got, oracle.exact_sum(x)), (got, oracle.exact_sum(x))
    assert 1 <= digits <= 84


def test_digits_cover_the_exponent_span(lib):
    # a column of similar magnitudes needs a handful of digits; the full float64 range fits
    _, d = host_sum(lib, np.linspace(1.0, 2.0, 1000))
    assert d <= 6  # 53 bits + 32 for the row count + a sign, in 28-bit digits, + 2
    _, d = host_sum(lib, np.array([5e-324, 1.7e308]))
    assert d <= 84


@pytest.mark.parametrize("dt", [np.float64, np.float32])
def test_exactly_rounded_on_random_columns(lib, dt):
    """Random lengths, exponent ranges, signs and cancellations, each against the rational sum."""
    rng = np.random.default_rng(2024 if dt == np.float64 else 2025)
    lim = 1000 if dt == np.float64 else 120
    for _ in range(150):
        n = int(rng.integers(1, 400))
        lo = int(rng.integers(-lim, lim))
        hi = min(lim, lo + int(rng.integers(0, 200)))
        x = (rng.standard_normal(n) * np.exp2(rng.integers(lo, hi + 1, n).astype(np.float64))).astype(dt)
        if rng.random() < 0.3:  # cancel most of the column
            x = np.concatenate([x, -x[: n // 2]])
        got, _ = host_sum(lib, x)
        assert same(got, exact(x)), (x.tolist(), got, exact(x))
