"""Pins for the CPU oracle: checks against things other than the oracle itself.

* exact floating-point sums against Python's math.fsum (Shewchuk's correctly
  rounded summation) and against fractions.Fraction, whose conversion to float
  is correctly rounded;
* integer folds against Python integers reduced mod 2^64 and closed forms;
* GROUP BY against brute force over every input of a tiny domain;
* invariants between grouped and ungrouped results.
"""
import itertools
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle

INT_DT = [np.int32, np.int64, np.uint32]


def _wrap64(v: int) -> int:
    v &= (1 << 64) - 1
    return v - (1 << 64) if v >> 63 else v


# ---------------------------------------------------------------------------
# Exact floating-point SUM
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("seed", range(6))
def test_exact_sum_f64_matches_fsum_wide_exponents(seed):
    rng = np.random.default_rng(seed)
    n = 5000
    x = rng.standard_normal(n) * np.exp2(rng.integers(-1070, 1000, n).astype(np.float64))
    x[rng.integers(0, n, 50)] = 0.0
    assert oracle.exact_sum(x) == math.fsum(x)


@pytest.mark.parametrize("seed", range(6))
def test_exact_sum_f32_matches_fsum(seed):
    rng = np.random.default_rng(100 + seed)
    n = 20000
    x = (rng.standard_normal(n) * np.exp2(rng.integers(-150, 126, n).astype(np.float64))).astype(np.float32)
    x = x[np.isfinite(x)]
    # float32 -> float64 is exact, so fsum of the widened values is the exact sum rounded once
    assert oracle.exact_sum(x) == math.fsum(x.astype(np.float64))


def test_exact_sum_against_fractions():
    rng = np.random.default_rng(7)
    for _ in range(20):
        x = rng.standard_normal(40) * np.exp2(rng.integers(-60, 60, 40).astype(np.float64))
        exact = float(sum((Fraction(float(v)) for v in x), Fraction(0)))
        assert oracle.exact_sum(x) == exact


def test_exact_sum_rounding_ties_and_subnormals():
    e = 2.0 ** -53
    assert oracle.exact_sum(np.array([1.0, e])) == 1.0                     # tie -> even
    assert oracle.exact_sum(np.array([1.0, e, 2.0 ** -200])) == 1.0 + 2 * e  # above tie -> up
    assert oracle.exact_sum(np.array([1.0 + 2 * e, e])) == 1.0 + 4 * e       # tie -> even (up)
    tiny = 5e-324
    assert oracle.exact_sum(np.array([tiny, tiny, tiny])) == 3 * tiny
    assert oracle.exact_sum(np.array([1e308, 1e308, -1e308])) == 1e308      # no intermediate overflow
    assert oracle.exact_sum(np.array([1e308, 1e308])) == math.inf
    x = np.array([3.0, -3.0] * 1000 + [0.5])
    assert oracle.exact_sum(x) == 0.5
    assert oracle.exact_sum(np.array([], dtype=np.float64)) == 0.0
    f = np.array([np.float32(2.0 ** -149)] * 7 + [np.float32(-(2.0 ** -149))], dtype=np.float32)
    assert oracle.exact_sum(f) == 6 * 2.0 ** -149


def test_exact_sum_many_terms_normalises():
    # more terms than one carry-free window: 3 * 2^30 powers of two would be slow,
    # so the carry path is exercised with large digits instead
    x = np.full(200000, 2.0 ** 52 + 1.0)
    assert oracle.exact_sum(x) == math.fsum(x)


# ---------------------------------------------------------------------------
# Ungrouped folds (Fig. 4: r = aggregate(r, input[i]))
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("dt", INT_DT)
def test_reduce_closed_forms_int(dt):
    n = 100003
    r = oracle.reduce(np.ones(n, dtype=dt))
    assert (r["count"], r["sum"], r["min"], r["max"], r["avg"]) == (n, n, 1, 1, 1.0)
    r = oracle.reduce(np.arange(n, dtype=dt))
    assert r["sum"] == n * (n - 1) // 2 and r["min"] == 0 and r["max"] == n - 1
    assert r["avg"] == float(n * (n - 1) // 2) / n
    c = 77
    r = oracle.reduce(np.full(n, c, dtype=dt))
    assert r["sum"] == c * n and r["min"] == r["max"] == c and r["avg"] == c


def test_reduce_int_wraps_mod_2_64():
    x = np.array([2 ** 63 - 1, 1, 5], dtype=np.int64)
    assert oracle.reduce(x)["sum"] == _wrap64(2 ** 63 - 1 + 1 + 5)
    x = np.array([-(2 ** 63), -1], dtype=np.int64)
    assert oracle.reduce(x)["sum"] == _wrap64(-(2 ** 63) - 1)
    u = np.full(5, 0xFFFFFFFF, dtype=np.uint32)  # zero-extended, not sign-extended
    r = oracle.reduce(u)
    assert r["sum"] == 5 * 0xFFFFFFFF and r["min"] == 0xFFFFFFFF
    i = np.array([np.iinfo(np.int32).min, np.iinfo(np.int32).max, -1], dtype=np.int32)
    r = oracle.reduce(i)
    assert r["sum"] == -(2 ** 31) + 2 ** 31 - 1 - 1 and r["min"] == -(2 ** 31) and r["max"] == 2 ** 31 - 1


@pytest.mark.parametrize("dt", INT_DT + [np.float32, np.float64])
def test_reduce_random_against_python(dt):
    rng = np.random.default_rng(3)
    if np.dtype(dt).kind == "f":
        x = (rng.standard_normal(3001) * 1e3).astype(dt)
    else:
        info = np.iinfo(dt)
        x = rng.integers(info.min, info.max, 3001, dtype=np.int64 if dt != np.uint32 else np.uint64,
                         endpoint=True).astype(dt)
    r = oracle.reduce(x)
    vals = [v.item() for v in x]
    assert r["count"] == len(vals)
    if np.dtype(dt).kind == "f":
        assert r["sum"] == math.fsum(float(v) for v in vals)
    else:
        assert r["sum"] == _wrap64(sum(vals))
    assert r["min"] == min(vals) and r["max"] == max(vals)
    assert r["avg"] == float(r["sum"]) / len(vals)


def test_reduce_signed_zero_order():
    r = oracle.reduce(np.array([0.0, -0.0, 0.0], dtype=np.float32))
    assert r["min"] == 0 and math.copysign(1, r["min"]) == -1
    assert r["max"] == 0 and math.copysign(1, r["max"]) == 1
    r = oracle.reduce(np.array([-0.0], dtype=np.float64))
    assert math.copysign(1, r["max"]) == -1


def test_reduce_empty():
    r = oracle.reduce(np.array([], dtype=np.int32))
    assert r["count"] == 0 and r["sum"] == 0 and math.isnan(r["avg"])
    assert r["min"] == np.iinfo(np.int64).max and r["max"] == np.iinfo(np.int64).min
    r = oracle.reduce(np.array([], dtype=np.float32))
    assert r["count"] == 0 and r["sum"] == 0.0 and r["min"] == math.inf and r["max"] == -math.inf


def test_reduce_avg_between_min_and_max():
    rng = np.random.default_rng(11)
    for dt in INT_DT + [np.float32, np.float64]:
        x = (rng.standard_normal(999) * 1e4).astype(dt) if np.dtype(dt).kind == "f" else \
            rng.integers(0, 2 ** 20, 999).astype(dt)
        r = oracle.reduce(x)
        assert r["min"] <= r["avg"] <= r["max"]


# ---------------------------------------------------------------------------
# GROUP BY
# ---------------------------------------------------------------------------

def _naive_groupby(keys, vals):
    """O(n * k) distinct-key scan in plain Python."""
    out = {}
    for k in sorted(set(int(k) for k in keys)):
        vs = [v.item() for kk, v in zip(keys, vals) if int(kk) == k]
        out[k] = vs
    return out


def _check_against_naive(keys, vals):
    g = oracle.groupby(keys, vals)
    ref = _naive_groupby(keys, vals)
    assert list(g.keys) == list(ref.keys())
    fp = vals.dtype.kind == "f"
    for j, (k, vs) in enumerate(ref.items()):
        assert g.count[j] == len(vs)
        if fp:
            assert g.sum[j] == math.fsum(vs)
        else:
            assert g.sum[j] == _wrap64(sum(vs))
        assert g.min[j] == min(vs) and g.max[j] == max(vs)
        assert g.avg[j] == float(g.sum[j]) / len(vs)


def test_groupby_brute_force_tiny_domain():
    key_dom = [0, 5, 0xFFFFFFFF]
    val_dom = [-2, 0, 3]
    for n in range(0, 5):
        for ks in itertools.product(key_dom, repeat=n):
            for vs in itertools.product(val_dom, repeat=n):
                k = np.array(ks, dtype=np.uint32)
                v = np.array(vs, dtype=np.int32)
                _check_against_naive(k, v)


@pytest.mark.parametrize("dt", [np.int64, np.uint32, np.float32, np.float64])
def test_groupby_random_against_naive(dt):
    rng = np.random.default_rng(5)
    keys = rng.integers(0, 17, 600).astype(np.uint32) * np.uint32(0x9E3779B1)
    vals = (rng.standard_normal(600) * 100).astype(dt) if np.dtype(dt).kind == "f" else \
        rng.integers(0, 2 ** 31, 600).astype(dt)
    _check_against_naive(keys, vals)


@pytest.mark.parametrize("dt", [np.int32, np.int64, np.uint32, np.float32, np.float64])
def test_groupby_invariants(dt):
    rng = np.random.default_rng(9)
    n = 50000
    keys = rng.integers(0, 2 ** 32, 700, dtype=np.uint64).astype(np.uint32)[rng.integers(0, 700, n)]
    vals = (rng.standard_normal(n) * 1e3).astype(dt) if np.dtype(dt).kind == "f" else \
        rng.integers(-(2 ** 20) if dt != np.uint32 else 0, 2 ** 20, n).astype(dt)
    g = oracle.groupby(keys, vals)
    r = oracle.reduce(vals)
    assert np.all(np.diff(g.keys.astype(np.int64)) > 0)
    assert g.count.sum() == n == r["count"]
    assert g.min.min() == r["min"] and g.max.max() == r["max"]
    assert np.all(g.min <= g.avg) and np.all(g.avg <= g.max)
    if np.dtype(dt).kind == "f":
        # each group sum is exact-then-rounded; their exact sum is within d ulps of the total
        assert abs(math.fsum(g.sum) - r["sum"]) <= len(g) * 2 ** -52 * np.abs(vals).astype(np.float64).sum()
    else:
        assert _wrap64(int(g.sum.astype(object).sum())) == r["sum"]


def test_groupby_single_key_equals_reduce_and_all_distinct_equals_rows():
    rng = np.random.default_rng(1)
    vals = rng.integers(-1000, 1000, 5000).astype(np.int64)
    g = oracle.groupby(np.full(5000, 42, dtype=np.uint32), vals)
    r = oracle.reduce(vals)
    assert len(g) == 1 and g.keys[0] == 42 and g.sum[0] == r["sum"] and g.count[0] == 5000
    keys = np.arange(5000, dtype=np.uint32)[::-1].copy()
    g = oracle.groupby(keys, vals)
    assert len(g) == 5000 and np.all(g.count == 1)
    assert np.array_equal(g.sum, vals[::-1]) and np.array_equal(g.min, g.max)


def test_groupby_selected_matches_full():
    rng = np.random.default_rng(2)
    keys = rng.integers(0, 300, 20000).astype(np.uint32)
    vals = (rng.standard_normal(20000) * 1e3).astype(np.float32)
    g = oracle.groupby(keys, vals)
    sel = g.keys[::7]
    s = oracle.groupby_selected(keys, vals, np.concatenate([sel, np.array([100000], dtype=np.uint32)]))
    idx = np.searchsorted(g.keys, sel)
    assert np.array_equal(s.keys[:-1], sel) and s.keys[-1] == 100000 and s.count[-1] == 0
    for f in ("count", "sum", "min", "max", "avg"):
        assert np.array_equal(getattr(s, f)[:-1], getattr(g, f)[idx])
