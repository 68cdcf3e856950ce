"""Pins for the oracle's composite-key, multi-column, filtered GROUP BY.

Checked against a brute-force Python definition on tiny inputs (exact
rational sums rounded once, Python integers mod 2^64), against the already
pinned single-key oracle where the definitions coincide, and on invariants.
"""
from fractions import Fraction

import numpy as np
import pytest

import oracle


def _brute(lo, hi, cols, filt):
    groups = {}
    for i in range(lo.size):
        if filt is not None:
            f, a, b = filt
            x = float(f[i]) if f.dtype.kind == "f" else int(f[i])
            if not (a <= x <= b):
                continue
        key = ((int(hi[i]) if hi is not None else 0) << 32) | int(lo[i])
        g = groups.setdefault(key, [[] for _ in cols])
        for c, col in enumerate(cols):
            g[c].append(col[i])
    keys = sorted(groups)
    out = {"keys": np.array(keys, dtype=np.uint64), "count": np.array([len(groups[k][0]) for k in keys], np.int64),
           "cols": []}
    for c, col in enumerate(cols):
        sums, mins, maxs, avgs = [], [], [], []
        for k in keys:
            xs = groups[k][c]
            if col.dtype.kind == "f":
                s = float(sum(Fraction(float(x)) for x in xs))  # exact, rounded once to float64
                mins.append(min(float(x) for x in xs))
                maxs.append(max(float(x) for x in xs))
            else:
                t = sum(int(x) for x in xs) % (1 << 64)
                s = t - (1 << 64) if t >= 1 << 63 else t
                mins.append(min(int(x) for x in xs))
                maxs.append(max(int(x) for x in xs))
            sums.append(s)
            avgs.append(float(s) / len(xs))
        out["cols"].append({"sum": sums, "min": mins, "max": maxs, "avg": avgs})
    return out


def _same(got, ref):
    assert np.array_equal(got["keys"], ref["keys"])
    assert np.array_equal(got["count"], ref["count"])
    for g, r in zip(got["cols"], ref["cols"]):
        for f in ("sum", "min", "max", "avg"):
            a = np.asarray(g[f])
            b = np.asarray(r[f], dtype=a.dtype)
            if a.dtype.kind == "f":
                assert np.array_equal(a.view(np.int64), b.view(np.int64)), f
            else:
                assert np.array_equal(a, b), f


def _tiny(seed, n=40):
    rng = np.random.default_rng(seed)
    lo = rng.integers(0, 4, n).astype(np.uint32)
    lo[rng.integers(0, n, 3)] = 0xFFFFFFFF
    hi = rng.integers(0, 3, n).astype(np.uint32)
    hi[rng.integers(0, n, 2)] = 0xFFFFFFFF
    cols = [rng.integers(-(2 ** 62), 2 ** 62, n, dtype=np.int64),
            (rng.standard_normal(n) * np.exp2(rng.integers(-30, 30, n))).astype(np.float32),
            rng.integers(0, 2 ** 32, n, dtype=np.uint64).astype(np.uint32),
            rng.standard_normal(n) * 1e10,
            rng.integers(-(2 ** 31), 2 ** 31, n, dtype=np.int64).astype(np.int32)]
    return lo, hi, cols


@pytest.mark.parametrize("seed", range(12))
def test_brute_force_on_tiny_inputs(seed):
    lo, hi, cols = _tiny(seed)
    rng = np.random.default_rng(100 + seed)
    fcol = cols[seed % len(cols)]
    vals = np.sort(fcol.astype(np.float64) if fcol.dtype.kind == "f" else fcol.astype(object))
    a, b = vals[rng.integers(0, vals.size)], vals[rng.integers(0, vals.size)]
    a, b = min(a, b), max(a, b)
    for filt in (None, (fcol, a, b)):
        for key_hi in (None, hi):
            ref = _brute(lo, key_hi, cols, filt)
            got = oracle.groupby_multi(lo, key_hi, cols, filt)
            _same(got, ref)


def test_one_column_without_filter_is_the_single_key_oracle():
    rng = np.random.default_rng(7)
    n = 50_000
    keys = rng.integers(0, 3000, n).astype(np.uint32)
    for x in (rng.integers(-(2 ** 62), 2 ** 62, n, dtype=np.int64), rng.standard_normal(n).astype(np.float32),
              rng.standard_normal(n)):
        got = oracle.groupby_multi(keys, None, [x])
        ref = oracle.groupby(keys, x)
        assert np.array_equal(got["keys"], ref.keys.astype(np.uint64))
        assert np.array_equal(got["count"], ref.count)
        for f in ("sum", "min", "max", "avg"):
            assert np.array_equal(np.asarray(got["cols"][0][f]).view(np.int64), getattr(ref, f).view(np.int64))


def test_filter_is_a_selection_of_rows():
    """A filtered GROUP BY equals the unfiltered one over the selected rows."""
    rng = np.random.default_rng(8)
    n = 30_000
    lo = rng.integers(0, 500, n).astype(np.uint32)
    hi = rng.integers(0, 3, n).astype(np.uint32)
    x = rng.standard_normal(n).astype(np.float32)
    f = rng.integers(-100, 100, n).astype(np.int32)
    got = oracle.groupby_multi(lo, hi, [x], (f, -20, 35))
    sel = (f >= -20) & (f <= 35)
    ref = oracle.groupby_multi(lo[sel], hi[sel], [x[sel]])
    _same(got, ref)
    assert int(got["count"].sum()) == int(sel.sum())
    # bounds are inclusive, and a filter no row passes leaves no group
    assert oracle.groupby_multi(lo, hi, [x], (f, 36, 35))["keys"].size == 0
    one = oracle.groupby_multi(lo, hi, [x], (f, 7, 7))
    assert int(one["count"].sum()) == int((f == 7).sum())
    # a filter every row passes changes nothing
    _same(oracle.groupby_multi(lo, hi, [x], (f, -100, 99)), oracle.groupby_multi(lo, hi, [x]))


def test_composite_key_orders_by_high_then_low_word():
    lo = np.array([5, 1, 5, 0xFFFFFFFF, 1, 0], dtype=np.uint32)
    hi = np.array([0, 1, 1, 0, 0xFFFFFFFF, 1], dtype=np.uint32)
    x = np.arange(6, dtype=np.int64)
    got = oracle.groupby_multi(lo, hi, [x])
    assert list(got["keys"]) == [5, 0xFFFFFFFF, (1 << 32) | 0, (1 << 32) | 1, (1 << 32) | 5, (0xFFFFFFFF << 32) | 1]
    assert list(got["cols"][0]["sum"]) == [0, 3, 5, 1, 2, 4]


def test_invariants_over_columns():
    rng = np.random.default_rng(9)
    n = 20_000
    lo = rng.integers(0, 700, n).astype(np.uint32)
    hi = rng.integers(0, 4, n).astype(np.uint32)
    a = rng.integers(-(2 ** 40), 2 ** 40, n, dtype=np.int64)
    b = rng.standard_normal(n)
    got = oracle.groupby_multi(lo, hi, [a, b, a])
    assert int(got["count"].sum()) == n
    assert int(np.asarray(got["cols"][0]["sum"]).sum()) == int(a.sum())
    assert np.array_equal(got["cols"][0]["sum"], got["cols"][2]["sum"])  # the same column twice
    assert min(got["cols"][1]["min"]) == b.min() and max(got["cols"][1]["max"]) == b.max()
    assert abs(sum(got["cols"][1]["sum"]) - oracle.exact_sum(b)) <= 1e-9 * np.abs(b).sum()
