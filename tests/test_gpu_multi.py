"""Parity of the fused multi-column GROUP BY (agg_groupby_multi) with the CPU oracle.

Composite keys, several value columns of mixed types, a range filter; keys,
counts, integer results and float MIN/MAX bit-identical to the oracle, float
sums and averages within the 1e-6 bar.
"""
import numpy as np
import pytest
import torch

import datagen as dg
import oracle
import paper_2606_10030_gb300 as agg
from tests.common import FP_REL

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _build():
    agg.build()
    agg.lib()


def make(case, seed=0):
    rng = np.random.default_rng(seed)
    if case == "empty":
        n = 0
    elif case == "one":
        n = 1
    else:
        n = {"few": 100_003, "many": 400_009, "zipf": 300_007, "sentinel": 50_001, "ragged": 33_333}[case]
    if case == "many":  # more groups than a block's shared-memory accumulators hold
        lo = dg.keys_uniform(n, 150_000, seed)
        hi = rng.integers(0, 2, n).astype(np.uint32)
    elif case == "zipf":
        lo = dg.keys_zipf(n, 20_000, 1.1, seed)
        hi = rng.integers(0, 3, n).astype(np.uint32)
    else:
        lo = dg.keys_uniform(n, 50, seed) if n else np.zeros(0, np.uint32)
        hi = rng.integers(0, 4, n).astype(np.uint32)
    if case == "sentinel":
        lo[::5] = 0xFFFFFFFF
        hi[::10] = 0xFFFFFFFF
    cols = [rng.integers(-(2 ** 62), 2 ** 62, n, dtype=np.int64),
            dg.values("f32", n, seed + 1) if n else np.zeros(0, np.float32),
            rng.integers(-(2 ** 31), 2 ** 31, n, dtype=np.int64).astype(np.int32),
            dg.values("f64", n, seed + 2) if n else np.zeros(0, np.float64)]
    return lo.astype(np.uint32), hi, cols


def run(lo, hi, cols, ops, filt):
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()  # noqa: E731
    f = None if filt is None else (dev(filt[0]), filt[1], filt[2])
    m = agg.agg_groupby_multi(dev(lo), dev(hi) if hi is not None else None, [(dev(c), o) for c, o in zip(cols, ops)],
                              f)
    res = m.to_host()
    m.free()
    return res


def check(res, lo, hi, cols, ops, filt):
    ref = oracle.groupby_multi(lo, hi, cols, filt)
    assert np.array_equal(res["keys"], ref["keys"])
    assert np.array_equal(res["count"], ref["count"])
    refa = oracle.groupby_multi(lo, hi, [np.abs(c) for c in cols], filt) if any(c.dtype.kind == "f" for c in cols) \
        else None
    for c, (col, op) in enumerate(zip(cols, ops)):
        g, r = res["cols"][c], ref["cols"][c]
        if op & (agg.AGG_SUM | agg.AGG_AVG):
            if col.dtype.kind == "f":
                bar = FP_REL * np.maximum(np.abs(r["sum"]), 2.0 ** -24 * refa["cols"][c]["sum"])
                assert np.all(np.abs(g["sum"] - r["sum"]) <= bar)
                assert np.all(np.abs(g["avg"] - r["avg"]) <= bar / np.maximum(ref["count"], 1))
            else:
                assert np.array_equal(g["sum"], r["sum"])
                assert np.array_equal(g["avg"].view(np.int64), r["avg"].view(np.int64))
        if op & (agg.AGG_MIN | agg.AGG_MAX):
            if col.dtype.kind == "f":
                assert np.array_equal(g["min"].view(np.int64), r["min"].view(np.int64))
                assert np.array_equal(g["max"].view(np.int64), r["max"].view(np.int64))
            else:
                assert np.array_equal(g["min"], r["min"]) and np.array_equal(g["max"], r["max"])


FILTERS = ["none", "int", "float", "nothing"]


def make_filter(kind, cols):
    if kind == "none":
        return None
    if kind == "int":
        return (cols[2], -(2 ** 30), 2 ** 29)  # about 3/8 of the int32 column passes
    if kind == "float":
        return (cols[1], -250.0, 1e9)
    return (cols[2], 5, 4)  # an empty range


@pytest.mark.parametrize("case", ["empty", "one", "few", "many", "zipf", "sentinel", "ragged"])
@pytest.mark.parametrize("fk", FILTERS)
@pytest.mark.parametrize("two_keys", [False, True])
def test_multi_parity(case, fk, two_keys):
    lo, hi, cols = make(case, seed=len(case))
    ops = [agg.AGG_ALL] * 4
    filt = make_filter(fk, cols)
    key_hi = hi if two_keys else None
    res = run(lo, key_hi, cols, ops, filt)
    check(res, lo, key_hi, cols, ops, filt)


@pytest.mark.parametrize("ncols", [1, 2, 3])
def test_multi_column_subsets_and_op_subsets(ncols):
    lo, hi, cols = make("zipf", seed=5)
    ops = [agg.AGG_SUM, agg.AGG_MIN | agg.AGG_MAX, agg.AGG_COUNT | agg.AGG_AVG][:ncols]
    pick = [cols[3], cols[0], cols[1]][:ncols]
    res = run(lo, hi, pick, ops, (cols[2], 0, 2 ** 31 - 1))
    check(res, lo, hi, pick, ops, (cols[2], 0, 2 ** 31 - 1))


def test_multi_matches_the_single_key_group_by():
    lo, _, cols = make("many", seed=8)
    res = run(lo, None, [cols[0]], [agg.AGG_ALL], None)
    g = agg.agg_groupby(torch.from_numpy(lo).cuda(), torch.from_numpy(cols[0]).cuda(), agg.AGG_ALL)
    r = g.to_host()
    g.free()
    assert np.array_equal(res["keys"], r["keys"].astype(np.uint64))
    for f in ("sum", "min", "max"):
        assert np.array_equal(res["cols"][0][f], r[f])


def test_multi_2p26_rows_two_keys_three_columns_filtered():
    """2^26 rows: low key over 4096 keys, high key over 16 values, int64 / float32 /
    float64 columns, a filter that keeps about half the rows."""
    from datagen import cuda as dgc
    n = 1 << 26
    lo = dgc.keys_uniform(n, 4096, 3)
    hi = dgc.keys_uniform(n, 16, 4)
    a = dgc.values("i64", n, 5)
    b = dgc.values("f32", n, 6)
    c = dgc.values("f64", n, 7)
    f = dgc.values("i32", n, 8)
    m = agg.agg_groupby_multi(lo, hi, [(a, agg.AGG_ALL), (b, agg.AGG_ALL), (c, agg.AGG_SUM)], (f, -(2 ** 19), 2 ** 19))
    res = m.to_host()
    m.free()
    h = lambda t: t.cpu().numpy()  # noqa: E731
    check(res, h(lo), h(hi), [h(a), h(b), h(c)], [agg.AGG_ALL, agg.AGG_ALL, agg.AGG_SUM], (h(f), -(2 ** 19), 2 ** 19))
    assert 0.45 * n < res["count"].sum() < 0.55 * n
