"""The key-partitioned parallel run of the oracle returns exactly the oracle's result."""
import numpy as np

import datagen as dg
import oracle
from tests import oracle_par


def test_key_classes_cover_every_key_once():
    keys = dg.keys_zipf(100_000, 5000, 1.0, 3)
    c = oracle_par.key_class(keys, 6)
    assert c.min() >= 0 and c.max() < 64 and len(np.unique(c)) > 32


def test_partitioned_groupby_is_the_oracle(tmp_path, monkeypatch):
    monkeypatch.setenv("AGG_ORACLE_CACHE", str(tmp_path))
    n = 300_007
    keys = dg.keys_zipf(n, 40_000, 1.0, 5)
    vals = dg.values("f32", n, 5)
    got = oracle_par.groupby(keys, vals, name="t_f32", classes_log2=3, workers=3)
    ref = oracle.groupby(keys, vals)
    assert np.array_equal(got["keys"], ref.keys) and np.array_equal(got["count"], ref.count)
    for f in ("sum", "min", "max", "avg"):
        assert np.array_equal(got[f].view(np.int64), getattr(ref, f).view(np.int64)), f
    refa = oracle.groupby(keys, np.abs(vals)).sum
    assert np.allclose(got["abs_sum"], refa, rtol=1e-12, atol=0)
    again = oracle_par.groupby(keys[:10], vals[:10], name="t_f32")  # served from the cache
    assert np.array_equal(again["keys"], got["keys"])


def test_row_range_selected_groupby_is_the_oracle(tmp_path, monkeypatch):
    monkeypatch.setenv("AGG_ORACLE_CACHE", str(tmp_path))
    n = 200_003
    keys = dg.keys_uniform(n, 3000, 6)
    vals = np.random.default_rng(6).integers(-(2 ** 62), 2 ** 62, n, dtype=np.int64)
    sel = np.concatenate([keys[:50], np.array([12345, 0xFFFFFFFF], dtype=np.uint32)])
    got = oracle_par.groupby_selected_int(keys, vals, sel, workers=4, min_rows=30_000)
    ref = oracle.groupby_selected(keys, vals, sel)
    assert np.array_equal(got["keys"], ref.keys) and np.array_equal(got["count"], ref.count)
    has = ref.count > 0
    assert np.array_equal(got["sum"], ref.sum)
    assert np.array_equal(got["min"][has], ref.min[has]) and np.array_equal(got["max"][has], ref.max[has])


def test_table_check_regenerates_the_seeded_table(tmp_path, monkeypatch):
    monkeypatch.setenv("AGG_ORACLE_CACHE", str(tmp_path))
    n = 150_001
    for D, s in ((3000, 0.0), (50_000, 0.5)):
        keys = dg.keys_zipf(n, D, s, 9) if s > 0 else dg.keys_uniform(n, D, 9)
        vals = dg.values("i64", n, 9)
        sel = np.concatenate([keys[::997], np.array([1, 2, 3], dtype=np.uint32)])
        got = oracle_par.table_check(n, D, s, "i64", 9, sel, rows_per_job=20_000, workers=4)
        ref = oracle.groupby_selected(keys, vals, sel)
        has = ref.count > 0
        assert np.array_equal(got["keys"], ref.keys) and np.array_equal(got["count"], ref.count)
        assert np.array_equal(got["sum"], ref.sum)
        assert np.array_equal(got["min"][has], ref.min[has]) and np.array_equal(got["max"][has], ref.max[has])
        r = oracle.reduce(vals)
        assert got["total"] == {"count": r["count"], "sum": r["sum"], "min": r["min"], "max": r["max"]}
        again = oracle_par.table_check(n, D, s, "i64", 9, sel, rows_per_job=20_000, workers=4, columns=(keys, vals))
        for f in ("keys", "count", "sum"):
            assert np.array_equal(again[f], got[f])
        assert again["total"] == got["total"]
