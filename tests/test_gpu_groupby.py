"""Parity of GROUP BY (agg_groupby, agg_groupby_host, agg_sketch) with the CPU oracle.

Keys, counts, integer sums and averages, and MIN/MAX must be bit-identical to
the oracle for every strategy; float sums and averages within the 1e-6 bar.
"""
import numpy as np
import pytest
import torch

import datagen as dg
import oracle
import paper_2606_10030_gb300 as agg
from oracle.sketch import sketch as oracle_sketch
from tests.common import FP_REL

pytestmark = pytest.mark.gpu

STRATS = [agg.AGG_STRAT_SMEM, agg.AGG_STRAT_GLOBAL, agg.AGG_STRAT_SORT, agg.AGG_STRAT_AUTO]
DTS = ["i32", "i64", "u32", "f32", "f64"]
NP = {"i32": np.int32, "i64": np.int64, "u32": np.uint32, "f32": np.float32, "f64": np.float64}


@pytest.fixture(scope="module", autouse=True)
def _build():
    agg.build()
    agg.lib()


def make_case(case: str, dt: str, seed: int = 0):
    rng = np.random.default_rng(seed)
    if case == "empty":
        keys = np.array([], dtype=np.uint32)
    elif case == "one":
        keys = np.array([123], dtype=np.uint32)
    elif case == "few":
        keys = dg.keys_uniform(1000, 7, seed)
    elif case == "uniform1k":
        keys = dg.keys_uniform(100_003, 1000, seed)
    elif case == "uniform50k":
        keys = dg.keys_uniform(300_007, 50_000, seed)
    elif case == "zipf":
        keys = dg.keys_zipf(200_003, 100_000, 1.0, seed)
    elif case == "distinct":
        keys = dg.domain_keys(seed, rng.permutation(70_001))
    elif case == "runs":  # sorted keys: long runs, whole warps on one key
        keys = np.sort(dg.keys_uniform(400_009, 300, seed))
    elif case == "onekey":  # every row on one key, the sentinel key in a tail run
        keys = np.full(262_147, 77, dtype=np.uint32)
        keys[-70_000:] = 0xFFFFFFFF
    elif case == "dense":  # keys in a narrow integer range: the sort needs fewer passes
        keys = (1000 + rng.integers(0, 50_000, 200_003)).astype(np.uint32)
    elif case == "highnarrow":  # a narrow range far from zero: digits of key - min
        keys = (0x80000000 + rng.integers(0, 300, 150_001)).astype(np.uint32)
    elif case == "sentinel":
        keys = dg.keys_uniform(50_001, 5, seed)
        keys[::3] = 0xFFFFFFFF
        keys[1::7] = 0
    else:
        raise ValueError(case)
    n = keys.size
    if dt in ("f32", "f64"):
        vals = dg.values(dt, n, seed + 1)
    elif dt == "i32":
        vals = rng.integers(-(2 ** 31), 2 ** 31, n, dtype=np.int64).astype(np.int32)
    elif dt == "u32":
        vals = rng.integers(0, 2 ** 32, n, dtype=np.uint64).astype(np.uint32)
    else:
        vals = rng.integers(-(2 ** 62), 2 ** 62, n, dtype=np.int64)
    return keys.astype(np.uint32), vals.astype(NP[dt])


def check_groups(res: dict, keys: np.ndarray, vals: np.ndarray, ops=agg.AGG_ALL):
    ref = oracle.groupby(keys, vals)
    assert np.array_equal(res["keys"], ref.keys)
    assert np.array_equal(res["count"], ref.count)
    fp = vals.dtype.kind == "f"
    if ops & (agg.AGG_SUM | agg.AGG_AVG):
        if fp:
            a = oracle.groupby(keys, np.abs(vals)).sum
            bar = FP_REL * np.maximum(np.abs(ref.sum), 2.0 ** -24 * a)
            assert np.all(np.abs(res["sum"] - ref.sum) <= bar)
            assert np.all(np.abs(res["avg"] - ref.avg) <= bar / ref.count)
        else:
            assert np.array_equal(res["sum"], ref.sum)
            assert np.array_equal(res["avg"].view(np.int64), ref.avg.view(np.int64))
    if ops & (agg.AGG_MIN | agg.AGG_MAX):
        if fp:
            assert np.array_equal(res["min"].view(np.int64), ref.min.view(np.int64))
            assert np.array_equal(res["max"].view(np.int64), ref.max.view(np.int64))
        else:
            assert np.array_equal(res["min"], ref.min) and np.array_equal(res["max"], ref.max)
    return ref


def run(keys, vals, strategy, ops=agg.AGG_ALL, **kw):
    k = torch.from_numpy(keys).cuda()
    v = torch.from_numpy(vals).cuda()
    g = agg.agg_groupby(k, v, ops, agg.options(strategy, **kw))
    res = g.to_host()
    meta = (g.strategy, g.retries, g.table_slots)
    g.free()
    return res, meta


CASES = ["empty", "one", "few", "uniform1k", "uniform50k", "zipf", "distinct", "sentinel", "runs", "onekey", "dense",
         "highnarrow"]


@pytest.mark.parametrize("strategy", STRATS)
@pytest.mark.parametrize("dt", DTS)
@pytest.mark.parametrize("case", CASES)
def test_groupby_parity(strategy, dt, case):
    keys, vals = make_case(case, dt, seed=len(case))
    res, meta = run(keys, vals, strategy)
    if strategy != agg.AGG_STRAT_AUTO:
        assert meta[0] == strategy
    check_groups(res, keys, vals)


@pytest.mark.parametrize("dt", DTS)
@pytest.mark.parametrize("ops", [agg.AGG_SUM, agg.AGG_COUNT, agg.AGG_MIN | agg.AGG_MAX, agg.AGG_AVG,
                                 agg.AGG_SUM | agg.AGG_COUNT | agg.AGG_MIN | agg.AGG_MAX])
def test_groupby_op_subsets(dt, ops):
    keys, vals = make_case("uniform1k", dt, seed=3)
    for s in STRATS[:3]:
        res, _ = run(keys, vals, s, ops)
        check_groups(res, keys, vals, ops)


@pytest.mark.parametrize("dt", DTS)
def test_strategies_return_identical_results(dt):
    keys, vals = make_case("zipf", dt, seed=11)
    outs = [run(keys, vals, s)[0] for s in STRATS[:3]]
    for o in outs[1:]:
        for f in ("keys", "count", "min", "max"):
            assert np.array_equal(o[f].view(np.int64) if o[f].dtype == np.float64 else o[f],
                                  outs[0][f].view(np.int64) if outs[0][f].dtype == np.float64 else outs[0][f])
        if dt in ("f32", "f64"):
            a = oracle.groupby(keys, np.abs(vals)).sum
            assert np.all(np.abs(o["sum"] - outs[0]["sum"]) <= 2 * FP_REL * np.maximum(np.abs(outs[0]["sum"]),
                                                                                     2.0 ** -24 * a))
        else:
            assert np.array_equal(o["sum"], outs[0]["sum"]) and np.array_equal(o["avg"], outs[0]["avg"])


def test_table_regrows_when_undersized():
    keys, vals = make_case("uniform50k", "i64", seed=5)
    res, meta = run(keys, vals, agg.AGG_STRAT_GLOBAL, table_slots=1024)
    assert meta[1] == 1 and meta[2] >= 65536  # a column this small regrows once, to 2n slots
    check_groups(res, keys, vals)
    res, meta = run(keys, vals, agg.AGG_STRAT_SMEM, table_slots=2048, smem_slots=256)
    assert meta[1] >= 1
    check_groups(res, keys, vals)


@pytest.mark.parametrize("strategy", [agg.AGG_STRAT_SMEM, agg.AGG_STRAT_GLOBAL])
def test_large_table_regrows_from_the_folded_fraction(strategy):
    """2^24 rows over about 2^22 keys into a 2^16-slot table: the first build stops when the table
    fills, and the next table is sized from the fraction of rows folded by then."""
    n = 1 << 24
    keys = dg.keys_uniform(n, 1 << 22, 7)
    vals = dg.values("i64", n, 7)
    res, meta = run(keys, vals, strategy, table_slots=1 << 16)
    assert 1 <= meta[1] <= 2
    check_groups(res, keys, vals)


@pytest.mark.parametrize("strategy", STRATS[:3])
def test_unaligned_columns_use_the_scalar_path(strategy):
    keys, vals = make_case("uniform1k", "i64", seed=6)
    k = torch.from_numpy(keys).cuda()
    v = torch.from_numpy(vals).cuda()
    g = agg.agg_groupby(k[1:], v[:-1], agg.AGG_ALL, agg.options(strategy))
    check_groups(g.to_host(), keys[1:], vals[:-1])
    g.free()
    g = agg.agg_groupby(k[3:], v[3:], agg.AGG_ALL, agg.options(strategy))
    check_groups(g.to_host(), keys[3:], vals[3:])
    g.free()


def test_config_2p26_rows_1024_keys_int64_bit_exact():
    """2^26 rows, uint32 keys uniform over 1024 random keys, int64 values in [0, 2^32):
    GROUP BY SUM/COUNT/MIN/MAX bit-exact (the shared-memory hash path)."""
    from datagen import cuda as dgc
    n = 1 << 26
    k = dgc.keys_uniform(n, 1024, 0)
    v = dgc.values("i64", n, 0)
    ops = agg.AGG_SUM | agg.AGG_COUNT | agg.AGG_MIN | agg.AGG_MAX
    g = agg.agg_groupby(k, v, ops)
    assert g.strategy == agg.AGG_STRAT_SMEM and g.num_groups == 1024
    res = g.to_host()
    g.free()
    kh, vh = k.cpu().numpy(), v.cpu().numpy()
    assert np.array_equal(kh, dg.keys_uniform(n, 1024, 0)[:n]) if n <= (1 << 20) else True
    check_groups(res, kh, vh, ops)


@pytest.mark.parametrize("dt", ["i64", "f32"])
@pytest.mark.parametrize("strategy", STRATS)
def test_host_fed_groupby(dt, strategy):
    n = 20_000_017  # three 8 Mi-row chunks
    keys = dg.keys_uniform(n, 3000, 2)
    vals = dg.values(dt, n, 2)
    g = agg.agg_groupby_host(torch.from_numpy(keys).pin_memory(), torch.from_numpy(vals).pin_memory(),
                             agg.AGG_ALL, agg.options(strategy))
    res = g.to_host()
    g.free()
    check_groups(res, keys, vals)


@pytest.mark.parametrize("partition", [-1, 1, 2])
def test_host_fed_groupby_high_cardinality(partition):
    """Partitioned plans copy the whole column and run the device path; -1 keeps per-chunk builds."""
    n = 20_000_017
    keys = dg.keys_zipf(n, 1 << 20, 1.0, 4)
    vals = dg.values("f32", n, 4)
    g = agg.agg_groupby_host(torch.from_numpy(keys).pin_memory(), torch.from_numpy(vals).pin_memory(),
                             agg.AGG_ALL, agg.options(agg.AGG_STRAT_SMEM, partition=partition))
    res = g.to_host()
    g.free()
    check_groups(res, keys, vals)


def _dev_consts():
    p = torch.cuda.get_device_properties(0)
    return float(p.shared_memory_per_block_optin), float(p.L2_cache_size)


@pytest.mark.parametrize("case", ["uniform1k", "zipf", "distinct", "sentinel", "few", "sorted", "tiny"])
@pytest.mark.parametrize("offset", [0, 12345, 2 ** 63 + 17])
def test_sketch_parity(case, offset):
    if case == "sorted":
        keys = np.sort(dg.keys_uniform(500_000, 3000, 1))
    elif case == "tiny":
        keys = dg.keys_uniform(1000, 40, 1)
    else:
        keys, _ = make_case(case, "i32", seed=2)
    smem, l2 = _dev_consts()
    ops = agg.AGG_SUM | agg.AGG_MIN
    got = agg.agg_sketch(torch.from_numpy(keys).cuda(), agg.AGG_F64, ops, offset).cpu().numpy()
    ref = oracle_sketch(keys, 8, 2, 1, 32, offset, smem, l2)
    assert np.allclose(got, ref, rtol=1e-5, atol=1e-6), (got, ref)


@pytest.mark.parametrize("levels", [1, 2])
@pytest.mark.parametrize("strategy", [agg.AGG_STRAT_SMEM, agg.AGG_STRAT_GLOBAL])
@pytest.mark.parametrize("dt", DTS)
@pytest.mark.parametrize("case", ["uniform50k", "zipf", "sentinel", "distinct", "runs"])
def test_hash_partitioned_build_parity(levels, strategy, dt, case):
    """Rows hash-partitioned (one or two levels) before the build, forced on for these small inputs."""
    keys, vals = make_case(case, dt, seed=21)
    res, meta = run(keys, vals, strategy, partition=levels)
    check_groups(res, keys, vals)
    res2, _ = run(keys, vals, strategy, partition=-1)
    assert np.array_equal(res["keys"], res2["keys"]) and np.array_equal(res["count"], res2["count"])


@pytest.mark.parametrize("items", [4, 8])
@pytest.mark.parametrize("tile", [0, 4096, 16384])
def test_items_per_thread_and_tile_rows(items, tile):
    keys, vals = make_case("uniform50k", "f64", seed=17)
    for strategy, part in ((agg.AGG_STRAT_SMEM, 1), (agg.AGG_STRAT_SMEM, -1), (agg.AGG_STRAT_GLOBAL, -1)):
        res, _ = run(keys, vals, strategy, items_per_thread=items, tile_rows=tile, partition=part)
        check_groups(res, keys, vals)


@pytest.mark.parametrize("dt", ["i32", "i64"])
@pytest.mark.parametrize("pattern", ["all_carry", "negative", "mixed"])
@pytest.mark.parametrize("tile", [0, 65536])
def test_tile_count_word_at_its_limits(dt, pattern, tile):
    """Tile builds keep a slot's count and its low word's carries in one 32-bit word: tiles of the
    largest size (65536 asks for 65532 rows) where one key takes every row and nearly every add
    carries, with values whose high words are zero, all ones (negative), or both."""
    n = 3 * 65536 + 11
    rng = np.random.default_rng(7)
    keys = np.where(rng.random(n) < 0.97, 12345, rng.integers(0, 2 ** 32, n)).astype(np.uint32)
    if pattern == "all_carry":
        v = np.full(n, 0xFFFFFFFF if dt == "i64" else 2 ** 31 - 1, np.int64)
    elif pattern == "negative":
        v = -rng.integers(1, 2 ** 31, n).astype(np.int64)
    else:
        v = rng.integers(-(2 ** 31), 2 ** 31 if dt == "i32" else 2 ** 40, n).astype(np.int64)
    vals = v.astype(np.int32 if dt == "i32" else np.int64)
    res, meta = run(keys, vals, agg.AGG_STRAT_SMEM, partition=1, tile_rows=tile)
    check_groups(res, keys, vals)


@pytest.mark.parametrize("later", ["same_keys", "new_keys"])
def test_host_fed_streamed_builds(later):
    """A host-fed column of two 2^23-row chunks whose first chunk recurs over 2^16 keys: each chunk is
    partitioned and built as it arrives into a table sized from the first chunk's count. With the
    same keys later the table holds; with 2^20 new keys in the second chunk it fills and the column
    is rebuilt over every piece from the count of all chunks. Both match the oracle."""
    n0, n1 = 1 << 23, 1 << 22
    k0 = dg.keys_uniform(n0, 1 << 16, 31)
    k1 = dg.keys_uniform(n1, 1 << 16, 31) if later == "same_keys" else \
        (dg.keys_uniform(n1, 1 << 20, 32) ^ np.uint32(0x9E3779B9))
    keys = np.concatenate([k0, k1]).astype(np.uint32)
    vals = dg.values("i64", n0 + n1, 33)
    g = agg.agg_groupby_host(torch.from_numpy(keys).pin_memory(), torch.from_numpy(vals).pin_memory(),
                             agg.AGG_ALL, agg.options(agg.AGG_STRAT_SMEM))
    res = g.to_host()
    retries = g.retries
    g.free()
    check_groups(res, keys, vals)
    assert (retries > 0) == (later == "new_keys")


@pytest.mark.parametrize("partition", [-1, 1])
@pytest.mark.parametrize("spread", ["two_words", "wide", "one_word"])
def test_int64_min_max_word_pairs(partition, spread):
    """Int64 MIN/MAX keep values that share the high word of a row the block (or tile) read first on
    32-bit (min, max) pairs and the others on 64-bit pairs, merged at the flush: values over two high
    words (signs mixed), over many, and over one, in the plain and the partitioned build."""
    n = (1 << 22) + 13
    rng = np.random.default_rng(41)
    keys = dg.keys_uniform(n, 1024, 41)
    if spread == "two_words":
        vals = rng.integers(-(2 ** 31), 2 ** 31, n).astype(np.int64)
    elif spread == "wide":
        vals = rng.integers(-(2 ** 62), 2 ** 62, n).astype(np.int64)
    else:
        vals = rng.integers(0, 2 ** 32, n).astype(np.int64)
        vals[::997] = -1 - vals[::997]  # a few rows on another high word
    res, _ = run(keys, vals, agg.AGG_STRAT_SMEM, partition=partition)
    check_groups(res, keys, vals)


def test_host_fed_streamed_build_with_a_small_table():
    """A host-fed column whose chunk-by-chunk build is given too small a table (agg_options.table_slots)
    fills it; the rebuild over every piece regrows the table and matches the oracle."""
    n = (1 << 23) + (1 << 21)
    keys = dg.keys_uniform(n, 1 << 16, 51)
    vals = dg.values("i64", n, 52)
    g = agg.agg_groupby_host(torch.from_numpy(keys).pin_memory(), torch.from_numpy(vals).pin_memory(),
                             agg.AGG_ALL, agg.options(agg.AGG_STRAT_SMEM, table_slots=4096))
    res = g.to_host()
    retries = g.retries
    g.free()
    check_groups(res, keys, vals)
    assert retries > 0
