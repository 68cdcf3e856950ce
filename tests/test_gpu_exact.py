"""Exact float GROUP BY sums (AGG_FLAG_EXACT_SUM): every group's SUM and AVG are
bit-identical to the oracle's exactly rounded sums, for every strategy and run.
"""
import numpy as np
import pytest
import torch

import datagen as dg
import oracle
import paper_2606_10030_gb300 as agg

pytestmark = pytest.mark.gpu

STRATS = [agg.AGG_STRAT_SMEM, agg.AGG_STRAT_GLOBAL, agg.AGG_STRAT_SORT, agg.AGG_STRAT_AUTO]
NP = {"f32": np.float32, "f64": np.float64}


@pytest.fixture(scope="module", autouse=True)
def _build():
    agg.build()
    agg.lib()


def make(case: str, dt: str, seed: int = 3):
    rng = np.random.default_rng(seed)
    if case == "few":
        keys = dg.keys_uniform(300_007, 16, seed)
        vals = dg.values(dt, keys.size, seed + 1)
    elif case == "many":
        keys = dg.keys_uniform((1 << 20) + 17, 50_000, seed)
        vals = dg.values(dt, keys.size, seed + 1)
    elif case == "zipf":
        keys = dg.keys_zipf(400_009, 100_000, 1.0, seed)
        vals = dg.values(dt, keys.size, seed + 1)
    elif case == "wide":  # exponents over a wide range inside each group
        keys = dg.keys_uniform(200_003, 300, seed)
        e = rng.integers(-100, 100, keys.size) if dt == "f32" else rng.integers(-600, 600, keys.size)
        vals = rng.standard_normal(keys.size) * np.exp2(e.astype(np.float64))
    elif case == "cancel":  # each group's rows cancel except a small residue
        base = dg.keys_uniform(100_000, 1000, seed)
        x = rng.standard_normal(base.size) * 1e6
        keys = np.concatenate([base, base[::-1], base[:1000]])
        vals = np.concatenate([x, -x[::-1], np.full(1000, 2.0 ** -20)])
    elif case == "sentinel":
        keys = dg.keys_uniform(50_001, 5, seed)
        keys[::3] = 0xFFFFFFFF
        keys[1::7] = 0
        vals = dg.values(dt, keys.size, seed + 1)
    else:
        raise ValueError(case)
    return keys.astype(np.uint32), np.asarray(vals).astype(NP[dt])


def run(keys, vals, strategy, ops=agg.AGG_ALL, flags=agg.AGG_FLAG_EXACT_SUM):
    g = agg.agg_groupby(torch.from_numpy(keys).cuda(), torch.from_numpy(vals).cuda(), ops,
                        agg.options(strategy, flags=flags))
    res = g.to_host()
    g.free()
    return res


def bits(a):
    return np.asarray(a, dtype=np.float64).view(np.int64)


@pytest.mark.parametrize("strategy", STRATS)
@pytest.mark.parametrize("dt", ["f32", "f64"])
@pytest.mark.parametrize("case", ["few", "many", "zipf", "wide", "cancel", "sentinel"])
def test_exact_sums_match_the_oracle_bit_for_bit(case, dt, strategy):
    keys, vals = make(case, dt)
    ref = oracle.groupby(keys, vals)
    res = run(keys, vals, strategy)
    assert np.array_equal(res["keys"], ref.keys)
    assert np.array_equal(res["count"], ref.count)
    assert np.array_equal(bits(res["sum"]), bits(ref.sum))
    assert np.array_equal(bits(res["avg"]), bits(ref.avg))
    assert np.array_equal(bits(res["min"]), bits(ref.min))
    assert np.array_equal(bits(res["max"]), bits(ref.max))


def test_exact_sums_are_identical_across_runs_and_strategies():
    keys, vals = make("zipf", "f32", seed=8)
    first = run(keys, vals, agg.AGG_STRAT_GLOBAL)
    for s in STRATS:
        for _ in range(2):
            r = run(keys, vals, s)
            assert np.array_equal(bits(r["sum"]), bits(first["sum"]))


@pytest.mark.parametrize("ops", [agg.AGG_SUM, agg.AGG_AVG, agg.AGG_SUM | agg.AGG_COUNT])
def test_exact_sums_with_a_subset_of_ops(ops):
    keys, vals = make("few", "f64", seed=4)
    ref = oracle.groupby(keys, vals)
    res = run(keys, vals, agg.AGG_STRAT_SMEM, ops=ops)
    if ops & agg.AGG_SUM:
        assert np.array_equal(bits(res["sum"]), bits(ref.sum))
    if ops & agg.AGG_AVG:
        assert np.array_equal(bits(res["avg"]), bits(ref.avg))


def test_exact_flag_on_an_all_zero_column():
    keys = dg.keys_uniform(10_007, 9, 1).astype(np.uint32)
    vals = np.zeros(keys.size, dtype=np.float64)
    vals[::2] = -0.0
    res = run(keys, vals, agg.AGG_STRAT_SORT)
    assert np.all(bits(res["sum"]) == 0)  # +0.0, the exact sum


def test_exact_flag_leaves_integer_columns_unchanged():
    keys = dg.keys_uniform(100_003, 500, 2).astype(np.uint32)
    vals = np.random.default_rng(2).integers(-(2 ** 40), 2 ** 40, keys.size)
    a = run(keys, vals, agg.AGG_STRAT_GLOBAL)
    b = run(keys, vals, agg.AGG_STRAT_GLOBAL, flags=0)
    assert np.array_equal(a["sum"], b["sum"]) and np.array_equal(bits(a["avg"]), bits(b["avg"]))


def test_exact_flag_rejects_non_finite_values():
    keys = dg.keys_uniform(5_001, 3, 1).astype(np.uint32)
    vals = np.ones(keys.size, dtype=np.float32)
    vals[1234] = np.inf
    with pytest.raises(agg.AggError) as e:
        run(keys, vals, agg.AGG_STRAT_SMEM)
    assert e.value.status == agg.AGG_ERR_INVALID


def test_exact_flag_rejected_on_the_host_path():
    keys = dg.keys_uniform(1000, 3, 1).astype(np.uint32)
    vals = np.ones(keys.size, dtype=np.float64)
    with pytest.raises(agg.AggError) as e:
        agg.agg_groupby_host(torch.from_numpy(keys), torch.from_numpy(vals), agg.AGG_ALL,
                             agg.options(agg.AGG_STRAT_AUTO, flags=agg.AGG_FLAG_EXACT_SUM))
    assert e.value.status == agg.AGG_ERR_INVALID


@pytest.mark.parametrize("strategy", STRATS)
@pytest.mark.parametrize("dt", ["f32", "f64"])
@pytest.mark.parametrize("case", ["many", "zipf", "wide", "cancel"])
def test_sum_error_is_the_distance_from_the_oracles_sum(strategy, dt, case):
    """AGG_FLAG_SUM_ERROR keeps the strategy's sums and reports |sum - oracle sum| per group."""
    keys, vals = make(case, dt)
    res = run(keys, vals, strategy, flags=agg.AGG_FLAG_SUM_ERROR)
    ref = oracle.groupby(keys, vals)
    assert np.array_equal(res["keys"], ref.keys)
    assert np.array_equal(res["sum_err"].view(np.int64), np.abs(res["sum"] - ref.sum).view(np.int64))
    # and the sums kept are the strategy's own (within the bar, not replaced)
    plain = run(keys, vals, strategy, flags=0)
    assert "sum_err" not in plain
    a = oracle.groupby(keys, np.abs(vals)).sum
    assert np.all(res["sum_err"] <= 1e-6 * np.maximum(np.abs(ref.sum), 2.0 ** -24 * a))


def test_sum_error_with_exact_sums_is_zero():
    keys, vals = make("zipf", "f32")
    res = run(keys, vals, agg.AGG_STRAT_AUTO, flags=agg.AGG_FLAG_SUM_ERROR | agg.AGG_FLAG_EXACT_SUM)
    ref = oracle.groupby(keys, vals)
    assert np.array_equal(res["sum"].view(np.int64), ref.sum.view(np.int64))
    assert np.all(res["sum_err"] == 0.0)


def test_sum_error_is_absent_for_integer_columns():
    keys = dg.keys_uniform(10_000, 30, 1)
    vals = dg.values("i64", keys.size, 1)
    g = agg.agg_groupby(torch.from_numpy(keys).cuda(), torch.from_numpy(vals).cuda(), agg.AGG_ALL,
                        agg.options(flags=agg.AGG_FLAG_SUM_ERROR))
    assert not g.has_sum_err
    g.free()
