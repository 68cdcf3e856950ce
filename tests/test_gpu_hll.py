"""HyperLogLog distinct estimate on the GPU against its oracle, and the plans it sizes."""
import numpy as np
import pytest
import torch

import datagen as dg
import oracle
import paper_2606_10030_gb300 as agg
from oracle.sketch import hll_estimate

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _build():
    agg.build()
    agg.lib()


def _cases():
    yield "empty", np.zeros(0, np.uint32)
    yield "one", np.array([7], np.uint32)
    yield "few", dg.keys_uniform(1_000_003, 1000, 1)
    yield "many", dg.keys_uniform(3_000_017, 1 << 20, 2)
    yield "zipf", dg.keys_zipf(2_000_003, 1 << 18, 1.2, 3)
    yield "distinct", np.arange(5_000_000, dtype=np.uint32) * np.uint32(2654435761)
    yield "sentinel", np.where(np.arange(100_001) % 3 == 0, 0xFFFFFFFF, np.arange(100_001)).astype(np.uint32)


@pytest.mark.parametrize("name,keys", list(_cases()))
@pytest.mark.parametrize("off", [0, 1, 3])
def test_distinct_estimate_matches_the_oracle(name, keys, off):
    k = keys[off:] if keys.size > off else keys
    got = agg.agg_distinct_estimate(torch.from_numpy(np.ascontiguousarray(k)).cuda())
    ref = hll_estimate(k)
    assert abs(got - ref) <= 1e-9 * max(1.0, ref), (got, ref)


@pytest.mark.parametrize("s", [1.0, 1.5])
def test_plans_from_the_count_need_no_regrowth(s):
    """A skewed column of 2^23 rows whose sample misses most of its 2^16 keys: the table is
    sized from the count (no regrowth), and every strategy returns the oracle's groups."""
    n, D = 1 << 23, 1 << 16
    keys = dg.keys_zipf(n, D, s, 5)
    vals = dg.values("i64", n, 5)
    k, v = torch.from_numpy(keys).cuda(), torch.from_numpy(vals).cuda()
    ref = oracle.groupby(keys, vals)
    for strategy in (agg.AGG_STRAT_AUTO, agg.AGG_STRAT_SMEM, agg.AGG_STRAT_GLOBAL):
        g = agg.agg_groupby(k, v, agg.AGG_ALL, agg.options(strategy))
        assert g.retries == 0 and g.table_slots <= 4 * D
        res = g.to_host()
        g.free()
        assert np.array_equal(res["keys"], ref.keys) and np.array_equal(res["count"], ref.count)
        assert np.array_equal(res["sum"], ref.sum) and np.array_equal(res["min"], ref.min)
        assert np.array_equal(res["max"], ref.max)


@pytest.mark.parametrize("strategy", [agg.AGG_STRAT_AUTO, agg.AGG_STRAT_LEARNED, agg.AGG_STRAT_SMEM])
@pytest.mark.parametrize("off", [0, 3])
def test_partition_counts_from_the_count_pass(strategy, off):
    """The distinct-count pass also counts each hash partition's rows, and the one-level
    partition then skips its own histogram: a ragged, misaligned column of about 2^22 rows
    over 2^17 keys (partitioned, counted) gives the oracle's groups."""
    n, D = (1 << 22) + 7, 1 << 17
    keys, vals = dg.keys_uniform(n, D, 11), dg.values("i64", n, 12)
    k, v = torch.from_numpy(keys).cuda()[off:], torch.from_numpy(vals).cuda()[off:]  # off: not 16-byte aligned
    ref = oracle.groupby(keys[off:], vals[off:])
    g = agg.agg_groupby(k, v, agg.AGG_ALL, agg.options(strategy, partition=1))
    res = g.to_host()
    g.free()
    assert np.array_equal(res["keys"], ref.keys) and np.array_equal(res["count"], ref.count)
    assert np.array_equal(res["sum"], ref.sum) and np.array_equal(res["min"], ref.min)
    assert np.array_equal(res["max"], ref.max)
