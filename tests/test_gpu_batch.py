"""Batched GROUP BY (persistent kernel + CUDA graph) against the CPU oracle."""
import numpy as np
import pytest
import torch

import datagen as dg
import paper_2606_10030_gb300 as agg
from datagen import cuda as dgc
from tests.test_gpu_groupby import check_groups

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _build():
    agg.build()
    agg.lib()


def _queries(nq, seed, log2_rows=(10, 18), log2_keys=(0, 16), strategies=(agg.AGG_STRAT_AUTO,)):
    qs = dg.batch_queries(nq, seed, log2_rows=log2_rows, log2_keys=log2_keys)
    out = []
    for i, q in enumerate(qs):
        k, v = dgc.group_column(q)
        out.append((k, v, q.ops, strategies[i % len(strategies)]))
    return out


def _check_all(plan, queries):
    for i, (k, v, ops, _) in enumerate(queries):
        g = plan.result(i)
        res = g.to_host()
        g.free()
        check_groups(res, k.cpu().numpy(), v.cpu().numpy(), ops)


@pytest.mark.parametrize("strategies", [(agg.AGG_STRAT_AUTO,), (agg.AGG_STRAT_SMEM,), (agg.AGG_STRAT_GLOBAL,),
                                        (agg.AGG_STRAT_SMEM, agg.AGG_STRAT_GLOBAL, agg.AGG_STRAT_SORT,
                                         agg.AGG_STRAT_LEARNED)])
def test_batch_matches_oracle(strategies):
    queries = _queries(40, 3, strategies=strategies)
    plan = agg.BatchPlan(queries)
    plan.run()
    _check_all(plan, queries)
    plan.free()


def test_batch_replays_the_graph_on_new_inputs():
    queries = _queries(24, 5, log2_keys=(4, 18))
    plan = agg.BatchPlan(queries)
    plan.run()
    _check_all(plan, queries)
    # overwrite the inputs in place: a replay recomputes from them
    for i, (k, v, ops, _) in enumerate(queries):
        v.copy_(torch.flip(v, [0]))
        k.copy_(torch.roll(k.view(torch.int32), 7).view(torch.uint32))
    plan.run()
    _check_all(plan, queries)
    plan.run()
    _check_all(plan, queries)
    plan.free()


def test_batch_with_empty_tiny_and_sentinel_queries():
    rng = np.random.default_rng(0)
    specs = []
    for n, dt in [(0, "i32"), (1, "f64"), (5, "u32"), (65536, "i64"), (65537, "f32"), (200_000, "i64")]:
        keys = dg.keys_uniform(n, max(1, n // 3), 9) if n else np.array([], np.uint32)
        if n > 3:
            keys[::5] = 0xFFFFFFFF
        vals = dg.values(dt, n, 9) if n else np.array([], dg.DTYPES[dt])
        specs.append((torch.from_numpy(keys).cuda(), torch.from_numpy(vals).cuda(), agg.AGG_ALL,
                      agg.AGG_STRAT_AUTO))
    plan = agg.BatchPlan(specs)
    plan.run()
    _check_all(plan, specs)
    plan.free()


def test_batch_regrows_a_table_the_sketch_undersized():
    # 99% of rows on one key, 1% spread over many distinct keys: the sample
    # covers the mass, so the estimate is small and the first table overflows
    n = 2_000_000
    keys = np.full(n, 12345, dtype=np.uint32)
    idx = np.arange(0, n, 100)
    keys[idx] = dg.domain_keys(3, np.arange(idx.size))
    vals = dg.values("i64", n, 3)
    q = [(torch.from_numpy(keys).cuda(), torch.from_numpy(vals).cuda(), agg.AGG_ALL, agg.AGG_STRAT_GLOBAL)]
    plan = agg.BatchPlan(q)
    plan.run()
    _check_all(plan, q)
    plan.free()


def test_batch_result_outlives_the_plan():
    queries = _queries(6, 8)
    plan = agg.BatchPlan(queries)
    plan.run()
    gs = [plan.result(i) for i in range(len(queries))]
    plan.free()
    for (k, v, ops, _), g in zip(queries, gs):
        check_groups(g.to_host(), k.cpu().numpy(), v.cpu().numpy(), ops)
        g.free()


def test_batch_tune_picks_a_tile_and_keeps_results():
    import oracle
    qs = dg.batch_queries(24, 5, log2_rows=(12, 20), log2_keys=(0, 16))
    cols = [dgc.group_column(q) for q in qs]
    plan = agg.BatchPlan([(k, v, q.ops, agg.AGG_STRAT_AUTO) for (k, v), q in zip(cols, qs)])
    tile = plan.tune(1)
    assert tile in (16384, 32768, 65536)
    plan.run()
    for i, ((k, v), q) in enumerate(zip(cols, qs)):
        g = plan.result(i)
        res = g.to_host()
        g.free()
        ref = oracle.groupby(k.cpu().numpy(), v.cpu().numpy())
        assert np.array_equal(res["keys"], ref.keys) and np.array_equal(res["count"], ref.count)
    plan.free()
