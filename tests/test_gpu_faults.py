"""Failure paths, injected on the host (no GPU fault): every device allocation
the library makes can fail; the call must report AGG_ERR_OOM, and later calls
must work and be correct."""
import numpy as np
import pytest
import torch

import datagen as dg
import paper_2606_10030_gb300 as agg
from tests.test_gpu_groupby import check_groups

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _build():
    agg.build()
    agg.lib()
    yield
    agg.lib().agg_debug_fail_alloc(0)


def _cols(n=300_000, D=60_000, dt="i64"):
    k = dg.keys_uniform(n, D, 4)
    v = dg.values(dt, n, 4)
    return k, v, torch.from_numpy(k).cuda(), torch.from_numpy(v).cuda()


@pytest.mark.parametrize("strategy", [agg.AGG_STRAT_SMEM, agg.AGG_STRAT_GLOBAL, agg.AGG_STRAT_SORT])
def test_groupby_reports_every_failed_allocation(strategy):
    k, v, kd, vd = _cols()
    L = agg.lib()
    failures = 0
    for countdown in range(1, 12):
        L.agg_debug_fail_alloc(countdown)
        try:
            g = agg.agg_groupby(kd, vd, agg.AGG_ALL, agg.options(strategy, partition=1))
            g.free()
        except agg.AggError as e:
            assert e.status == agg.AGG_ERR_OOM, e
            failures += 1
        L.agg_debug_fail_alloc(0)
        torch.cuda.synchronize()
        g = agg.agg_groupby(kd, vd, agg.AGG_ALL, agg.options(strategy))
        check_groups(g.to_host(), k, v)
        g.free()
    assert failures >= 1


def test_batch_and_training_report_failed_allocations():
    k, v, kd, vd = _cols(100_000, 5000, "f32")
    L = agg.lib()
    for countdown in range(1, 6):
        L.agg_debug_fail_alloc(countdown)
        try:
            plan = agg.BatchPlan([(kd, vd, agg.AGG_ALL, agg.AGG_STRAT_AUTO)] * 3)
            plan.run()
            plan.free()
        except agg.AggError as e:
            assert e.status == agg.AGG_ERR_OOM
        L.agg_debug_fail_alloc(0)
    plan = agg.BatchPlan([(kd, vd, agg.AGG_ALL, agg.AGG_STRAT_AUTO)] * 3)
    plan.run()
    for i in range(3):
        g = plan.result(i)
        check_groups(g.to_host(), k, v)
        g.free()
    plan.free()
    X = torch.randn(300, 16, device="cuda")
    y = torch.randint(0, 3, (300,), device="cuda", dtype=torch.int32)
    p = torch.zeros(agg.lib().agg_mlp_param_count(), device="cuda")
    m, vv = torch.zeros_like(p), torch.zeros_like(p)
    L.agg_debug_fail_alloc(1)
    with pytest.raises(agg.AggError) as ei:
        agg.agg_mlp_train(p, m, vv, X, y, epochs=1)
    assert ei.value.status == agg.AGG_ERR_OOM
    L.agg_debug_fail_alloc(0)
    agg.agg_mlp_train(p, m, vv, X, y, epochs=1)


def test_reduce_host_reports_failed_allocation():
    x = dg.values("i32", 1 << 22, 1)
    L = agg.lib()
    torch.cuda.synchronize()
    s = torch.cuda.Stream()  # a new stream needs new scratch, so the allocation happens
    L.agg_debug_fail_alloc(1)
    with pytest.raises(agg.AggError) as ei:
        agg.agg_reduce_host(torch.from_numpy(x).pin_memory(), agg.AGG_ALL, stream=s)
    assert ei.value.status == agg.AGG_ERR_OOM
    L.agg_debug_fail_alloc(0)
    r = agg.agg_reduce_host(torch.from_numpy(x).pin_memory(), agg.AGG_ALL, stream=s).as_dict()
    assert r["sum"] == int(x.astype(np.int64).sum())
