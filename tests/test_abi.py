"""The C-ABI library loads, exports every entry point declared in include/*.h,
and rejects bad arguments before touching the GPU (no GPU needed)."""
import ctypes
import glob
import os
import re

import pytest

import paper_2606_10030_gb300 as agg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        names += re.findall(r"^[A-Za-z_][\w \*]*?\b(agg_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def L():
    agg.build()
    return agg.lib()


def test_header_declares_entry_points():
    names = declared_functions()
    assert "agg_reduce" in names and "agg_reduce_host" in names and "agg_last_error" in names


def test_every_declared_symbol_is_exported(L):
    for name in declared_functions():
        assert hasattr(L, name), name
        assert name in agg.SIGNATURES, f"binding lacks {name}"


def test_version(L):
    assert L.agg_version() == 101


def test_reduce_rejects_bad_arguments_without_launching(L):
    p = ctypes.c_void_p(0x1000)
    out = ctypes.c_void_p(0x2000)
    assert L.agg_reduce(p, 10, 9, agg.AGG_SUM, out, None) == agg.AGG_ERR_INVALID
    assert "dtype" in agg.last_error()
    assert L.agg_reduce(p, 10, agg.AGG_I32, 0, out, None) == agg.AGG_ERR_INVALID
    assert L.agg_reduce(p, 10, agg.AGG_I32, 64, out, None) == agg.AGG_ERR_INVALID
    assert L.agg_reduce(p, -1, agg.AGG_I32, agg.AGG_SUM, out, None) == agg.AGG_ERR_INVALID
    assert L.agg_reduce(None, 10, agg.AGG_I32, agg.AGG_SUM, out, None) == agg.AGG_ERR_INVALID
    assert L.agg_reduce(p, 10, agg.AGG_I32, agg.AGG_SUM, None, None) == agg.AGG_ERR_INVALID
    assert L.agg_reduce(ctypes.c_void_p(0x1002), 10, agg.AGG_I32, agg.AGG_SUM, out, None) == agg.AGG_ERR_INVALID
    assert "aligned" in agg.last_error()
    assert L.agg_reduce_host(p, 10, agg.AGG_F64, 0, out, None) == agg.AGG_ERR_INVALID


def test_scalar_struct_layout():
    assert agg.SCALAR_BYTES == 80


def test_groupby_batch_and_network_reject_bad_arguments_without_launching(L):
    out = ctypes.c_void_p()
    k = ctypes.c_void_p(0x1000)
    v = ctypes.c_void_p(0x2000)
    assert L.agg_groupby(k, v, 10, 7, agg.AGG_SUM, None, ctypes.byref(out), None) == agg.AGG_ERR_INVALID
    assert L.agg_groupby(k, v, 10, agg.AGG_I32, 0, None, ctypes.byref(out), None) == agg.AGG_ERR_INVALID
    assert L.agg_groupby(k, v, 1 << 32, agg.AGG_I32, agg.AGG_SUM, None, ctypes.byref(out), None) == agg.AGG_ERR_INVALID
    assert "2^32" in agg.last_error()
    assert L.agg_groupby(None, v, 10, agg.AGG_I32, agg.AGG_SUM, None, ctypes.byref(out), None) == agg.AGG_ERR_INVALID
    assert L.agg_groupby(k, v, 10, agg.AGG_I32, agg.AGG_SUM, None, None, None) == agg.AGG_ERR_INVALID
    assert L.agg_groupby(ctypes.c_void_p(0x1002), v, 10, agg.AGG_I32, agg.AGG_SUM, None, ctypes.byref(out),
                         None) == agg.AGG_ERR_INVALID
    assert L.agg_groupby(k, ctypes.c_void_p(0x2004), 10, agg.AGG_I64, agg.AGG_SUM, None, ctypes.byref(out),
                         None) == agg.AGG_ERR_INVALID
    for bad in [dict(strategy=9), dict(table_slots=1000), dict(smem_slots=100), dict(smem_slots=16384),
                dict(block_threads=100), dict(blocks_per_sm=-1)]:
        o = agg.options(**bad) if "strategy" not in bad else agg.options(bad["strategy"])
        assert L.agg_groupby(k, v, 10, agg.AGG_I32, agg.AGG_SUM, ctypes.byref(o), ctypes.byref(out),
                             None) == agg.AGG_ERR_INVALID, bad
    o = agg.options(flags=4)
    assert L.agg_groupby(k, v, 10, agg.AGG_F32, agg.AGG_SUM, ctypes.byref(o), ctypes.byref(out),
                         None) == agg.AGG_ERR_INVALID
    assert "flags" in agg.last_error()
    for kw in (dict(items_per_thread=5), dict(tile_rows=1000), dict(tile_rows=1 << 17)):
        o = agg.options(**kw)
        assert L.agg_groupby(k, v, 10, agg.AGG_I32, agg.AGG_SUM, ctypes.byref(o), ctypes.byref(out),
                             None) == agg.AGG_ERR_INVALID, kw
    for f in (agg.AGG_FLAG_EXACT_SUM, agg.AGG_FLAG_SUM_ERROR):  # the exact float sums read device columns
        o = agg.options(flags=f)
        assert L.agg_groupby_host(k, v, 10, agg.AGG_F32, agg.AGG_SUM, ctypes.byref(o), ctypes.byref(out),
                                  None) == agg.AGG_ERR_INVALID
    assert L.agg_groupby_host(k, v, 10, 9, agg.AGG_SUM, None, ctypes.byref(out), None) == agg.AGG_ERR_INVALID
    assert L.agg_sketch(k, 10, 9, agg.AGG_SUM, 0, v, None) == agg.AGG_ERR_INVALID
    assert L.agg_sketch(k, 10, agg.AGG_I32, agg.AGG_SUM, 0, None, None) == agg.AGG_ERR_INVALID
    r = agg.AggTuneResult()
    assert L.agg_autotune(k, v, 0, agg.AGG_I32, agg.AGG_SUM, 1, ctypes.byref(r), None) == agg.AGG_ERR_INVALID
    assert L.agg_groups_to_host(None, None, None, None, None, None, None, None) == agg.AGG_ERR_INVALID
    # batches
    q = (agg.AggQuery * 2)()
    q[0].keys, q[0].vals, q[0].n, q[0].dtype, q[0].ops = 0x1000, 0x2000, 10, agg.AGG_I32, agg.AGG_SUM
    q[1].keys, q[1].vals, q[1].n, q[1].dtype, q[1].ops = 0x1000, 0x2000, 10, 11, agg.AGG_SUM
    plan = ctypes.c_void_p()
    assert L.agg_batch_plan_create(q, 2, ctypes.byref(plan), None) == agg.AGG_ERR_INVALID
    assert "query 1" in agg.last_error()
    assert L.agg_batch_plan_create(q, 70000, ctypes.byref(plan), None) == agg.AGG_ERR_INVALID
    assert L.agg_batch_run(None, None) == agg.AGG_ERR_INVALID
    # network
    f = ctypes.c_void_p(0x3000)
    assert L.agg_mlp_grad(f, None, None, f, f, 0, f, f, None) == agg.AGG_ERR_INVALID
    assert L.agg_mlp_grad(f, None, None, f, f, 257, f, f, None) == agg.AGG_ERR_INVALID
    assert L.agg_mlp_grad(f, f, None, f, f, 10, f, f, None) == agg.AGG_ERR_INVALID
    assert L.agg_mlp_adam(f, f, f, f, 0, 1e-3, 0.9, 0.999, 1e-8, None) == agg.AGG_ERR_INVALID
    import numpy as np
    p = np.zeros(5443, np.float32)
    z = np.zeros(16, np.float32)
    assert L.agg_selector_set(p.ctypes.data_as(ctypes.c_void_p), z.ctypes.data_as(ctypes.c_void_p),
                              z.ctypes.data_as(ctypes.c_void_p)) == agg.AGG_ERR_INVALID
    assert "std" in agg.last_error()


def test_rule_strategy_is_a_host_call(L):
    import numpy as np
    f = np.zeros(16, np.float32)
    f[0] = 20
    f[4] = 1024 / 4096
    f[5] = 0.0
    f[6] = 0.1
    f[12] = 10
    assert agg.agg_rule_strategy(f, agg.AGG_SUM) == agg.AGG_STRAT_SMEM
    # all-distinct sample: a flat column whose key count the sample leaves open
    f[4], f[5], f[6], f[8], f[12] = 1.0, 1.0, 0.0, 8 / 4096, 21
    assert agg.agg_rule_strategy(f, agg.AGG_SUM) == agg.AGG_STRAT_SORT
    f[0] = 16  # ... on a small column: one global table
    assert agg.agg_rule_strategy(f, agg.AGG_SUM) == agg.AGG_STRAT_GLOBAL
    # flat with repeats (about 65536 keys, f2 well above 2): partitioned shared-memory build
    f[0], f[4], f[5], f[6], f[8], f[12] = 28, 3970 / 4096, 3846 / 4096, 124 / 4096, 17 / 4096, 20
    assert agg.agg_rule_strategy(f, agg.AGG_SUM) == agg.AGG_STRAT_SMEM
    # flat with few repeats (Chao1 about 7e5): sort below 2^28 rows, partitioned tables from there on
    f[5], f[6] = 4060 / 4096, 11 / 4096
    assert agg.agg_rule_strategy(f, agg.AGG_SUM) == agg.AGG_STRAT_SMEM
    f[0] = 26
    assert agg.agg_rule_strategy(f, agg.AGG_SUM) == agg.AGG_STRAT_SORT
    f[0], f[5], f[6] = 28, 3846 / 4096, 124 / 4096
    # skewed and far from covered, on 2^28 rows: partitioned shared-memory build
    f[8] = 0.2
    assert agg.agg_rule_strategy(f, agg.AGG_SUM) == agg.AGG_STRAT_SMEM
    # ... on 2^22 rows the partition pass does not pay: sort
    f[0] = 22
    assert agg.agg_rule_strategy(f, agg.AGG_SUM) == agg.AGG_STRAT_SORT
    # ... on a small column: shared-memory tables keep the hot keys
    f[0] = 16
    assert agg.agg_rule_strategy(f, agg.AGG_SUM) == agg.AGG_STRAT_SMEM
    # a hot head covering 94 % of the mass and a long tail, on 2^30 rows: sort
    f[0], f[4], f[5], f[6], f[8] = 30, 400 / 4096, 250 / 4096, 60 / 4096, 0.65
    assert agg.agg_rule_strategy(f, agg.AGG_SUM) == agg.AGG_STRAT_SORT
    # a skewed sample of a small domain (most seen keys repeat): shared-memory tables
    f[4], f[5], f[6], f[8] = 900 / 4096, 200 / 4096, 200 / 4096, 0.1
    assert agg.agg_rule_strategy(f, agg.AGG_SUM) == agg.AGG_STRAT_SMEM
    # a sample covering 98 % of the mass of a large column: shared-memory tables
    f[0], f[4], f[5], f[6], f[8] = 28, 2000 / 4096, 80 / 4096, 200 / 4096, 0.01
    assert agg.agg_rule_strategy(f, agg.AGG_SUM) == agg.AGG_STRAT_SMEM


def test_multi_rejects_bad_arguments_without_launching(L):
    k = ctypes.c_void_p(0x1000)
    cols = (agg.AggColumn * 5)()
    for c in cols:
        c.data, c.dtype, c.ops = 0x2000, agg.AGG_I64, agg.AGG_SUM
    out = ctypes.c_void_p()
    ok_args = lambda **kw: dict(dict(lo=k, hi=None, n=10, cols=cols, ncols=1, filt=None, out=ctypes.byref(out)), **kw)  # noqa: E731

    def call(**kw):
        a = ok_args(**kw)
        return L.agg_groupby_multi(a["lo"], a["hi"], a["n"], a["cols"], a["ncols"], a["filt"], a["out"], None)

    assert call(ncols=0) == agg.AGG_ERR_INVALID
    assert call(ncols=5) == agg.AGG_ERR_INVALID
    assert call(n=-1) == agg.AGG_ERR_INVALID
    assert call(lo=None) == agg.AGG_ERR_INVALID
    assert call(lo=ctypes.c_void_p(0x1002)) == agg.AGG_ERR_INVALID
    assert call(out=None) == agg.AGG_ERR_INVALID
    cols[0].dtype = 9
    assert call() == agg.AGG_ERR_INVALID and "dtype" in agg.last_error()
    cols[0].dtype, cols[0].ops = agg.AGG_I64, 0
    assert call() == agg.AGG_ERR_INVALID and "ops" in agg.last_error()
    cols[0].ops = agg.AGG_SUM
    cols[0].data = 0x2004  # not 8-byte aligned for int64
    assert call() == agg.AGG_ERR_INVALID
    cols[0].data = 0x2000
    r = agg.AggRange()
    r.data, r.dtype = 0x3000, 11
    assert call(filt=ctypes.byref(r)) == agg.AGG_ERR_INVALID
    assert L.agg_multi_to_host(None, None, None, 0, None, None, None, None) == agg.AGG_ERR_INVALID
    L.agg_multi_free(None)
