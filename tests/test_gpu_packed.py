"""Scans of frame-of-reference bit-packed columns (on device and end to end) against the oracle."""
import numpy as np
import pytest
import torch

import datagen as dg
import oracle
import paper_2606_10030_gb300 as agg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _build():
    agg.build()
    agg.lib()


def columns():
    rng = np.random.default_rng(1)
    for n in (0, 1, 1023, 1024, 1025, 3_000_007):
        yield f"narrow{n}", dg.values("i32", n, 2)  # uniform in [-2^20, 2^20): 21 bits a value
    yield "full_i64", rng.integers(-(2 ** 63), 2 ** 63 - 1, 400_000, dtype=np.int64, endpoint=True)
    yield "u32", rng.integers(0, 2 ** 32, 500_001, dtype=np.uint64).astype(np.uint32)
    yield "i64_0_2p32", dg.values("i64", 1_000_003, 3)
    yield "constant", np.full(70_000, -123456789, dtype=np.int64)
    runs = np.repeat(rng.integers(-1000, 1000, 300), 1000).astype(np.int32)
    yield "runs", runs
    yield "extremes", np.array([np.iinfo(np.int32).min, np.iinfo(np.int32).max] * 5000, dtype=np.int32)


def same(got: dict, ref: dict, ops):
    assert got["count"] == ref["count"]
    if ops & (agg.AGG_SUM | agg.AGG_AVG):
        assert got["sum"] == ref["sum"]
        assert np.float64(got["avg"]).tobytes() == np.float64(ref["avg"]).tobytes()
    if ops & (agg.AGG_MIN | agg.AGG_MAX):
        assert got["min"] == ref["min"] and got["max"] == ref["max"]


@pytest.mark.parametrize("name,x", list(columns()))
@pytest.mark.parametrize("ops", [agg.AGG_ALL, agg.AGG_SUM, agg.AGG_MIN | agg.AGG_MAX])
def test_packed_scans_match_the_oracle(name, x, ops):
    ref = oracle.reduce(x)
    p = agg.agg_pack_for(torch.from_numpy(x))
    same(agg.agg_reduce_packed_host(p, ops).as_dict(), ref, ops)
    dev = p.to("cuda")
    same(agg.decode_scalar(agg.agg_reduce_packed(dev, ops)).as_dict(), ref, ops)


def test_packed_host_scan_over_many_chunks():
    """2^26 + 5 int32 rows: several 16 Mi-value chunks through the copy ring."""
    x = dg.values("i32", (1 << 26) + 5, 4)
    p = agg.agg_pack_for(torch.from_numpy(x))
    assert p.nbytes < 0.7 * x.nbytes  # 21 of 32 bits
    same(agg.agg_reduce_packed_host(p, agg.AGG_ALL).as_dict(), oracle.reduce(x), agg.AGG_ALL)
