"""The NVML energy counter on the GPU: it can be read, and it grows over half a second of scans."""
import time

import pytest
import torch

import paper_2606_10030_gb300 as agg
from datagen import cuda as dgc

pytestmark = pytest.mark.gpu


def test_energy_counter_grows_under_load():
    agg.build()
    col = dgc.values("i32", 1 << 28, 0)
    out = torch.empty(agg.SCALAR_BYTES, dtype=torch.uint8, device="cuda")
    torch.cuda.synchronize()
    e0 = agg.agg_energy_counter(torch.cuda.current_device())
    t0 = time.perf_counter()
    while time.perf_counter() - t0 < 0.5:
        for _ in range(20):
            agg.agg_reduce(col, agg.AGG_ALL, out=out)
        torch.cuda.synchronize()
    e1 = agg.agg_energy_counter(torch.cuda.current_device())
    # a GB300 draws well over 50 W even when idle: at least 25 J over half a second
    assert e1 - e0 >= 25_000, (e0, e1)
