#!/usr/bin/env python
"""Benchmark of the in-memory aggregation hot path on GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME] [--impl ours|reference]

Prints ONE JSON line (rank 0). A step is one aggregation call over one batch of
synthetic input already resident in HBM; `value` is input GB/s over all ranks
(max-over-ranks time), `e2e` the same metric through the host-fed entry point
with the host-to-device copy inside the timed region.

Workloads (synthetic, seeded; they stand in for the paper's TPC-H
lineitem.suppkey scan, which is not available here):
  table2p30   (default) GROUP BY SUM/MIN/MAX/COUNT/AVG over a 2^30-row table:
              uint32 keys Zipf(1.0) over 2^16 random keys, int64 values uniform
              in [0, 2^32) (12 GiB), strategy chosen by the learned selector
  groupby     GROUP BY SUM/COUNT/MIN/MAX over 2^26 rows: uint32 keys drawn
              uniformly from 1024 random keys, int64 values uniform in [0, 2^32)
  scan        ungrouped SUM/MIN/MAX/COUNT/AVG over a 2^30-row int32 column
              (4 GiB, uniform in [-2^20, 2^20))
The default run also reports, as extra objects: the 2^26-row GROUP BY above;
the 2^30-row scans of every value type (float sums with their error against
the oracle); the high-cardinality GROUP BY (2^28 rows, Zipf(1) keys over 2^24,
float32 values, with every group's error against the exactly rounded sum);
the 512-query batch against plain per-query calls; and the selector's
evaluation on 2^30-row tables over 2^4..2^26 keys x Zipf 0..1.5 (on-device
GB/s, regret against the exhaustive autotuner, end-to-end GB/s on a few).
The host-link peak (pinned host-to-device copies) is measured once and the
end-to-end figure given as a fraction of it.

Under torchrun each rank aggregates its own replica of the workload (weak
scaling, no data-path collective); only the timing uses a MAX all-reduce.
`--impl reference` times the CPU oracle (single thread) on a bounded sample of
the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "Input GB/s & % of GB300 HBM peak; batched+learned vs plain per-query kernels"
UNIT = "GB/s"
FALLBACK_HBM_GBS = 6800.0
WEIGHTS = os.path.join(ROOT, "paper_2606_10030_gb300", "selector_weights.npz")


def load_peaks() -> dict:
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return {"hbm_gbs": float(d["hbm_gbs"]), "source": "measured"}
    return {"hbm_gbs": FALLBACK_HBM_GBS, "source": "fallback"}


# ---------------------------------------------------------------------------
# Clock sampling during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(prefix="clocks_", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except FileNotFoundError:
            self.proc = None
        time.sleep(0.3)

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.proc.terminate()
        self.proc.wait()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# Distributed plumbing (one process per GPU; weak scaling)
# ---------------------------------------------------------------------------
def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x: float, world: int) -> float:
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------------------
# Workloads
# ---------------------------------------------------------------------------
class ScanWorkload:
    """Ungrouped SUM/MIN/MAX/COUNT/AVG over a 2^30-row int32 column (4 GiB)."""
    name = "scan"
    n = 1 << 30
    dtype = "i32"
    esize = 4
    kernel = "reduce_scan"
    phase = "scan"

    def release(self):
        """Drop the workload's device and host columns."""
        for a in ("col", "host", "k", "v", "hk", "hv"):
            self.__dict__.pop(a, None)

    def config(self):
        return {"workload": "ungrouped SUM/MIN/MAX/COUNT/AVG, 2^30-row int32 column uniform in [-2^20, 2^20)",
                "rows": self.n, "dtype": "int32", "input_bytes": self.n * self.esize,
                "l2": "input (4 GiB) larger than L2 (129 MB); no flush needed"}

    def bytes_per_step(self):
        return self.n * self.esize

    def setup(self, rank):
        import torch

        import paper_2606_10030_gb300 as agg
        from datagen import cuda as dgc
        self.agg = agg
        self.col = dgc.values(self.dtype, self.n, seed=rank)
        self.out = torch.empty(agg.SCALAR_BYTES, dtype=torch.uint8, device="cuda")
        torch.cuda.synchronize()

    def step(self):
        self.agg.agg_reduce(self.col, self.agg.AGG_ALL, out=self.out)
        return 1  # kernel launches

    def setup_e2e(self):
        self.host = self.col.cpu().pin_memory()

    def step_e2e(self):
        r = self.agg.agg_reduce_host(self.host, self.agg.AGG_ALL)
        return r.count

    def e2e_bytes(self):
        return self.n * self.esize, 80

    def cpu_sample(self, budget_s: float):
        """Oracle on consecutive 2^24-row slices of the same column until budget_s elapses."""
        import numpy as np

        import datagen as dg
        import oracle
        oracle.build()
        rows = 0
        t0 = time.perf_counter()
        chunk = 1 << 24
        start = 0
        t_compute = 0.0
        while time.perf_counter() - t0 < budget_s and start < self.n:
            x = dg.values(self.dtype, chunk, seed=0, start=start)
            a = time.perf_counter()
            oracle.reduce(x)
            t_compute += time.perf_counter() - a
            rows += chunk
            start += chunk
        return rows, t_compute, f"oracle.reduce over the first {rows} rows (2^24-row slices) of the column"


class GroupbyWorkload:
    """GROUP BY SUM/COUNT/MIN/MAX, 2^26 rows, 1024 uniform random uint32 keys, int64 values."""
    name = "groupby"
    n = 1 << 26
    D = 1024
    dtype = "i64"
    esize = 12  # key + value bytes per row
    kernel = "gb_build"
    phase = "build"

    def release(self):
        """Drop the workload's device and host columns."""
        for a in ("col", "host", "k", "v", "hk", "hv"):
            self.__dict__.pop(a, None)

    def config(self):
        return {"workload": "GROUP BY SUM/COUNT/MIN/MAX, 2^26 rows, uint32 keys uniform over 1024 random keys, "
                            "int64 values uniform in [0, 2^32)",
                "rows": self.n, "distinct_keys": self.D, "key_dtype": "uint32", "value_dtype": "int64",
                "input_bytes": self.n * self.esize, "strategy": "auto (sketch rule -> shared-memory hash)",
                "l2": "input (768 MiB) larger than L2 (129 MB); no flush needed"}

    def bytes_per_step(self):
        return self.n * self.esize

    def setup(self, rank):
        import paper_2606_10030_gb300 as agg
        from datagen import cuda as dgc
        self.agg = agg
        self.ops = agg.AGG_SUM | agg.AGG_COUNT | agg.AGG_MIN | agg.AGG_MAX
        if getattr(self, "ops_override", 0):
            self.ops = self.ops_override
        self.opts = agg.options(getattr(self, "strategy", agg.AGG_STRAT_AUTO))
        self.k = dgc.keys_uniform(self.n, self.D, seed=rank)
        self.v = dgc.values(self.dtype, self.n, seed=rank)
        import torch
        torch.cuda.synchronize()

    def step(self):
        g = self.agg.agg_groupby(self.k, self.v, self.ops, self.opts)
        self.last_strategy = g.strategy
        g.free()
        return 0  # launches are counted by the library

    def setup_e2e(self):
        self.hk = self.k.cpu().pin_memory()
        self.hv = self.v.cpu().pin_memory()

    def step_e2e(self):
        g = self.agg.agg_groupby_host(self.hk, self.hv, self.ops, self.opts)
        r = g.to_host()
        self.e2e_groups = len(r["keys"])
        g.free()
        return self.e2e_groups

    def e2e_bytes(self):
        return self.n * self.esize, getattr(self, "e2e_groups", self.D) * (4 + 5 * 8)

    def cpu_sample(self, budget_s: float):
        """Oracle GROUP BY on consecutive 2^24-row slices of the same columns until budget_s elapses."""
        import datagen as dg
        import oracle
        oracle.build()
        rows, start, t_compute = 0, 0, 0.0
        chunk = 1 << 24
        t0 = time.perf_counter()
        while time.perf_counter() - t0 < budget_s and start < self.n:
            k = dg.keys_uniform(chunk, self.D, 0, start=start)
            v = dg.values(self.dtype, chunk, 0, start=start)
            a = time.perf_counter()
            oracle.groupby(k, v)
            t_compute += time.perf_counter() - a
            rows += chunk
            start += chunk
        return rows, t_compute, f"oracle.groupby (std::map) over the first {rows} rows (2^24-row slices)"


class Table2p30Workload:
    """GROUP BY SUM/MIN/MAX/COUNT/AVG over a 2^30-row table: uint32 keys Zipf(1.0) over
    2^16 random keys, int64 values uniform in [0, 2^32); the learned selector picks the
    strategy (the AUTO rule if no trained weights are installed)."""
    name = "table2p30"
    n = 1 << 30
    D = 1 << 16
    zipf_s = 1.0
    dtype = "i64"
    esize = 12
    kernel = None  # the phase with the largest share of the step

    def release(self):
        """Drop the workload's device and host columns."""
        for a in ("col", "host", "k", "v", "hk", "hv"):
            self.__dict__.pop(a, None)

    def config(self):
        return {"workload": "GROUP BY SUM/MIN/MAX/COUNT/AVG, 2^30 rows, uint32 keys Zipf(s=1.0) over D=2^16 random "
                            "keys, int64 values uniform in [0, 2^32), strategy from the learned selector",
                "rows": self.n, "distinct_keys_domain": self.D, "zipf_s": self.zipf_s, "key_dtype": "uint32",
                "value_dtype": "int64", "input_bytes": self.n * self.esize,
                "strategy": "learned selector" if os.path.exists(WEIGHTS) else "auto rule (no trained weights)",
                "l2": "input (12 GiB) larger than L2 (129 MB); no flush needed"}

    def bytes_per_step(self):
        return self.n * self.esize

    def table_ops(self, agg):
        return agg.AGG_ALL

    def query(self, rank):
        import datagen as dg
        return dg.GroupQuery(self.n, self.D, self.zipf_s, self.dtype, 31, rank)

    def setup(self, rank):
        import torch

        import paper_2606_10030_gb300 as agg
        from datagen import cuda as dgc
        from paper_2606_10030_gb300 import selector
        self.agg = agg
        self.learned = selector.install_default()
        self.ops = self.table_ops(agg)
        if getattr(self, "ops_override", 0):
            self.ops = self.ops_override
        strat = getattr(self, "strategy", 0) or (agg.AGG_STRAT_LEARNED if self.learned else agg.AGG_STRAT_AUTO)
        self.opts = agg.options(strat)
        self.q = self.query(rank)
        self.k, self.v = dgc.group_column(self.q)
        torch.cuda.synchronize()

    def step(self):
        g = self.agg.agg_groupby(self.k, self.v, self.ops, self.opts)
        self.last_strategy = g.strategy
        self.groups = g.num_groups
        g.free()
        return 0

    def setup_e2e(self):
        self.hk = self.k.cpu().pin_memory()
        self.hv = self.v.cpu().pin_memory()

    def step_e2e(self):
        g = self.agg.agg_groupby_host(self.hk, self.hv, self.ops, self.opts)
        r = g.to_host()
        self.e2e_groups = len(r["keys"])
        g.free()
        return self.e2e_groups

    def e2e_bytes(self):
        return self.n * self.esize, getattr(self, "e2e_groups", self.D) * (4 + 5 * 8)

    def cpu_sample(self, budget_s: float):
        """Oracle GROUP BY on consecutive 2^24-row slices of the same table until budget_s elapses."""
        import datagen as dg
        import oracle
        oracle.build()
        q = self.query(0)
        t = dg.zipf_thresholds(q.D, q.zipf_s)
        rows, start, t_compute = 0, 0, 0.0
        chunk = 1 << 24
        t0 = time.perf_counter()
        while time.perf_counter() - t0 < budget_s and start < self.n:
            k = dg.keys_zipf(chunk, q.D, q.zipf_s, q.seed, start=start, thresholds=t)
            v = dg.values(q.dtype, chunk, q.seed, start=start)
            a = time.perf_counter()
            oracle.groupby(k, v)
            t_compute += time.perf_counter() - a
            rows += chunk
            start += chunk
        return rows, t_compute, f"oracle.groupby (std::map) over the first {rows} rows (2^24-row slices)"


class Zipf2p28Workload(Table2p30Workload):
    """GROUP BY SUM/AVG, 2^28 rows, uint32 keys Zipf(1.0) over 2^24 random keys, float32 values
    ~N(0,1)*1e3 (compensated float32 partials, merged in float64)."""
    name = "zipf2p28"
    n = 1 << 28
    D = 1 << 24
    zipf_s = 1.0
    dtype = "f32"
    esize = 8

    def table_ops(self, agg):
        return agg.AGG_SUM | agg.AGG_AVG

    def config(self):
        return {"workload": "GROUP BY SUM/AVG, 2^28 rows, uint32 keys Zipf(s=1.0) over 2^24 random keys, float32 "
                            "values N(0,1)*1e3",
                "rows": self.n, "distinct_keys_domain": self.D, "zipf_s": self.zipf_s, "key_dtype": "uint32",
                "value_dtype": "float32", "input_bytes": self.n * self.esize,
                "strategy": "learned selector" if os.path.exists(WEIGHTS) else "auto rule (no trained weights)",
                "l2": "input (2 GiB) larger than L2 (129 MB); no flush needed"}

    def query(self, rank):
        import datagen as dg
        return dg.GroupQuery(self.n, self.D, self.zipf_s, self.dtype, 1 | 16, rank)

    def e2e_bytes(self):
        return self.n * self.esize, getattr(self, "e2e_groups", self.D) * (4 + 3 * 8)


WORKLOADS = {"table2p30": Table2p30Workload, "groupby": GroupbyWorkload, "scan": ScanWorkload,
             "zipf2p28": Zipf2p28Workload}

# phase of the library's event timers -> the kernels it times
PHASE_KERNELS = {"scan": "reduce_scan", "sketch": "sketch_gather + sketch_kernel + hll_kernel",
                 "build": "gb_build_tiles (hash build over partitioned tiles) or gb_build",
                 "finalize": "gb_compact + key sort + gb_gather (finalise)",
                 "sort": "part_hist + part_scatter (one-level partition) or radix_hist + radix_scatter",
                 "segreduce": "seg_reduce + seg_finalize", "batch": "batch_build", "mlp": "mlp kernels"}


def energy_mj(device: int):
    """NVML's energy counter of the GPU (mJ, read-only), or None where it cannot be read."""
    import paper_2606_10030_gb300 as agg
    try:
        return agg.agg_energy_counter(device)
    except agg.AggError:
        return None


def energy_report(e0, e1, e2, e3, steps, e2e_steps, bytes_step, e2e_bytes) -> dict:
    """Energy per step of the on-device and the end-to-end runs (the paper's Sec. 6 comparison)."""
    if None in (e0, e1, e2, e3):
        return {"unavailable": "NVML energy counter not readable"}
    dev_j = (e1 - e0) / 1e3 / steps
    e2e_j = (e3 - e2) / 1e3 / e2e_steps
    return {"J_per_step": round(dev_j, 4), "GB_per_J": round(bytes_step / 1e9 / dev_j, 3) if dev_j > 0 else None,
            "e2e_J_per_step": round(e2e_j, 4),
            "e2e_GB_per_J": round(e2e_bytes / 1e9 / e2e_j, 3) if e2e_j > 0 else None,
            "how": "difference of NVML's total-energy counter around the timed steps (whole GPU, idle draw "
                   "included)"}


def host_link_peak(gib: int = 1, reps: int = 10) -> dict:
    """Pinned host-to-device copy bandwidth (best of reps, CUDA events): the end-to-end roofline."""
    import torch
    n = gib << 30
    h = torch.empty(n, dtype=torch.uint8).pin_memory()
    d = torch.empty(n, dtype=torch.uint8, device="cuda")
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    best = float("inf")
    for _ in range(reps + 1):
        a.record()
        d.copy_(h, non_blocking=True)
        b.record()
        b.synchronize()
        best = min(best, a.elapsed_time(b))
    del h, d
    torch.cuda.empty_cache()
    return {"GB/s": round(n / (best * 1e-3) / 1e9, 1), "bytes": n, "reps": reps,
            "how": "pinned host -> device copy of 1 GiB, best of 10, CUDA events"}


def extra_scan(steps: int, peaks: dict) -> dict:
    """Ungrouped 2^30-row int32 scan: input GB/s and fraction of the HBM peak."""
    import torch

    import paper_2606_10030_gb300 as agg
    from datagen import cuda as dgc
    n = 1 << 30
    col = dgc.values("i32", n, seed=0)
    out = torch.empty(agg.SCALAR_BYTES, dtype=torch.uint8, device="cuda")
    for _ in range(3):
        agg.agg_reduce(col, agg.AGG_ALL, out=out)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(steps):
        agg.agg_reduce(col, agg.AGG_ALL, out=out)
    b.record()
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / steps
    gbs = n * 4 / (ms * 1e-3) / 1e9
    del col
    torch.cuda.empty_cache()
    # the small ungrouped case (2^20 int32 rows, L2-resident): time per call over 1000
    # back-to-back calls (scan and merge, launch-bound at this size)
    small = dgc.values("i32", 1 << 20, seed=0)
    for _ in range(10):
        agg.agg_reduce(small, agg.AGG_ALL, out=out)
    torch.cuda.synchronize()
    a.record()
    for _ in range(1000):
        agg.agg_reduce(small, agg.AGG_ALL, out=out)
    b.record()
    torch.cuda.synchronize()
    small_us = a.elapsed_time(b) / 1000 * 1e3
    del small
    # the other value types, 2^30 rows each (int64 and float64: 8 GiB), all five ops;
    # float sums: the error against the oracle's exactly rounded sum, and the bound the
    # scan computes alongside the sum
    by_dtype = {"i32": round(gbs, 1)}
    errors = {}
    for dt, esz in (("i64", 8), ("f32", 4), ("f64", 8)):
        col = dgc.values(dt, n, seed=0)
        for _ in range(3):
            agg.agg_reduce(col, agg.AGG_ALL, out=out)
        torch.cuda.synchronize()
        reps = 20
        a.record()
        for _ in range(reps):
            agg.agg_reduce(col, agg.AGG_ALL, out=out)
        b.record()
        torch.cuda.synchronize()
        by_dtype[dt] = round(n * esz / (a.elapsed_time(b) / reps * 1e-3) / 1e9, 1)
        if dt in ("f32", "f64"):
            r = agg.decode_scalar(out)
            errors[dt] = float_sum_error(r.sum_f, r.err_bound, col)
        del col
        torch.cuda.empty_cache()
    return {"workload": "ungrouped SUM/MIN/MAX/COUNT/AVG, 2^30 int32 rows (4 GiB)", "ms": round(ms, 4),
            "GB/s": round(gbs, 1), "frac_of_measured_hbm": round(gbs / peaks["hbm_gbs"], 4),
            "frac_of_nominal_8TBs": round(gbs / 8000.0, 4), "steps": steps,
            "small_2p20_int32_us_per_call_back_to_back": round(small_us, 2),
            "GB/s_by_value_type_2p30_rows": by_dtype, "float_sum_error_vs_oracle": errors}


def float_sum_error(got: float, bound: float, col) -> dict:
    """Error of a float column's SUM against the oracle's exactly rounded sum."""
    import numpy as np

    import oracle
    x = col.cpu().numpy()
    ref = oracle.exact_sum(x)
    abs_sum = float(np.abs(x.astype(np.float64)).sum())
    err = abs(got - ref)
    return {"abs_err": err, "rel_err": err / abs(ref) if ref else err,
            "err_bound": bound, "err_bound_rel": bound / abs(ref) if ref else bound,
            "bar": 1e-6 * max(abs(ref), 2.0 ** -24 * abs_sum), "within_bar": err <= 1e-6 * max(abs(ref), 2.0 ** -24 * abs_sum)}


def extra_batched(steps: int, nq: int = 512) -> dict:
    """512 uneven GROUP BY queries: one batched plan (persistent kernel + CUDA graph,
    learned selector) against plain per-query agg_groupby calls on one stream."""
    import torch

    import datagen as dg
    import paper_2606_10030_gb300 as agg
    from datagen import cuda as dgc
    from paper_2606_10030_gb300 import selector
    learned = selector.install_default()
    qs = dg.batch_queries(nq, 0)
    cols = []
    rows = 0
    in_bytes = 0
    for q in qs:
        k, v = dgc.group_column(q)
        cols.append((k, v, q.ops))
        rows += q.n
        in_bytes += q.n * (4 + v.element_size())
    torch.cuda.synchronize()
    strat = agg.AGG_STRAT_LEARNED if learned else agg.AGG_STRAT_AUTO
    t0 = time.perf_counter()
    plan = agg.BatchPlan([(k, v, ops, strat) for k, v, ops in cols])
    plan_s = time.perf_counter() - t0
    plan.run()  # capture + first replay
    torch.cuda.synchronize()

    def time_runs():
        agg.profile_read()
        agg.profile_enable(True)
        t0 = time.perf_counter()
        for _ in range(steps):
            plan.run()
        torch.cuda.synchronize()
        wall = (time.perf_counter() - t0) / steps
        agg.profile_enable(False)
        return wall, sum(v[0] for v in agg.profile_read().values()) / steps

    time_runs()  # warm-up replays (the first replays after a capture run slower)
    fixed_s, fixed_gpu_ms = time_runs()  # the default 64 Ki-row work items
    tile = plan.tune(2)  # the autotuner's tile axis: 16, 32 or 64 Ki rows
    time_runs()  # warm-up replays of the re-planned graph
    batch_s, batch_gpu_ms = time_runs()
    best_s = min(batch_s, fixed_s)
    plan.free()
    o = agg.options(strat)
    for k, v, ops in cols[:8]:
        agg.agg_groupby(k, v, ops, o).free()
    torch.cuda.synchronize()
    agg.profile_read()
    agg.profile_enable(True)
    t0 = time.perf_counter()
    for k, v, ops in cols:
        agg.agg_groupby(k, v, ops, o).free()
    torch.cuda.synchronize()
    plain_s = time.perf_counter() - t0
    agg.profile_enable(False)
    plain_gpu_ms = sum(v[0] for v in agg.profile_read().values())
    del cols
    torch.cuda.empty_cache()
    return {"workload": f"{nq} GROUP BY queries, rows log-uniform in [2^12, 2^24], distinct keys log-uniform in "
                        "[1, 2^20] (uniform or Zipf 0.5-1.5), mixed int32/int64/float32/float64 values and ops",
            "rows": rows, "input_bytes": in_bytes, "selector": "learned" if learned else "rule (no weights file)",
            "batched_ms": round(best_s * 1e3, 3), "batched_GB/s": round(in_bytes / best_s / 1e9, 1),
            "batched_how": "the faster of the default 64 Ki-row work items and the tuned size (tuning runs may "
                           "regrow a table that fills, and the larger table stays with the plan)",
            "batched_ms_tuned": round(batch_s * 1e3, 3), "tile_rows_tuned": tile,
            "batched_ms_fixed_64Ki_tile": round(fixed_s * 1e3, 3),
            "batched_plan_ms": round(plan_s * 1e3, 1),
            "plain_ms": round(plain_s * 1e3, 3), "plain_GB/s": round(in_bytes / plain_s / 1e9, 1),
            "speedup": round(plain_s / best_s, 2),
            "gpu_ms": {"batched_tuned": round(batch_gpu_ms, 3), "batched_fixed_64Ki_tile": round(fixed_gpu_ms, 3),
                       "plain": round(plain_gpu_ms, 3),
                       "how": "sum of the library's per-phase CUDA-event times (kernels only)"},
            "steps": steps}


def extra_zipf(steps: int) -> dict:
    """GROUP BY SUM/AVG, 2^28 rows, Zipf(1) keys over 2^24 random keys, float32 N(0,1)*1e3."""
    import numpy as np
    import torch

    import paper_2606_10030_gb300 as agg
    from datagen import cuda as dgc
    n, D = 1 << 28, 1 << 24
    k = dgc.keys_zipf(n, D, 1.0, 0)
    v = dgc.values("f32", n, 0)
    ops = agg.AGG_SUM | agg.AGG_AVG
    g = agg.agg_groupby(k, v, ops)
    strategy = agg.STRATEGY_NAMES[g.strategy]
    d = g.num_groups
    g.free()
    torch.cuda.synchronize()
    res = {}
    for name, strat in [("auto", agg.AGG_STRAT_AUTO), ("smem", agg.AGG_STRAT_SMEM),
                        ("global", agg.AGG_STRAT_GLOBAL), ("sort", agg.AGG_STRAT_SORT)]:
        o = agg.options(strat)
        agg.agg_groupby(k, v, ops, o).free()
        t0 = time.perf_counter()
        for _ in range(steps):
            agg.agg_groupby(k, v, ops, o).free()
        torch.cuda.synchronize()
        ms = (time.perf_counter() - t0) * 1e3 / steps
        res[name] = {"ms": round(ms, 3), "GB/s": round(n * 8 / (ms * 1e-3) / 1e9, 1)}
        # every group's error against its exactly rounded sum (one extra pass, untimed)
        g = agg.agg_groupby(k, v, ops, agg.options(strat, flags=agg.AGG_FLAG_SUM_ERROR))
        r = g.to_host()
        g.free()
        nz = np.abs(r["sum"]) > 0
        rel = r["sum_err"][nz] / np.abs(r["sum"][nz])
        res[name]["sum_error"] = {"groups": int(r["keys"].size), "max_abs_err": float(r["sum_err"].max()),
                                  "max_rel_err": float(rel.max()), "groups_rel_err_over_1e-6": int((rel > 1e-6).sum())}
    del k, v
    torch.cuda.empty_cache()
    return {"workload": "GROUP BY SUM/AVG, 2^28 rows, Zipf(1.0) keys over 2^24, float32 values",
            "groups": d, "auto_strategy": strategy, "per_strategy": res, "steps": steps}



def extra_groupby_2p26(steps: int, peaks: dict) -> dict:
    """GROUP BY SUM/COUNT/MIN/MAX, 2^26 rows over 1024 uniform keys, int64 values: the step and its build kernel."""
    import torch

    import paper_2606_10030_gb300 as agg
    W = GroupbyWorkload()
    W.setup(0)
    for _ in range(5):
        W.step()
    torch.cuda.synchronize()
    agg.profile_read()
    agg.profile_enable(True)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(steps):
        W.step()
    b.record()
    torch.cuda.synchronize()
    prof = agg.profile_read()
    agg.profile_enable(False)
    ms = a.elapsed_time(b) / steps
    build_ms = prof["build"][0] / max(1, prof["build"][1])
    by = W.bytes_per_step()
    del W
    torch.cuda.empty_cache()
    return {"workload": GroupbyWorkload().config()["workload"], "ms": round(ms, 4),
            "GB/s": round(by / (ms * 1e-3) / 1e9, 1), "frac_of_measured_hbm": round(by / (ms * 1e-3) / 1e9 /
                                                                                      peaks["hbm_gbs"], 4),
            "build_kernel": "gb_build", "build_ms": round(build_ms, 4),
            "build_GB/s": round(by / (build_ms * 1e-3) / 1e9, 1),
            "build_frac_of_measured_hbm": round(by / (build_ms * 1e-3) / 1e9 / peaks["hbm_gbs"], 4),
            "phases_ms_per_step": {k: round(v[0] / steps, 4) for k, v in prof.items() if v[1]}, "steps": steps}


def extra_table_grid(link: dict) -> dict:
    """The learned selector on 2^30-row uint32/int64 tables, 2^4..2^26 keys x Zipf 0..1.5:
    on-device GB/s of its choice, regret against the exhaustive autotuner (and the AUTO
    rule's), end-to-end GB/s from pinned host memory on four tables."""
    from paper_2606_10030_gb300 import selector
    if not selector.install_default():
        return {"skipped": "no trained selector weights"}
    ev = selector.evaluate_large(30, e2e_tables=4, log=lambda *a: None)
    for r in ev["tables"]:
        if "e2e_GBps" in r:
            r["e2e_frac_of_link"] = round(r["e2e_GBps"] / link["GB/s"], 4)
    ev["workload"] = ("GROUP BY SUM/MIN/MAX/COUNT/AVG over 2^30-row tables, uint32 keys over D = 2^4, 2^6, ..., "
                      "2^26 random keys, uniform or Zipf s in {0.5, 1.0, 1.5}, int64 values; one table per (D, s)")
    return ev


def extra_compressed(link: dict, steps: int = 10) -> dict:
    """The paper's scan shape (int32 uniform in [-2^20, 2^20): 21 of 32 bits) packed by frame of
    reference: end to end from pinned host memory, plain and packed, and the on-device packed scan."""
    import torch

    import paper_2606_10030_gb300 as agg
    from datagen import cuda as dgc
    n = 1 << 28
    col = dgc.values("i32", n, 0)
    host = col.cpu()
    raw = n * 4
    t0 = time.perf_counter()
    p = agg.agg_pack_for(host)
    enc_s = time.perf_counter() - t0
    hp = host.pin_memory()
    del col
    torch.cuda.empty_cache()

    def timed(fn, reps):
        fn()
        torch.cuda.synchronize()
        a = time.perf_counter()
        for _ in range(reps):
            fn()
        torch.cuda.synchronize()
        return (time.perf_counter() - a) / reps

    plain_s = timed(lambda: agg.agg_reduce_host(hp, agg.AGG_ALL), steps)
    packed_s = timed(lambda: agg.agg_reduce_packed_host(p, agg.AGG_ALL), steps)
    dev = p.to("cuda")
    out = torch.empty(agg.SCALAR_BYTES, dtype=torch.uint8, device="cuda")
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for _ in range(3):
        agg.agg_reduce_packed(dev, agg.AGG_ALL, out=out)
    a.record()
    for _ in range(50):
        agg.agg_reduce_packed(dev, agg.AGG_ALL, out=out)
    b.record()
    torch.cuda.synchronize()
    dev_ms = a.elapsed_time(b) / 50
    del dev, hp
    torch.cuda.empty_cache()
    e2e_packed = raw / packed_s / 1e9
    return {"workload": "ungrouped SUM/MIN/MAX/COUNT/AVG, 2^28 int32 rows uniform in [-2^20, 2^20), frame-of-reference "
                        "bit-packed (1024-value frames)",
            "raw_bytes": raw, "packed_bytes": p.nbytes, "ratio": round(raw / p.nbytes, 3),
            "encode_s_host": round(enc_s, 2),
            "e2e_plain_GB/s": round(raw / plain_s / 1e9, 1), "e2e_packed_input_GB/s": round(e2e_packed, 1),
            "e2e_packed_frac_of_link": round(e2e_packed / link["GB/s"], 3), "link_peak_GB/s": link["GB/s"],
            "device_packed_ms": round(dev_ms, 4), "device_packed_input_GB/s": round(raw / (dev_ms * 1e-3) / 1e9, 1),
            "device_packed_bytes_GB/s": round(p.nbytes / (dev_ms * 1e-3) / 1e9, 1), "steps": steps}


def extra_multi(steps: int = 10) -> dict:
    """Fused filter -> multi-column GROUP BY: 2^26 rows, key (hi over 16, lo over 4096 random keys),
    int64 / float32 / float64 value columns, a range filter on an int32 column keeping half."""
    import torch

    import paper_2606_10030_gb300 as agg
    from datagen import cuda as dgc
    n = 1 << 26
    lo, hi = dgc.keys_uniform(n, 4096, 3), dgc.keys_uniform(n, 16, 4)
    a, b, c, f = dgc.values("i64", n, 5), dgc.values("f32", n, 6), dgc.values("f64", n, 7), dgc.values("i32", n, 8)
    cols = [(a, agg.AGG_ALL), (b, agg.AGG_ALL), (c, agg.AGG_SUM)]
    filt = (f, -(2 ** 19), 2 ** 19)
    m = agg.agg_groupby_multi(lo, hi, cols, filt)
    groups = m.num_groups
    m.free()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        agg.agg_groupby_multi(lo, hi, cols, filt).free()
    torch.cuda.synchronize()
    ms = (time.perf_counter() - t0) * 1e3 / steps
    in_bytes = n * (4 + 4 + 8 + 4 + 8 + 4)
    del lo, hi, a, b, c, f
    torch.cuda.empty_cache()
    return {"workload": "GROUP BY (hi, lo) over 2^26 rows, 3 value columns (int64 all ops, float32 all ops, float64 "
                        "SUM), filter -2^19 <= int32 <= 2^19 (about half the rows)",
            "groups": groups, "ms": round(ms, 3), "input_bytes": in_bytes, "GB/s": round(in_bytes / (ms * 1e-3) / 1e9, 1),
            "steps": steps}


def kernel_traffic(kernel: str, workload: str):
    """DRAM bytes per launch from a committed ncu summary, if it matches the current kernel source."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    try:
        d = json.load(open(p)).get(f"{kernel}:{workload}")
    except Exception:
        return None
    if not d:
        return None
    src = os.path.join(ROOT, d["source"])
    if not os.path.exists(src) or code_sha256(src) != d["code_sha256"]:
        return None
    return d["dram_bytes_per_launch"]


def code_sha256(path: str) -> str:
    """sha256 of a source file's code: // comments, trailing blanks and empty lines removed (a
    comment edit does not change the kernel the recorded counters describe)."""
    import hashlib
    import re
    lines = []
    for line in open(path, encoding="utf-8").read().splitlines():
        line = re.sub(r"//.*$", "", line).rstrip()
        if line:
            lines.append(line)
    return hashlib.sha256("\n".join(lines).encode()).hexdigest()


def run_ours(args):
    import torch

    rank, world, local = dist_setup()
    torch.cuda.set_device(local)
    W = WORKLOADS[args.workload]()
    if args.rows:
        W.n = args.rows
    if args.strategy:
        W.strategy = args.strategy
    if args.ops:
        W.ops_override = args.ops
    W.setup(rank)
    peaks = load_peaks()
    stream = torch.cuda.current_stream()
    import paper_2606_10030_gb300 as agg
    for _ in range(args.warmup):
        W.step()
    torch.cuda.synchronize()
    agg.profile_read()
    sampler = ClockSampler(local)
    sampler.start()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    barrier(world)
    torch.cuda.synchronize()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    agg.profile_enable(True)
    launches0 = agg.launch_count()
    e0 = energy_mj(local)
    t0.record(stream)
    launches = 0
    for i in range(args.steps):
        evs[i][0].record(stream)
        launches += W.step()
        evs[i][1].record(stream)
    t1.record(stream)
    torch.cuda.synchronize()
    e1 = energy_mj(local)
    launches = agg.launch_count() - launches0
    prof = agg.profile_read()
    agg.profile_enable(False)
    barrier(world)
    clocks = sampler.stop()
    ms = t0.elapsed_time(t1)
    ms = max_over_ranks(ms, world)
    # the dominant kernel: the workload's, or the phase with the largest share of the step
    phase = W.phase if W.kernel else max(prof, key=lambda k: prof[k][0])
    kernel = W.kernel or PHASE_KERNELS.get(phase, phase)
    ph_ms, ph_calls = prof.get(phase, (0.0, 0))
    if ph_calls == 0:  # a strategy without this phase: time the whole step
        ph_ms, ph_calls = ms, args.steps
    per_launch_ms = ph_ms / max(1, ph_calls)
    bytes_step = W.bytes_per_step()
    value = world * bytes_step * args.steps / (ms * 1e-3) / 1e9
    achieved = bytes_step / (per_launch_ms * 1e-3) / 1e9

    # end to end through the host-fed entry point
    W.setup_e2e()
    e2e_steps = max(1, min(args.steps, args.e2e_steps))
    for _ in range(2):  # warm-up calls (the first ones allocate the pipeline's buffers)
        W.step_e2e()
    torch.cuda.synchronize()
    barrier(world)
    e2 = energy_mj(local)
    a = time.perf_counter()
    step_s = []
    for _ in range(e2e_steps):
        t0 = time.perf_counter()
        W.step_e2e()  # synchronous: host -> device copies, kernels, result read back
        step_s.append(time.perf_counter() - t0)
    e2e_s = max_over_ranks(time.perf_counter() - a, world)
    torch.cuda.synchronize()
    e3 = energy_mj(local)
    h2d, d2h = W.e2e_bytes()
    e2e_mean = world * h2d * e2e_steps / e2e_s / 1e9
    # the host link is shared with other jobs on the machine: the median step is the figure,
    # the mean over all steps is reported beside it
    e2e_value = world * h2d / max_over_ranks(statistics.median(step_s), world) / 1e9
    strategy = agg.STRATEGY_NAMES.get(getattr(W, "last_strategy", -1), None)
    W.release()
    torch.cuda.empty_cache()
    link = host_link_peak()

    extra = {}
    if rank == 0 and world == 1 and not args.no_extra and W.name == "table2p30":
        extra["groupby_2p26"] = extra_groupby_2p26(200, peaks)
        extra["scan"] = extra_scan(200, peaks)
        extra["zipf"] = extra_zipf(5)
        extra["batched"] = extra_batched(5)
        extra["compressed"] = extra_compressed(link)
        extra["multi"] = extra_multi()
        extra["table2p30_grid"] = extra_table_grid(link)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        rows, t, sample = W.cpu_sample(args.cpu_budget)
        cpu = {"value": rows * W.esize / t / 1e9, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample}
    if rank == 0:
        line = {
            "metric": METRIC, "value": round(value, 2), "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": W.dtype, "data": "synthetic (seeded SplitMix64)",
            "config": W.config(),
            "rows_per_s": world * W.n * args.steps / (ms * 1e-3),
            "roofline": {"bound": "hbm", "achieved": round(achieved, 2), "peak": peaks["hbm_gbs"], "unit": "GB/s",
                         "frac": round(achieved / peaks["hbm_gbs"], 4),
                         "traffic": kernel_traffic(W.kernel or phase, W.name),
                         "kernel": kernel, "phase": phase, "strategy": strategy,
                         "ms_per_launch": round(per_launch_ms, 4),
                         "achieved_how": "input bytes of the step / mean CUDA-event time of the phase per launch",
                         "peak_source": peaks["source"] + " (hbm_gbs, burst copy)"},
            "e2e": {"value": round(e2e_value, 2), "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "steps": e2e_steps, "mean_GB/s": round(e2e_mean, 2),
                    "how": "median of the per-step times (each step synchronous) over the timed steps, after 2 "
                           "warm-up calls; mean_GB/s = all steps' bytes / their total time",
                    "link_peak_GB/s": link["GB/s"],
                    "frac_of_link": round(e2e_value / world / link["GB/s"], 4), "link_how": link["how"]},
            "gpu_launches": launches,
            "energy": energy_report(e0, e1, e2, e3, args.steps, e2e_steps, bytes_step, h2d),
            "phases_ms_per_step": {k: round(v[0] / args.steps, 4) for k, v in prof.items() if v[1]},
            "extra": extra,
            "clocks": clocks,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)


def run_reference(args):
    """The CPU oracle, single-threaded, on a bounded sample of the same workload."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    W = WORKLOADS[args.workload]()
    if args.rows:
        W.n = args.rows
    per_step = max(0.1, args.cpu_budget / max(1, args.steps + args.warmup))
    for _ in range(args.warmup):
        W.cpu_sample(per_step)
    rows_t, t_t = 0, 0.0
    sample = ""
    for _ in range(args.steps):
        rows, t, sample = W.cpu_sample(per_step)
        rows_t += rows
        t_t += t
    v = rows_t * W.esize / t_t / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": round(v, 3), "unit": UNIT,
            "n_gpus": int(os.environ.get("WORLD_SIZE", "1")), "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * t_t / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": W.dtype, "data": "synthetic (seeded SplitMix64)",
            "config": W.config(),
            "cpu_baseline": {"value": round(v, 3), "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"per step: {sample}"},
            "e2e": {"value": round(v, 3), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--workload", default="table2p30", choices=sorted(WORKLOADS))
    ap.add_argument("--no-extra", action="store_true", help="skip the extra scan and Zipf measurements")
    ap.add_argument("--strategy", type=int, default=0, help="GROUP BY strategy (0 auto, 1 smem, 2 global, 3 sort)")
    ap.add_argument("--ops", type=int, default=0, help="override the ops bitmask (diagnostics)")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--cpu-budget", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--rows", type=int, default=0, help="override the workload's row count (small profiling cases)")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
