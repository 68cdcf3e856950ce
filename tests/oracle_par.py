"""The CPU oracle on inputs of hundreds of millions of rows (test infrastructure).

A GROUP BY result is a function of each key's rows alone, so the key space can
be split into P classes and every class given to its own host process: a
process selects the rows whose key falls in its class (in row order) and
runs ``oracle.groupby`` on them unchanged. The classes' groups are disjoint;
concatenated and ordered by key they are the oracle's result for the whole
column, float sums included (every group is still folded by one accumulator
in row order). Nothing here aggregates: the only arithmetic is the class of a
key and, for the tolerance bar of float sums, a float64 sum of |x| per group.

The pool is started with ``spawn`` (a pool forked after the first GPU call can
hang). Inputs are shared with the workers through ``.npy`` files; results are
cached on disk under ``AGG_ORACLE_CACHE`` (default: a folder in the system
temporary directory) by a caller-chosen name, so that several tests of one
run can reuse the oracle's result for the same seeded input.
"""
from __future__ import annotations

import multiprocessing as mp
import os
import tempfile

import numpy as np

CHUNK = 1 << 24  # rows a worker reads at a time


def cache_dir() -> str:
    base = "/dev/shm" if os.path.isdir("/dev/shm") and os.access("/dev/shm", os.W_OK) else tempfile.gettempdir()
    d = os.environ.get("AGG_ORACLE_CACHE") or os.path.join(base, "agg_oracle_cache")
    os.makedirs(d, exist_ok=True)
    return d


def key_class(keys: np.ndarray, bits: int) -> np.ndarray:
    """Class of each key: the top `bits` bits of key * 0x9E3779B1 mod 2^32 (Fibonacci hashing)."""
    with np.errstate(over="ignore"):
        return (keys.astype(np.uint32) * np.uint32(0x9E3779B1)) >> np.uint32(32 - bits)


def _class_worker(args):
    kpath, vpath, bits, cls, with_abs = args
    import oracle
    keys = np.load(kpath, mmap_mode="r")
    vals = np.load(vpath, mmap_mode="r")
    ks, vs = [], []
    for a in range(0, keys.size, CHUNK):
        k = np.asarray(keys[a:a + CHUNK])
        m = key_class(k, bits) == cls
        ks.append(k[m])
        vs.append(np.asarray(vals[a:a + CHUNK])[m])
    k = np.concatenate(ks) if ks else np.zeros(0, np.uint32)
    v = np.concatenate(vs) if vs else np.zeros(0, vals.dtype)
    g = oracle.groupby(k, v)
    out = {"keys": g.keys, "count": g.count, "sum": g.sum, "min": g.min, "max": g.max, "avg": g.avg}
    if with_abs:
        idx = np.searchsorted(g.keys, k)
        out["abs_sum"] = np.bincount(idx, weights=np.abs(v.astype(np.float64)), minlength=g.keys.size)
    return out


def groupby(keys: np.ndarray, vals: np.ndarray, name: str | None = None, classes_log2: int = 6,
            workers: int | None = None) -> dict:
    """The oracle's full GROUP BY of (keys, vals) as arrays in ascending key order.

    For float values the result also holds ``abs_sum`` (sum of |x| per group,
    float64) for the tolerance bar. With a name, the result is cached on disk.
    """
    path = os.path.join(cache_dir(), f"{name}.npz") if name else None
    if path and os.path.exists(path):
        d = np.load(path)
        return {k: d[k] for k in d.files}
    with tempfile.TemporaryDirectory(dir=cache_dir()) as tmp:
        kpath, vpath = os.path.join(tmp, "k.npy"), os.path.join(tmp, "v.npy")
        np.save(kpath, np.ascontiguousarray(keys, dtype=np.uint32))
        np.save(vpath, np.ascontiguousarray(vals))
        with_abs = vals.dtype.kind == "f"
        jobs = [(kpath, vpath, classes_log2, c, with_abs) for c in range(1 << classes_log2)]
        workers = workers or min(len(jobs), os.cpu_count() or 1)
        with mp.get_context("spawn").Pool(workers) as pool:
            parts = pool.map(_class_worker, jobs, chunksize=1)
    out = {f: np.concatenate([p[f] for p in parts]) for f in parts[0]}
    order = np.argsort(out["keys"], kind="stable")
    out = {f: a[order] for f, a in out.items()}
    if path:
        np.savez(path, **out)
    return out


def _selected_worker(args):
    kpath, vpath, a, b, sel = args
    import oracle
    keys = np.load(kpath, mmap_mode="r")
    vals = np.load(vpath, mmap_mode="r")
    g = oracle.groupby_selected(np.asarray(keys[a:b]), np.asarray(vals[a:b]), sel)
    return g.keys, g.count, g.sum, g.min, g.max


def groupby_selected_int(keys: np.ndarray, vals: np.ndarray, sel: np.ndarray, workers: int | None = None,
                         min_rows: int = CHUNK) -> dict:
    """``oracle.groupby_selected`` over an integer column, on row ranges in parallel.

    Integer COUNT, SUM (mod 2^64), MIN and MAX of a group over the whole column
    are the count sum, wrapped sum, min and max of its row ranges' results.
    """
    assert vals.dtype.kind in "iu"
    sel = np.unique(np.asarray(sel, dtype=np.uint32))
    with tempfile.TemporaryDirectory(dir=cache_dir()) as tmp:
        kpath, vpath = os.path.join(tmp, "k.npy"), os.path.join(tmp, "v.npy")
        np.save(kpath, np.ascontiguousarray(keys, dtype=np.uint32))
        np.save(vpath, np.ascontiguousarray(vals))
        n = keys.size
        workers = workers or (os.cpu_count() or 1)
        step = max(min_rows, -(-n // workers))
        jobs = [(kpath, vpath, a, min(n, a + step), sel) for a in range(0, n, step)]
        with mp.get_context("spawn").Pool(min(workers, len(jobs))) as pool:
            parts = pool.map(_selected_worker, jobs, chunksize=1)
    cnt = np.zeros(sel.size, np.int64)
    s = np.zeros(sel.size, np.uint64)
    mn = np.full(sel.size, np.iinfo(np.int64).max, np.int64)
    mx = np.full(sel.size, np.iinfo(np.int64).min, np.int64)
    for k, c, sm, lo, hi in parts:
        assert np.array_equal(k, sel)
        cnt += c
        with np.errstate(over="ignore"):
            s += sm.view(np.uint64)
        has = c > 0
        mn[has] = np.minimum(mn[has], lo[has])
        mx[has] = np.maximum(mx[has], hi[has])
    return {"keys": sel, "count": cnt, "sum": s.view(np.int64), "min": mn, "max": mx}


def _table_rows(spec, a: int, b: int, thresholds):
    """Rows [a, b) of a seeded table, from the shared input generators."""
    import datagen as dg
    n_keys, s, dtype, seed = spec
    count = b - a
    if s > 0:
        u = dg.draws(seed, dg.STREAM_KEYS, a, count)
        order = np.argsort(u, kind="stable")  # sorted needles: one sweep through the thresholds
        idx = np.empty(count, np.uint64)
        idx[order] = dg.zipf_pick(u[order], thresholds)
        keys = dg.domain_keys(seed, idx.astype(np.uint32))
    else:
        keys = dg.keys_uniform(count, n_keys, seed, start=a)
    return keys, dg.values(dtype, count, seed, start=a)


def _table_worker(args):
    spec, a, b, tpath, sel = args
    import oracle
    if isinstance(spec, tuple) and len(spec) == 2:  # row ranges of stored columns
        keys = np.asarray(np.load(spec[0], mmap_mode="r")[a:b])
        vals = np.asarray(np.load(spec[1], mmap_mode="r")[a:b])
    else:
        thresholds = np.load(tpath, mmap_mode="r") if tpath else None
        keys, vals = _table_rows(spec, a, b, thresholds)
    g = oracle.groupby_selected(keys, vals, sel)
    r = oracle.reduce(vals)
    return (g.keys, g.count, g.sum, g.min, g.max), (r["count"], r["sum"], r["min"], r["max"])


def table_check(n: int, n_keys: int, s: float, dtype: str, seed: int, sel: np.ndarray, rows_per_job: int = CHUNK,
                workers: int | None = None, columns=None) -> dict:
    """Oracle results for a seeded integer table of up to billions of rows.

    Each job takes a row range, regenerated with the seeded generators (the
    same draws the GPU generator makes; uniform keys are cheap to redraw) or,
    when ``columns`` = (keys, vals) is given, read from a copy of them, and
    runs ``oracle.groupby_selected`` and ``oracle.reduce`` on it; the ranges'
    integer results are merged as in ``groupby_selected_int``. Returns the
    selected groups and the ungrouped count, sum (mod 2^64), min and max of
    the whole column.
    """
    import datagen as dg
    assert dtype in ("i32", "i64", "u32")
    sel = np.unique(np.asarray(sel, dtype=np.uint32))
    with tempfile.TemporaryDirectory(dir=cache_dir()) as tmp:
        tpath = None
        if columns is not None:
            spec = (os.path.join(tmp, "k.npy"), os.path.join(tmp, "v.npy"))
            np.save(spec[0], np.ascontiguousarray(columns[0], dtype=np.uint32))
            np.save(spec[1], np.ascontiguousarray(columns[1]))
        elif s > 0:
            tpath = os.path.join(tmp, "thresholds.npy")
            np.save(tpath, dg.zipf_thresholds(n_keys, s))
        if columns is None:
            spec = (n_keys, s, dtype, seed)
        jobs = [(spec, a, min(n, a + rows_per_job), tpath, sel) for a in range(0, n, rows_per_job)]
        workers = workers or (os.cpu_count() or 1)
        with mp.get_context("spawn").Pool(min(workers, len(jobs))) as pool:
            parts = pool.map(_table_worker, jobs, chunksize=1)
    cnt = np.zeros(sel.size, np.int64)
    sm = np.zeros(sel.size, np.uint64)
    mn = np.full(sel.size, np.iinfo(np.int64).max, np.int64)
    mx = np.full(sel.size, np.iinfo(np.int64).min, np.int64)
    total = {"count": 0, "sum": 0, "min": None, "max": None}
    for (k, c, s_, lo, hi), (rc, rs, rmin, rmax) in parts:
        assert np.array_equal(k, sel)
        cnt += c
        with np.errstate(over="ignore"):
            sm += s_.view(np.uint64)
        has = c > 0
        mn[has] = np.minimum(mn[has], lo[has])
        mx[has] = np.maximum(mx[has], hi[has])
        total["count"] += rc
        total["sum"] = (total["sum"] + rs) % (1 << 64)
        total["min"] = rmin if total["min"] is None else min(total["min"], rmin)
        total["max"] = rmax if total["max"] is None else max(total["max"], rmax)
    if total["sum"] >= 1 << 63:
        total["sum"] -= 1 << 64
    return {"keys": sel, "count": cnt, "sum": sm.view(np.int64), "min": mn, "max": mx, "total": total}
