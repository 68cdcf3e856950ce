"""Seeded synthetic inputs for the aggregation tests and benchmarks.

This module is shared by the CPU oracle and the CUDA path as the only common
piece: it draws columns and holds none of the aggregation arithmetic.

Every random number comes from SplitMix64 (Steele, Lea and Flood, "Fast
splittable pseudorandom number generators", OOPSLA 2014) used as a counter-based
generator: the i-th draw of stream ``s`` under seed ``seed`` is the i-th output
of a SplitMix64 sequence whose start state is itself one SplitMix64 output of
``seed`` and ``s``. Any row can therefore be generated independently, on the
host (NumPy, here) or on the GPU (``datagen/datagen.cu``), with bit-identical
integer draws.

Workload shapes (the paper's TPC-H ``lineitem.suppkey`` scan is not available
here, so these stand in for it):

* ungrouped integer column, values uniform in [-2^20, 2^20)          (2^20 rows)
* GROUP BY with 1024 random uint32 keys drawn uniformly, int64 values
  uniform in [0, 2^32)                                               (2^26 rows)
* GROUP BY with 2^24 random uint32 keys drawn Zipf(s=1), float32 values
  N(0, 1) * 1e3                                                      (2^28 rows)
* batches of 512 queries of mixed sizes, cardinalities and dtypes
* 2^30-row uint32 / int64 selector evaluation tables
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

M64 = (1 << 64) - 1
GAMMA = 0x9E3779B97F4A7C15
MIX1 = 0xBF58476D1CE4E5B9
MIX2 = 0x94D049BB133111EB

# Stream ids, fixed so that the GPU generator draws the same numbers.
STREAM_KEYS = 1
STREAM_VALS = 2
STREAM_VALS2 = 3
STREAM_DOMAIN = 7

DTYPES = {"i32": np.int32, "i64": np.int64, "u32": np.uint32, "f32": np.float32, "f64": np.float64}
DTYPE_CODE = {"i32": 0, "i64": 1, "u32": 2, "f32": 3, "f64": 4}


def _u64(x):
    return np.asarray(x, dtype=np.uint64)


def mix64(z):
    """SplitMix64 output function (the finaliser of the published generator)."""
    z = _u64(z)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * np.uint64(MIX1)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(MIX2)
    return z ^ (z >> np.uint64(31))


def mix64_int(z: int) -> int:
    z &= M64
    z = ((z ^ (z >> 30)) * MIX1) & M64
    z = ((z ^ (z >> 27)) * MIX2) & M64
    return z ^ (z >> 31)


def stream_state(seed: int, stream: int) -> int:
    """Start state of stream ``stream`` under ``seed``."""
    return mix64_int((seed + GAMMA * (stream + 1)) & M64)


def draws(seed: int, stream: int, start: int, count: int) -> np.ndarray:
    """Draws start..start+count-1 of one stream, as uint64."""
    st = np.uint64(stream_state(seed, stream))
    i = np.arange(start + 1, start + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return mix64(st + np.uint64(GAMMA) * i)


def perm32(x):
    """A bijection of uint32 (Wellons' "lowbias32" integer hash)."""
    x = np.asarray(x, dtype=np.uint32)
    with np.errstate(over="ignore"):
        x = x ^ (x >> np.uint32(16))
        x = x * np.uint32(0x7FEB352D)
        x = x ^ (x >> np.uint32(15))
        x = x * np.uint32(0x846CA68B)
        x = x ^ (x >> np.uint32(16))
    return x


def domain_salt(seed: int) -> int:
    return stream_state(seed, STREAM_DOMAIN) & 0xFFFFFFFF


def domain_keys(seed: int, idx) -> np.ndarray:
    """The idx-th key of a seeded domain of distinct uint32 keys."""
    return perm32(np.asarray(idx, dtype=np.uint32) ^ np.uint32(domain_salt(seed)))


def bounded(u, r: int) -> np.ndarray:
    """Map uint64 draws onto [0, r) for r <= 2^32 (multiply-shift on the top 32 bits)."""
    assert 0 < r <= (1 << 32)
    hi = _u64(u) >> np.uint64(32)
    with np.errstate(over="ignore"):
        return (hi * np.uint64(r)) >> np.uint64(32)


def zipf_thresholds(D: int, s: float) -> np.ndarray:
    """uint64 thresholds T[r] = floor(CDF(r) * 2^64) of Zipf(s) over ranks 1..D.

    A draw u picks rank index j = #{r : T[r] <= u}, clamped to D - 1.
    """
    r = np.arange(1, D + 1, dtype=np.float64)
    w = r ** (-float(s)) if s != 0 else np.ones(D)
    cdf = np.cumsum(w)
    cdf /= cdf[-1]
    t = np.empty(D, dtype=np.uint64)
    full = cdf >= 1.0
    t[~full] = (cdf[~full] * 2.0 ** 64).astype(np.uint64)
    t[full] = np.uint64(M64)
    return t


def zipf_pick(u, thresholds: np.ndarray) -> np.ndarray:
    j = np.searchsorted(thresholds, _u64(u), side="right")
    return np.minimum(j, len(thresholds) - 1).astype(np.uint64)


def keys_uniform(n: int, D: int, seed: int, start: int = 0) -> np.ndarray:
    idx = bounded(draws(seed, STREAM_KEYS, start, n), D)
    return domain_keys(seed, idx.astype(np.uint32))


def keys_zipf(n: int, D: int, s: float, seed: int, start: int = 0, thresholds=None) -> np.ndarray:
    t = zipf_thresholds(D, s) if thresholds is None else thresholds
    idx = zipf_pick(draws(seed, STREAM_KEYS, start, n), t)
    return domain_keys(seed, idx.astype(np.uint32))


def unit_open(u) -> np.ndarray:
    """uint64 -> float64 in (0, 1): (top 53 bits + 0.5) * 2^-53."""
    return ((_u64(u) >> np.uint64(11)).astype(np.float64) + 0.5) * (2.0 ** -53)


def unit_closed_open(u) -> np.ndarray:
    """uint64 -> float64 in [0, 1): top 53 bits * 2^-53."""
    return (_u64(u) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def values(dtype: str, n: int, seed: int, dist: str = "default", start: int = 0) -> np.ndarray:
    """A value column.

    dist "default": i32 uniform [-2^20, 2^20); i64 and u32 uniform [0, 2^32);
    f32/f64 N(0, 1) * 1e3 (Box-Muller, computed in float64).
    """
    u = draws(seed, STREAM_VALS, start, n)
    if dtype == "i32":
        return (bounded(u, 1 << 21).astype(np.int64) - (1 << 20)).astype(np.int32)
    if dtype == "i64":
        return (u >> np.uint64(32)).astype(np.int64)
    if dtype == "u32":
        return (u >> np.uint64(32)).astype(np.uint32)
    if dtype in ("f32", "f64"):
        u2 = draws(seed, STREAM_VALS2, start, n)
        z = np.sqrt(-2.0 * np.log(unit_open(u))) * np.cos(2.0 * np.pi * unit_closed_open(u2))
        z = z * 1e3
        return z.astype(np.float32) if dtype == "f32" else z
    raise ValueError(dtype)


# ---------------------------------------------------------------------------
# Workload recipes
# ---------------------------------------------------------------------------

@dataclass
class GroupQuery:
    """One group-by query of a batch (rows, key distribution, value dtype, ops)."""
    n: int
    D: int
    zipf_s: float   # 0 = uniform keys
    dtype: str
    ops: int
    seed: int


def batch_queries(nq: int = 512, base_seed: int = 0, log2_rows=(12, 24), log2_keys=(0, 20),
                  ops_bits: int = 5) -> list[GroupQuery]:
    """Seeded batch of uneven group-by queries.

    rows log-uniform in [2^12, 2^24], distinct keys log-uniform in [1, 2^20]
    (capped by rows), keys uniform or Zipf with s ~ U[0.5, 1.5], value dtype
    uniform over {i32, i64, f32, f64}, ops a random non-empty subset of
    {SUM, MIN, MAX, COUNT, AVG}.
    """
    out = []
    for j in range(nq):
        seed = mix64_int(base_seed * GAMMA + j + 1)
        d = draws(seed, 11, 0, 6)
        f = unit_closed_open(d)
        lr = log2_rows[0] + f[0] * (log2_rows[1] - log2_rows[0])
        n = int(round(2.0 ** lr))
        lk = log2_keys[0] + f[1] * (log2_keys[1] - log2_keys[0])
        D = max(1, min(n, int(round(2.0 ** lk))))
        zipf = 0.0 if f[2] < 0.5 else 0.5 + f[3]
        dtype = ["i32", "i64", "f32", "f64"][int(bounded(d[4:5], 4)[0])]
        ops = 1 + int(bounded(d[5:6], (1 << ops_bits) - 1)[0])
        out.append(GroupQuery(n, D, zipf, dtype, ops, seed))
    return out


def group_column(q: GroupQuery, start: int = 0, count: int | None = None):
    """Keys and values of one query (NumPy; for the sizes the CPU handles)."""
    count = q.n - start if count is None else count
    if q.zipf_s > 0:
        keys = keys_zipf(count, q.D, q.zipf_s, q.seed, start)
    else:
        keys = keys_uniform(count, q.D, q.seed, start)
    vals = values(q.dtype, count, q.seed, start=start)
    return keys, vals


def log2_ceil(x: int) -> int:
    return max(0, math.ceil(math.log2(max(1, x))))
