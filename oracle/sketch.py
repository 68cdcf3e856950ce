"""Oracle of the 16-feature key sketch (test infrastructure only), float64 NumPy.

The sketch summarises a strided sample of m = min(n, 4096) keys for the
strategy selectors. Its distinct-count estimate is GEE (Charikar, Chaudhuri,
Motwani and Narasayya, "Towards estimation error guarantees for distinct
values", PODS 2000): D = sqrt(n/m) * f1 + sum_{j>=2} f_j, where f_j is the
number of keys seen exactly j times in the sample. The selector's related-work
anchor is the processing-time model for aggregation of Sec. 7.

Features, in order:
  0 log2 n             1 value bytes       2 popcount(ops)     3 float values
  4 d/m (distinct fraction of the sample)  5 f1/m              6 f2/m
  7 top-1 share        8 top-8 share
  9 slope of ln(count_r) on ln(r) over the top min(d, 32) ranks (least squares)
 10 entropy of the sample / ln m           11 fraction of sampled rows equal to the next row
 12 log2 of GEE (clipped to [1, n])
 13 log2(1 + 2 * GEE * slot_bytes / shared memory per block)
 14 log2(1 + 2 * GEE * slot_bytes / L2 bytes)
 15 log2(max key - min key + 1) over the sample
"""
from __future__ import annotations

import math

import numpy as np

SAMPLE = 4096


def sample_positions(n: int, offset: int) -> np.ndarray:
    m = min(n, SAMPLE)
    stride = n // m
    return np.array([(offset + j * stride) % n for j in range(m)], dtype=np.int64)


def sketch(keys: np.ndarray, vbytes: int, nops: int, fp: int, slot_bytes: int, offset: int,
           smem_bytes: float, l2_bytes: float) -> np.ndarray:
    keys = np.asarray(keys, dtype=np.uint32)
    n = keys.size
    f = np.zeros(16, dtype=np.float64)
    f[1], f[2], f[3] = vbytes, nops, fp
    if n == 0:
        return f
    m = min(n, SAMPLE)
    pos = sample_positions(n, offset)
    s = keys[pos]
    nxt = pos + 1
    ok = nxt < n
    adj = int(np.count_nonzero(keys[nxt[ok]] == s[ok]))
    _, counts = np.unique(s, return_counts=True)
    d = counts.size
    f1 = int(np.count_nonzero(counts == 1))
    f2 = int(np.count_nonzero(counts == 2))
    top = np.sort(counts)[::-1].astype(np.float64)
    f[0] = math.log2(n)
    f[4] = d / m
    f[5] = f1 / m
    f[6] = f2 / m
    f[7] = top[0] / m
    f[8] = top[:8].sum() / m
    R = min(d, 32)
    if R >= 2:
        x = np.log(np.arange(1, R + 1, dtype=np.float64))
        y = np.log(top[:R])
        f[9] = (R * np.dot(x, y) - x.sum() * y.sum()) / (R * np.dot(x, x) - x.sum() ** 2)
    p = counts / m
    f[10] = float(-(p * np.log(p)).sum() / math.log(m)) if m > 1 else 0.0
    f[11] = adj / m
    gee = math.sqrt(n / m) * f1 + (d - f1)
    gee = min(max(gee, 1.0), float(n))
    f[12] = math.log2(gee)
    tb = 2.0 * gee * slot_bytes
    f[13] = math.log2(1.0 + tb / smem_bytes)
    f[14] = math.log2(1.0 + tb / l2_bytes)
    f[15] = math.log2(float(int(s.max()) - int(s.min())) + 1.0)
    return f


# ---------------------------------------------------------------------------
# HyperLogLog distinct-count estimate (Flajolet, Fusy, Gandouet and Meunier,
# "HyperLogLog: the analysis of a near-optimal cardinality estimation
# algorithm", AofA 2007), over every key of a column. The GROUP BY planner
# sizes its tables from it when the sample does not cover a large column.
# Hash of a key: MurmurHash3's 32-bit finaliser (a bijection of uint32); the
# top p = 14 bits pick one of m = 2^14 registers, which keeps the largest rank
# (position of the first one bit, from 1) of the remaining 18 bits (19 when
# they are all zero).
# ---------------------------------------------------------------------------
HLL_P = 14


def _fmix32(x: np.ndarray) -> np.ndarray:
    x = np.asarray(x, dtype=np.uint32).copy()
    with np.errstate(over="ignore"):
        x ^= x >> np.uint32(16)
        x *= np.uint32(0x85EBCA6B)
        x ^= x >> np.uint32(13)
        x *= np.uint32(0xC2B2AE35)
        x ^= x >> np.uint32(16)
    return x


def hll_registers(keys: np.ndarray, p: int = HLL_P) -> np.ndarray:
    """The m = 2^p registers after adding every key."""
    m = 1 << p
    h = _fmix32(keys).astype(np.int64)
    idx = h >> (32 - p)
    w = (h << p) & 0xFFFFFFFF  # the remaining 32 - p bits, at the top of a 32-bit word
    rank = np.full(h.size, 32 - p + 1, dtype=np.int64)
    nz = w != 0
    # position of the leading one bit of w, from 1: 32 - bit_length(w) + 1
    bl = np.floor(np.log2(w[nz].astype(np.float64))).astype(np.int64) + 1  # exact for w < 2^32
    rank[nz] = 32 - bl + 1
    reg = np.zeros(m, dtype=np.int64)
    np.maximum.at(reg, idx, rank)
    return reg


def hll_estimate(keys: np.ndarray, p: int = HLL_P) -> float:
    """alpha_m m^2 / sum 2^-M_j; linear counting m ln(m / V) below 5m/2 when V registers are
    zero; above 2^32 / 30, the 32-bit hash space correction -2^32 ln(1 - E / 2^32)."""
    if np.asarray(keys).size == 0:
        return 0.0
    m = 1 << p
    reg = hll_registers(keys, p)
    alpha = 0.7213 / (1.0 + 1.079 / m)
    e = alpha * m * m / float(np.sum(np.ldexp(1.0, -reg)))
    zeros = int(np.count_nonzero(reg == 0))
    if e <= 2.5 * m and zeros > 0:
        e = m * math.log(m / zeros)
    elif e > 2.0 ** 32 / 30.0:
        e = -(2.0 ** 32) * math.log(1.0 - e / 2.0 ** 32)
    return e
