"""Pins for the key-sketch oracle: closed forms on constructed samples."""
import math

import numpy as np
import pytest

from oracle.sketch import SAMPLE, sample_positions, sketch

ARGS = dict(vbytes=8, nops=4, fp=0, slot_bytes=32, offset=0, smem_bytes=232448.0, l2_bytes=132120576.0)


def test_all_distinct_sample():
    keys = np.arange(SAMPLE, dtype=np.uint32) * np.uint32(7)
    f = sketch(keys, **ARGS)
    assert f[0] == 12 and f[4] == 1 and f[5] == 1 and f[6] == 0
    assert f[7] == 1 / SAMPLE and f[8] == 8 / SAMPLE
    assert f[9] == 0                         # all counts 1: flat rank-frequency
    assert abs(f[10] - 1.0) < 1e-12          # uniform over m keys: entropy ln m
    assert f[11] == 0
    assert f[12] == 12                       # GEE = sqrt(1) * m + 0 = m
    assert f[15] == math.log2(7 * (SAMPLE - 1) + 1)


def test_constant_column():
    keys = np.full(100000, 5, dtype=np.uint32)
    f = sketch(keys, **ARGS)
    assert f[4] == 1 / SAMPLE and f[5] == 0 and f[7] == 1 and f[8] == 1
    assert f[9] == 0 and f[10] == 0 and f[11] == 1
    assert f[12] == 0                        # GEE = 0 + (1 - 0) = 1
    assert f[15] == 0
    assert f[13] == math.log2(1 + 2 * 32 / 232448.0)


def test_two_equal_halves_entropy_and_gee():
    keys = np.repeat(np.array([1, 9], dtype=np.uint32), SAMPLE // 2)
    f = sketch(keys, **ARGS)
    assert abs(f[10] - math.log(2) / math.log(SAMPLE)) < 1e-12
    assert f[7] == 0.5 and f[8] == 1.0
    # two counts of m/2: the slope over R=2 ranks is ln(1)/ln(2) = 0
    assert f[9] == 0
    assert f[15] == math.log2(9)


def test_gee_scales_singletons_by_sqrt_n_over_m():
    n = SAMPLE * 64                          # stride 64: each sampled key distinct
    keys = np.arange(n, dtype=np.uint32)
    f = sketch(keys, **ARGS)
    assert f[12] == math.log2(math.sqrt(64) * SAMPLE)


def test_known_slope_on_constructed_frequencies():
    # counts 512/r for r = 1..32 (a Zipf(1) profile): slope -1 up to rounding of the counts
    counts = [int(round(512 / r)) for r in range(1, 33)]
    keys = np.concatenate([np.full(c, r, dtype=np.uint32) for r, c in enumerate(counts)])
    keys = np.concatenate([keys, np.arange(10 ** 6, 10 ** 6 + SAMPLE - keys.size, dtype=np.uint32)])
    assert keys.size == SAMPLE
    f = sketch(keys, **ARGS)
    x = np.log(np.arange(1, 33))
    top = np.sort(np.array(counts + [1] * (SAMPLE - sum(counts))))[::-1][:32].astype(float)
    y = np.log(top)
    expect = np.polyfit(x, y, 1)[0]
    assert abs(f[9] - expect) < 1e-12 and -1.1 < f[9] < -0.9


def test_sample_positions_wrap_and_small_n():
    assert list(sample_positions(10, 3)) == list(range(3, 10)) + [0, 1, 2]
    p = sample_positions(SAMPLE * 3 + 5, 2 ** 63)
    assert p.size == SAMPLE and p.max() < SAMPLE * 3 + 5


def test_empty():
    f = sketch(np.array([], dtype=np.uint32), **ARGS)
    assert f[1] == 8 and f[2] == 4 and f[0] == 0 and np.all(f[4:] == 0)


def test_table_size_features_on_closed_form_cases():
    """Features 13 and 14 compare the estimated table (2 x GEE slots of slot_bytes)
    with shared memory and with L2. The byte counts below are chosen so that the
    expected values are integers: a wrong slot size, a missing factor 2, or the
    two memories swapped gives a different number."""
    # constant column: GEE = 1, table = 2 * 1 * 32 = 64 bytes
    args = dict(ARGS, smem_bytes=64.0, l2_bytes=64.0 / 7.0)
    f = sketch(np.full(50000, 3, dtype=np.uint32), **args)
    assert f[13] == 1.0            # log2(1 + 64 / 64)
    assert f[14] == 3.0            # log2(1 + 64 / (64/7)) = log2(8)
    # all sampled keys distinct with stride 1: GEE = m = 4096, table = 2 * 4096 * 32 = 2^18 bytes
    args = dict(ARGS, smem_bytes=float(2 ** 18), l2_bytes=float(2 ** 18) / 3.0)
    f = sketch(np.arange(SAMPLE, dtype=np.uint32), **args)
    assert f[12] == 12.0
    assert f[13] == 1.0            # log2(1 + 1)
    assert f[14] == 2.0            # log2(1 + 3)
    # n = 64 m distinct keys: GEE = 8 m = 2^15, table = 2^21 bytes; L2 of 2^21 / 15 bytes
    args = dict(ARGS, slot_bytes=32, smem_bytes=float(2 ** 21) / 3.0, l2_bytes=float(2 ** 21) / 15.0)
    f = sketch(np.arange(SAMPLE * 64, dtype=np.uint32), **args)
    assert f[13] == 2.0 and f[14] == 4.0
    # slot bytes enter linearly: 16-byte slots halve the table
    args = dict(ARGS, slot_bytes=16, smem_bytes=float(2 ** 20), l2_bytes=float(2 ** 20) / 3.0)
    f = sketch(np.arange(SAMPLE * 64, dtype=np.uint32), **args)
    assert f[13] == 1.0 and f[14] == 2.0


def test_hll_closed_forms():
    from oracle.sketch import hll_estimate, hll_registers
    assert hll_estimate(np.array([], dtype=np.uint32)) == 0.0
    one = hll_registers(np.full(1000, 12345, dtype=np.uint32))
    assert np.count_nonzero(one) == 1 and 1 <= one.max() <= 19
    # one key: linear counting with V = m - 1 zero registers gives m ln(m / (m - 1)) ~ 1
    m = 1 << 14
    assert abs(hll_estimate(np.full(10, 7, dtype=np.uint32)) - m * math.log(m / (m - 1))) < 1e-9


def test_hll_ignores_repeats_and_order():
    from oracle.sketch import hll_estimate
    rng = np.random.default_rng(4)
    keys = rng.integers(0, 2 ** 32, 50_000, dtype=np.uint64).astype(np.uint32)
    rep = np.concatenate([keys, keys[::3], keys[::7]])
    rng.shuffle(rep)
    assert hll_estimate(rep) == hll_estimate(np.unique(keys))


def test_hll_registers_of_known_hashes():
    """Register and rank worked out by hand from MurmurHash3's finaliser: fmix32(1) =
    0x514E28B7 (register 0x514E28B7 >> 18 = 5203; low 18 bits 0x228B7 >= 2^17, so the
    first of the 18 bits is one: rank 1); fmix32(0) = 0 (register 0, no one bit among the
    18: rank 19); and the rank rule, 18 - bit_length(low 18 bits) + 1, on a few more keys."""
    from oracle.sketch import _fmix32, hll_registers
    assert int(_fmix32(np.array([1], dtype=np.uint32))[0]) == 0x514E28B7
    reg = hll_registers(np.array([1], dtype=np.uint32))
    assert reg[5203] == 1 and np.count_nonzero(reg) == 1
    # the rank rule on more keys (their registers may also hold other keys' larger ranks)
    keys = np.arange(1 << 16, dtype=np.uint32)
    h = _fmix32(keys).astype(np.int64)
    reg = hll_registers(keys)
    for k in (3, 77, 4096, 65535):
        low = int(h[k]) & 0x3FFFF
        rank = 18 - low.bit_length() + 1 if low else 19
        assert reg[int(h[k]) >> 18] >= rank
    reg = hll_registers(np.array([0], dtype=np.uint32))
    assert reg[0] == 19 and np.count_nonzero(reg) == 1


@pytest.mark.parametrize("d", [300, 20_000, 200_000, 3_000_000])
def test_hll_within_its_error_bound(d):
    """Relative standard error 1.04 / sqrt(m) = 0.81%; allow five of them."""
    from oracle.sketch import hll_estimate
    keys = np.arange(d, dtype=np.uint64).astype(np.uint32) * np.uint32(2654435761)
    assert abs(hll_estimate(keys) / d - 1.0) < 5 * 1.04 / math.sqrt(1 << 14)
