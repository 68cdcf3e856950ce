"""The frame-of-reference encoder (host code, no GPU): a round trip through a
NumPy decoder written from the format's description, and minimal bit widths."""
import ctypes

import numpy as np
import pytest
import torch

import paper_2606_10030_gb300 as agg

FRAME = agg.AGG_PACK_FRAME


def decode(p: agg.Packed) -> np.ndarray:
    """Frames: 24-byte descriptors {int64 ref, uint32 bits, uint32 0, uint64 first word},
    then (16-byte aligned) the 32-bit words, least significant bit first."""
    info = p.info
    raw = p.buf.numpy()[: info.bytes].tobytes()
    nf = info.nframes
    desc = np.frombuffer(raw[: nf * 24], dtype=np.dtype([("ref", "<i8"), ("bits", "<u4"), ("z", "<u4"), ("w", "<u8")]))
    woff = (nf * 24 + 15) // 16 * 16
    words = np.frombuffer(raw[woff:], dtype="<u4")
    out = []
    for f in range(nf):
        cnt = min(FRAME, info.n - f * FRAME)
        b = int(desc["bits"][f])
        ref = int(desc["ref"][f])
        w0 = int(desc["w"][f])
        stream = int.from_bytes(words[w0: w0 + 32 * b + 2].tobytes(), "little")
        for i in range(cnt):
            x = (stream >> (i * b)) & ((1 << b) - 1) if b else 0
            out.append(ref + x)
    return np.array(out, dtype=np.int64)


def cases():
    rng = np.random.default_rng(0)
    yield "narrow_i32", rng.integers(-(2 ** 20), 2 ** 20, 5000).astype(np.int32)
    yield "full_i64", rng.integers(-(2 ** 63), 2 ** 63 - 1, 3000, dtype=np.int64, endpoint=True)
    yield "u32", rng.integers(0, 2 ** 32, 2100, dtype=np.uint64).astype(np.uint32)
    yield "constant", np.full(2500, -7, dtype=np.int64)
    yield "one", np.array([42], dtype=np.int32)
    yield "empty", np.zeros(0, dtype=np.int32)
    yield "extremes", np.array([np.iinfo(np.int64).min, np.iinfo(np.int64).max] * 700, dtype=np.int64)
    mix = rng.integers(0, 5, 4096).astype(np.int64)
    mix[1024:2048] = rng.integers(0, 2 ** 40, 1024)
    yield "mixed_frames", mix


@pytest.mark.parametrize("name,x", list(cases()))
def test_round_trip_and_minimal_widths(name, x):
    agg.build()
    p = agg.agg_pack_for(torch.from_numpy(x))
    assert p.info.n == x.size and p.info.nframes == (x.size + FRAME - 1) // FRAME
    assert np.array_equal(decode(p), x.astype(np.int64))
    raw = p.buf.numpy()[: p.info.bytes].tobytes()
    for f in range(p.info.nframes):
        seg = x[f * FRAME:(f + 1) * FRAME].astype(object)
        rng_ = int(max(seg)) - int(min(seg))
        bits = int.from_bytes(raw[f * 24 + 8: f * 24 + 12], "little")
        assert bits == rng_.bit_length(), (f, bits, rng_)
    # the buffer ends in eight zero bytes
    assert raw[-8:] == bytes(8)


def test_encoder_rejects_a_short_buffer():
    agg.build()
    x = np.arange(5000, dtype=np.int64) * 1000
    info = agg.AggPackedInfo()
    buf = np.zeros(64, dtype=np.uint8)
    st = agg.lib().agg_pack_for(x.ctypes.data_as(ctypes.c_void_p), x.size, agg.AGG_I64,
                                ctypes.c_void_p((buf.ctypes.data + 15) // 16 * 16), 32, ctypes.byref(info))
    assert st == agg.AGG_ERR_INVALID and "bytes" in agg.last_error()
    assert agg.lib().agg_pack_for(x.ctypes.data_as(ctypes.c_void_p), x.size, agg.AGG_F32, None, 0,
                                  ctypes.byref(info)) == agg.AGG_ERR_INVALID
