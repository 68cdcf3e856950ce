"""Seeded generators: known-answer vector and empirical shape checks."""
import os

import numpy as np

import datagen as dg

GOLD = os.path.join(os.path.dirname(__file__), "golden", "splitmix64_kat.txt")


def test_splitmix64_known_answer():
    vals = [int(l) for l in open(GOLD) if l.strip() and not l.startswith("#")]
    state, expect = vals[0], vals[1:]
    got = []
    for _ in expect:
        state = (state + dg.GAMMA) & dg.M64
        got.append(dg.mix64_int(state))
    assert got == expect
    # the vectorised counter form gives the same sequence
    st0 = vals[0]
    z = dg.mix64(np.uint64(st0) + np.uint64(dg.GAMMA) * np.arange(1, 6, dtype=np.uint64))
    assert [int(v) for v in z] == expect


def test_draws_are_counter_based():
    a = dg.draws(3, 2, 0, 1000)
    b = dg.draws(3, 2, 400, 100)
    assert np.array_equal(a[400:500], b)
    assert not np.array_equal(dg.draws(3, 1, 0, 10), dg.draws(3, 2, 0, 10))


def test_perm32_is_a_bijection():
    x = np.arange(1 << 20, dtype=np.uint32)
    assert np.unique(dg.perm32(x)).size == x.size
    assert np.unique(dg.domain_keys(5, np.arange(1 << 16))).size == 1 << 16


def test_uniform_values_ranges():
    v = dg.values("i32", 1 << 18, 0)
    assert v.min() >= -(1 << 20) and v.max() < (1 << 20)
    assert abs(v.mean()) < 5e3
    v = dg.values("i64", 1 << 18, 0)
    assert v.min() >= 0 and v.max() < (1 << 32)


def test_normal_values_shape():
    v = dg.values("f32", 1 << 18, 1).astype(np.float64)
    assert abs(v.mean()) < 10 and abs(v.std() - 1e3) < 10


def test_uniform_keys_hit_the_domain():
    k = dg.keys_uniform(1 << 18, 1024, 0)
    dom = dg.domain_keys(0, np.arange(1024))
    assert np.unique(k).size == 1024 and np.isin(k, dom).all()


def test_zipf_rank_frequency_slope():
    D, s = 1 << 12, 1.0
    t = dg.zipf_thresholds(D, s)
    assert np.all(np.diff(t.astype(np.float64)) >= 0) and t[-1] == np.uint64(dg.M64)
    k = dg.keys_zipf(1 << 20, D, s, 4, thresholds=t)
    _, cnt = np.unique(k, return_counts=True)
    cnt = np.sort(cnt)[::-1][:64].astype(np.float64)
    slope = np.polyfit(np.log(np.arange(1, 65)), np.log(cnt), 1)[0]
    assert abs(slope + s) < 0.1
    # top key share ~ 1 / H(D)
    share = cnt[0] / (1 << 20)
    assert abs(share - 1.0 / np.sum(1.0 / np.arange(1, D + 1))) < 0.01


def test_batch_queries_recipe():
    qs = dg.batch_queries(512, 0)
    assert len(qs) == 512
    n = np.array([q.n for q in qs])
    assert n.min() >= 1 << 12 and n.max() <= 1 << 24
    assert all(1 <= q.D <= min(q.n, 1 << 20) for q in qs)
    assert set(q.dtype for q in qs) == {"i32", "i64", "f32", "f64"}
    assert all(1 <= q.ops <= 31 for q in qs)
    assert all(q.zipf_s == 0 or 0.5 <= q.zipf_s <= 1.5 for q in qs)
    assert qs[7].seed == dg.batch_queries(8, 0)[7].seed
