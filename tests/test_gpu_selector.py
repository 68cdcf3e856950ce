"""The selector network's kernels against the float64 oracle, the autotuner,
and what the trained selector gains over the strategy choice without it."""
import numpy as np
import pytest
import torch

import datagen as dg
import oracle
import paper_2606_10030_gb300 as agg
from oracle import mlp as omlp
from paper_2606_10030_gb300 import selector

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _build():
    agg.build()
    agg.lib()


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def test_forward_matches_oracle():
    rng = np.random.default_rng(0)
    p = (rng.standard_normal(omlp.N_PARAMS) * 0.3).astype(np.float32)
    X = (rng.standard_normal((700, 16)) * 3 + 1).astype(np.float32)
    mean, std = X.mean(axis=0).astype(np.float32), (X.std(axis=0) + 0.1).astype(np.float32)
    got = agg.agg_mlp_forward(_dev(p), _dev(X), _dev(mean), _dev(std)).cpu().numpy()
    ref, _ = omlp.forward(p.astype(np.float64), X, mean, std)
    assert np.allclose(got, ref, rtol=1e-4, atol=1e-6)
    got_raw = agg.agg_mlp_forward(_dev(p), _dev(X)).cpu().numpy()
    assert np.allclose(got_raw, omlp.forward(p.astype(np.float64), X)[0], rtol=1e-4, atol=1e-6)


@pytest.mark.parametrize("B", [1, 17, 256])
def test_gradient_matches_oracle(B):
    rng = np.random.default_rng(B)
    p = (rng.standard_normal(omlp.N_PARAMS) * 0.3).astype(np.float32)
    X = rng.standard_normal((B, 16)).astype(np.float32)
    y = rng.integers(0, 3, B).astype(np.int32)
    mean, std = np.zeros(16, np.float32), np.ones(16, np.float32) * 1.5
    g, loss = agg.agg_mlp_grad(_dev(p), _dev(X), _dev(y), _dev(mean), _dev(std))
    L, gr = omlp.loss_and_grad(p.astype(np.float64), X, y, mean, std)
    assert abs(float(loss.item()) - L) <= 1e-4 * max(1.0, abs(L))
    g = g.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(g - gr) <= 1e-4 * np.linalg.norm(gr) + 1e-7
    assert np.all(np.abs(g - gr) <= 1e-4 * np.abs(gr) + 1e-4 * np.abs(gr).max())


def test_adam_matches_oracle():
    rng = np.random.default_rng(9)
    p = rng.standard_normal(omlp.N_PARAMS).astype(np.float32)
    g = rng.standard_normal(omlp.N_PARAMS).astype(np.float32)
    m = (rng.standard_normal(omlp.N_PARAMS) * 0.1).astype(np.float32)
    v = np.abs(rng.standard_normal(omlp.N_PARAMS) * 0.1).astype(np.float32)
    pd, md, vd = _dev(p), _dev(m), _dev(v)
    agg.agg_mlp_adam(pd, _dev(g), md, vd, 7, lr=1e-2)
    rp, rm, rv = omlp.adam(p.astype(np.float64), g, m, v, 7, lr=1e-2)
    assert np.allclose(pd.cpu().numpy(), rp, rtol=1e-5, atol=1e-6)
    assert np.allclose(md.cpu().numpy(), rm, rtol=1e-5, atol=1e-7)
    assert np.allclose(vd.cpu().numpy(), rv, rtol=1e-5, atol=1e-7)


def test_training_on_the_gpu_fits_a_separable_problem():
    rng = np.random.default_rng(3)
    X = rng.standard_normal((2000, 16)).astype(np.float32)
    y = ((X[:, 0] > 0).astype(int) + (X[:, 3] > 0.5).astype(int)).astype(np.int32)
    params, mean, std, losses = selector.train(X, y, epochs=40, lr=3e-3, seed=1)
    assert losses[-1] < 0.25 * losses[0]
    pred = selector.predict(params, mean, std, X)
    assert (pred == y).mean() > 0.95
    # the oracle agrees with the trained network's predictions
    ref = omlp.forward(params.astype(np.float64), X, mean, std)[0].argmax(axis=1)
    assert (ref == pred).mean() > 0.995


def test_autotune_times_every_candidate_and_caches():
    agg.lib().agg_autotune_clear()
    keys = torch.from_numpy(dg.keys_uniform(1 << 20, 500, 0)).cuda()
    vals = torch.from_numpy(dg.values("i64", 1 << 20, 0)).cuda()
    r = agg.agg_autotune(keys, vals, agg.AGG_ALL, reps=2)
    assert r.ncand >= 7 and 0 <= r.best < r.ncand
    assert set(list(r.items_per_thread)[:r.ncand]) >= {4, 8} and 16384 in list(r.tile_rows)[:r.ncand]
    ms = np.array(list(r.ms)[:r.ncand])
    assert np.all(ms > 0) and ms[r.best] == ms.min()
    assert set(list(r.strategy)[:r.ncand]) == {agg.AGG_STRAT_SMEM, agg.AGG_STRAT_GLOBAL, agg.AGG_STRAT_SORT}
    assert agg.lib().agg_autotune_cache_size() == 1
    # AUTOTUNE uses the cache and returns the oracle's result
    g = agg.agg_groupby(keys, vals, agg.AGG_ALL, agg.options(agg.AGG_STRAT_AUTOTUNE))
    res = g.to_host()
    g.free()
    ref = oracle.groupby(keys.cpu().numpy(), vals.cpu().numpy())
    assert np.array_equal(res["keys"], ref.keys) and np.array_equal(res["sum"], ref.sum)
    assert agg.lib().agg_autotune_cache_size() == 1


def test_autotune_cache_save_and_load(tmp_path):
    agg.lib().agg_autotune_clear()
    keys = torch.from_numpy(dg.keys_uniform(300_000, 70_000, 1)).cuda()
    vals = torch.from_numpy(dg.values("f32", 300_000, 1)).cuda()
    agg.agg_autotune(keys, vals, agg.AGG_SUM)
    p = str(tmp_path / "tune.txt").encode()
    assert agg.lib().agg_autotune_save(p) == 0
    agg.lib().agg_autotune_clear()
    assert agg.lib().agg_autotune_cache_size() == 0
    assert agg.lib().agg_autotune_load(p) == 0
    assert agg.lib().agg_autotune_cache_size() == 1


def test_learned_strategy_returns_exact_results():
    rng = np.random.default_rng(4)
    X = rng.standard_normal((300, 16)).astype(np.float32)
    y = rng.integers(0, 3, 300).astype(np.int32)
    params, mean, std, _ = selector.train(X, y, epochs=2, seed=0)
    selector.install(params, mean, std)
    assert agg.lib().agg_selector_installed() == 1
    keys = dg.keys_zipf(400_000, 20_000, 1.1, 2)
    vals = dg.values("f64", 400_000, 2)
    g = agg.agg_groupby(torch.from_numpy(keys).cuda(), torch.from_numpy(vals).cuda(), agg.AGG_ALL,
                        agg.options(agg.AGG_STRAT_LEARNED))
    assert g.strategy in (agg.AGG_STRAT_SMEM, agg.AGG_STRAT_GLOBAL, agg.AGG_STRAT_SORT)
    res = g.to_host()
    g.free()
    ref = oracle.groupby(keys, vals)
    assert np.array_equal(res["keys"], ref.keys) and np.array_equal(res["count"], ref.count)
    assert np.array_equal(res["min"], ref.min) and np.array_equal(res["max"], ref.max)
    agg.lib().agg_selector_clear()


def test_trained_selector_gain_over_the_method_without_it():
    """Train on autotuner labels of seeded distributions and compare, on held-out
    distributions, the total time of the learned choice with the AUTO rule's and
    with every fixed strategy (regret = t(choice) / t(best) - 1)."""
    qs = selector.sample_queries(480, seed=11, log2_rows=(16, 21))
    X, y, T, ops = selector.label(qs)
    params, mean, std, losses = selector.train(X[:400], y[:400], epochs=120, lr=2e-3, seed=11)
    ev = selector.evaluate(params, mean, std, X[400:], T[400:], ops[400:])
    print("selector evaluation", ev)
    assert losses[-1] < losses[0]
    fixed_best = min(ev[k]["total_ms"] for k in ("smem", "global", "sort"))
    assert ev["learned"]["total_ms"] <= fixed_best
    assert ev["learned"]["mean_regret"] <= ev["rule"]["mean_regret"] + 0.05


def test_shipped_selector_beats_the_rule_on_fresh_distributions():
    """The installed network (trained on 20000 autotuner-labelled distributions) on 96 distributions
    it never saw (another seed; 2^16-2^24 rows): its choices cost no more in total than the best
    fixed strategy, and its mean regret is below the AUTO rule's."""
    params, mean, std = selector.load(selector.DEFAULT_WEIGHTS)
    qs = selector.sample_queries(96, seed=424242, log2_rows=(16, 24))
    X, y, T, ops = selector.label(qs)
    ev = selector.evaluate(params, mean, std, X, T, ops)
    print("shipped selector on fresh distributions", ev)
    fixed_best = min(ev[k]["total_ms"] for k in ("smem", "global", "sort"))
    assert ev["learned"]["total_ms"] <= fixed_best
    assert ev["learned"]["mean_regret"] < ev["rule"]["mean_regret"]
