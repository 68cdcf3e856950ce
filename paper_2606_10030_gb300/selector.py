"""Training pipeline of the learned GROUP BY strategy selector.

1. Seeded training distributions (rows, distinct keys, Zipf skew, value dtype,
   ops) are generated on the GPU.
2. The autotuner times every strategy on each one (agg_autotune); the label
   is the fastest of SMEM, GLOBAL and SORT, and the features are the key
   sketch the library computes for the query.
3. The 16 -> 64 -> 64 -> 3 network is trained on the GPU by the library's
   own kernels (agg_mlp_train), on standardised features.
4. The weights are installed for AGG_STRAT_LEARNED (agg_selector_set) and
   can be saved to / loaded from an .npz file.

Run ``python -m paper_2606_10030_gb300.selector --samples N --out FILE`` on a
GPU to train from scratch.
"""
from __future__ import annotations

import argparse
import math
import os
import time

import numpy as np

from . import (AGG_ALL, AGG_STRAT_GLOBAL, AGG_STRAT_SMEM, AGG_STRAT_SORT, agg_autotune, agg_mlp_forward,
               agg_mlp_train, agg_rule_strategy, agg_selector_set, lib)

CLASS_OF_STRATEGY = {AGG_STRAT_SMEM: 0, AGG_STRAT_GLOBAL: 1, AGG_STRAT_SORT: 2}
STRATEGY_OF_CLASS = {v: k for k, v in CLASS_OF_STRATEGY.items()}
DEFAULT_WEIGHTS = os.path.join(os.path.dirname(os.path.abspath(__file__)), "selector_weights.npz")


def sample_queries(count: int, seed: int, log2_rows=(16, 24), log2_keys=(0, 26), max_s=1.5):
    """Seeded training distributions: rows and distinct keys log-uniform, Zipf s ~ U[0, max_s]."""
    import datagen as dg
    out = []
    for j in range(count):
        qs = dg.mix64_int(seed * dg.GAMMA + j + 1)
        f = dg.unit_closed_open(dg.draws(qs, 13, 0, 6))
        n = int(round(2.0 ** (log2_rows[0] + f[0] * (log2_rows[1] - log2_rows[0]))))
        D = max(1, min(n, int(round(2.0 ** (log2_keys[0] + f[1] * (log2_keys[1] - log2_keys[0]))))))
        s = float(f[2] * max_s)
        dtype = ["i32", "i64", "f32", "f64"][int(f[3] * 4) % 4]
        ops = 1 + int(f[4] * 31) % 31
        out.append(dg.GroupQuery(n, D, s if s > 0.05 else 0.0, dtype, ops, qs))
    return out


def label(queries, reps: int = 1, log_every: int = 0, checkpoint: str = ""):
    """Features, labels and per-strategy best times (ms) from the autotuner.

    With a checkpoint path, the arrays labelled so far are saved there every
    log_every queries (a long labelling run keeps its progress)."""
    import torch

    from datagen import cuda as dgc
    X = np.zeros((len(queries), 16), np.float32)
    y = np.zeros(len(queries), np.int32)
    T = np.zeros((len(queries), 3), np.float32)
    ops_all = np.zeros(len(queries), np.int64)
    t0 = time.time()
    maxn = max(q.n for q in queries)
    kbuf = torch.empty(maxn, dtype=torch.uint32, device="cuda")
    vbufs = {}
    for i, q in enumerate(queries):
        if q.dtype not in vbufs:
            vbufs[q.dtype] = torch.empty(maxn, dtype=dgc.torch_dtype(q.dtype), device="cuda")
        k, v = dgc.group_column(q, out_keys=kbuf[:q.n], out_vals=vbufs[q.dtype][:q.n])
        r = agg_autotune(k, v, q.ops, reps)
        X[i] = np.array(list(r.features), np.float32)
        T[i] = np.array(list(r.best_ms_per_strategy), np.float32)
        y[i] = int(np.argmin(T[i]))
        ops_all[i] = q.ops
        if log_every and (i + 1) % log_every == 0:
            print(f"labelled {i + 1}/{len(queries)} in {time.time() - t0:.1f}s", flush=True)
            if checkpoint:
                np.savez(checkpoint, X=X[:i + 1], y=y[:i + 1], T=T[:i + 1], ops=ops_all[:i + 1])
    return X, y, T, ops_all


def init_params(seed: int) -> np.ndarray:
    """He-uniform weights (bound sqrt(6 / fan_in)) from SplitMix64 draws, zero biases."""
    import datagen as dg
    parts = []
    for k, (fan_in, fan_out) in enumerate([(16, 64), (64, 64), (64, 3)]):
        u = dg.unit_closed_open(dg.draws(seed, 100 + k, 0, fan_in * fan_out))
        b = math.sqrt(6.0 / fan_in)
        parts.append(((2.0 * u - 1.0) * b).astype(np.float32))
        parts.append(np.zeros(fan_out, np.float32))
    p = np.concatenate(parts)
    assert p.size == lib().agg_mlp_param_count()
    return p


def standardisation(X: np.ndarray):
    mean = X.mean(axis=0).astype(np.float32)
    std = np.maximum(X.std(axis=0), 1e-3).astype(np.float32)
    return mean, std


def train(X: np.ndarray, y: np.ndarray, epochs: int = 60, batch: int = 256, lr: float = 2e-3, seed: int = 0):
    """Train on the GPU; returns (params, mean, std, per-epoch loss)."""
    import torch
    mean, std = standardisation(X)
    dev = "cuda"
    p = torch.from_numpy(init_params(seed)).to(dev)
    m = torch.zeros_like(p)
    v = torch.zeros_like(p)
    xd = torch.from_numpy(np.ascontiguousarray(X, np.float32)).to(dev)
    yd = torch.from_numpy(np.ascontiguousarray(y, np.int32)).to(dev)
    md = torch.from_numpy(mean).to(dev)
    sd = torch.from_numpy(std).to(dev)
    losses = agg_mlp_train(p, m, v, xd, yd, md, sd, epochs=epochs, batch=batch, lr=lr, seed=seed)
    return p.cpu().numpy(), mean, std, losses


def predict(params, mean, std, X: np.ndarray) -> np.ndarray:
    import torch
    dev = "cuda"
    probs = agg_mlp_forward(torch.from_numpy(params).to(dev), torch.from_numpy(np.ascontiguousarray(X, np.float32))
                            .to(dev), torch.from_numpy(mean).to(dev), torch.from_numpy(std).to(dev))
    return probs.cpu().numpy().argmax(axis=1)


def evaluate(params, mean, std, X, T, ops) -> dict:
    """Regret t(choice)/t(best) - 1 of the network, the AUTO rule and each fixed strategy."""
    best = T.min(axis=1)
    learned = predict(params, mean, std, X)
    rule = np.array([CLASS_OF_STRATEGY[agg_rule_strategy(X[i], int(ops[i]))] for i in range(len(X))])
    res = {}
    for name, choice in [("learned", learned), ("rule", rule), ("smem", np.zeros(len(X), int)),
                         ("global", np.ones(len(X), int)), ("sort", np.full(len(X), 2))]:
        t = T[np.arange(len(X)), choice]
        reg = t / best - 1.0
        res[name] = {"mean_regret": float(reg.mean()), "p95_regret": float(np.percentile(reg, 95)),
                     "total_ms": float(t.sum()), "accuracy": float((choice == T.argmin(axis=1)).mean())}
    res["best_total_ms"] = float(best.sum())
    return res


def install(params, mean, std) -> None:
    agg_selector_set(params, mean, std)


def save(path, params, mean, std, **meta) -> None:
    np.savez(path, params=params, mean=mean, std=std, **{k: np.asarray(v) for k, v in meta.items()})


def load(path=DEFAULT_WEIGHTS):
    d = np.load(path)
    return d["params"], d["mean"], d["std"]


def install_default() -> bool:
    if not os.path.exists(DEFAULT_WEIGHTS):
        return False
    install(*load(DEFAULT_WEIGHTS))
    return True


def evaluate_large(log2_rows: int = 30, log2_keys=range(4, 27, 2), skews=(0.0, 0.5, 1.0, 1.5),
                   e2e_tables: int = 4, seed: int = 7, log=print) -> dict:
    """Regret of the installed selector against the exhaustive autotuner on large
    uint32-key / int64-value tables, on the device; and end-to-end GB/s from pinned
    host memory (AGG_STRAT_LEARNED through agg_groupby_host) on a few of them."""
    import torch

    import datagen as dg
    from datagen import cuda as dgc

    from . import AGG_ALL, AGG_STRAT_LEARNED, agg_groupby_host, options
    n = 1 << log2_rows
    ops = AGG_ALL
    rows = []
    k = torch.empty(n, dtype=torch.uint32, device="cuda")
    v = torch.empty(n, dtype=torch.int64, device="cuda")
    e2e_done = 0
    for lk in log2_keys:
        for sk in skews:
            D = 1 << lk
            q = dg.GroupQuery(n, D, sk, "i64", ops, dg.mix64_int(seed * 1000 + lk * 10 + int(sk * 2)))
            dgc.group_column(q, out_keys=k, out_vals=v)
            r = agg_autotune(k, v, ops, 1)
            f = np.array(list(r.features), np.float32)
            T = np.array(list(r.best_ms_per_strategy), np.float64)
            probs = agg_mlp_forward(*[torch.from_numpy(a).cuda() for a in load()[:1]],
                                    torch.from_numpy(f[None]).cuda(),
                                    *[torch.from_numpy(a).cuda() for a in load()[1:]]).cpu().numpy()[0]
            learned = int(probs.argmax())
            rule = CLASS_OF_STRATEGY[agg_rule_strategy(f, ops)]
            row = {"log2_keys": lk, "zipf_s": sk, "ms": T.round(3).tolist(), "best": int(T.argmin()),
                   "learned": learned, "rule": rule, "learned_regret": float(T[learned] / T.min() - 1),
                   "rule_regret": float(T[rule] / T.min() - 1),
                   "learned_GBps": float(n * 12 / (T[learned] * 1e-3) / 1e9),
                   "best_GBps": float(n * 12 / (T.min() * 1e-3) / 1e9)}
            if e2e_done < e2e_tables and lk in (4, 12, 20, 26) and sk == 1.0:
                hk, hv = k.cpu().pin_memory(), v.cpu().pin_memory()
                g = agg_groupby_host(hk, hv, ops, options(AGG_STRAT_LEARNED))
                g.free()
                torch.cuda.synchronize()
                dts = []
                for _ in range(3):  # the median of three calls: the host link is shared
                    t0 = time.perf_counter()
                    g = agg_groupby_host(hk, hv, ops, options(AGG_STRAT_LEARNED))
                    res = g.to_host()
                    g.free()
                    dts.append(time.perf_counter() - t0)
                dt = sorted(dts)[1]
                row["e2e_GBps"] = float(n * 12 / dt / 1e9)
                row["e2e_groups"] = int(len(res["keys"]))
                del hk, hv
                e2e_done += 1
            rows.append(row)
            log(row)
    lr = np.array([r["learned_regret"] for r in rows])
    rr = np.array([r["rule_regret"] for r in rows])
    total_learned_ms = float(sum(r["ms"][r["learned"]] for r in rows))
    return {"tables": rows, "rows_per_table": n, "learned_mean_regret": float(lr.mean()),
            "learned_p95_regret": float(np.percentile(lr, 95)), "rule_mean_regret": float(rr.mean()),
            "rule_p95_regret": float(np.percentile(rr, 95)),
            "learned_classes": np.bincount([r["learned"] for r in rows], minlength=3).tolist(),
            "best_classes": np.bincount([r["best"] for r in rows], minlength=3).tolist(),
            "learned_GBps_all_tables": float(len(rows) * n * 12 / (total_learned_ms * 1e-3) / 1e9)}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--samples", type=int, default=2000)
    ap.add_argument("--holdout", type=int, default=400)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--max-log2-rows", type=int, default=24)
    ap.add_argument("--epochs", type=int, default=80)
    ap.add_argument("--out", default=DEFAULT_WEIGHTS)
    ap.add_argument("--evaluate-large", default="", help="write the large-table evaluation (JSON) to this path")
    ap.add_argument("--large-log2-rows", type=int, default=30)
    ap.add_argument("--checkpoint", default="", help="save the labelled arrays here as labelling proceeds")
    ap.add_argument("--data", default="", help="train on labelled arrays saved earlier (skips labelling)")
    args = ap.parse_args()
    if args.evaluate_large:
        import json
        install_default()
        ev = evaluate_large(args.large_log2_rows)
        with open(args.evaluate_large, "w") as f:
            json.dump(ev, f, indent=1)
        print({k: v for k, v in ev.items() if k != "tables"})
        return
    if args.data:
        d = np.load(args.data)
        X, y, T, ops = d["X"], d["y"], d["T"], d["ops"]
    else:
        qs = sample_queries(args.samples + args.holdout, args.seed, log2_rows=(16, args.max_log2_rows))
        X, y, T, ops = label(qs, log_every=500, checkpoint=args.checkpoint)
    ntr = min(args.samples, len(X) - max(1, args.holdout))
    params, mean, std, losses = train(X[:ntr], y[:ntr], epochs=args.epochs, seed=args.seed)
    ev = evaluate(params, mean, std, X[ntr:], T[ntr:], ops[ntr:])
    print("loss first/last epoch", float(losses[0]), float(losses[-1]))
    print("held-out", ev)
    save(args.out, params, mean, std, train_samples=ntr, holdout=args.holdout, seed=args.seed,
         max_log2_rows=args.max_log2_rows, label_counts=np.bincount(y[:ntr], minlength=3))
    np.savez(os.path.splitext(args.out)[0] + "_data.npz", X=X, y=y, T=T, ops=ops)


if __name__ == "__main__":
    main()
