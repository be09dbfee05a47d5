"""Training data, training and regret evaluation of the learned tuner.

Run on a GPU:

    python -m paper_1112_5588_gb300.tuner_data generate --n-train 800 --n-test 200 --out timings.npz
    python -m paper_1112_5588_gb300.tuner_data train timings.npz --model tuner_mlp.json
    python -m paper_1112_5588_gb300.tuner_data evaluate timings.npz --model tuner_mlp.json
    python -m paper_1112_5588_gb300.tuner_data recheck timings.npz --model tuner_mlp.json --count 200

`generate` draws seeded synthetic matrices (N log-uniform, Zipf(s) row
lengths with s uniform in [1.5, 3] and a cap drawn from {64, ..., 1024},
columns uniform over the matrix or within a band), computes the features of
each pattern and times the full candidate space (b in {32, 64, 128, 256} x
threads per row in {1, 2, 4, 8} x {fp64, fp32, bf16}) with the exhaustive
sweep. `train` fits the cost model (log of the kernel time) on the training
matrices in libpjds's CUDA kernels. `evaluate` reports the regret of the
model's choice against the sweep's best on the held-out matrices, for each
precision separately (the precision is the caller's choice; the tuner picks b
and threads per row within it) and over all candidates. `recheck` rebuilds
the first `--count` held-out matrices from their stored parameters, times
the candidate space again with the library as it is now, and reports the
model's regret on those fresh timings and their agreement with the stored
ones (the model is not retrained).
"""
from __future__ import annotations

import argparse
import json
import sys
import time

import numpy as np

DTYPES = ("f64", "f32", "bf16")


def matrix_params(i: int, seed: int, n_lo: float, n_hi: float) -> dict:
    """Deterministic parameters of the i-th synthetic matrix."""
    rng = np.random.default_rng([seed, i])
    n = int(np.exp(rng.uniform(np.log(n_lo), np.log(n_hi))))
    return {"n": n, "s": float(rng.uniform(1.5, 3.0)), "len_max": int(rng.choice([64, 128, 256, 512, 1024])),
            "banded": bool(rng.random() < 0.5), "bw": int(max(64, n * 10 ** rng.uniform(-4, -1))),
            "seed": int(seed * 100003 + i)}


def make_matrix(p: dict):
    import synth
    return synth.zipf_rows(p["n"], s=p["s"], len_max=min(p["len_max"], p["n"]), banded=p["banded"], bw=p["bw"],
                           seed=p["seed"])


def generate(n_train: int, n_test: int, seed: int = 2024, n_lo: float = 1e4, n_hi: float = 2e6, reps: int = 3,
             log=sys.stderr) -> dict:
    from . import learned, tune
    cands = tune.default_space(DTYPES)
    n_all = n_train + n_test
    feats = np.zeros((n_all, 8), np.float32)
    times = np.full((n_all, len(cands)), np.nan, np.float64)
    params = []
    t0 = time.time()
    for i in range(n_all):
        p = matrix_params(i, seed if i < n_train else seed + 1, n_lo, n_hi)
        A = make_matrix(p)
        feats[i] = learned.features(A)
        entries, _ = tune.sweep(A, cands, reps=reps, flush_bytes=0)
        for c, e in enumerate(entries):
            if e["status"] == 0 and e["us"] > 0:
                times[i, c] = e["us"]
        params.append(p)
        if (i + 1) % 50 == 0:
            print(f"[tuner_data] {i + 1}/{n_all} matrices, {time.time() - t0:.0f} s", file=log, flush=True)
    return {"features": feats, "times_us": times, "n_train": n_train,
            "cands": json.dumps(cands), "params": json.dumps(params)}


def samples(data: dict, rows):
    """(X, y) over (matrix, candidate) pairs with a valid time; y = log(us)."""
    from . import learned
    cands = json.loads(str(data["cands"]))
    X, y = [], []
    for i in rows:
        enc = learned.encode(data["features"][i], cands)
        ok = np.isfinite(data["times_us"][i])
        X.append(enc[ok])
        y.append(np.log(data["times_us"][i][ok]))
    return np.concatenate(X).astype(np.float32), np.concatenate(y).astype(np.float32)


def train(data: dict, epochs: int = 400, batch: int = 1024, lr: float = 2e-3, seed: int = 1):
    from . import learned
    n_train = int(data["n_train"])
    X, y = samples(data, range(n_train))
    m = learned.init(seed)
    learned.fit_scaling(m, X, y)
    hist = learned.train(m, X, y, epochs=epochs, batch=batch, lr=lr, seed=seed)
    return m, hist


def evaluate(data: dict, m) -> dict:
    """Regret of the model's choice on the held-out matrices."""
    from . import learned
    cands = json.loads(str(data["cands"]))
    n_train = int(data["n_train"])
    dt_of = np.array([DTYPES.index(c["dtype"]) for c in cands])
    out = {}
    groups = {"all": np.ones(len(cands), bool)}
    groups.update({d: dt_of == k for k, d in enumerate(DTYPES)})
    rows = range(n_train, len(data["times_us"]))
    preds = {i: learned.predict(m, learned.encode(data["features"][i], cands)) for i in rows}
    for name, sel in groups.items():
        reg, default_reg = [], []
        for i in rows:
            t = data["times_us"][i].copy()
            t[~sel] = np.nan
            if not np.any(np.isfinite(t)):
                continue
            p = preds[i].astype(np.float64).copy()
            p[~(sel & np.isfinite(t))] = np.inf
            best = np.nanmin(t)
            reg.append(t[int(np.argmin(p))] / best - 1.0)
            # the paper's mapping for comparison: b = 32, one thread per row
            j0 = [c for c in range(len(cands)) if sel[c] and cands[c]["b"] == 32 and cands[c]["threads_per_row"] == 1]
            if j0 and np.isfinite(t[j0[0]]):
                default_reg.append(t[j0[0]] / best - 1.0)
        reg = np.array(reg)
        out[name] = {"matrices": int(len(reg)), "mean_regret": float(reg.mean()),
                     "median_regret": float(np.median(reg)), "p90_regret": float(np.percentile(reg, 90)),
                     "within_5pct": float(np.mean(reg <= 0.05)),
                     "paper_mapping_mean_regret": float(np.mean(default_reg)) if default_reg else None}
    return out


def recheck(data: dict, m, count: int, reps: int = 3, log=sys.stderr) -> dict:
    """Fresh sweep of held-out matrices; regret of `m` on the new timings."""
    from . import tune
    cands = json.loads(str(data["cands"]))
    n_train = int(data["n_train"])
    params = json.loads(str(data["params"]))
    rows = list(range(n_train, min(len(params), n_train + count)))
    fresh = {k: np.asarray(v).copy() for k, v in data.items()}
    ratios = []
    t0 = time.time()
    for k, i in enumerate(rows):
        A = make_matrix(params[i])
        entries, _ = tune.sweep(A, cands, reps=reps, flush_bytes=0)
        t = np.full(len(cands), np.nan)
        for c, e in enumerate(entries):
            if e["status"] == 0 and e["us"] > 0:
                t[c] = e["us"]
        old = data["times_us"][i]
        ok = np.isfinite(t) & np.isfinite(old)
        ratios.extend((t[ok] / old[ok]).tolist())
        fresh["times_us"][i] = t
        if (k + 1) % 50 == 0:
            print(f"[tuner_data] recheck {k + 1}/{len(rows)}, {time.time() - t0:.0f} s", file=log, flush=True)
    fresh["times_us"] = fresh["times_us"][: n_train + len(rows)]
    fresh["features"] = fresh["features"][: n_train + len(rows)]
    r = np.array(ratios)
    return {"matrices": len(rows), "new_over_stored_time": {"median": float(np.median(r)),
                                                             "p10": float(np.percentile(r, 10)),
                                                             "p90": float(np.percentile(r, 90))},
            "regret_on_fresh_timings": evaluate(fresh, m)}


def main(argv=None) -> int:
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    sub = ap.add_subparsers(dest="cmd", required=True)
    g = sub.add_parser("generate")
    g.add_argument("--n-train", type=int, default=800)
    g.add_argument("--n-test", type=int, default=200)
    g.add_argument("--seed", type=int, default=2024)
    g.add_argument("--n-lo", type=float, default=1e4)
    g.add_argument("--n-hi", type=float, default=2e6)
    g.add_argument("--out", required=True)
    t = sub.add_parser("train")
    t.add_argument("data")
    t.add_argument("--model", required=True)
    t.add_argument("--epochs", type=int, default=400)
    t.add_argument("--batch", type=int, default=1024)
    t.add_argument("--lr", type=float, default=2e-3)
    e = sub.add_parser("evaluate")
    e.add_argument("data")
    e.add_argument("--model", required=True)
    r = sub.add_parser("recheck")
    r.add_argument("data")
    r.add_argument("--model", required=True)
    r.add_argument("--count", type=int, default=200)
    a = ap.parse_args(argv)
    if a.cmd == "generate":
        d = generate(a.n_train, a.n_test, a.seed, a.n_lo, a.n_hi)
        np.savez_compressed(a.out, **d)
        print(json.dumps({"saved": a.out, "matrices": a.n_train + a.n_test}))
    elif a.cmd == "train":
        from . import learned
        d = dict(np.load(a.data, allow_pickle=False))
        m, hist = train(d, a.epochs, a.batch, a.lr)
        ev = evaluate(d, m)
        learned.save(m, a.model, {"epochs": a.epochs, "batch": a.batch, "lr": a.lr, "final_loss": float(hist[-1]),
                                  "data": a.data, "heldout": ev})
        print(json.dumps({"model": a.model, "loss_first": float(hist[0]), "loss_last": float(hist[-1]),
                          "heldout": ev}))
    elif a.cmd == "recheck":
        from . import learned
        d = dict(np.load(a.data, allow_pickle=False))
        print(json.dumps(recheck(d, learned.load(a.model), a.count)))
    else:
        from . import learned
        d = dict(np.load(a.data, allow_pickle=False))
        print(json.dumps(evaluate(d, learned.load(a.model))))
    return 0


if __name__ == "__main__":
    sys.exit(main())
