"""Training data, training and regret evaluation of the learned tuner.

Run on a GPU:

    python -m paper_1112_5588_gb300.tuner_data generate --n-train 800 --n-test 200 --out timings.npz
    python -m paper_1112_5588_gb300.tuner_data train timings.npz --model tuner_mlp.json
    python -m paper_1112_5588_gb300.tuner_data evaluate timings.npz --model tuner_mlp.json
    python -m paper_1112_5588_gb300.tuner_data recheck timings.npz --model tuner_mlp.json --count 200
    python -m paper_1112_5588_gb300.tuner_data plan-eval timings.npz --rows train --out plan_train.npz
    python -m paper_1112_5588_gb300.tuner_data plan-eval timings.npz --rows test --out plan_test.npz
    python -m paper_1112_5588_gb300.tuner_data plan-fit plan_train.npz plan_test.npz      # CPU

`generate` draws seeded synthetic matrices (N log-uniform in [10k, 20M] by
default, Zipf(s) row lengths with s uniform in [1.5, 3] and a cap drawn from
{64, ..., 1024}, columns uniform over the matrix or within a band), computes
the features of each pattern and times the full candidate space (b in {32,
64, 128, 256} x threads per row in {1, 2, 4, 8} x tile order in {sorted,
traversal table}, plus the per-tile mapping for each b, x {fp64, fp32, bf16}:
108 candidates) with the exhaustive sweep. `train` fits the cost model (log of the kernel time) on the training
matrices in libpjds's CUDA kernels and stores their feature range in the
model (outside it pjds_tune_pick falls back to the sweep). `evaluate` reports the regret of the
model's choice against the sweep's best on the held-out matrices, for each
precision separately (the precision is the caller's choice; the tuner picks b,
threads per row, tile order or the per-tile mapping within it) and over all
candidates, beside the regret of the paper's fixed mapping and of the
library's default mapping. `recheck` rebuilds
the first `--count` held-out matrices from their stored parameters, times
the candidate space again with the library as it is now, and reports the
model's regret on those fresh timings and their agreement with the stored
ones (the model is not retrained).

`plan-eval` times, for each matrix and precision, the stored timings' best
uniform candidate and the per-tile mapping at the same b in one sweep (L2
flushed), and records how far the uniform rule's own pick is from the best
in the stored timings. `plan-fit` chooses, per precision, the row count from
which the default takes the per-tile mapping (fitted on the training
matrices, reported on the held-out ones).
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


def generate(n_train: int, n_test: int, seed: int = 2024, n_lo: float = 1e4, n_hi: float = 2e7, reps: int = 3,
             log=sys.stderr, checkpoint: str | None = None, resume: dict | None = None) -> dict:
    """Time the candidate space (tune.default_space: 36 candidates per
    precision) on n_train + n_test synthetic matrices; with `checkpoint`, the
    data gathered so far is saved there every 100 matrices; `resume` (such a
    checkpoint, same arguments) continues after its last matrix."""
    from . import learned, tune
    cands = tune.default_space(DTYPES)
    n_all = n_train + n_test
    feats = np.zeros((n_all, 8), np.float32)
    times = np.full((n_all, len(cands)), np.nan, np.float64)
    sizes = np.zeros((n_all, 3), np.int64)  # n_rows, nnz, longest row
    params = []
    if resume is not None:
        if json.loads(str(resume["cands"])) != cands:
            raise ValueError("the checkpoint was taken over another candidate space")
        params = json.loads(str(resume["params"]))
        k0 = len(params)
        feats[:k0], times[:k0], sizes[:k0] = resume["features"], resume["times_us"], resume["sizes"]
    t0 = time.time()

    def pack(k):
        return {"features": feats[:k], "times_us": times[:k], "sizes": sizes[:k], "n_train": min(n_train, k),
                "cands": json.dumps(cands), "params": json.dumps(params[:k])}
    for i in range(len(params), n_all):
        p = matrix_params(i, seed if i < n_train else seed + 1, n_lo, n_hi)
        A = make_matrix(p)
        feats[i] = learned.features(A)
        sizes[i] = (A.n_rows, A.nnz, int(np.diff(A.row_ptr).max()))
        entries, _ = tune.sweep(A, cands, reps=reps, flush_bytes=0)
        for c, e in enumerate(entries):
            if e["status"] == 0 and e["us"] > 0:
                times[i, c] = e["us"]
        params.append(p)
        if (i + 1) % 50 == 0:
            print(f"[tuner_data] {i + 1}/{n_all} matrices, {time.time() - t0:.0f} s", file=log, flush=True)
        if checkpoint and (i + 1) % 100 == 0:
            np.savez_compressed(checkpoint, **pack(i + 1))
    return pack(n_all)


def default_index(cands, n_rows: int, nnz: int, n_max: int, dtype: str) -> int:
    """Index of the candidate pjds_spmv's default mapping runs for a matrix of
    these sizes at b = 32 (include/pjds.h): the per-tile mapping when the
    longest row exceeds 4 times the mean and n_rows reaches 2^16 / 2^17 / 2^18
    (fp64 / fp32 / bf16), else the uniform threads per row with the traversal
    table from 2^20 rows when the longest row is at most 4 times the mean."""
    spread = n_max * n_rows > 4 * nnz
    min_rows = {"f64": 1 << 16, "f32": 1 << 17, "bf16": 1 << 18}[dtype]
    for k, c in enumerate(cands):
        if c["dtype"] != dtype or c["b"] != 32:
            continue
        if spread and n_rows >= min_rows:
            if c["plan"] == 1:
                return k
            continue
        order = 1 if n_rows >= (1 << 20) and not spread else -1
        if c["plan"] != 1 and c["threads_per_row"] == uniform_threads(n_rows, nnz, n_max, dtype) and \
                c["tile_order"] == order:
            return k
    return -1


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
    learned.fit_range(m, np.asarray(data["features"][:n_train], np.float32))
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
    sizes = data.get("sizes")
    for name, sel in groups.items():
        reg, paper_reg, lib_reg = [], [], []
        for i in rows:
            t = data["times_us"][i].copy()
            t[~sel] = np.nan
            if not np.any(np.isfinite(t)):
                continue
            p = preds[i].astype(np.float64).copy()
            p[~(sel & np.isfinite(t))] = np.inf
            best = np.nanmin(t)
            reg.append(t[int(np.argmin(p))] / best - 1.0)
            # the paper's mapping for comparison: b = 32, one thread per row, sorted order
            j0 = [c for c in range(len(cands)) if sel[c] and cands[c]["b"] == 32 and cands[c]["threads_per_row"] == 1
                  and cands[c].get("plan", 0) != 1 and cands[c].get("tile_order", -1) in (0, -1)]
            if j0 and np.isfinite(t[j0[0]]):
                paper_reg.append(t[j0[0]] / best - 1.0)
            # the library's default mapping (pjds_spmv), when the sizes are stored
            if sizes is not None and name in DTYPES:
                k = default_index(cands, *[int(v) for v in sizes[i]], name)
                if k >= 0 and np.isfinite(t[k]):
                    lib_reg.append(t[k] / best - 1.0)
        reg = np.array(reg)
        out[name] = {"matrices": int(len(reg)), "mean_regret": float(reg.mean()),
                     "median_regret": float(np.median(reg)), "p90_regret": float(np.percentile(reg, 90)),
                     "within_5pct": float(np.mean(reg <= 0.05)),
                     "paper_mapping_mean_regret": float(np.mean(paper_reg)) if paper_reg else None,
                     "library_default_mean_regret": float(np.mean(lib_reg)) if lib_reg else None}
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


def uniform_threads(n_rows: int, nnz: int, n_max: int, dtype: str) -> int:
    """Threads per row of pjds_spmv's uniform mapping (api.cu): the longest
    row's chain against the product's stream time, ratio = n_max * 2^20 /
    (nnz * entry bytes); 1 below 2, 2 below 8, 4 below 64, else 8; doubled
    while n_rows * T < 2^17."""
    entry = {"f64": 12, "f32": 8, "bf16": 6}[dtype]
    num, den = n_max * 2**20, max(nnz, 1) * entry
    t = 1 if num < 2 * den else 2 if num < 8 * den else 4 if num < 64 * den else 8
    while t < 8 and n_rows * t < 2**17:
        t *= 2
    return t


def plan_eval(data: dict, rows, reps: int = 3, log=sys.stderr) -> dict:
    """Per matrix row i and precision: the re-timed best uniform candidate,
    the per-tile mapping at its b (one sweep, L2 flushed), and the uniform
    rule's stored time over the stored best."""
    from . import tune
    cands = json.loads(str(data["cands"]))
    params = json.loads(str(data["params"]))
    stored = data["times_us"]
    # the uniform candidates in sorted order (the full candidate space also
    # holds the traversal-table and per-tile entries)
    ci = {(c["b"], c["dtype"], c["threads_per_row"]): k for k, c in enumerate(cands)
          if c.get("plan", 0) != 1 and c.get("tile_order", 0) in (0, -1)}
    out = {"i": [], "n": []}
    for dt in DTYPES:
        out[f"{dt}_uniform_us"], out[f"{dt}_plan_us"], out[f"{dt}_rule_over_best"] = [], [], []
    t0 = time.time()
    for k, i in enumerate(rows):
        A = make_matrix(params[i])
        lens = np.diff(A.row_ptr)
        test = []
        for dt in DTYPES:
            idx = [k for k in ci.values() if cands[k]["dtype"] == dt]
            best = min(idx, key=lambda c: stored[i, c])
            cand = {key: cands[best][key] for key in ("b", "dtype", "rows_per_thread", "threads_per_row",
                                                      "block_threads", "unroll", "staged")}
            test += [cand, {"b": cand["b"], "dtype": dt, "plan": 1}]
        entries, _ = tune.sweep(A, test, reps=reps)
        out["i"].append(i)
        out["n"].append(A.n_rows)
        for j, dt in enumerate(DTYPES):
            u, p = entries[2 * j], entries[2 * j + 1]
            ok = u["status"] == 0 and p["status"] == 0
            t_rule = uniform_threads(A.n_rows, A.nnz, int(lens.max()), dt)
            best_stored = np.nanmin([stored[i, k] for k in ci.values() if cands[k]["dtype"] == dt])
            out[f"{dt}_uniform_us"].append(u["us"] if ok else np.nan)
            out[f"{dt}_plan_us"].append(p["us"] if ok else np.nan)
            out[f"{dt}_rule_over_best"].append(stored[i, ci[(32, dt, t_rule)]] / best_stored)
        if (k + 1) % 200 == 0:
            print(f"[tuner_data] plan-eval {k + 1}/{len(rows)}, {time.time() - t0:.0f} s", file=log, flush=True)
    return {key: np.asarray(v) for key, v in out.items()}


def plan_fit(train: dict, test: dict) -> dict:
    """Per precision, the power-of-two row count from which taking the
    per-tile mapping (else the uniform rule) minimises the geometric mean of
    the time over the best uniform candidate on the training matrices; that
    mean on the held-out matrices, beside the uniform rule alone and the plan
    always."""
    def score(d, dt, thr):
        u, p, r = d[f"{dt}_uniform_us"], d[f"{dt}_plan_us"], d[f"{dt}_rule_over_best"]
        ok = np.isfinite(u) & np.isfinite(p) & np.isfinite(r)
        t = np.where(d["n"] >= thr, p, u * r)
        return float(np.exp(np.mean(np.log(t[ok] / u[ok]))))
    res = {}
    for dt in DTYPES:
        cands = [2 ** k for k in range(14, 23)]
        thr = min(cands, key=lambda t: score(train, dt, t))
        res[dt] = {"min_rows": thr, "train": round(score(train, dt, thr), 3), "test": round(score(test, dt, thr), 3),
                   "test_rule_only": round(score(test, dt, float("inf")), 3),
                   "test_plan_always": round(score(test, dt, 0), 3)}
    return res


def main(argv=None) -> int:
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    sub = ap.add_subparsers(dest="cmd", required=True)
    g = sub.add_parser("generate")
    g.add_argument("--n-train", type=int, default=800)
    g.add_argument("--n-test", type=int, default=200)
    g.add_argument("--seed", type=int, default=2024)
    g.add_argument("--n-lo", type=float, default=1e4)
    g.add_argument("--n-hi", type=float, default=2e7)
    g.add_argument("--out", required=True)
    g.add_argument("--checkpoint", default=None)
    g.add_argument("--resume", default=None, help="a checkpoint of the same command to continue from")
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
    pe = sub.add_parser("plan-eval")
    pe.add_argument("data")
    pe.add_argument("--rows", choices=["train", "test"], required=True)
    pe.add_argument("--out", required=True)
    pf = sub.add_parser("plan-fit")
    pf.add_argument("train")
    pf.add_argument("test")
    a = ap.parse_args(argv)
    if a.cmd == "generate":
        d = generate(a.n_train, a.n_test, a.seed, a.n_lo, a.n_hi, checkpoint=a.checkpoint,
                     resume=dict(np.load(a.resume, allow_pickle=False)) if a.resume else None)
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
    elif a.cmd == "plan-eval":
        d = dict(np.load(a.data, allow_pickle=False))
        nt = int(d["n_train"])
        rows = range(0, nt) if a.rows == "train" else range(nt, len(d["times_us"]))
        np.savez_compressed(a.out, **plan_eval(d, rows))
        print(json.dumps({"saved": a.out, "matrices": len(rows)}))
    elif a.cmd == "plan-fit":
        print(json.dumps(plan_fit(dict(np.load(a.train)), dict(np.load(a.test)))))
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
