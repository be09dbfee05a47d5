"""Run one pJDS product case a few times, for profiling under ncu.

    python -m paper_1112_5588_gb300.profile_cases --matrix stencil --g 100 --dtype f64 --permuted --staged --reps 3

Builds one seeded synthetic matrix, converts it, uploads it and launches the
chosen product `--reps` times (after `--warmup` launches) on the current
stream, then prints one JSON line with the CUDA-event time of each launch.
Matrices: hmep (--n rows), stencil (--g grid), dlr (--n rows, 144/row), zipf
(--n rows). Kinds: spmv (default), ellr, spmm (--k right-hand sides);
cg (one mixed-precision CG solve of `--reps` inner steps in the permuted
basis, fp64 outer matrix, --dtype inner matrix, no graph) and lanczos
(`--reps` steps, no graph) on the stencil; batch (--mats Zipf matrices with
N log-uniform in [10k, --n], one persistent launch per repetition); mlp (the
learned tuner's cost model trained for `--reps` epochs on the committed
timing data, then inference over the candidates of the held-out matrices).
"""
from __future__ import annotations

import argparse
import json
import sys

import numpy as np


def main(argv=None) -> int:
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--matrix", choices=["hmep", "stencil", "dlr", "zipf"], default="hmep")
    ap.add_argument("--n", type=int, default=2_000_000)
    ap.add_argument("--g", type=int, default=100)
    ap.add_argument("--dtype", choices=["f64", "f32", "bf16"], default="f64")
    ap.add_argument("--kind", choices=["spmv", "ellr", "spmm", "cg", "lanczos", "batch", "mlp"], default="spmv")
    ap.add_argument("--mats", type=int, default=64)
    ap.add_argument("--k", type=int, default=8)
    ap.add_argument("--permuted", action="store_true")
    ap.add_argument("--staged", action="store_true")
    ap.add_argument("--threads-per-row", type=int, default=0)
    ap.add_argument("--rows-per-thread", type=int, default=0)
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=2)
    ap.add_argument("--seed", type=int, default=1234)
    a = ap.parse_args(argv)

    import torch

    import synth
    from . import batch, krylov, pjds

    dev = torch.device("cuda")
    if a.kind == "mlp":
        return run_mlp(a, torch)
    if a.kind == "batch":
        return run_batch(a, torch, synth, batch, pjds, dev)
    if a.kind in ("cg", "lanczos"):
        return run_krylov(a, torch, synth, krylov, pjds, dev)
    if a.matrix == "hmep":
        A = synth.hmep_like(n=a.n, seed=a.seed)
    elif a.matrix == "stencil":
        A = synth.stencil27(g=a.g, seed=a.seed)
    elif a.matrix == "dlr":
        A = synth.block_dense(n_brow=max(1, a.n // 4), bs=4, nb=36, frac=0.05, seed=a.seed)
    else:
        A = synth.zipf_rows(a.n, s=2.0, len_max=512, seed=a.seed)
    if a.kind == "ellr":
        D = pjds.ellr_create(A.n_rows, A.n_cols, A.row_ptr, A.col, A.val, dtype=a.dtype).to_device(dev)
    else:
        D = pjds.pjds_create(A.n_rows, A.n_cols, A.row_ptr, A.col, A.val, b=32, dtype=a.dtype,
                             permute_cols=a.permuted).to_device(dev)
    if a.kind == "spmm":
        X = torch.rand(A.n_cols, a.k, device=dev, dtype=D.vec_dtype)
        Y = torch.empty(A.n_rows, a.k, device=dev, dtype=D.vec_dtype)
        run = lambda: batch.spmm(D, X, Y)  # noqa: E731
    else:
        x = torch.from_numpy(synth.vector(A.n_cols, seed=a.seed)).to(dev, D.vec_dtype)
        y = torch.empty(A.n_rows, device=dev, dtype=D.vec_dtype)
        if a.kind == "ellr":
            run = lambda: pjds.ellr_spmv(D, x, y)  # noqa: E731
        else:
            kw = dict(staged=1 if a.staged else 0, threads_per_row=a.threads_per_row,
                      rows_per_thread=a.rows_per_thread)
            run = lambda: pjds.pjds_spmv_cfg(D, x, y, **kw)  # noqa: E731
    for _ in range(a.warmup):
        run()
    torch.cuda.synchronize()
    times = []
    for _ in range(a.reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        run()
        e1.record()
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1) * 1e3)
    status = pjds.pjds_device_status() if a.staged else 0
    print(json.dumps({"matrix": a.matrix, "n_rows": A.n_rows, "nnz": A.nnz, "dtype": a.dtype, "kind": a.kind,
                      "permuted": a.permuted, "staged": a.staged, "us": [round(t, 2) for t in times],
                      "device_status": status}))
    return 0 if status == 0 else 1


def _timed(torch, run, reps, warmup):
    for _ in range(warmup):
        run()
    torch.cuda.synchronize()
    times = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        run()
        e1.record()
        torch.cuda.synchronize()
        times.append(round(e0.elapsed_time(e1) * 1e3, 2))
    return times


def run_mlp(a, torch) -> int:
    import os
    import time
    from . import learned, tuner_data
    data = dict(np.load(os.path.join(os.path.dirname(__file__), "data", "tuner_timings_gb300.npz"),
                        allow_pickle=False))
    X, y = tuner_data.samples(data, range(int(data["n_train"])))
    m = learned.init(1)
    learned.fit_scaling(m, X, y)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    hist = learned.train(m, X, y, epochs=a.reps, batch=1024, lr=2e-3, seed=1)
    t_train = time.perf_counter() - t0
    cands = __import__("json").loads(str(data["cands"]))
    rows = range(int(data["n_train"]), len(data["times_us"]))
    enc = np.concatenate([learned.encode(data["features"][i], cands) for i in rows])
    learned.predict(m, enc)
    t0 = time.perf_counter()
    learned.predict(m, enc)
    t_pred = time.perf_counter() - t0
    print(json.dumps({"kind": "mlp", "samples": int(len(y)), "epochs": a.reps, "train_s": round(t_train, 3),
                      "s_per_epoch": round(t_train / max(a.reps, 1), 4), "loss_first": float(hist[0]),
                      "loss_last": float(hist[-1]), "predict_rows": int(len(enc)), "predict_us": round(t_pred * 1e6, 1)}))
    return 0


def run_batch(a, torch, synth, batch, pjds, dev) -> int:
    rng = np.random.default_rng(a.seed)
    sizes = np.exp(rng.uniform(np.log(10_000), np.log(max(a.n, 10_001)), a.mats)).astype(int)
    devs, xs, ys, nnz = [], [], [], 0
    for m, n in enumerate(sizes):
        M = synth.zipf_rows(int(n), s=2.0, len_max=512, seed=a.seed + m)
        nnz += M.nnz
        devs.append(pjds.pjds_create(M.n_rows, M.n_cols, M.row_ptr, M.col, M.val, b=32,
                                     dtype=a.dtype).to_device(dev))
        xs.append(torch.from_numpy(synth.vector(M.n_cols, seed=m)).to(dev, devs[-1].vec_dtype))
        ys.append(torch.empty(M.n_rows, dtype=devs[-1].vec_dtype, device=dev))
    B = batch.Batch(devs, xs, ys)
    times = _timed(torch, lambda: B.run(use_graph=False), a.reps, a.warmup)
    info = B.info()
    B.destroy()
    print(json.dumps({"kind": "batch", "n_mats": a.mats, "total_rows": int(sizes.sum()), "nnz": int(nnz),
                      "dtype": a.dtype, **info, "us": times}))
    return 0


def run_krylov(a, torch, synth, krylov, pjds, dev) -> int:
    A = synth.stencil27(g=a.g, seed=a.seed)
    H64 = pjds.pjds_create(A.n_rows, A.n_cols, A.row_ptr, A.col, A.val, b=32, dtype="f64", permute_cols=True)
    D64 = H64.to_device(dev)
    H64.destroy()
    if a.kind == "cg":
        Dlo = D64 if a.dtype == "f64" else pjds.pjds_create(
            A.n_rows, A.n_cols, A.row_ptr, A.col, A.val, b=32, dtype=a.dtype, permute_cols=True).to_device(dev)
        b = torch.from_numpy(synth.vector(A.n_rows, seed=a.seed)).to(dev)
        x = torch.zeros_like(b)

        def run():
            x.zero_()
            krylov.cg_solve(D64, Dlo, b, x, max_outer=1, inner_iters=a.reps, use_graph=False)
        times = _timed(torch, run, 1, a.warmup)
    else:
        D = D64 if a.dtype == "f64" else pjds.pjds_create(
            A.n_rows, A.n_cols, A.row_ptr, A.col, A.val, b=32, dtype=a.dtype, permute_cols=True).to_device(dev)
        v0 = torch.from_numpy(synth.vector(A.n_rows, seed=a.seed)).to(dev, D.vec_dtype)
        times = _timed(torch, lambda: krylov.lanczos(D, v0, a.reps, use_graph=False), 1, a.warmup)
    print(json.dumps({"kind": a.kind, "matrix": f"stencil g={a.g}", "n_rows": A.n_rows, "nnz": A.nnz,
                      "dtype": a.dtype, "steps": a.reps, "us_total": times}))
    return 0


if __name__ == "__main__":
    sys.exit(main())
