"""Exhaustive autotuner on the GPU: every valid candidate is timed, invalid
ones are recorded and skipped, the best one is the fastest, and the best
configuration's product matches the oracle."""
import numpy as np
import pytest

import synth
from tests import parity

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_1112_5588_gb300 import build
    build.build()
    from paper_1112_5588_gb300 import pjds, tune
    return torch, pjds, tune


def test_sweep_and_best_candidate_parity(mods, oracle_lib):
    torch, pjds, tune = mods
    A = synth.zipf_rows(50_000, s=2.0, len_max=512, seed=5)
    cands = tune.default_space(("f64", "f32")) + [
        {"b": 48, "dtype": "f64"},                                 # not a multiple of 32
        {"b": 32, "dtype": "f64", "rows_per_thread": 4},
        {"b": 32, "dtype": "f64", "threads_per_row": 2, "unroll": 16},  # unroll not available for T=2
    ]
    entries, best = tune.sweep(A, cands, reps=3, flush_bytes=64 << 20)
    assert len(entries) == len(cands)
    assert entries[-3]["status"] == -1 and entries[-3]["us"] < 0
    assert entries[-1]["status"] == -1 and entries[-1]["us"] < 0
    valid = [i for i, e in enumerate(entries) if e["status"] == 0]
    assert len(valid) == len(cands) - 2
    assert all(entries[i]["us"] > 0 for i in valid)
    assert best == min(valid, key=lambda i: entries[i]["us"])
    assert entries[-2]["rows_per_thread"] == 4 and entries[-2]["threads_per_row"] == 1
    # the winner's configuration gives the oracle's product
    e = entries[best]
    H = pjds.pjds_create(A.n_rows, A.n_cols, A.row_ptr, A.col, A.val, b=e["b"], dtype=e["dtype"])
    D = H.to_device("cuda")
    x = synth.vector(A.n_cols, seed=9)
    xt = torch.from_numpy(x).to("cuda", D.vec_dtype)
    y = torch.empty(A.n_rows, dtype=D.vec_dtype, device="cuda")
    pjds.pjds_spmv_cfg(D, xt, y, rows_per_thread=e["rows_per_thread"], threads_per_row=e["threads_per_row"],
                       block_threads=e["block_threads"], unroll=e["unroll"])
    torch.cuda.synchronize()
    yo = y.double().cpu().numpy()
    if e["dtype"] == "f64":
        r = parity.check_fp64(yo, oracle_lib.crs_spmv(A, x), oracle_lib.crs_absmv(A, x), np.diff(A.row_ptr))
    else:
        Ar = A._replace(val=oracle_lib.round_f32(A.val))
        xd = x.astype(np.float32).astype(np.float64)
        r = parity.check_fp32(yo, oracle_lib.crs_spmv(Ar, xd), oracle_lib.crs_absmv(Ar, xd), np.diff(A.row_ptr))
    assert r["ok"], (e, r)


def test_sweep_times_the_per_tile_mapping(mods, oracle_lib):
    # plan candidates run the matrix's per-tile mapping; on widely spread rows
    # (Zipf s = 2, 1M rows: 1.4-1.7x over the best uniform count) it wins
    torch, pjds, tune = mods
    A = synth.zipf_rows(1_000_000, s=2.0, len_max=512, seed=6)
    cands = [c for c in tune.default_space(("f64",)) if c["plan"] == 1 or c["tile_order"] == -1]
    assert sum(c.get("plan", 0) == 1 for c in cands) == 4 and len(cands) == 20
    entries, best = tune.sweep(A, cands, reps=7)
    for c, e in zip(cands, entries):
        assert e["status"] == 0 and e["us"] > 0, e
        assert e["plan"] == (1 if c.get("plan") == 1 else -1), (c, e)
    assert entries[best]["plan"] == 1, [(e["b"], e["threads_per_row"], e["plan"], round(e["us"], 1)) for e in entries]
    # the winning candidate's product against the oracle
    e = entries[best]
    H = pjds.pjds_create(A.n_rows, A.n_cols, A.row_ptr, A.col, A.val, b=e["b"], dtype="f64")
    D = H.to_device("cuda")
    x = synth.vector(A.n_cols, seed=6)
    y = torch.full((A.n_rows,), float("nan"), dtype=torch.float64, device="cuda")
    pjds.pjds_spmv_cfg(D, torch.from_numpy(x).cuda(), y, plan=1)
    torch.cuda.synchronize()
    r = parity.check_fp64(y.cpu().numpy(), oracle_lib.crs_spmv(A, x), oracle_lib.crs_absmv(A, x), np.diff(A.row_ptr))
    assert r["ok"], r
