"""Cases for the checked build (run by tests/test_gpu_checked.py in a process
with PJDS_LIBRARY=checked, which loads libpjds_checked.so).

Clean: every mapping of the product with device-side extent checks (one and
T threads per row, several rows per thread, tile order, per-tile mapping,
64-bit offsets), the pattern product, ELLPACK-R, the block product (also with
paired rows on a block-structured matrix) and the batched launch, on ragged,
spread, banded and block-dense matrices, must leave the check word at 0 and
match the oracle (fp64; fp32 bounds for the paired block product).

Planted: an index put out of range in a device copy of a matrix (a column
beyond n_cols, a perm entry beyond n_rows, a jagged-diagonal offset beyond
the stored entries, a block longer than the longest row) must be recorded
with its code and skipped: the kernels check each index before the access.

Prints one JSON line.
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

CFGS = [dict(), dict(threads_per_row=1), dict(rows_per_thread=2), dict(rows_per_thread=4), dict(threads_per_row=2),
        dict(threads_per_row=4), dict(threads_per_row=8), dict(tile_order=1), dict(plan=1), dict(index64=1),
        dict(plan=1, index64=1), dict(rows_per_thread=2, index64=1)]
CODE_SHIFT = 56


def split(w):
    return w >> CODE_SHIFT, w & ((1 << CODE_SHIFT) - 1)


def main():
    assert os.environ.get("PJDS_LIBRARY") == "checked"
    import torch

    import oracle
    import synth
    from paper_1112_5588_gb300 import batch, pjds
    from synth import tiny
    from tests import parity
    assert pjds.LIB_PATH.endswith("libpjds_checked.so")
    oracle.build()
    assert pjds.pjds_check_word(clear=True) == 0

    mats = {
        "ragged": tiny.random_lengths(1037, 1037, max_len=90, seed=61, p_empty=0.2),
        "zipf": synth.zipf_rows(70_000, s=1.8, len_max=600, seed=62),
        "hmep": synth.hmep_like(n=30_011, seed=63),
        "full_row": tiny.one_full_row(900, full_row=37),
    }
    res = {"clean": [], "planted": {}}

    def run(D, xt, cfg):
        y = torch.full((D.n_rows,), float("nan"), dtype=D.vec_dtype, device="cuda")
        pjds.pjds_spmv_cfg(D, xt, y, **cfg)
        torch.cuda.synchronize()
        return y

    for name, A in mats.items():
        x = synth.vector(A.n_cols, seed=64)
        yref, absax, lens = oracle.crs_spmv(A, x), oracle.crs_absmv(A, x), np.diff(A.row_ptr)
        for dt in ("f64", "f32", "bf16"):
            for b in (32, 128):
                H = pjds.pjds_create(A.n_rows, A.n_cols, A.row_ptr, A.col, A.val, b=b, dtype=dt)
                D = H.to_device("cuda")
                H.destroy()
                xt = torch.from_numpy(x).to("cuda", D.vec_dtype)
                for cfg in CFGS:
                    y = run(D, xt, cfg)
                    w = pjds.pjds_check_word(clear=True)
                    ok = bool(torch.isfinite(y).all())
                    if dt == "f64":
                        ok = ok and parity.check_fp64(y.cpu().numpy(), yref, absax, lens)["ok"]
                    res["clean"].append([name, dt, b, cfg, w, ok])
                # the pattern product (the gather ceiling) with one and two rows per thread
                for cfg in (dict(threads_per_row=1), dict(rows_per_thread=2)):
                    y = torch.full((D.n_rows,), float("nan"), dtype=D.vec_dtype, device="cuda")
                    pjds.pjds_spmv_pattern(D, xt, y, **cfg)
                    torch.cuda.synchronize()
                    w = pjds.pjds_check_word(clear=True)
                    res["clean"].append([name, dt, b, dict(pattern=1, **cfg), w, bool(torch.isfinite(y).all())])
            E = pjds.ellr_create(A.n_rows, A.n_cols, A.row_ptr, A.col, A.val, dtype=dt).to_device("cuda")
            y = torch.full((A.n_rows,), float("nan"), dtype=E.vec_dtype, device="cuda")
            pjds.ellr_spmv(E, torch.from_numpy(x).to("cuda", E.vec_dtype), y)
            torch.cuda.synchronize()
            w = pjds.pjds_check_word(clear=True)
            ok = bool(torch.isfinite(y).all())
            if dt == "f64":
                ok = ok and parity.check_fp64(y.cpu().numpy(), yref, absax, lens)["ok"]
            res["clean"].append([name, dt, 0, "ellr", w, ok])

    # SpMM: k right-hand sides
    for name, A in mats.items():
        lens = np.diff(A.row_ptr)
        for dt, ks in (("f64", (2, 8)), ("f32", (4, 32))):
            D = pjds.pjds_create(A.n_rows, A.n_cols, A.row_ptr, A.col, A.val, b=32, dtype=dt).to_device("cuda")
            for k in ks:
                X = np.stack([synth.vector(A.n_cols, seed=70 + c) for c in range(k)], axis=1)
                Y = torch.full((A.n_rows, k), float("nan"), dtype=D.vec_dtype, device="cuda")
                batch.spmm(D, torch.from_numpy(np.ascontiguousarray(X)).to("cuda", D.vec_dtype), Y)
                torch.cuda.synchronize()
                w = pjds.pjds_check_word(clear=True)
                ok = bool(torch.isfinite(Y).all())
                if dt == "f64":
                    Yr = oracle.crs_spmm(A, X)
                    S = np.abs(oracle.crs_spmm(A._replace(val=np.abs(A.val)), np.abs(X)))
                    Yg = Y.cpu().numpy()
                    ok = ok and all(parity.check_fp64(Yg[:, c], Yr[:, c], S[:, c], lens)["ok"] for c in range(k))
                res["clean"].append([name, dt, 32, f"spmm k={k}", w, ok])

    # the batched launch over all four matrices, with the built-in rule and given lanes
    devs = [pjds.pjds_create(A.n_rows, A.n_cols, A.row_ptr, A.col, A.val, b=32).to_device("cuda")
            for A in mats.values()]
    xs = [torch.from_numpy(synth.vector(A.n_cols, seed=65)).cuda() for A in mats.values()]
    for kw in (dict(), dict(lanes=[1, 8, 2, 4]), dict(rule=(4, 16, 64))):
        ys = [torch.full((A.n_rows,), float("nan"), dtype=torch.float64, device="cuda") for A in mats.values()]
        B = batch.Batch(devs, xs, ys, **kw)
        B.run(use_graph=False)
        torch.cuda.synchronize()
        w = pjds.pjds_check_word(clear=True)
        ok = all(parity.check_fp64(y.cpu().numpy(), oracle.crs_spmv(A, xv.cpu().numpy()),
                                   oracle.crs_absmv(A, xv.cpu().numpy()), np.diff(A.row_ptr))["ok"]
                 for A, xv, y in zip(mats.values(), xs, ys))
        B.destroy()
        res["clean"].append(["batch", "f64", 32, kw.get("lanes") and "lanes" or kw.get("rule") and "rule" or "default",
                             w, ok])

    # paired rows (block-structured, 2^18 rows of 64: pair_share 1000): the
    # single product (two rows per thread), the paired block product and its
    # pattern product
    Pm = synth.block_dense(70_000, 4, 16, 0.05, seed=67)
    lens = np.diff(Pm.row_ptr)
    for dt, k in (("f32", 8), ("bf16", 16)):
        D = pjds.pjds_create(Pm.n_rows, Pm.n_cols, Pm.row_ptr, Pm.col, Pm.val, b=32, dtype=dt).to_device("cuda")
        assert D.pair_share >= 500 and pjds.pjds_spmv_resolve(D)["rows_per_thread"] == 2
        xt = torch.from_numpy(synth.vector(Pm.n_cols, seed=68)).to("cuda", D.vec_dtype)
        y = run(D, xt, {})
        res["clean"].append(["paired", dt, 32, "spmv", pjds.pjds_check_word(clear=True), bool(torch.isfinite(y).all())])
        X = np.stack([synth.vector(Pm.n_cols, seed=80 + c) for c in range(k)], axis=1).astype(np.float32)
        Xt = torch.from_numpy(np.ascontiguousarray(X)).cuda()
        for fn, tag in ((batch.spmm, "spmm"), (batch.spmm_pattern, "spmm_pattern")):
            Y = torch.full((Pm.n_rows, k), float("nan"), device="cuda")
            fn(D, Xt, Y)
            torch.cuda.synchronize()
            w = pjds.pjds_check_word(clear=True)
            ok = bool(torch.isfinite(Y).all())
            if tag == "spmm":
                Ar = Pm._replace(val=oracle.round_f32(Pm.val) if dt == "f32" else oracle.round_bf16(Pm.val))
                Xd = X.astype(np.float64)
                Yr, S = oracle.crs_spmm(Ar, Xd), oracle.crs_spmm(Ar._replace(val=np.abs(Ar.val)), np.abs(Xd))
                Yg = Y.double().cpu().numpy()
                ok = ok and all(parity.check_fp32(Yg[:, c], Yr[:, c], S[:, c], lens)["ok"] for c in (0, k - 1))
            res["clean"].append(["paired", dt, 32, f"{tag} k={k}", w, ok])
    # a column beyond n_cols in the paired block product: recorded and skipped
    D = pjds.pjds_create(Pm.n_rows, Pm.n_cols, Pm.row_ptr, Pm.col, Pm.val, b=32, dtype="f32").to_device("cuda")
    D.col[1] = Pm.n_cols + 11
    Y = torch.empty(Pm.n_rows, 8, device="cuda")
    batch.spmm(D, torch.rand(Pm.n_cols, 8, device="cuda"), Y)
    torch.cuda.synchronize()
    res["planted"]["paired_column"] = [[{}, *split(pjds.pjds_check_word(clear=True))]]
    res["paired_n_cols"] = Pm.n_cols

    # planted indices (fp64, original basis)
    A = mats["ragged"]
    H = pjds.pjds_create(A.n_rows, A.n_cols, A.row_ptr, A.col, A.val, b=32)
    x = synth.vector(A.n_cols, seed=66)
    mapping = [dict(threads_per_row=1), dict(rows_per_thread=2), dict(threads_per_row=4), dict(plan=1), dict()]

    def planted(mutate):
        out = []
        for cfg in mapping:
            D = H.to_device("cuda")
            mutate(D)
            xt = torch.from_numpy(x).cuda()
            pjds.pjds_check_word(clear=True)
            run(D, xt, cfg)
            out.append([cfg, *split(pjds.pjds_check_word(clear=True))])
        return out

    res["n"] = {"n_rows": A.n_rows, "n_cols": A.n_cols, "n_stored": H.n_stored, "n_max": H.n_max}
    res["planted"]["column"] = planted(lambda D: D.col.__setitem__(0, A.n_cols + 5))
    res["planted"]["perm"] = planted(lambda D: D.perm.__setitem__(3, A.n_rows + 7))
    res["planted"]["offset"] = planted(lambda D: D.col_start.__setitem__(1, H.n_stored + 1000))
    res["planted"]["block"] = planted(lambda D: D.block_len.__setitem__(0, H.n_max + 3))
    # a planted column changes at most the one row that holds it
    D = H.to_device("cuda")
    xt = torch.from_numpy(x).cuda()
    y0 = run(D, xt, dict(threads_per_row=1))
    D.col[0] = A.n_cols + 5
    y1 = run(D, xt, dict(threads_per_row=1))
    pjds.pjds_check_word(clear=True)
    res["column_rows_changed"] = int((y0 != y1).sum().item())
    # ELLPACK-R with a column beyond n_cols
    E = pjds.ellr_create(A.n_rows, A.n_cols, A.row_ptr, A.col, A.val).to_device("cuda")
    k = int(np.argmax(np.diff(A.row_ptr) > 0))
    E.col[k] = A.n_cols + 9
    y = torch.empty(A.n_rows, dtype=torch.float64, device="cuda")
    pjds.ellr_spmv(E, torch.from_numpy(x).cuda(), y)
    torch.cuda.synchronize()
    res["planted"]["ellr_column"] = [[{}, *split(pjds.pjds_check_word(clear=True))]]
    # SpMM with a column beyond n_cols
    D = H.to_device("cuda")
    D.col[0] = A.n_cols + 5
    Y = torch.empty(A.n_rows, 4, dtype=torch.float64, device="cuda")
    batch.spmm(D, torch.rand(A.n_cols, 4, dtype=torch.float64, device="cuda"), Y)
    torch.cuda.synchronize()
    res["planted"]["spmm_column"] = [[{}, *split(pjds.pjds_check_word(clear=True))]]
    print(json.dumps(res))


if __name__ == "__main__":
    main()
