"""GPU batched products: pjds_spmm against the oracle's block product and,
column by column, bit for bit against pjds_spmv with one thread per row; the
persistent multi-matrix launch against the oracle and the single products."""
import numpy as np
import pytest

import synth
from synth import tiny
from tests import parity

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_1112_5588_gb300 import build
    build.build()
    from paper_1112_5588_gb300 import batch, pjds
    return torch, pjds, batch


SHAPES = [("dlr", lambda: synth.block_dense(n_brow=3000, bs=4, nb=36, frac=0.05, seed=3)),
          ("zipf", lambda: synth.zipf_rows(20_000, s=2.0, len_max=512, seed=4)),
          ("ragged", lambda: tiny.random_lengths(1037, 900, max_len=70, seed=5, p_empty=0.2))]


@pytest.mark.parametrize("dtype,k", [("f64", 2), ("f64", 8), ("f64", 32), ("f32", 4), ("f32", 16), ("f32", 32),
                                     ("f32", 128), ("bf16", 8)])
@pytest.mark.parametrize("name,make", SHAPES, ids=[s[0] for s in SHAPES])
def test_spmm_matches_oracle_and_columnwise_spmv(mods, oracle_lib, dtype, k, name, make):
    torch, pjds, batch = mods
    A = make()
    X = np.random.default_rng(k).uniform(-1, 1, (A.n_cols, k))
    if dtype != "f64":
        X = X.astype(np.float32).astype(np.float64)
    H = pjds.pjds_create(A.n_rows, A.n_cols, A.row_ptr, A.col, A.val, b=32, dtype=dtype)
    D = H.to_device("cuda")
    Xt = torch.from_numpy(X).to("cuda", D.vec_dtype).contiguous()
    Yt = torch.full((A.n_rows, k), float("nan"), dtype=D.vec_dtype, device="cuda")
    batch.spmm(D, Xt, Yt)
    torch.cuda.synchronize()
    Y = Yt.double().cpu().numpy()
    Ar = A if dtype == "f64" else A._replace(
        val=oracle_lib.round_f32(A.val) if dtype == "f32" else oracle_lib.round_bf16(A.val))
    Yr = oracle_lib.crs_spmm(Ar, X)
    S = oracle_lib.crs_spmm(Ar._replace(val=np.abs(Ar.val)), np.abs(X))
    lens = np.diff(A.row_ptr)
    check = parity.check_fp64 if dtype == "f64" else parity.check_fp32
    for c in range(k):
        r = check(Y[:, c], Yr[:, c], S[:, c], lens)
        assert r["ok"], (c, r)
    # same arithmetic as the single product, column by column
    for c in (0, k - 1):
        y1 = torch.empty(A.n_rows, dtype=D.vec_dtype, device="cuda")
        pjds.pjds_spmv_cfg(D, Xt[:, c].contiguous(), y1, threads_per_row=1, rows_per_thread=1)
        torch.cuda.synchronize()
        assert torch.equal(y1, Yt[:, c].contiguous())


def test_spmm_permuted_basis_and_k1(mods):
    torch, pjds, batch = mods
    A = synth.stencil27(g=16, seed=2)
    H = pjds.pjds_create(A.n_rows, A.n_cols, A.row_ptr, A.col, A.val, b=32, dtype="f32", permute_cols=True)
    D = H.to_device("cuda")
    X = torch.rand(A.n_rows, 8, device="cuda")
    Y = torch.empty_like(X)
    batch.spmm(D, X, Y)
    for c in range(8):
        y1 = torch.empty(A.n_rows, device="cuda")
        pjds.pjds_spmv_cfg(D, X[:, c].contiguous(), y1, threads_per_row=1)
        torch.cuda.synchronize()
        assert torch.equal(y1, Y[:, c].contiguous())
    X1 = X[:, :1].contiguous()
    Y1 = torch.empty(A.n_rows, 1, device="cuda")
    batch.spmm(D, X1, Y1)
    y1 = torch.empty(A.n_rows, device="cuda")
    pjds.pjds_spmv(D, X1.reshape(-1), y1)
    torch.cuda.synchronize()
    assert torch.equal(Y1.reshape(-1), y1)


def test_spmm_rejects_bad_k(mods):
    torch, pjds, batch = mods
    A = tiny.random_lengths(64, 64, max_len=8, seed=1)
    D = pjds.pjds_create(A.n_rows, A.n_cols, A.row_ptr, A.col, A.val, dtype="f32").to_device("cuda")
    for k in (3, 6, 132):
        with pytest.raises(pjds.PjdsError):
            batch.spmm(D, torch.zeros(64, k, device="cuda"), torch.zeros(64, k, device="cuda"))


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("graph", [True, False])
def test_batch_uneven_matrices(mods, oracle_lib, dtype, graph):
    torch, pjds, batch = mods
    rng = np.random.default_rng(7)
    sizes = np.exp(rng.uniform(np.log(300), np.log(60_000), 24)).astype(int)
    mats, devs, xs, ys, xh = [], [], [], [], []
    for m, n in enumerate(sizes):
        A = synth.zipf_rows(int(n), s=2.0, len_max=512, seed=100 + m) if m % 3 else \
            tiny.random_lengths(int(n), int(n), max_len=min(40, int(n)), seed=m, p_empty=0.1)
        H = pjds.pjds_create(A.n_rows, A.n_cols, A.row_ptr, A.col, A.val, b=32, dtype=dtype,
                             permute_cols=(m % 4 == 1))
        D = H.to_device("cuda")
        x = synth.vector(A.n_cols, seed=m)
        if dtype == "f32":
            x = x.astype(np.float32).astype(np.float64)
        xin = x[H.perm] if m % 4 == 1 else x
        mats.append((A, H.perm.copy(), m % 4 == 1))
        devs.append(D)
        xs.append(torch.from_numpy(xin).to("cuda", D.vec_dtype))
        ys.append(torch.full((A.n_rows,), float("nan"), dtype=D.vec_dtype, device="cuda"))
        xh.append(x)
    B = batch.Batch(devs, xs, ys)
    info = B.info()
    # one-lane tiles hold 512 rows (two per thread), 8-lane tiles 32
    assert sum((A.n_rows + 511) // 512 for A, _, _ in mats) <= info["n_tiles"] <= sum(
        (A.n_rows + 31) // 32 for A, _, _ in mats)
    for _ in range(2):
        for y in ys:
            y.fill_(float("nan"))
        B.run(use_graph=graph)
        torch.cuda.synchronize()
        for (A, perm, permuted), x, y, D in zip(mats, xh, ys, devs):
            got = y.double().cpu().numpy()
            if permuted:
                g2 = np.empty_like(got)
                g2[perm] = got
                got = g2
            Ar = A if dtype == "f64" else A._replace(val=oracle_lib.round_f32(A.val))
            check = parity.check_fp64 if dtype == "f64" else parity.check_fp32
            r = check(got, oracle_lib.crs_spmv(Ar, x), oracle_lib.crs_absmv(Ar, x), np.diff(A.row_ptr))
            assert r["ok"], r
    # bit for bit the single product with the built-in rule's lanes: rows whose
    # block has >= 256 entries with 8 threads per row, >= 64 with 4, >= 16 with
    # 2, the others with one thread per row
    for m in (2, 5):
        A, perm, permuted = mats[m]
        H = pjds.pjds_create(A.n_rows, A.n_cols, A.row_ptr, A.col, A.val, b=32, dtype=dtype, permute_cols=permuted)
        bl = H.block_len[np.arange(A.n_rows) // 32]
        lanes = np.where(bl >= 256, 8, np.where(bl >= 64, 4, np.where(bl >= 16, 2, 1)))
        out_row = np.arange(A.n_rows) if permuted else H.perm  # output row of sorted row i
        want = np.full(A.n_rows, np.nan)
        for t in (1, 2, 4, 8):
            yt = torch.empty_like(ys[m])
            if t == 1:
                pjds.pjds_spmv_cfg(devs[m], xs[m], yt, threads_per_row=1, tile_order=-1)
            else:
                pjds.pjds_spmv_cfg(devs[m], xs[m], yt, threads_per_row=t, unroll=4, tile_order=-1)
            torch.cuda.synchronize()
            want[out_row[lanes == t]] = yt.double().cpu().numpy()[out_row[lanes == t]]
        assert np.array_equal(want, ys[m].double().cpu().numpy()), m
        assert (lanes > 1).any() or m == 2
    B.destroy()


@pytest.mark.parametrize("dtype,k", [("f32", 16), ("f32", 32), ("f64", 8), ("f64", 16)])
def test_spmm_two_chunk_lanes(mods, oracle_lib, dtype, k):
    # 160k rows of 144 entries: enough threads for lanes of two 16-byte chunks;
    # every column against the oracle, and bit for bit against pjds_spmv
    torch, pjds, batch = mods
    A = synth.block_dense(n_brow=40_000, bs=4, nb=36, frac=0.05, seed=11)
    X = np.random.default_rng(k).uniform(-1, 1, (A.n_cols, k))
    if dtype != "f64":
        X = X.astype(np.float32).astype(np.float64)
    D = pjds.pjds_create(A.n_rows, A.n_cols, A.row_ptr, A.col, A.val, b=32, dtype=dtype).to_device("cuda")
    Xt = torch.from_numpy(X).to("cuda", D.vec_dtype).contiguous()
    Yt = torch.full((A.n_rows, k), float("nan"), dtype=D.vec_dtype, device="cuda")
    batch.spmm(D, Xt, Yt)
    torch.cuda.synchronize()
    Ar = A if dtype == "f64" else A._replace(val=oracle_lib.round_f32(A.val))
    Yr = oracle_lib.crs_spmm(Ar, X)
    S = oracle_lib.crs_spmm(Ar._replace(val=np.abs(Ar.val)), np.abs(X))
    Y = Yt.double().cpu().numpy()
    check = parity.check_fp64 if dtype == "f64" else parity.check_fp32
    lens = np.diff(A.row_ptr)
    for c in range(k):
        r = check(Y[:, c], Yr[:, c], S[:, c], lens)
        assert r["ok"], (c, r)
    for c in range(k):
        y1 = torch.empty(A.n_rows, dtype=D.vec_dtype, device="cuda")
        pjds.pjds_spmv_cfg(D, Xt[:, c].contiguous(), y1, threads_per_row=1, rows_per_thread=1, tile_order=-1)
        torch.cuda.synchronize()
        assert torch.equal(y1, Yt[:, c].contiguous()), c


def test_batch_given_lanes(mods, oracle_lib):
    # lanes per row given per matrix (as an autotuner would): every row equals
    # the oracle, and bit for bit pjds_spmv_cfg with threads_per_row = lanes
    torch, pjds, batch = mods
    makes = [lambda: synth.zipf_rows(30_000, s=2.0, len_max=300, seed=31),
             lambda: synth.hmep_like(n=40_000, seed=32),
             lambda: tiny.random_lengths(1037, 1037, max_len=90, seed=33, p_empty=0.2),
             lambda: synth.zipf_rows(12_000, s=1.6, len_max=512, seed=34),
             lambda: synth.banded_uniform(n=20_000, seed=35),
             lambda: tiny.random_lengths(333, 500, max_len=40, seed=36)]
    lanes = [1, 2, 4, 8, 0, 2]
    mats, devs, xs, ys = [], [], [], []
    for k, make in enumerate(makes):
        A = make()
        D = pjds.pjds_create(A.n_rows, A.n_cols, A.row_ptr, A.col, A.val, b=32).to_device("cuda")
        mats.append(A)
        devs.append(D)
        xs.append(torch.from_numpy(synth.vector(A.n_cols, seed=k)).cuda())
        ys.append(torch.full((A.n_rows,), float("nan"), dtype=torch.float64, device="cuda"))
    B = batch.Batch(devs, xs, ys, lanes=lanes)
    B.run(use_graph=True)
    torch.cuda.synchronize()
    for A, D, x, y, ln in zip(mats, devs, xs, ys, lanes):
        xh = x.cpu().numpy()
        r = parity.check_fp64(y.cpu().numpy(), oracle_lib.crs_spmv(A, xh), oracle_lib.crs_absmv(A, xh),
                              np.diff(A.row_ptr))
        assert r["ok"], (ln, r)
        if ln:
            y1 = torch.empty_like(y)
            pjds.pjds_spmv_cfg(D, x, y1, threads_per_row=ln, unroll=4, tile_order=-1)
            torch.cuda.synchronize()
            assert torch.equal(y1, y), ln
    B.destroy()
    with pytest.raises(pjds.PjdsError):
        batch.Batch(devs, xs, ys, lanes=[1, 2, 3, 8, 0, 2])


def test_batch_rule_and_rule_tuner(mods, oracle_lib):
    # tiles by a block-length rule: every rule gives oracle-exact rows; the
    # built-in rule given explicitly is bit for bit the default plan; the
    # tuner times each rule and picks the fastest
    torch, pjds, batch = mods
    mats, devs, xs, ys = [], [], [], []
    for k in range(10):
        A = synth.zipf_rows(int(5_000 + 7_000 * k), s=1.8 + 0.05 * k, len_max=400, seed=60 + k)
        devs.append(pjds.pjds_create(A.n_rows, A.n_cols, A.row_ptr, A.col, A.val, b=32).to_device("cuda"))
        xs.append(torch.from_numpy(synth.vector(A.n_cols, seed=k)).cuda())
        ys.append(torch.full((A.n_rows,), float("nan"), dtype=torch.float64, device="cuda"))
        mats.append(A)
    B0 = batch.Batch(devs, xs, ys)
    B0.run(use_graph=False)
    torch.cuda.synchronize()
    y_default = [y.clone() for y in ys]
    B0.destroy()
    for rule in (batch.DEFAULT_RULES[0], (4, 16, 64), (2, 8, 32), (batch.NEVER, batch.NEVER, 1)):
        for y in ys:
            y.fill_(float("nan"))
        B = batch.Batch(devs, xs, ys, rule=rule)
        B.run(use_graph=True)
        torch.cuda.synchronize()
        for A, x, y in zip(mats, xs, ys):
            xh = x.cpu().numpy()
            r = parity.check_fp64(y.cpu().numpy(), oracle_lib.crs_spmv(A, xh), oracle_lib.crs_absmv(A, xh),
                                  np.diff(A.row_ptr))
            assert r["ok"], (rule, r)
        if rule == batch.DEFAULT_RULES[0]:
            assert all(torch.equal(a, b) for a, b in zip(y_default, ys))
        B.destroy()
    rules = batch.DEFAULT_RULES[:4]
    best, timings = batch.tune_rule(devs, xs, ys, rules=rules, reps=3, flush_bytes=0)
    assert len(timings) == 4 and all(us > 0 for _, us in timings)
    assert best == min(timings, key=lambda t: t[1])[0]


def test_batch_degenerate_matrices(mods, oracle_lib):
    # a matrix without rows, one whose rows are all empty, a one-row matrix
    # and two ordinary ones in one launch, with each way of choosing lanes
    torch, pjds, batch = mods
    makes = [lambda: tiny.from_lengths([], 5), lambda: tiny.from_lengths([0] * 77, 9),
             lambda: tiny.from_lengths([3], 4, seed=1), lambda: synth.zipf_rows(3_000, s=2.0, len_max=300, seed=71),
             lambda: tiny.random_lengths(515, 600, max_len=70, seed=72, p_empty=0.3)]
    mats, devs, xs = [], [], []
    for k, make in enumerate(makes):
        A = make()
        mats.append(A)
        devs.append(pjds.pjds_create(A.n_rows, A.n_cols, A.row_ptr, A.col, A.val, b=32).to_device("cuda"))
        xs.append(torch.from_numpy(synth.vector(A.n_cols, seed=k)).cuda())
    for kw in (dict(), dict(rule=(4, 16, 64)), dict(lanes=[1, 2, 4, 8, 0])):
        ys = [torch.full((A.n_rows,), float("nan"), dtype=torch.float64, device="cuda") for A in mats]
        B = batch.Batch(devs, xs, ys, **kw)
        B.run(use_graph=True)
        torch.cuda.synchronize()
        for A, x, y in zip(mats, xs, ys):
            if A.n_rows == 0:
                continue
            xh = x.cpu().numpy()
            r = parity.check_fp64(y.cpu().numpy(), oracle_lib.crs_spmv(A, xh), oracle_lib.crs_absmv(A, xh),
                                  np.diff(A.row_ptr))
            assert r["ok"], (kw, r)
        B.destroy()
