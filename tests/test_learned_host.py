"""Learned tuner host logic: features, candidate encoding, model init and scaling."""
import numpy as np
import pytest

import synth
from synth import tiny


@pytest.fixture(scope="module")
def L():
    from paper_1112_5588_gb300 import build
    build.build()
    from paper_1112_5588_gb300 import learned
    return learned


def test_features_against_numpy(L):
    for A in (synth.zipf_rows(5000, s=1.7, len_max=300, seed=2), tiny.random_lengths(300, 900, max_len=50, seed=1),
              synth.hmep_like(n=20_000, seed=3)):
        f = L.features(A)
        lens = np.diff(A.row_ptr).astype(np.float64)
        rows = np.repeat(np.arange(A.n_rows), np.diff(A.row_ptr))
        d = np.abs(A.col.astype(np.float64) - rows)
        mu, sd = lens.mean(), lens.std()
        want = [np.log10(A.n_rows), np.log10(A.nnz), np.log2(1 + mu), sd / mu, ((lens - mu) ** 3).mean() / sd ** 3,
                np.log2(1 + lens.max()), d.mean() / A.n_rows, np.mean(d <= 64)]
        assert np.allclose(f, want, rtol=1e-5, atol=1e-6), (f, want)


def test_encode(L):
    f = np.arange(8, dtype=np.float32)
    cands = [{"b": 32, "dtype": "f64", "threads_per_row": 1}, {"b": 256, "dtype": "bf16", "threads_per_row": 8},
             {"b": 64, "dtype": "f32", "threads_per_row": 0}]
    X = L.encode(f, cands)
    assert X.shape == (3, 15)
    assert np.array_equal(X[:, :8], np.tile(f, (3, 1)))
    assert np.array_equal(X[:, 8:], [[0, 0, 1, 0, 0, 0, 0], [3, 3, 0, 0, 1, 0, 0], [1, 0, 0, 1, 0, 0, 0]])
    # the per-tile mapping (threads per row does not apply) and the traversal table
    X = L.encode(f, [{"b": 64, "dtype": "f64", "plan": 1, "threads_per_row": 8, "tile_order": 1},
                     {"b": 128, "dtype": "bf16", "threads_per_row": 2, "tile_order": 1},
                     {"b": 128, "dtype": "bf16", "threads_per_row": 2, "tile_order": -1}])
    assert np.array_equal(X[:, 8:], [[1, 0, 1, 0, 0, 1, 0], [2, 1, 0, 0, 1, 0, 1], [2, 1, 0, 0, 1, 0, 0]])


def test_init_and_scaling(L):
    m = L.init(5)
    w1 = np.array(m.w1)
    assert np.all(np.abs(w1) <= np.sqrt(6 / 15)) and w1.std() > 0.3
    assert np.array_equal(np.array(L.init(5).w2), np.array(m.w2))
    X = np.random.default_rng(0).standard_normal((100, 15)).astype(np.float32) * 3 + 1
    X[:, 4] = 2.0  # constant column keeps std 1
    y = np.random.default_rng(1).standard_normal(100).astype(np.float32)
    L.fit_scaling(m, X, y)
    assert np.allclose(m.in_mean, X.mean(0), atol=1e-5)
    assert np.allclose(np.array(m.in_std)[[0, 1, 2, 3, 5]], X.std(0)[[0, 1, 2, 3, 5]], rtol=1e-5)
    assert m.in_std[4] == 1.0
    assert m.out_mean == pytest.approx(y.mean(), abs=1e-6) and m.out_std == pytest.approx(y.std(), rel=1e-5)


def test_feature_range(L):
    m = L.init(3)
    assert np.all(np.array(m.feat_lo) > np.array(m.feat_hi))  # none set
    F = np.random.default_rng(2).standard_normal((50, 8)).astype(np.float32)
    L.fit_range(m, F)
    assert np.array_equal(np.array(m.feat_lo, np.float32), F.min(0))
    assert np.array_equal(np.array(m.feat_hi, np.float32), F.max(0))


def test_model_json_roundtrip(L, tmp_path):
    m = L.init(9)
    p = tmp_path / "m.json"
    L.save(m, str(p), {"note": "test"})
    m2 = L.load(str(p))
    assert np.array_equal(np.array(m.w2), np.array(m2.w2)) and m.b3 == m2.b3


def test_committed_model_and_data_are_consistent(L):
    import json
    import os
    here = os.path.dirname(L.MODEL_PATH)
    m = L.load()
    assert len(m.w1) == 64 * 15 and len(m.w2) == 64 * 64 and m.out_std > 0
    meta = json.load(open(L.MODEL_PATH))["meta"]
    for d in ("f64", "f32", "bf16"):
        assert meta["heldout"][d]["mean_regret"] <= 0.05
    data = np.load(os.path.join(here, "data", "tuner_timings_full_gb300.npz"))
    assert data["features"].shape == (2200, 8) and data["times_us"].shape == (2200, 108)
    assert int(data["n_train"]) == 2000
    assert np.isfinite(data["times_us"]).mean() > 0.99
    # the model's feature range is the training matrices' range
    F = data["features"][:2000]
    assert np.allclose(np.array(m.feat_lo), F.min(0)) and np.allclose(np.array(m.feat_hi), F.max(0))


def test_pick_needs_the_sweep_outside_the_range(L):
    # the range check runs on the host: outside the model's range, or without
    # a model, pjds_tune_pick needs the sweep's arena and says so (no GPU work)
    import ctypes
    from paper_1112_5588_gb300 import pjds, tune
    A = synth.hmep_like(n=20_000, seed=5)
    rp, col, val = pjds._crs_args(A.row_ptr, A.col, A.val)
    cands = tune.default_space(("f64",))
    m = L.init(1)
    L.fit_range(m, np.zeros((4, 8), np.float32))  # a range no matrix of 20k rows lies in
    for model in (ctypes.byref(m), None):
        out = L.Pick()
        rc = L._lib.pjds_tune_pick(A.n_rows, A.n_cols, rp.ctypes.data, col.ctypes.data, val.ctypes.data, model,
                                   tune._to_cands(cands), len(cands), 3, None, 0, None, 0, None, 0,
                                   ctypes.byref(out), None)
        assert rc == -1 and "sweep arena" in pjds.lib().pjds_last_error().decode()
    assert out.n_outside == 0  # no model: nothing compared
    out = L.Pick()
    L._lib.pjds_tune_pick(A.n_rows, A.n_cols, rp.ctypes.data, col.ctypes.data, val.ctypes.data, ctypes.byref(m),
                          tune._to_cands(cands), len(cands), 3, None, 0, None, 0, None, 0, ctypes.byref(out), None)
    assert out.n_outside >= 3  # N, nnz and the mean row length at least
