"""Host-side evidence for the per-tile mapping's size thresholds.

The committed plan-eval data (GB300 timings of the per-tile mapping and of
each precision's best uniform candidate on the tuner data's 2,000 training
and 200 held-out matrices) must reproduce the thresholds libpjds uses, and
the Python mirror of the uniform threads-per-row rule must agree with the
library's own resolve.
"""
import os

import numpy as np
import pytest

import synth
from synth import tiny

DATA = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_1112_5588_gb300", "data")


@pytest.fixture(scope="module")
def td():
    from paper_1112_5588_gb300 import tuner_data
    return tuner_data


def test_plan_fit_reproduces_the_library_thresholds(td):
    train = dict(np.load(os.path.join(DATA, "plan_eval_gb300_train.npz")))
    test = dict(np.load(os.path.join(DATA, "plan_eval_gb300_test.npz")))
    assert len(train["n"]) == 2000 and len(test["n"]) == 200
    fit = td.plan_fit(train, test)
    assert {dt: fit[dt]["min_rows"] for dt in fit} == {"f64": 1 << 16, "f32": 1 << 17, "bf16": 1 << 18}
    # the held-out figures the library's comments quote
    assert [fit[dt]["test"] for dt in ("f64", "f32", "bf16")] == [0.87, 0.941, 0.98]
    for dt in fit:
        assert fit[dt]["test"] < fit[dt]["test_rule_only"] and fit[dt]["test"] < fit[dt]["test_plan_always"]


def test_uniform_rule_mirror_matches_the_library(td):
    from paper_1112_5588_gb300 import pjds
    mats = [synth.zipf_rows(70_000, s=2.0, len_max=512, seed=3), synth.hmep_like(n=40_000, seed=4),
            tiny.random_lengths(5_000, 3_000, max_len=300, seed=5), synth.banded_uniform(n=300_000, seed=6),
            synth.block_dense(8_000, 4, 36, 0.05, seed=7)]
    for A in mats:
        n_max = int(np.diff(A.row_ptr).max())
        for dt in ("f64", "f32", "bf16"):
            H = pjds.pjds_create(A.n_rows, A.n_cols, A.row_ptr, A.col, A.val, b=32, dtype=dt)
            assert pjds.pjds_spmv_resolve(H, plan=-1)["threads_per_row"] == \
                td.uniform_threads(A.n_rows, A.nnz, n_max, dt), (A.n_rows, dt)
            H.destroy()
