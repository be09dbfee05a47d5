"""The committed cost model, evaluated with the CUDA inference kernel on the
committed held-out timings: mean regret against the exhaustive sweep <= 5%
for every precision (the blueprint's target), and far below the paper's fixed
mapping (b = 32, one thread per row)."""
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_heldout_regret_of_committed_model():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_1112_5588_gb300 import build
    build.build()
    from paper_1112_5588_gb300 import learned, tuner_data
    here = os.path.dirname(learned.MODEL_PATH)
    data = dict(np.load(os.path.join(here, "data", "tuner_timings_gb300.npz")))
    ev = tuner_data.evaluate(data, learned.load())
    for d in ("f64", "f32", "bf16"):
        assert ev[d]["matrices"] == 200
        assert ev[d]["mean_regret"] <= 0.05, ev[d]
        assert ev[d]["paper_mapping_mean_regret"] > 5 * ev[d]["mean_regret"]


def test_choose_returns_a_valid_candidate():
    import synth
    from paper_1112_5588_gb300 import learned
    A = synth.zipf_rows(200_000, s=1.8, len_max=512, seed=9)
    i, cand, pred = learned.choose(A)
    assert 0 <= i < 48 and len(pred) == 48 and np.all(pred > 0)
    assert cand["b"] in (32, 64, 128, 256) and cand["threads_per_row"] in (1, 2, 4, 8)
