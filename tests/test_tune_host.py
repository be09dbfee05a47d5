"""Autotuner host logic: candidate space and arena sizing (no GPU)."""
import numpy as np
import pytest

import synth
from synth import tiny


@pytest.fixture(scope="module")
def T():
    from paper_1112_5588_gb300 import build
    build.build()
    from paper_1112_5588_gb300 import tune
    return tune


def test_default_space(T):
    s = T.default_space(("f64", "f32", "bf16"))
    assert len(s) == 108
    uni = [c for c in s if c["plan"] != 1]
    assert {c["b"] for c in s} == {32, 64, 128, 256}
    assert {c["threads_per_row"] for c in uni} == {1, 2, 4, 8}
    assert {c["tile_order"] for c in uni} == {-1, 1}
    assert {c["dtype"] for c in s} == {"f64", "f32", "bf16"}
    # every (b, threads per row, tile order) once per dtype, then the per-tile mapping for every b
    for d in ("f64", "f32", "bf16"):
        keys = [T.cand_key(c) for c in s if c["dtype"] == d]
        assert len(keys) == len(set(keys)) == 36
        assert sum(k.endswith("_plan") for k in keys) == 4
    assert len(T.default_space()) == 36 and len(T.default_space(plan=False)) == 32


@pytest.mark.parametrize("make", [lambda: synth.zipf_rows(20_000, s=1.8, len_max=400, seed=2),
                                  lambda: tiny.random_lengths(999, 300, max_len=80, seed=4, p_empty=0.3),
                                  lambda: synth.hmep_like(n=30_000, seed=1)])
def test_arena_bytes_covers_every_candidate(T, make):
    from paper_1112_5588_gb300 import pjds
    A = make()
    cands = T.default_space(("f64", "bf16"))
    need = T.arena_bytes(A, cands)
    a256 = lambda b: (b + 255) // 256 * 256  # noqa: E731
    worst = 0
    for c in cands:
        H = pjds.pjds_create(A.n_rows, A.n_cols, A.row_ptr, A.col, A.val, b=c["b"], dtype=c["dtype"])
        vb = {"f64": 8, "f32": 4, "bf16": 2}[c["dtype"]]
        m = a256(4 * H.n_rows) + a256(4 * H.n_blocks) + a256(8 * (H.n_max + 1)) + a256(4 * H.n_stored) + \
            a256(vb * H.n_stored) + a256(4 * (H.n_pad // 32)) + a256(16 * (H.n_pad // 32))
        assert 16 * H.n_plan <= 16 * (H.n_pad // 32)  # the plan's room: one entry per 32 rows at most
        worst = max(worst, m)
    assert need == worst + a256(8 * A.n_cols) + a256(8 * A.n_rows)
