"""The checked build (libpjds_checked.so, device-side extent checks) on the GPU.

The cases run in a child process that loads the checked library
(tests/checked_cases.py): clean runs of every instrumented mapping must leave
the check word at 0 and match the oracle; indices planted out of range in a
device copy of a matrix must be recorded with their code and skipped.
"""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
DIAG, OFFSET, COLUMN, ROW, BLOCK = 1, 2, 3, 4, 5


@pytest.fixture(scope="module")
def res():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_1112_5588_gb300 import build
    build.build(checked=True)
    env = dict(os.environ, PJDS_LIBRARY="checked")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "tests", "checked_cases.py")], env=env, cwd=ROOT,
                       capture_output=True, text=True, timeout=1200)
    assert r.returncode == 0, r.stderr[-3000:]
    return json.loads(r.stdout.strip().splitlines()[-1])


def test_clean_runs_leave_the_check_word_at_zero(res):
    assert len(res["clean"]) >= 4 * 3 * 2 * 12
    bad = [c for c in res["clean"] if c[4] != 0 or not c[5]]
    assert not bad, bad[:10]


def test_planted_column_is_recorded_and_skipped(res):
    n = res["n"]
    for cfg, code, idx in res["planted"]["column"] + res["planted"]["ellr_column"] + res["planted"]["spmm_column"]:
        assert code == COLUMN and idx in (n["n_cols"] + 5, n["n_cols"] + 9), (cfg, code, idx)
    assert res["column_rows_changed"] == 1


def test_planted_perm_entry_is_recorded(res):
    n = res["n"]
    for cfg, code, idx in res["planted"]["perm"]:
        assert (code, idx) == (ROW, n["n_rows"] + 7), cfg


def test_planted_offset_is_recorded(res):
    n = res["n"]
    for cfg, code, idx in res["planted"]["offset"]:
        assert code == OFFSET and idx >= n["n_stored"], (cfg, code, idx)


def test_planted_block_length_is_recorded(res):
    # diagonals past the last one (code 1), or the end sentinel's offset (code 2)
    n = res["n"]
    for cfg, code, idx in res["planted"]["block"]:
        assert (code == DIAG and idx >= n["n_max"] + 1) or (code == OFFSET and idx >= n["n_stored"]), (cfg, code, idx)


def test_paired_block_product_column_is_recorded(res):
    # the block product with one thread per pair of rows checks both rows' columns
    for cfg, code, idx in res["planted"]["paired_column"]:
        assert (code, idx) == (COLUMN, res["paired_n_cols"] + 11), (cfg, code, idx)
    assert any(c[0] == "paired" for c in res["clean"])
