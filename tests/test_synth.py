"""Seeded synthetic inputs: determinism and the shapes they promise."""
import numpy as np

import synth


def _valid_crs(A):
    assert A.row_ptr[0] == 0 and np.all(np.diff(A.row_ptr) >= 0)
    assert A.nnz == len(A.col) == len(A.val)
    assert np.all((A.col >= 0) & (A.col < A.n_cols))
    for i in range(0, A.n_rows, max(1, A.n_rows // 200)):
        c = A.col[A.row_ptr[i]:A.row_ptr[i + 1]]
        assert np.all(np.diff(c) > 0), "columns ascending and distinct within a row"


def test_banded_uniform_shape_and_determinism():
    A = synth.banded_uniform(n=20_000, seed=1234)
    B = synth.banded_uniform(n=20_000, seed=1234)
    C = synth.banded_uniform(n=20_000, seed=99)
    assert np.array_equal(A.col, B.col) and np.array_equal(A.val, B.val)
    assert not np.array_equal(A.row_ptr, C.row_ptr)
    _valid_crs(A)
    lens = np.diff(A.row_ptr)
    assert lens.min() >= 5 and lens.max() <= 40 and 21.5 < lens.mean() < 23.5
    rows = np.repeat(np.arange(A.n_rows), lens)
    assert np.all(np.abs(A.col - rows) <= 2000)
    assert np.all(np.isin(np.arange(A.n_rows), A.col[A.col == rows]))  # diagonal present
    assert A.val.min() >= -1 and A.val.max() < 1


def test_hmep_like_symmetric_pattern_small():
    A = synth.hmep_like(n=50_000, offsets=(1, 64, 4096), seed=5)
    _valid_crs(A)
    lens = np.diff(A.row_ptr)
    assert 14.0 < lens.mean() < 16.0
    rows = np.repeat(np.arange(A.n_rows), lens).astype(np.int64)
    key = rows * A.n_cols + A.col
    keyT = A.col.astype(np.int64) * A.n_cols + rows
    assert np.array_equal(np.sort(key), np.sort(keyT)), "pattern symmetric"
    off = A.col - rows
    band = np.isin(off, [0, 1, -1, 64, -64, 4096, -4096])
    assert np.all(np.abs(off[~band]) <= A.n_rows // 8)
    assert 0.0 < A.param < 1.0


def test_stencil27_spd_structure():
    A = synth.stencil27(g=12, p_drop=0.1, seed=3)
    _valid_crs(A)
    assert A.n_rows == 12 ** 3
    d = np.zeros((A.n_rows, A.n_cols))
    rows = np.repeat(np.arange(A.n_rows), np.diff(A.row_ptr))
    d[rows, A.col] = A.val
    assert np.array_equal(d, d.T)
    off = d - np.diag(np.diag(d))
    assert np.allclose(np.diag(d), np.abs(off).sum(1) + 1.0, rtol=1e-14, atol=0)
    assert np.all(np.linalg.eigvalsh(d) > 0)
    assert np.diff(A.row_ptr).max() <= 27


def test_block_dense_rows():
    A = synth.block_dense(n_brow=2000, bs=4, nb=36, frac=0.05, seed=2)
    _valid_crs(A)
    lens = np.diff(A.row_ptr)
    assert np.all(lens % 4 == 0) and lens.max() == 144


def test_zipf_rows():
    A = synth.zipf_rows(30_000, s=2.0, len_max=512, seed=4)
    _valid_crs(A)
    lens = np.diff(A.row_ptr)
    assert lens.min() >= 1 and lens.max() <= 512
    assert np.mean(lens == 1) > 0.5  # Zipf(2): P(1) = 1/zeta(2) ~ 0.61


def test_vector():
    x = synth.vector(1000, seed=1)
    assert np.array_equal(x, synth.vector(1000, seed=1))
    assert x.min() >= -1 and x.max() < 1 and abs(x.mean()) < 0.1
