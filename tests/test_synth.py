"""Generators: symmetric CSR, sorted columns, degree and value recipes (CPU only)."""
import numpy as np
import pytest

import synth


def _check_csr(m):
    assert m.rowptr[0] == 0 and np.all(np.diff(m.rowptr) >= 1)
    rows = np.repeat(np.arange(m.n), np.diff(m.rowptr))
    for i in range(0, m.n, max(1, m.n // 50)):
        c = m.col[m.rowptr[i]:m.rowptr[i + 1]]
        assert np.all(np.diff(c) > 0)
    # symmetric pattern and values: sort (col,row) keys and compare with (row,col)
    k1 = rows.astype(np.int64) * m.n + m.col
    k2 = m.col.astype(np.int64) * m.n + rows
    o2 = np.argsort(k2)
    assert np.array_equal(k1, k2[o2])
    assert np.array_equal(m.val, m.val[o2])
    d = m.val[rows == m.col]
    assert d.size == m.n and np.all(d != 0)


def test_grid2d_shape():
    m = synth.grid2d(32, -1.0, 4.5)
    _check_csr(m)
    assert m.n == 1024 and m.num_edges == 3968 and m.nnz == 4992


def test_random_sym_recipe():
    m = synth.random_sym(4096, 8, 1.1, 2)
    _check_csr(m)
    deg = np.diff(m.rowptr) - 1
    assert deg.min() >= 8 and 15.0 < deg.mean() < 16.1
    rows = np.repeat(np.arange(m.n), np.diff(m.rowptr))
    off = rows != m.col
    assert np.all(np.abs(m.val[off]) < 1.0)
    absrow = np.bincount(rows[off], np.abs(m.val[off]), minlength=m.n)
    assert np.allclose(m.val[~off], 1.1 * absrow, rtol=1e-15)


def test_random_sym_deterministic():
    a = synth.random_sym(1000, 3, 1.2, 5)
    b = synth.random_sym(1000, 3, 1.2, 5)
    assert np.array_equal(a.col, b.col) and np.array_equal(a.val, b.val)


def test_grid3d_recipe():
    m = synth.grid3d(8, 1.05, 3)
    _check_csr(m)
    assert m.num_edges == 6 * 8 * 8 * 7
    rows = np.repeat(np.arange(m.n), np.diff(m.rowptr))
    off = rows != m.col
    assert np.all(m.val[off] < 0)


def test_rgg_batch_recipe():
    mats = synth.rgg_batch(16, 1024, 65536, 2.0, 4)
    for m in mats:
        _check_csr(m)
        assert 1024 <= m.n <= 65536
    big = synth.block_diag(mats)
    _check_csr(big)
    assert big.meta["offsets"][-1] == big.n == sum(m.n for m in mats)
    avg = sum(m.num_edges for m in mats) / big.n
    assert 4.5 < avg < 6.5


def test_tree_is_tree():
    m = synth.random_tree(50, 1)
    _check_csr(m)
    assert m.num_edges == 2 * 49


def test_random_rect_shape_and_rows():
    J = synth.random_rect(500, 70, 6, 9)
    assert (J.m, J.k, J.nnz) == (500, 70, 3000)
    for r in range(J.m):
        c = J.col[J.rowptr[r]:J.rowptr[r + 1]]
        assert np.all(np.diff(c) > 0) and c.min() >= 0 and c.max() < J.k
    assert np.all(J.val != 0.0) and np.all(np.isfinite(J.val))
    J2 = synth.random_rect(500, 70, 6, 9)
    assert np.array_equal(J.col, J2.col) and np.array_equal(J.val, J2.val)


def test_dense_generators():
    """dense_dd: symmetric, diagonal diag_factor x the off-diagonal row sum (1 for n = 1);
    rbf_kernel_system: exactly symmetric, the Gaussian kernel off the diagonal, the weighted
    diagonal; both seeded."""
    A = synth.dense_dd(50, 1.1, 3)
    assert np.array_equal(A, A.T)
    off = np.abs(A).sum(axis=1) - np.abs(np.diag(A))
    assert np.allclose(np.diag(A), 1.1 * off)
    assert np.array_equal(A, synth.dense_dd(50, 1.1, 3))
    assert synth.dense_dd(1, 1.1, 0)[0, 0] == 1.0
    K = synth.rbf_kernel_system(300, 3, 0.2, 1.1, 4)
    assert np.array_equal(K, K.T)
    X = np.random.default_rng(4).uniform(0.0, 1.0, size=(300, 3))
    i, j = 5, 17
    assert np.isclose(K[i, j], np.exp(-np.sum((X[i] - X[j]) ** 2) / (2 * 0.2 ** 2)), rtol=1e-14)
    assert np.allclose(np.diag(K), 1.1 * (K.sum(axis=1) - np.diag(K)))
    assert np.all(K > 0)
    assert np.array_equal(K, synth.rbf_kernel_system(300, 3, 0.2, 1.1, 4, block=64))
