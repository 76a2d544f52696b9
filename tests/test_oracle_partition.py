"""Pins for the oracle's block bookkeeping and block products (Sec. 2.1,
the block products and sums of Algorithm 1): against numpy.array_split, exact reassembly and
dense FP64 products."""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle
from paper_1812_01307_gb300 import synth


@pytest.mark.parametrize("L,K", [(10, 3), (60, 4), (360, 8), (7, 7), (5, 1), (3, 5), (512, 8)])
def test_split_bounds_matches_numpy_array_split(L, K):
    sizes = [len(a) for a in np.array_split(np.arange(L), K)]
    assert np.array_equal(np.diff(oracle.split_bounds(L, K)), sizes)


def test_partition_units():
    rb, cb = oracle.partition(60 * 91, 64 * 64, 4, 4, row_unit=91, col_unit=64)
    assert np.array_equal(rb, np.array([0, 15, 30, 45, 60]) * 91)
    assert np.array_equal(cb, np.array([0, 16, 32, 48, 64]) * 64)
    rb, cb = oracle.partition(7 * 5, 6 * 6, 3, 4, row_unit=5, col_unit=6)
    assert np.array_equal(rb, np.array([0, 3, 5, 7]) * 5)
    assert np.array_equal(cb, np.array([0, 2, 4, 5, 6]) * 6)


def _tiny(n=8, na=12, nb=13):
    A = synth.parallel_beam_csr(n, na, nb)
    return A, A.to_scipy()


@pytest.mark.parametrize("M,N", [(1, 1), (3, 4), (4, 4), (12, 8)])
def test_blocks_reassemble_A_exactly(M, N):
    A, S = _tiny()
    rb, cb = oracle.partition(S.shape[0], S.shape[1], M, N, 13, 8)
    blocks = oracle.split_blocks(A, rb, cb)
    back = sp.bmat(blocks).tocsr()
    assert (back != S).nnz == 0


@pytest.mark.parametrize("M,N", [(1, 1), (3, 2), (4, 4)])
def test_block_products_against_dense(M, N):
    A, S = _tiny()
    D = S.toarray()
    rng = np.random.default_rng(3)
    x = rng.standard_normal(S.shape[1])
    r = rng.standard_normal(S.shape[0])
    rb, cb = oracle.partition(S.shape[0], S.shape[1], M, N, 13, 8)
    blocks = oracle.split_blocks(A, rb, cb)
    z, gh = oracle.block_products(blocks, rb, cb, x, r)
    for i in range(M):
        for j in range(N):
            Dij = D[rb[i]:rb[i + 1], cb[j]:cb[j + 1]]
            assert np.allclose(z[i][j], Dij @ x[cb[j]:cb[j + 1]], rtol=1e-13, atol=1e-13)
            assert np.allclose(gh[i][j], 2 * Dij.T @ r[rb[i]:rb[i + 1]], rtol=1e-13, atol=1e-13)
    y = rng.standard_normal(S.shape[0])
    assert np.allclose(oracle.reduce_residual(y, z, rb), y - D @ x, rtol=1e-12, atol=1e-12)
    assert np.allclose(oracle.reduce_gradient(gh, cb, S.shape[1]), 2 * D.T @ r, rtol=1e-12, atol=1e-12)


def test_pair_order_does_not_change_products():
    A, S = _tiny()
    rng = np.random.default_rng(0)
    x = rng.standard_normal(S.shape[1])
    r = rng.standard_normal(S.shape[0])
    rb, cb = oracle.partition(S.shape[0], S.shape[1], 4, 4, 13, 8)
    blocks = oracle.split_blocks(A, rb, cb)
    z1, g1 = oracle.block_products(blocks, rb, cb, x, r)
    pairs = [(i, j) for i in range(4) for j in range(4)]
    order = [pairs[k] for k in rng.permutation(16)]
    z2, g2 = oracle.block_products(blocks, rb, cb, x, r, order)
    for i in range(4):
        for j in range(4):
            assert np.array_equal(z1[i][j], z2[i][j]) and np.array_equal(g1[i][j], g2[i][j])
