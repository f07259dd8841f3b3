"""Oracle pins: block-sparse SVD with truncation (paper Sec. 9.1 / 9.2).

The printed values (tests/golden/svd_pins.txt) fix the dense example's
singular values and the outcome of keepdim / min_blockdim on the symmetric
example; reconstruction, orthogonality and the Eckart-Young identity
(squared truncation error = sum of the dropped squared values) pin the rest.
"""
import os

import numpy as np
import pytest

from oracle.svd import kept_counts, matrix_blocks, reconstruct, svd_truncate
from oracle.symtensor import IN, OUT, Bond, BlockTensor, Symmetry, U1

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "svd_pins.txt")
SYM = (Symmetry(U1),)


def golden(key):
    for line in open(GOLDEN):
        if line.startswith(key + " "):
            return [float(x) for x in line.split()[1:]]
    raise KeyError(key)


def dense_example():
    """Sec. 9.1 listing: arange(2*2*6) reshaped (a, b, c) = (2, 2, 6), permuted to (c, a, b), rowrank 1."""
    M = np.arange(24, dtype=np.float64).reshape(2, 2, 6).transpose(2, 0, 1)
    bonds = [Bond.make(0, [((), 6)]), Bond.make(0, [((), 2)]), Bond.make(0, [((), 2)])]
    return BlockTensor(bonds, {(0, 0, 0): M.copy()})


def test_dense_example_singular_values_match_the_paper():
    T = dense_example()
    svals, U, S, V = svd_truncate(T, 1)
    got = np.concatenate(svals)
    want = golden("dense_full")
    assert len(got) == 4
    assert np.allclose(got[:2], want[:2], rtol=5e-6, atol=0)
    assert np.all(got[2:] < 1e-12 * got[0])          # rank 2: the printed tails are rounding noise
    svals, U, S, V, err = svd_truncate(T, 1, keepdim=3, err=1e-10, return_err=1)
    assert np.allclose(np.concatenate(svals), golden("dense_trunc"), rtol=5e-6, atol=0)
    assert err < 1e-12 * got[0]


def symmetric_example(values):
    """Sec. 9.2 listing bonds: a, b IN {+1:2, -1:2}, c OUT {+2:2, 0:4, -2:2}, rowrank 2, filled so
    that the blocks of S (ascending charge) have the given singular values."""
    a = Bond.make(IN, [((1,), 2), ((-1,), 2)], SYM)
    c = Bond.make(OUT, [((2,), 2), ((0,), 4), ((-2,), 2)], SYM)
    T = BlockTensor([a, a, c])
    rng = np.random.default_rng(4)
    for (g, rl, cl, M), s in zip(matrix_blocks(T, 2), values):
        m, n = M.shape
        q1, _ = np.linalg.qr(rng.standard_normal((m, m)))
        q2, _ = np.linalg.qr(rng.standard_normal((n, n)))
        k = len(s)
        M = q1[:, :k] @ np.diag(s) @ q2[:, :k].T
        for t, r0, mm in rl:
            for u, c0, nn in cl:
                T.blocks[t + u] = M[r0:r0 + mm, c0:c0 + nn].reshape(T.block_shape(t + u))
    return T


PRINTED = None


def printed_blocks():
    return [golden("sym_block0"), golden("sym_block1"), golden("sym_block2")]


def test_symmetric_example_block_structure():
    T = symmetric_example(printed_blocks())
    svals, U, S, V = svd_truncate(T, 2)
    assert [len(s) for s in svals] == [2, 4, 2]
    for s, w in zip(svals, printed_blocks()):
        assert np.allclose(s, w, rtol=1e-12)


def test_symmetric_keepdim_drops_a_whole_block_as_printed():
    T = symmetric_example(printed_blocks())
    svals, U, S, V, err = svd_truncate(T, 2, keepdim=4, err=1e-10, return_err=1)
    assert [list(np.round(s, 5)) for s in svals] == [[round(x, 5) for x in golden("sym_keep4_block0")],
                                                    [round(x, 5) for x in golden("sym_keep4_block1")]]
    assert U.bonds[-1].sectors == (((-2,), 1), ((0,), 3))       # the third block is gone from the new leg
    assert err == pytest.approx(max(printed_blocks()[2]))


def test_symmetric_min_blockdim_keeps_every_block_as_printed():
    T = symmetric_example(printed_blocks())
    svals, U, S, V, err = svd_truncate(T, 2, keepdim=4, err=1e-10, min_blockdim=[1, 1, 1], return_err=1)
    want = [golden("sym_min_block0"), golden("sym_min_block1"), golden("sym_min_block2")]
    assert [len(s) for s in svals] == [len(w) for w in want]
    for s, w in zip(svals, want):
        assert np.allclose(s, w, rtol=1e-12)


def test_kept_counts_rules():
    s = [np.array([5.0, 1.0]), np.array([4.0, 3.0, 0.5]), np.array([0.2])]
    assert kept_counts(s)[0] == [2, 3, 1]
    assert kept_counts(s, keepdim=3)[0] == [1, 2, 0]
    assert kept_counts(s, err=0.9)[0] == [2, 2, 0]
    assert kept_counts(s, keepdim=3, min_blockdim=[0, 0, 1])[0] == [1, 1, 1]
    k, dropped = kept_counts(s, keepdim=2)
    assert k == [1, 1, 0] and dropped == [3.0, 1.0, 0.5, 0.2]


def _random_symmetric(seed):
    a = Bond.make(IN, [((1,), 3), ((-1,), 2), ((0,), 2)], SYM)
    s = Bond.make(IN, [((1,), 1), ((-1,), 1)], SYM)
    b = Bond.make(OUT, [((0,), 3), ((1,), 2), ((2,), 2), ((-1,), 4)], SYM)
    T = BlockTensor([a, s, s, b])
    rng = np.random.default_rng(seed)
    for q in T.keys():
        T.blocks[q] = rng.standard_normal(T.block_shape(q))
    return T


def test_full_svd_reconstructs_and_is_orthogonal():
    T = _random_symmetric(1)
    svals, U, S, V = svd_truncate(T, 2)
    R = reconstruct(U, S, V, T.bonds)
    num = sum(float(np.sum((R.blocks[q] - T.blocks[q]) ** 2)) for q in T.keys())
    den = sum(float(np.sum(T.blocks[q] ** 2)) for q in T.keys())
    assert np.sqrt(num / den) < 1e-13
    for g, rl, cl, M in matrix_blocks(U, 2):
        assert np.allclose(M.T @ M, np.eye(M.shape[1]), atol=1e-13)
    for g, rl, cl, M in matrix_blocks(V, 1):
        assert np.allclose(M @ M.T, np.eye(M.shape[0]), atol=1e-13)


def test_truncation_error_is_the_dropped_weight():
    """Eckart-Young per block: ||T - U S V||_F^2 equals the sum of the dropped s^2."""
    T = _random_symmetric(2)
    svals, U, S, V, dropped = svd_truncate(T, 2, keepdim=5, return_err=2)
    R = reconstruct(U, S, V, T.bonds)
    num = sum(float(np.sum((R.blocks[q] - T.blocks[q]) ** 2)) for q in T.keys())
    assert num == pytest.approx(float(np.sum(dropped ** 2)), rel=1e-10)
    assert sum(len(s) for s in svals) == 5
