"""Pins for the oracle's BHHB (two-level block) products (CPU only)."""

import itertools

import numpy as np
import pytest

import oracle


def rnd(rng, shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def loop_block_y(Hgen, Xs, n, N):
    """Y[i_1, j_1] = sum over all (i_p, j_p) of Hgen[sum i, sum j] prod X_p[i_p, j_p]."""
    m = len(n)
    Y = np.zeros((n[0], N[0]), dtype=complex)
    for i1 in range(n[0]):
        for j1 in range(N[0]):
            acc = 0
            for ii in itertools.product(*[range(k) for k in n[1:]]):
                for jj in itertools.product(*[range(k) for k in N[1:]]):
                    t = Hgen[i1 + sum(ii), j1 + sum(jj)]
                    for p in range(m - 1):
                        t = t * Xs[p][ii[p], jj[p]]
                    acc += t
            Y[i1, j1] = acc
    return Y


BLOCK_CASES = [
    ([2, 3], [3, 2]),
    ([3, 2, 2], [2, 2, 3]),
    ([2, 2, 2], [2, 2, 2]),
    ([1, 3, 2], [3, 1, 2]),
    ([2, 2, 1, 2], [1, 2, 2, 2]),
]


@pytest.mark.parametrize("n,N", BLOCK_CASES)
def test_block_loops_tensor_fft_agree(n, N):
    rng = np.random.default_rng(sum(n) + 3 * sum(N))
    m = len(n)
    Hgen = rnd(rng, (sum(n) - m + 1, sum(N) - m + 1))
    Xs = [rnd(rng, (n[p], N[p])) for p in range(m)]
    ref = loop_block_y(Hgen, Xs[1:], n, N)
    np.testing.assert_allclose(oracle.brute_block_y(Hgen, Xs[1:], n, N), ref, atol=1e-12)
    np.testing.assert_allclose(oracle.fast_block_y(Hgen, Xs[1:], n, N), ref, atol=1e-11)
    a_ref = np.sum(oracle.vec(Xs[0]) * oracle.vec(ref))
    np.testing.assert_allclose(oracle.brute_block_alpha(Hgen, Xs, n, N), a_ref, rtol=1e-12)
    np.testing.assert_allclose(oracle.fast_block_alpha(Hgen, Xs, n, N), a_ref, rtol=1e-11)


def test_block_with_single_block_is_one_level_product():
    # N_p = 1 for all p: the BHHB tensor is the Hankel tensor of column 0
    rng = np.random.default_rng(1)
    n, N = [4, 3, 5], [1, 1, 1]
    Hgen = rnd(rng, (sum(n) - 2, 1))
    Xs = [rnd(rng, (k, 1)) for k in n[1:]]
    Y = oracle.fast_block_y(Hgen, Xs, n, N)
    y = oracle.fast_y(Hgen[:, 0], [X[:, 0] for X in Xs], n)
    np.testing.assert_allclose(Y[:, 0], y, atol=1e-12)


def test_block_with_unit_blocks_is_product_along_j():
    # n_p = 1 for all p: blocks are scalars; the tensor is Hankel in j with
    # generating vector row 0 of Hgen
    rng = np.random.default_rng(2)
    n, N = [1, 1, 1], [4, 3, 5]
    Hgen = rnd(rng, (1, sum(N) - 2))
    Xs = [rnd(rng, (1, k)) for k in N[1:]]
    Y = oracle.fast_block_y(Hgen, Xs, n, N)
    y = oracle.fast_y(Hgen[0], [X[0] for X in Xs], N)
    np.testing.assert_allclose(Y[0], y, atol=1e-12)


def test_separable_generator_and_rank_one_blocks_factor():
    # Hgen = u v^T and X_p = a_p b_p^T: Y = (H(u) a_2 ... a_m)(H(v) b_2 ... b_m)^T
    rng = np.random.default_rng(3)
    n, N = [3, 4, 2], [5, 2, 3]
    m = 3
    u, v = rnd(rng, sum(n) - m + 1), rnd(rng, sum(N) - m + 1)
    a = [rnd(rng, k) for k in n[1:]]
    b = [rnd(rng, k) for k in N[1:]]
    Xs = [np.outer(a[p], b[p]) for p in range(m - 1)]
    Y = oracle.fast_block_y(np.outer(u, v), Xs, n, N)
    ref = np.outer(oracle.fast_y(u, a, n), oracle.fast_y(v, b, N))
    np.testing.assert_allclose(Y, ref, atol=1e-11)


def test_block_index_convention_column_major():
    # T[i_1 + n_1 j_1, ...] = Hgen[sum i, sum j] with vec stacking columns
    n, N = [2, 3], [3, 2]
    Hgen = np.arange(4 * 4).reshape(4, 4)
    T = oracle.bhhb_tensor(Hgen, n, N)
    for I1 in range(6):
        for I2 in range(6):
            i1, j1 = I1 % 2, I1 // 2
            i2, j2 = I2 % 3, I2 // 3
            assert T[I1, I2] == Hgen[i1 + i2, j1 + j2]
    X = np.arange(6).reshape(2, 3)
    np.testing.assert_array_equal(oracle.vec(X), [0, 3, 1, 4, 2, 5])
    np.testing.assert_array_equal(oracle.unvec(oracle.vec(X), 2, 3), X)


def test_block_padding_independence():
    rng = np.random.default_rng(4)
    n, N = [3, 3, 2], [2, 3, 3]
    Hgen = rnd(rng, (6, 6))
    Xs = [rnd(rng, (n[p], N[p])) for p in (1, 2)]
    ref = oracle.fast_block_y(Hgen, Xs, n, N)
    np.testing.assert_allclose(oracle.fast_block_y(Hgen, Xs, n, N, P=16, Q=32), ref, atol=1e-12)
