"""Pins for the oracle's level-k block Hankel layer (Section 2.2, end of
Section 3): the explicit tensor against Hankel / BHHB tensors and against
the recursive definition (block Hankel with level-(k-1) blocks), the
diagonalisation of level-k anti-circulant tensors by Kronecker products of
Fourier matrices, fast products against the definition, integer exactness,
and gradients against finite differences and the adjoint identity."""

import itertools

import numpy as np
import pytest

import oracle
from oracle import level as lv


def crand(rng, shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def case(sizes, seed=0):
    rng = np.random.default_rng(seed)
    G = crand(rng, lv.gen_shape(sizes))
    Xs = [crand(rng, lv.mode_shape(sizes, p)) for p in range(len(sizes[0]))]
    return G, Xs


def test_level1_is_a_hankel_tensor():
    rng = np.random.default_rng(1)
    dims = [3, 4, 2]
    h = crand(rng, sum(dims) - 2)
    np.testing.assert_array_equal(lv.level_tensor(h, [dims]), oracle.hankel_tensor(h, dims))


def test_level2_is_a_bhhb_tensor():
    rng = np.random.default_rng(2)
    n, N = [2, 3, 2], [3, 1, 2]
    H = crand(rng, (sum(n) - 2, sum(N) - 2))
    np.testing.assert_array_equal(lv.level_tensor(H, [n, N]), oracle.bhhb_tensor(H, n, N))


def test_level3_is_block_hankel_with_bhhb_blocks():
    # Section 2.2: block (j_1..j_m) of a level-3 tensor is the BHHB tensor
    # generated by the slice G[:, :, j_1 + ... + j_m]
    rng = np.random.default_rng(3)
    sizes = [[2, 3, 2], [2, 1, 2], [2, 3, 1]]
    G = crand(rng, lv.gen_shape(sizes))
    inner = [sizes[0][p] * sizes[1][p] for p in range(3)]
    T = np.zeros([inner[p] * sizes[2][p] for p in range(3)], dtype=complex)
    for j in itertools.product(*[range(sizes[2][p]) for p in range(3)]):
        blk = oracle.bhhb_tensor(G[:, :, sum(j)], sizes[0], sizes[1])
        T[tuple(slice(j[p] * inner[p], (j[p] + 1) * inner[p]) for p in range(3))] = blk
    np.testing.assert_array_equal(lv.level_tensor(G, sizes), T)


@pytest.mark.parametrize("shape,m", [((2, 4, 2), 2), ((2, 2, 4), 3)])
def test_level3_anticirculant_is_diagonalised_by_kronecker_fourier(shape, m):
    # Section 2.2: C = D (F_{n3} (x) F_{n2} (x) F_{n1})^m, diag(D) from ifftn
    rng = np.random.default_rng(4)
    C = crand(rng, shape)
    np.testing.assert_allclose(lv.diagonal_form(C, m), lv.anticirculant_level_tensor(C, m), atol=1e-11)


@pytest.mark.parametrize("sizes", [
    [[3, 2, 4], [2, 3, 1], [2, 2, 3]],     # level 3, order 3, ragged
    [[2, 5], [3, 2], [1, 2], [2, 2]],      # level 4, order 2
    [[4, 3, 2, 2], [2, 2, 3, 1]],          # level 2, order 4
])
def test_fast_level_products_match_the_definition(sizes):
    G, Xs = case(sizes, seed=len(sizes))
    y = lv.fast_level_y(G, Xs[1:], sizes)
    assert y.shape == lv.mode_shape(sizes, 0)
    np.testing.assert_allclose(y, lv.brute_level_y(G, Xs[1:], sizes), atol=1e-11)
    np.testing.assert_allclose(lv.fast_level_alpha(G, Xs, sizes), lv.brute_level_alpha(G, Xs, sizes), atol=1e-10)
    # any padded lengths >= the generating sizes give the same result
    Ps = tuple(2 * oracle.next_pow2(v) for v in lv.gen_shape(sizes))
    np.testing.assert_allclose(lv.fast_level_y(G, Xs[1:], sizes, Ps), y, atol=1e-11)


def test_integer_inputs_give_exact_integers():
    rng = np.random.default_rng(5)
    sizes = [[3, 2, 2], [2, 2, 3], [2, 3, 2]]
    G = rng.integers(-3, 4, lv.gen_shape(sizes)).astype(float)
    Xs = [rng.integers(-3, 4, lv.mode_shape(sizes, p)).astype(float) for p in range(3)]
    y = lv.fast_level_y(G, Xs[1:], sizes)
    np.testing.assert_array_equal(np.round(y.real), lv.brute_level_y(G, Xs[1:], sizes).real)
    assert np.abs(y - np.round(y.real)).max() < 1e-9


def test_level_grads():
    sizes = [[2, 3, 2], [3, 2, 2], [2, 2, 1]]
    G, Xs = case(sizes, seed=6)
    rng = np.random.default_rng(7)
    Gy = crand(rng, lv.mode_shape(sizes, 0))
    bG, bX = lv.brute_level_grads(G, Xs[1:], sizes, Gy)
    fG, fX = lv.fast_level_grads(G, Xs[1:], sizes, Gy)
    np.testing.assert_allclose(fG, bG, atol=1e-10)
    for a, b in zip(fX, bX):
        np.testing.assert_allclose(a, b, atol=1e-10)

    # the real loss L = Re <Gy, y>; its gradient in PyTorch's convention is
    # dL/dRe + i dL/dIm, checked by central differences
    def loss(G_, Xs_):
        return np.real(np.sum(np.conj(Gy) * lv.brute_level_y(G_, Xs_, sizes)))

    eps = 1e-6
    for idx in [(0, 0, 0), (3, 2, 1)]:
        for unit in (1.0, 1j):
            Gp, Gm = G.copy(), G.copy()
            Gp[idx] += eps * unit
            Gm[idx] -= eps * unit
            fd = (loss(Gp, Xs[1:]) - loss(Gm, Xs[1:])) / (2 * eps)
            want = bG[idx].real if unit == 1.0 else bG[idx].imag
            assert abs(fd - want) < 1e-6
    for q, idx in [(0, (2, 1, 1)), (1, (1, 1, 0))]:
        for unit in (1.0, 1j):
            Xp = [X.copy() for X in Xs[1:]]
            Xm = [X.copy() for X in Xs[1:]]
            Xp[q][idx] += eps * unit
            Xm[q][idx] -= eps * unit
            fd = (loss(G, Xp) - loss(G, Xm)) / (2 * eps)
            want = bX[q][idx].real if unit == 1.0 else bX[q][idx].imag
            assert abs(fd - want) < 1e-6
