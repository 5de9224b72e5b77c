"""Pins for the FP64 oracle's one-level products (CPU only).

Each test checks the oracle against something other than itself: nested
loops over index tuples (the definition of Section 1), library routines
(numpy FFT, scipy's Hankel matrix), closed forms (Vandermonde generators of
Section 4.1, Corollary 2.2), the printed examples of Section 2, Theorem 2.1,
exact integer arithmetic, and invariances of the multilinear map.
"""

import numpy as np
import pytest
import scipy.linalg

import oracle
from conftest import golden
from paper_1401_6238_gb300 import workloads as wl


def rand(rng, shape, cplx):
    v = rng.standard_normal(shape)
    if cplx:
        v = v + 1j * rng.standard_normal(shape)
    return v


# ---------------------------------------------------------------- oracle FFT

@pytest.mark.parametrize("L", [1, 2, 4, 8, 64, 1024])
def test_fft_matches_numpy_and_dft_matrix(L):
    rng = np.random.default_rng(L)
    a = rand(rng, (3, L), True)
    np.testing.assert_allclose(oracle.fft(a), np.fft.fft(a), atol=1e-12 * max(L, 1))
    np.testing.assert_allclose(oracle.ifft(a), np.fft.ifft(a), atol=1e-12)
    if L <= 64:
        j = np.arange(L)
        F = np.exp(-2j * np.pi * np.outer(j, j) / L)  # F_n of Section 2.1
        np.testing.assert_allclose(oracle.fft(a[0]), F @ a[0], atol=1e-12 * L)
        np.testing.assert_allclose(F @ F.conj().T, L * np.eye(L), atol=1e-9)


def test_fft2_matches_numpy():
    rng = np.random.default_rng(0)
    A = rand(rng, (16, 8), True)
    np.testing.assert_allclose(oracle.fft2(A), np.fft.fft2(A), atol=1e-11)
    np.testing.assert_allclose(oracle.ifft2(A), np.fft.ifft2(A), atol=1e-13)


def test_fft_rejects_non_power_of_two():
    with pytest.raises(ValueError):
        oracle.fft(np.ones(12))


# ------------------------------------------------- definition vs loops vs FFT

CASES = [
    ([3], False), ([4, 3], False), ([2, 5], True), ([3, 3, 3], False),
    ([2, 4, 3], True), ([4, 1, 2], False), ([2, 2, 3, 2], True),
    ([3, 2, 2, 1], False), ([2, 2, 2, 2, 2], False), ([1, 3, 2, 2, 2], True),
]


@pytest.mark.parametrize("dims,cplx", CASES)
def test_loops_tensor_fft_agree(dims, cplx):
    rng = np.random.default_rng(sum(dims) * 7 + len(dims))
    d = oracle.d_of(dims)
    h = rand(rng, d, cplx)
    xs = [rand(rng, n, cplx) for n in dims]
    y_loop = oracle.loop_y(h, xs[1:], dims)
    y_brute = oracle.brute_y(h, xs[1:], dims)
    y_fast = oracle.fast_y(h, xs[1:], dims)
    np.testing.assert_allclose(y_brute, y_loop, rtol=1e-13, atol=1e-13)
    np.testing.assert_allclose(y_fast, y_loop, rtol=1e-12, atol=1e-12)
    a_loop = oracle.loop_alpha(h, xs, dims)
    np.testing.assert_allclose(oracle.brute_alpha(h, xs, dims), a_loop, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(oracle.fast_alpha(h, xs, dims), a_loop, rtol=1e-12, atol=1e-12)


def test_order_two_is_hankel_matrix_vector_product():
    # m = 2: H is the n_1 x n_2 Hankel matrix with first column h[0:n_1] and
    # last row h[n_1-1:]; y = H x_2 is a textbook matrix-vector product.
    rng = np.random.default_rng(2)
    for n1, n2 in [(5, 9), (16, 3), (33, 64)]:
        h = rng.standard_normal(n1 + n2 - 1)
        x = rng.standard_normal(n2)
        Hm = scipy.linalg.hankel(h[:n1], h[n1 - 1:])
        np.testing.assert_allclose(oracle.fast_y(h, [x], [n1, n2]).real, Hm @ x, rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(oracle.brute_y(h, [x], [n1, n2]), Hm @ x, rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("m,n,a", [(3, 64, 0.97), (4, 20, 0.9), (5, 7, -0.8), (3, 9, 1.05)])
def test_vandermonde_closed_form(m, n, a):
    # h_k = a^k gives the rank-1 Vandermonde decomposition of Section 4.1:
    # H = a-vector^{(x) m}, so H x^{m-1} = (sum_i a^i x_i)^{m-1} [a^i]_i and
    # H x^m = (sum_i a^i x_i)^m.
    dims = [n] * m
    d = oracle.d_of(dims)
    h = wl.vandermonde_h(a, d)
    x = np.random.default_rng(1).standard_normal(n)
    s = np.sum(a ** np.arange(n) * x)
    y_ref = s ** (m - 1) * a ** np.arange(n)
    scale = np.max(np.abs(y_ref))
    np.testing.assert_allclose(oracle.fast_y(h, [x] * (m - 1), dims).real, y_ref, atol=1e-12 * scale)
    np.testing.assert_allclose(oracle.fast_alpha(h, [x] * m, dims).real, s ** m, rtol=1e-11)
    if n ** m <= 300000:
        np.testing.assert_allclose(oracle.brute_y(h, [x] * (m - 1), dims), y_ref, atol=1e-12 * scale)


def test_plain_case_vandermonde_and_brute():
    dims, h, x = wl.plain_case(seed=0)
    y_b = oracle.brute_y(h, [x, x], dims)
    y_f = oracle.fast_y(h, [x, x], dims)
    np.testing.assert_allclose(y_f.real, y_b, rtol=0, atol=1e-11 * np.max(np.abs(y_b)))
    assert np.max(np.abs(y_f.imag)) < 1e-11 * np.max(np.abs(y_b))


def test_mode_permutation_symmetry():
    rng = np.random.default_rng(5)
    dims = [4, 3, 5, 2]
    d = oracle.d_of(dims)
    h = rng.standard_normal(d)
    xs = [rng.standard_normal(n) for n in dims]
    y = oracle.fast_y(h, xs[1:], dims)
    # permuting (n_p, x_p) over modes 2..m leaves y unchanged
    for perm in [(2, 0, 1), (1, 2, 0), (0, 2, 1)]:
        pd = [dims[0]] + [dims[1 + p] for p in perm]
        px = [xs[1 + p] for p in perm]
        np.testing.assert_allclose(oracle.fast_y(h, px, pd), y, atol=1e-12)
    # permuting all m modes leaves alpha unchanged
    a = oracle.fast_alpha(h, xs, dims)
    for perm in [(3, 2, 1, 0), (1, 0, 3, 2), (2, 3, 0, 1)]:
        np.testing.assert_allclose(oracle.fast_alpha(h, [xs[p] for p in perm], [dims[p] for p in perm]), a, rtol=1e-12)


def test_alpha_is_inner_product_with_x1():
    # alpha = H x_1 x_2 ... x_m = sum_i x_1[i] y_i, no conjugation (Section 2.1)
    rng = np.random.default_rng(6)
    dims = [6, 4, 5]
    d = oracle.d_of(dims)
    h = rand(rng, d, True)
    xs = [rand(rng, n, True) for n in dims]
    y = oracle.fast_y(h, xs[1:], dims)
    np.testing.assert_allclose(oracle.fast_alpha(h, xs, dims), np.sum(xs[0] * y), rtol=1e-12)


@pytest.mark.parametrize("dims", [[5, 5, 5], [8, 3, 6], [4, 4, 4, 4], [3, 3, 3, 3, 3]])
def test_small_integers_exact(dims):
    # integer inputs: the direct sum is exact in FP64; the FFT result must
    # round to it exactly
    h, xs = wl.integer_case(dims, seed=len(dims))
    y_exact = oracle.loop_y(h, xs[1:], dims)
    assert np.all(y_exact == np.rint(y_exact))
    y_fast = oracle.fast_y(h, xs[1:], dims)
    np.testing.assert_array_equal(np.rint(y_fast.real), y_exact)
    a_exact = oracle.loop_alpha(h, xs, dims)
    assert np.rint(oracle.fast_alpha(h, xs, dims).real) == a_exact


@pytest.mark.parametrize("m,n", [(3, 4), (4, 4), (3, 8), (5, 2), (4, 6)])
def test_corollary_2_2_eigenpairs(m, n):
    # anti-circulant C with compressed generating vector c:
    # C 1^{m-1} = n^{m-2} (1^T c) 1, and for even n
    # C 1~^{m-1} = n^{m-2} (1~^T c) 1~ with 1~ = [1, -1, 1, -1, ...]
    c = np.random.default_rng(m * n).standard_normal(n)
    h = oracle.anticirculant_generating_vector(c, m)
    dims = [n] * m
    one = np.ones(n)
    np.testing.assert_allclose(oracle.brute_y(h, [one] * (m - 1), dims), n ** (m - 2) * c.sum() * one, rtol=1e-12)
    alt = (-1.0) ** np.arange(n)
    np.testing.assert_allclose(oracle.brute_y(h, [alt] * (m - 1), dims), n ** (m - 2) * (alt @ c) * alt,
                               rtol=1e-12, atol=1e-12)
    if n & (n - 1) == 0:  # the unpadded anti-circulant procedure (oracle FFT needs 2^k)
        np.testing.assert_allclose(oracle.anticirculant_y(c, [one] * (m - 1)).real, n ** (m - 2) * c.sum() * one,
                                   rtol=1e-12)
        np.testing.assert_allclose(oracle.anticirculant_y(c, [alt] * (m - 1)).real, n ** (m - 2) * (alt @ c) * alt,
                                   rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("m,n", [(2, 4), (3, 4), (3, 8), (4, 2)])
def test_theorem_2_1_diagonalisation(m, n):
    # C = D x_1 F_n x_2 F_n ... x_m F_n with diag(D) = ifft(c)
    rng = np.random.default_rng(m + 10 * n)
    c = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    j = np.arange(n)
    F = np.exp(-2j * np.pi * np.outer(j, j) / n)
    D = np.zeros([n] * m, dtype=complex)
    dd = oracle.ifft(c)
    for k in range(n):
        D[(k,) * m] = dd[k]
    C = D
    for p in range(1, m + 1):
        C = oracle.mode_product(C, F, p)
    C_ref = oracle.hankel_tensor(oracle.anticirculant_generating_vector(c, m), [n] * m)
    np.testing.assert_allclose(C, C_ref, atol=1e-12)
    # and the unpadded anti-circulant products of Section 3 agree with it
    xs = [rng.standard_normal(n) for _ in range(m)]
    np.testing.assert_allclose(oracle.anticirculant_y(c, xs[1:]),
                               oracle.brute_y(oracle.anticirculant_generating_vector(c, m), xs[1:], [n] * m),
                               atol=1e-11)
    np.testing.assert_allclose(oracle.anticirculant_alpha(c, xs),
                               oracle.brute_alpha(oracle.anticirculant_generating_vector(c, m), xs, [n] * m),
                               atol=1e-11)


def test_printed_anticirculant_examples():
    # Section 2 prints a 3x3 anti-circulant matrix and the mode-1 unfolding
    # of a 3x3x3 anti-circulant tensor; with c = [0, 1, 2] the entries are
    # the indices of c.
    c = np.arange(3)
    M = oracle.hankel_tensor(oracle.anticirculant_generating_vector(c, 2), [3, 3])
    np.testing.assert_array_equal(M, golden("anticirculant_3x3.txt"))
    T = oracle.hankel_tensor(oracle.anticirculant_generating_vector(c, 3), [3, 3, 3])
    unfold = np.concatenate([T[:, :, k] for k in range(3)], axis=1)
    np.testing.assert_array_equal(unfold, golden("anticirculant_3x3x3_unfold1.txt"))
    # the circulant matrix printed beside it is not Hankel (it is Toeplitz)
    circ = golden("circulant_3x3.txt")
    assert not np.array_equal(circ, M)
    np.testing.assert_array_equal(circ, (np.arange(3)[:, None] - np.arange(3)[None, :]) % 3)


def test_linearity_in_h_and_each_x():
    rng = np.random.default_rng(8)
    dims = [5, 4, 6]
    d = oracle.d_of(dims)
    h1, h2 = rng.standard_normal(d), rng.standard_normal(d)
    xs = [rng.standard_normal(n) for n in dims[1:]]
    a, b = 0.7, -1.3
    np.testing.assert_allclose(oracle.fast_y(a * h1 + b * h2, xs, dims),
                               a * oracle.fast_y(h1, xs, dims) + b * oracle.fast_y(h2, xs, dims), atol=1e-12)
    x2b = rng.standard_normal(dims[2])
    np.testing.assert_allclose(oracle.fast_y(h1, [xs[0], a * xs[1] + b * x2b], dims),
                               a * oracle.fast_y(h1, xs, dims) + b * oracle.fast_y(h1, [xs[0], x2b], dims), atol=1e-12)


def test_any_embedding_length_at_least_d():
    # the paper pads to exactly d_H; every L >= d_H gives the same product
    rng = np.random.default_rng(9)
    dims = [6, 6, 6]  # d_H = 16, a power of two, so L = d_H itself is testable
    d = oracle.d_of(dims)
    assert d == 16
    h = rng.standard_normal(d)
    xs = [rng.standard_normal(6) for _ in range(2)]
    ref = oracle.loop_y(h, xs, dims)
    for L in (16, 32, 128):
        np.testing.assert_allclose(oracle.fast_y(h, xs, dims, L=L).real, ref, atol=1e-12)
    with pytest.raises(ValueError):
        oracle.fast_y(h, xs, dims, L=8)


def test_planted_mistakes_are_caught():
    # Each plausible slip in the fast procedure makes the comparison with the
    # definition fail: the pins above are sharp enough to see it.
    rng = np.random.default_rng(10)
    dims = [5, 3, 4]
    d = oracle.d_of(dims)
    h = rng.standard_normal(d) + 1j * rng.standard_normal(d)
    xs = [rng.standard_normal(n) + 1j * rng.standard_normal(n) for n in dims[1:]]
    ref = oracle.loop_y(h, xs, dims)
    L = 16

    def pad(v):
        out = np.zeros(L, complex)
        out[: len(v)] = v
        return out

    good = oracle.fft(oracle.ifft(pad(h)) * oracle.fft(pad(xs[0])) * oracle.fft(pad(xs[1])))[:5]
    np.testing.assert_allclose(good, ref, atol=1e-12)
    wrong = {
        "fft of h instead of ifft (the convolution form)":
            oracle.fft(oracle.fft(pad(h)) * oracle.fft(pad(xs[0])) * oracle.fft(pad(xs[1])))[:5] / L,
        "conjugated x":
            oracle.fft(oracle.ifft(pad(h)) * oracle.fft(pad(np.conj(xs[0]))) * oracle.fft(pad(xs[1])))[:5],
        "dropped mode":
            oracle.fft(oracle.ifft(pad(h)) * oracle.fft(pad(xs[0])))[:5],
        "inverse transform at the end":
            oracle.ifft(oracle.ifft(pad(h)) * oracle.fft(pad(xs[0])) * oracle.fft(pad(xs[1])))[:5] * L,
    }
    for name, y in wrong.items():
        assert np.max(np.abs(y - ref)) > 1e-3 * np.max(np.abs(ref)), name


def test_pool_matches_serial_oracle():
    # the process-pool helper the full-batch parity checks use returns the
    # serial oracle's outputs, in order
    from oracle import pool
    from paper_1401_6238_gb300 import workloads as wl
    b = wl.batched_square(count=9, seed=3, n_lo=16, n_hi=80)
    tensors = [b.tensor(i) for i in range(len(b))]
    par = pool.square_refs(tensors, procs=2)
    for (m, n, h, x), y in zip(tensors, par):
        np.testing.assert_array_equal(y, oracle.fast_y(h, [x] * (m - 1), [n] * m).real)
