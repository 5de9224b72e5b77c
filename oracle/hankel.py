"""Hankel tensor-vector products, FP64 CPU oracle (test infrastructure only).

Notation follows the paper: an order-m Hankel tensor H of size
n_1 x ... x n_m has entries ``H[i_1, ..., i_m] = h[i_1 + ... + i_m]``
(0-based, Section 1), where the generating vector h has length
``d_H = n_1 + ... + n_m - m + 1``.  The two products of Section 3 are

    y     = H x_2 x_3 ... x_m    (mode products 2..m, a vector of length n_1)
    alpha = H x_1 x_2 ... x_m    (mode products 1..m, a scalar)

with the paper's mode product of Section 2.1, which never conjugates:
``(A x_p M)[..., j, ...] = sum_{i_p} A[..., i_p, ...] M[i_p, j]``.

Three independent ways to compute them live here:

* ``loop_*``  -- the definition as nested loops over every index tuple
  (pure Python, tiny sizes only);
* ``brute_*`` -- the explicit tensor from the definition, then one mode
  product per mode (numpy ``tensordot`` as the contraction primitive);
* ``fast_*``  -- the Section 3 procedure: embed H in the anti-circulant tensor
  of Theorem 2.1 at a power-of-two length L >= d_H, then
  ``y~ = fft(ifft(h~) .* fft(x~_2) .* ... .* fft(x~_m))``, ``y = y~[0:n_1]``
  and ``alpha = ifft(h~)^T (fft(x~_1) .* ... .* fft(x~_m))`` (a plain
  transpose, no conjugation).

Reading taken where the paper is specific to one length: it pads to exactly
L = d_H; any L >= d_H gives the same y and alpha because every index sum that
enters y or alpha is at most d_H - 1, so no wrap-around occurs.  The oracle
uses the next power of two.

Parity: pinned in ``tests/test_oracle.py`` (loops vs tensor vs FFT, m = 2
against ``scipy.linalg.hankel``, Vandermonde closed form, mode-permutation
symmetry, alpha = <x_1, y>, exact small-integer cases, Corollary 2.2
eigenpairs, Theorem 2.1 diagonalisation, the printed 3x3 and 3x3x3 examples).
"""

import itertools

import numpy as np

from .fft import fft, ifft, next_pow2


def d_of(dims):
    """Length of the generating vector, d_H = sum(n_k) - m + 1 (Section 1)."""
    dims = [int(n) for n in dims]
    if not dims or min(dims) < 1:
        raise ValueError("dims must be a non-empty list of positive sizes")
    return sum(dims) - len(dims) + 1


def hankel_tensor(h, dims):
    """Explicit Hankel tensor H[i_1..i_m] = h[i_1 + ... + i_m] (Section 1)."""
    h = np.asarray(h)
    d = d_of(dims)
    if h.shape[-1] != d:
        raise ValueError("generating vector has length %d, expected d_H = %d" % (h.shape[-1], d))
    s = np.zeros([1] * len(dims), dtype=np.int64)
    for p, n in enumerate(dims):
        shape = [1] * len(dims)
        shape[p] = n
        s = s + np.arange(n).reshape(shape)
    return h[s]


def mode_product(A, M, p):
    """Mode-p product of Section 2.1, p 1-based; M has shape (n_p, n_p').

    ``(A x_p M)[i_1..j..i_m] = sum_{i_p} A[i_1..i_p..i_m] M[i_p, j]``: the
    summed index of M is its FIRST one and nothing is conjugated.
    """
    A = np.asarray(A)
    M = np.asarray(M)
    ax = p - 1
    out = np.tensordot(A, M, axes=([ax], [0]))  # new axis is last
    return np.moveaxis(out, -1, ax)


def _check(h, xs, dims, first_mode):
    m = len(dims)
    if len(xs) != m - first_mode + 1:
        raise ValueError("expected %d vectors, got %d" % (m - first_mode + 1, len(xs)))
    for p, x in zip(range(first_mode, m + 1), xs):
        if np.asarray(x).shape != (dims[p - 1],):
            raise ValueError("x_%d must have length n_%d = %d" % (p, p, dims[p - 1]))
    if np.asarray(h).shape != (d_of(dims),):
        raise ValueError("h must have length d_H = %d" % d_of(dims))


def loop_y(h, xs, dims):
    """y = H x_2 ... x_m by nested loops over every index tuple (tiny sizes)."""
    _check(h, xs, dims, 2)
    m = len(dims)
    y = [0.0] * dims[0]
    for i1 in range(dims[0]):
        acc = 0.0
        for rest in itertools.product(*[range(n) for n in dims[1:]]):
            term = h[i1 + sum(rest)]
            for p in range(m - 1):
                term = term * xs[p][rest[p]]
            acc = acc + term
        y[i1] = acc
    return np.array(y)


def loop_alpha(h, xs, dims):
    """alpha = H x_1 ... x_m by nested loops over every index tuple."""
    _check(h, xs, dims, 1)
    acc = 0.0
    for idx in itertools.product(*[range(n) for n in dims]):
        term = h[sum(idx)]
        for p in range(len(dims)):
            term = term * xs[p][idx[p]]
        acc = acc + term
    return acc


def brute_y(h, xs, dims):
    """y = H x_2 ... x_m from the explicit tensor, one mode product per mode."""
    _check(h, xs, dims, 2)
    A = hankel_tensor(np.asarray(h), dims)
    for p in range(len(dims), 1, -1):  # contract the last mode first
        A = mode_product(A, np.asarray(xs[p - 2]).reshape(-1, 1), p)[..., 0]
    return A


def brute_alpha(h, xs, dims):
    """alpha = H x_1 ... x_m from the explicit tensor."""
    _check(h, xs, dims, 1)
    y = brute_y(h, xs[1:], dims)
    return mode_product(y, np.asarray(xs[0]).reshape(-1, 1), 1)[0]


def _pad(v, L):
    out = np.zeros(L, dtype=np.complex128)
    v = np.asarray(v)
    out[: v.shape[0]] = v
    return out


def fast_y(h, xs, dims, L=None):
    """Fast y = H x_2 ... x_m by the anti-circulant embedding of Section 3.

    x~_p = [x_p; 0] (length L), y~ = fft(ifft(h~) .* fft(x~_2) .* ... ),
    y = y~[0:n_1].  Returns complex128; for real inputs the imaginary part is
    rounding noise.
    """
    _check(h, xs, dims, 2)
    d = d_of(dims)
    L = next_pow2(d) if L is None else int(L)
    if L < d:
        raise ValueError("embedding length L must be >= d_H")
    acc = ifft(_pad(h, L))
    for x in xs:
        acc = acc * fft(_pad(x, L))
    return fft(acc)[: dims[0]]


def fast_alpha(h, xs, dims, L=None):
    """Fast alpha = ifft(h~)^T (fft(x~_1) .* ... .* fft(x~_m)) (Section 3)."""
    _check(h, xs, dims, 1)
    d = d_of(dims)
    L = next_pow2(d) if L is None else int(L)
    if L < d:
        raise ValueError("embedding length L must be >= d_H")
    prod = np.ones(L, dtype=np.complex128)
    for x in xs:
        prod = prod * fft(_pad(x, L))
    return np.sum(ifft(_pad(h, L)) * prod)


def anticirculant_generating_vector(c, m):
    """Periodic generating vector of the anti-circulant tensor (Section 2).

    An order-m anti-circulant tensor of dimension n with compressed generating
    vector c is the square Hankel tensor whose generating vector (length
    m(n-1)+1) satisfies h_k = c[k mod n].
    """
    c = np.asarray(c)
    n = c.shape[0]
    return c[np.arange(m * (n - 1) + 1) % n]


def anticirculant_y(c, xs):
    """y = C x_2 ... x_m for an anti-circulant C, no padding (Section 3).

    y = fft(ifft(c) .* fft(x_2) .* ... .* fft(x_m)); n must be a power of two
    for the oracle FFT.
    """
    acc = ifft(np.asarray(c, dtype=np.complex128))
    for x in xs:
        acc = acc * fft(np.asarray(x, dtype=np.complex128))
    return fft(acc)


def anticirculant_alpha(c, xs):
    """alpha = ifft(c)^T (fft(x_1) .* ... .* fft(x_m)) (Section 3)."""
    prod = np.ones(np.asarray(c).shape[0], dtype=np.complex128)
    for x in xs:
        prod = prod * fft(np.asarray(x, dtype=np.complex128))
    return np.sum(ifft(np.asarray(c, dtype=np.complex128)) * prod)
