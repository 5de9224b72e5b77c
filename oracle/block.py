"""BHHB (block Hankel with Hankel blocks) products, FP64 CPU oracle.

TEST INFRASTRUCTURE ONLY.

Section 2.2: an order-m BHHB tensor of size (n_1 N_1) x ... x (n_m N_m) with
blocks of size n_1 x ... x n_m is fixed by its generating matrix
``Hgen`` of size (n_1+...+n_m-m+1) x (N_1+...+N_m-m+1): block
(j_1, ..., j_m) is the Hankel tensor generated by column ``j_1 + ... + j_m``
of Hgen, so with the column-major index ``I_p = i_p + n_p j_p`` of Section 3

    T[I_1, ..., I_m] = Hgen[i_1 + ... + i_m, j_1 + ... + j_m].

Vectors are ``x_p = vec(X_p)`` with ``X_p`` of size n_p x N_p, vec stacking
columns (Section 3).  The products are y = T x_2 ... x_m (returned as the
n_1 x N_1 matrix vec^{-1}(y), which the paper allows) and alpha =
T x_1 ... x_m.

The fast forms follow Section 3: embed twice (each Hankel block in an
anti-circulant block, then the block level), so the BAAB tensor's compressed
generating matrix is Hgen zero-padded to P x Q, and

    Y~ = fft2(ifft2(H~) .* fft2(X~_2) .* ... .* fft2(X~_m)),  Y = Y~[0:n_1, 0:N_1]
    alpha = <ifft2(H~), fft2(X~_1) .* ... .* fft2(X~_m)>,   <A,B> = sum A_jk B_jk.

Reading: the alpha procedure printed in Section 3 lists the padded factors
for p = 2..m only; the product needs x_1 as well, so the oracle takes
p = 1..m as in the one-level alpha procedure.  P >= sum(n)-m+1 and
Q >= sum(N)-m+1 are powers of two here (the embedding argument of the
one-level case applies per axis).
Parity: pinned in ``tests/test_oracle_block.py``.
"""

import numpy as np

from .fft import fft2, ifft2, next_pow2
from .hankel import mode_product


def vec(A):
    """Column-stacking vectorisation vec(A) (Section 3)."""
    return np.asarray(A).T.reshape(-1)


def unvec(v, n, N):
    """vec^{-1}_{n,N}(v): columns v[0:n], v[n:2n], ... (Section 3)."""
    return np.asarray(v).reshape(N, n).T


def _gen_shape(n, N):
    m = len(n)
    return sum(n) - m + 1, sum(N) - m + 1


def bhhb_tensor(Hgen, n, N):
    """Explicit BHHB tensor T[i_p + n_p j_p]_p = Hgen[sum i_p, sum j_p]."""
    Hgen = np.asarray(Hgen)
    if Hgen.shape != _gen_shape(n, N):
        raise ValueError("generating matrix must be %s, got %s" % (_gen_shape(n, N), Hgen.shape))
    m = len(n)
    si = np.zeros([1] * m, dtype=np.int64)
    sj = np.zeros([1] * m, dtype=np.int64)
    for p in range(m):
        shape = [1] * m
        shape[p] = n[p] * N[p]
        I = np.arange(n[p] * N[p])
        si = si + (I % n[p]).reshape(shape)
        sj = sj + (I // n[p]).reshape(shape)
    return Hgen[si, sj]


def brute_block_y(Hgen, Xs, n, N):
    """Y = vec^{-1}(T vec(X_2) ... vec(X_m)) from the explicit tensor."""
    T = bhhb_tensor(Hgen, n, N)
    m = len(n)
    for p in range(m, 1, -1):
        T = mode_product(T, vec(Xs[p - 2]).reshape(-1, 1), p)[..., 0]
    return unvec(T, n[0], N[0])


def brute_block_alpha(Hgen, Xs, n, N):
    """alpha = T vec(X_1) ... vec(X_m) from the explicit tensor."""
    Y = brute_block_y(Hgen, Xs[1:], n, N)
    return np.sum(vec(Y) * vec(Xs[0]))


def _pad2(A, P, Q):
    out = np.zeros((P, Q), dtype=np.complex128)
    A = np.asarray(A)
    out[: A.shape[0], : A.shape[1]] = A
    return out


def _sizes(n, N, P, Q):
    d1, d2 = _gen_shape(n, N)
    P = next_pow2(d1) if P is None else int(P)
    Q = next_pow2(d2) if Q is None else int(Q)
    if P < d1 or Q < d2:
        raise ValueError("padded plane must be at least the generating matrix size")
    return P, Q


def fast_block_y(Hgen, Xs, n, N, P=None, Q=None):
    """Fast BHHB y by 2D FFTs (Section 3); returns the n_1 x N_1 matrix."""
    P, Q = _sizes(n, N, P, Q)
    acc = ifft2(_pad2(Hgen, P, Q))
    for X in Xs:
        acc = acc * fft2(_pad2(X, P, Q))
    return fft2(acc)[: n[0], : N[0]]


def fast_block_alpha(Hgen, Xs, n, N, P=None, Q=None):
    """Fast BHHB alpha = <ifft2(H~), prod_{p=1..m} fft2(X~_p)> (Section 3)."""
    P, Q = _sizes(n, N, P, Q)
    prod = np.ones((P, Q), dtype=np.complex128)
    for X in Xs:
        prod = prod * fft2(_pad2(X, P, Q))
    return np.sum(ifft2(_pad2(Hgen, P, Q)) * prod)
