"""Level-k block Hankel tensors and their fast products, FP64 CPU oracle.

TEST INFRASTRUCTURE ONLY.

Section 2.2: a block Hankel tensor whose blocks are level-(k-1) block Hankel
tensors is a level-k block Hankel tensor (level 1: Hankel, level 2: BHHB),
and its generating data is an order-k tensor G.  Each mode p has a size
n_p^(l) per level l = 1..k; with the index of mode p written in mixed radix,
level 1 innermost (the column-major order of the BHHB case, Section 3),

    I_p = a_p^(1) + n_p^(1) (a_p^(2) + n_p^(2) (a_p^(3) + ...)),

the tensor is

    T[I_1, ..., I_m] = G[sum_p a_p^(1), ..., sum_p a_p^(k)],

with G of size sum_p n_p^(l) - m + 1 along level l.  Here ``sizes[l][p]`` is
n_{p+1}^(l+1), arrays are numpy arrays of shape (n^(1), ..., n^(k)) and
vec() stacks them in column-major order.

A level-k block anti-circulant tensor is diagonalised by the Kronecker
product of k Fourier matrices (Section 2.2), so the fast products of
Section 3 carry over with k-dimensional FFTs (the paper states this at the
end of Section 3 without writing it out):

    Y~    = fftn(ifftn(G~) .* fftn(X~_2) .* ... .* fftn(X~_m)),
    Y     = Y~[0:n_1^(1), ..., 0:n_1^(k)],
    alpha = <ifftn(G~), fftn(X~_1) .* ... .* fftn(X~_m)>,

G~ and X~_p zero-padded to P_1 x ... x P_k with P_l >= sum_p n_p^(l) - m + 1
(powers of two here).  Gradients follow the convention of ``grad``
(PyTorch's, the adjoint J^H g): grad_G = (G_y correlated with conj(Z))
cropped, Z the k-dimensional full convolution of X_2 .. X_m;
grad_X_p = conj(product with conj(G_y) in mode 1, X_q elsewhere, mode p free).
Parity: pinned in tests/test_oracle_level.py.
"""

import itertools

import numpy as np

from .fft import fftn, ifftn, next_pow2
from .hankel import mode_product


def gen_shape(sizes):
    """Shape of the generating tensor: sum_p n_p^(l) - m + 1 per level."""
    return tuple(int(sum(s)) - len(s) + 1 for s in sizes)


def mode_shape(sizes, p):
    """Shape (n_p^(1), ..., n_p^(k)) of mode p's arrays (p 0-based)."""
    return tuple(int(s[p]) for s in sizes)


def vec(A):
    return np.asarray(A).reshape(-1, order="F")


def unvec(v, shape):
    return np.asarray(v).reshape(shape, order="F")


def level_tensor(G, sizes):
    """Explicit level-k block Hankel tensor from its generating tensor."""
    G = np.asarray(G)
    k, m = len(sizes), len(sizes[0])
    if G.shape != gen_shape(sizes):
        raise ValueError("generating tensor must be %s, got %s" % (gen_shape(sizes), G.shape))
    sums = [np.zeros([1] * m, dtype=np.int64) for _ in range(k)]
    for p in range(m):
        total = int(np.prod(mode_shape(sizes, p)))
        shape = [1] * m
        shape[p] = total
        rest = np.arange(total)
        for l in range(k):
            sums[l] = sums[l] + (rest % sizes[l][p]).reshape(shape)
            rest = rest // sizes[l][p]
    return G[tuple(sums)]


def brute_level_y(G, Xs, sizes):
    """Y = unvec(T vec(X_2) ... vec(X_m)) from the explicit tensor."""
    T = level_tensor(G, sizes)
    m = len(sizes[0])
    for p in range(m, 1, -1):
        T = mode_product(T, vec(Xs[p - 2]).reshape(-1, 1), p)[..., 0]
    return unvec(T, mode_shape(sizes, 0))


def brute_level_alpha(G, Xs, sizes):
    """alpha = T vec(X_1) ... vec(X_m) from the explicit tensor."""
    return np.sum(vec(brute_level_y(G, Xs[1:], sizes)) * vec(Xs[0]))


def _lengths(sizes, Ps):
    g = gen_shape(sizes)
    Ps = tuple(next_pow2(v) for v in g) if Ps is None else tuple(int(v) for v in Ps)
    if any(P < v for P, v in zip(Ps, g)):
        raise ValueError("padded lengths must cover the generating tensor")
    return Ps


def _pad(A, Ps):
    out = np.zeros(Ps, dtype=np.complex128)
    A = np.asarray(A)
    out[tuple(slice(0, s) for s in A.shape)] = A
    return out


def fast_level_y(G, Xs, sizes, Ps=None):
    """Fast level-k y by k-dimensional FFTs."""
    Ps = _lengths(sizes, Ps)
    acc = ifftn(_pad(G, Ps))
    for X in Xs:
        acc = acc * fftn(_pad(X, Ps))
    return fftn(acc)[tuple(slice(0, s) for s in mode_shape(sizes, 0))]


def fast_level_alpha(G, Xs, sizes, Ps=None):
    """Fast level-k alpha = <ifftn(G~), prod_{p=1..m} fftn(X~_p)>."""
    Ps = _lengths(sizes, Ps)
    prod = np.ones(Ps, dtype=np.complex128)
    for X in Xs:
        prod = prod * fftn(_pad(X, Ps))
    return np.sum(ifftn(_pad(G, Ps)) * prod)


def _convn_full(Xs):
    """k-dimensional full convolution X_2 * ... * X_m by direct summation."""
    out = np.ones((1,) * np.asarray(Xs[0]).ndim, dtype=np.complex128)
    for X in Xs:
        X = np.asarray(X, dtype=np.complex128)
        nxt = np.zeros(tuple(a + b - 1 for a, b in zip(out.shape, X.shape)), dtype=np.complex128)
        for idx in np.ndindex(*out.shape):
            nxt[tuple(slice(i, i + s) for i, s in zip(idx, X.shape))] += out[idx] * X
        out = nxt
    return out


def brute_level_grads(G, Xs, sizes, Gy):
    """(grad_G, [grad_X_2 .. grad_X_m]) from the explicit tensor."""
    G = np.asarray(G, dtype=np.complex128)
    Gy = np.asarray(Gy, dtype=np.complex128)
    m = len(sizes[0])
    Z = _convn_full(Xs)
    grad_G = np.zeros(G.shape, dtype=np.complex128)
    for c in np.ndindex(*G.shape):
        acc = 0.0
        for i in np.ndindex(*Gy.shape):
            s = tuple(a - b for a, b in zip(c, i))
            if all(0 <= v < z for v, z in zip(s, Z.shape)):
                acc += Gy[i] * np.conj(Z[s])
        grad_G[c] = acc
    T = level_tensor(G, sizes)
    grads = []
    for p in range(2, m + 1):
        A = T
        for q in range(m, 0, -1):
            if q == p:
                continue
            v = vec(np.conj(Gy)) if q == 1 else vec(np.asarray(Xs[q - 2], dtype=np.complex128))
            A = np.squeeze(mode_product(A, v.reshape(-1, 1), q), axis=q - 1)
        grads.append(unvec(np.conj(A), mode_shape(sizes, p - 1)))
    return grad_G, grads


def fast_level_grads(G, Xs, sizes, Gy, Ps=None):
    """The same gradients by k-dimensional FFTs."""
    Ps = _lengths(sizes, Ps)
    m = len(sizes[0])
    spec = fftn(_pad(Gy, Ps))
    for X in Xs:
        spec = spec * fftn(_pad(np.conj(np.asarray(X, dtype=np.complex128)), Ps))
    grad_G = ifftn(spec)[tuple(slice(0, s) for s in gen_shape(sizes))]
    Gh = ifftn(_pad(G, Ps))
    grads = []
    for p in range(2, m + 1):
        acc = Gh * fftn(_pad(np.conj(np.asarray(Gy, dtype=np.complex128)), Ps))
        for q in range(2, m + 1):
            if q != p:
                acc = acc * fftn(_pad(Xs[q - 2], Ps))
        grads.append(np.conj(fftn(acc)[tuple(slice(0, s) for s in mode_shape(sizes, p - 1))]))
    return grad_G, grads


def anticirculant_level_tensor(C, m):
    """Level-k block anti-circulant tensor of order m with compressed
    generating tensor C (shape (n^(1), ..., n^(k)), every mode the same):
    T[I_1..I_m] = C[(sum_p a_p^(1)) mod n^(1), ..., (sum_p a_p^(k)) mod n^(k)]."""
    C = np.asarray(C)
    shape = C.shape
    total = int(np.prod(shape))
    digits = []
    rest = np.arange(total)
    for s in shape:
        digits.append(rest % s)
        rest = rest // s
    idx = []
    for l, s in enumerate(shape):
        acc = np.zeros([1] * m, dtype=np.int64)
        for p in range(m):
            sh = [1] * m
            sh[p] = total
            acc = acc + digits[l].reshape(sh)
        idx.append(acc % s)
    return C[tuple(idx)]


def kron_fourier(shape):
    """F_{n^(k)} (x) ... (x) F_{n^(1)} for vec in column-major order."""
    F = np.ones((1, 1), dtype=np.complex128)
    for n in shape:
        Fn = np.exp(-2j * np.pi * np.outer(np.arange(n), np.arange(n)) / n)
        F = np.kron(Fn, F)
    return F


def diagonal_form(C, m):
    """D (F (x) ... (x) F)^m with diag(D) = vec(ifftn(C)): the diagonalisation
    of Section 2.2, evaluated entry by entry for a small tensor."""
    F = kron_fourier(np.asarray(C).shape)
    dvec = vec(ifftn(C))
    n = F.shape[0]
    T = np.zeros((n,) * m, dtype=np.complex128)
    for I in itertools.product(range(n), repeat=m):
        T[I] = np.sum(dvec * np.prod([F[:, i] for i in I], axis=0))
    return T
