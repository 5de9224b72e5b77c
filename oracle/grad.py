"""Gradients of the Hankel and BHHB products, FP64 CPU oracle.

TEST INFRASTRUCTURE ONLY.

The paper gives no gradients; these follow from the definition of y in
Section 1 / Section 3 and are stated here so that a reader can check them.
Write z = x_2 * x_3 * ... * x_m (full linear convolution, length
d_H - n_1 + 1), so that y_i = sum_s h[i + s] z[s] (a correlation of h with z).

Given the upstream gradient g of a real loss with respect to y, in PyTorch's
convention for complex tensors (grad = dL/dRe + i dL/dIm, so a map y = A v
back-propagates as A^H g):

    grad_h[j]   = sum_i g_i conj(z[j - i])                     j in [0, d_H)
    grad_x_p[j] = conj( (H x_1 conj(g) x_q x_q ... )[j] )      q != 1, p;
                  the product leaves mode p free.

For real data every conj is the identity.  With one vector x in all modes
2..m (the y = H x^{m-1} case of Section 2.1) grad_x = sum_p grad_x_p =
(m-1) conj(H x_1 conj(g) x_3 x ... x_m x), by the symmetry of a square
Hankel tensor.

The BHHB case is the same with 2D convolutions: Z = X_2 ** ... ** X_m
(2D full convolution), grad_Hgen[a, b] = sum_{i,j} G[i, j] conj(Z[a-i, b-j]),
grad_X_p = conj(block product with conj(G) in mode 1, X_q elsewhere, mode p
free), reshaped by vec^{-1}.

``brute_*`` compute these from the explicit tensors; ``fast_*`` by FFTs.
Parity: pinned in ``tests/test_oracle_grad.py`` against FP64 central finite
differences, the adjoint (dot-product) identity and Euler's identity.
"""

import numpy as np

from .block import bhhb_tensor, unvec, vec
from .fft import fft, fft2, ifft, ifft2, next_pow2
from .hankel import d_of, fast_y, hankel_tensor, mode_product


def _conv_full(xs):
    """z = x_2 * ... * x_m: sum over index tuples with a fixed index sum."""
    out = np.ones(1, dtype=np.complex128)
    for x in xs:
        x = np.asarray(x, dtype=np.complex128)
        nxt = np.zeros(out.shape[0] + x.shape[0] - 1, dtype=np.complex128)
        for s, v in enumerate(out):
            nxt[s: s + x.shape[0]] += v * x
        out = nxt
    return out


def brute_grads(h, xs, dims, g):
    """(grad_h, [grad_x_2, ..., grad_x_m]) from the explicit tensor."""
    dims = list(dims)
    m = len(dims)
    d = d_of(dims)
    g = np.asarray(g, dtype=np.complex128)
    z = _conv_full(xs)
    grad_h = np.zeros(d, dtype=np.complex128)
    for j in range(d):
        for i in range(dims[0]):
            s = j - i
            if 0 <= s < z.shape[0]:
                grad_h[j] += g[i] * np.conj(z[s])
    T = hankel_tensor(np.asarray(h, dtype=np.complex128), dims)
    grads_x = []
    for p in range(2, m + 1):
        A = T
        # contract every mode except p, the last mode first so axes stay put
        for q in range(m, 0, -1):
            if q == p:
                continue
            v = np.conj(g) if q == 1 else np.asarray(xs[q - 2], dtype=np.complex128)
            A = mode_product(A, v.reshape(-1, 1), q)
            A = np.squeeze(A, axis=q - 1)
        grads_x.append(np.conj(A))
    return grad_h, grads_x


def fast_grads(h, xs, dims, g, L=None):
    """Same gradients by FFT at a power-of-two length L >= d_H."""
    dims = list(dims)
    m = len(dims)
    d = d_of(dims)
    L = next_pow2(d) if L is None else int(L)
    g = np.asarray(g, dtype=np.complex128)
    gt = np.zeros(L, dtype=np.complex128)
    gt[: dims[0]] = g
    spec = fft(gt)
    for x in xs:
        xt = np.zeros(L, dtype=np.complex128)
        xt[: len(x)] = np.conj(np.asarray(x, dtype=np.complex128))
        spec = spec * fft(xt)
    grad_h = ifft(spec)[:d]  # linear convolution g * conj(z); length d_H <= L, no wrap
    grads_x = []
    for p in range(2, m + 1):
        # the Hankel tensor with modes (p, 1, others) has the same generating
        # vector; its mode-1 output is the mode-p output of the original
        others = [q for q in range(2, m + 1) if q != p]
        pdims = [dims[p - 1], dims[0]] + [dims[q - 1] for q in others]
        pvecs = [np.conj(g)] + [xs[q - 2] for q in others]
        grads_x.append(np.conj(fast_y(h, pvecs, pdims, L=L)))
    return grad_h, grads_x


def _conv2_full(Xs):
    out = np.ones((1, 1), dtype=np.complex128)
    for X in Xs:
        X = np.asarray(X, dtype=np.complex128)
        nxt = np.zeros((out.shape[0] + X.shape[0] - 1, out.shape[1] + X.shape[1] - 1), dtype=np.complex128)
        for a in range(out.shape[0]):
            for b in range(out.shape[1]):
                nxt[a: a + X.shape[0], b: b + X.shape[1]] += out[a, b] * X
        out = nxt
    return out


def brute_block_grads(Hgen, Xs, n, N, G):
    """(grad_Hgen, [grad_X_2..grad_X_m]) for the BHHB y, from explicit tensors."""
    m = len(n)
    G = np.asarray(G, dtype=np.complex128)
    Z = _conv2_full(Xs)
    Hgen = np.asarray(Hgen, dtype=np.complex128)
    grad_H = np.zeros(Hgen.shape, dtype=np.complex128)
    for a in range(Hgen.shape[0]):
        for b in range(Hgen.shape[1]):
            acc = 0.0
            for i in range(n[0]):
                for j in range(N[0]):
                    s, t = a - i, b - j
                    if 0 <= s < Z.shape[0] and 0 <= t < Z.shape[1]:
                        acc += G[i, j] * np.conj(Z[s, t])
            grad_H[a, b] = acc
    T = bhhb_tensor(Hgen, n, N)
    grads_X = []
    for p in range(2, m + 1):
        A = T
        for q in range(m, 0, -1):
            if q == p:
                continue
            v = vec(np.conj(G)) if q == 1 else vec(np.asarray(Xs[q - 2], dtype=np.complex128))
            A = np.squeeze(mode_product(A, v.reshape(-1, 1), q), axis=q - 1)
        grads_X.append(unvec(np.conj(A), n[p - 1], N[p - 1]))
    return grad_H, grads_X


def fast_block_grads(Hgen, Xs, n, N, G, P=None, Q=None):
    """Same BHHB gradients by 2D FFTs on a power-of-two P x Q plane."""
    m = len(n)
    d1, d2 = sum(n) - m + 1, sum(N) - m + 1
    P = next_pow2(d1) if P is None else int(P)
    Q = next_pow2(d2) if Q is None else int(Q)
    G = np.asarray(G, dtype=np.complex128)

    def pad(A):
        out = np.zeros((P, Q), dtype=np.complex128)
        out[: A.shape[0], : A.shape[1]] = A
        return out

    spec = fft2(pad(G))
    for X in Xs:
        spec = spec * fft2(pad(np.conj(np.asarray(X, dtype=np.complex128))))
    grad_H = ifft2(spec)[:d1, :d2]
    Hh = ifft2(pad(np.asarray(Hgen, dtype=np.complex128)))
    grads_X = []
    for p in range(2, m + 1):
        # mode-p output of the product with conj(G) in mode 1: the embedded
        # BAAB tensor is symmetric under mode permutations, so this is the
        # block y-procedure with mode p moved to the front.
        acc = Hh * fft2(pad(np.conj(G)))
        for q in range(2, m + 1):
            if q != p:
                acc = acc * fft2(pad(np.asarray(Xs[q - 2], dtype=np.complex128)))
        grads_X.append(np.conj(fft2(acc)[: n[p - 1], : N[p - 1]]))
    return grad_H, grads_X
