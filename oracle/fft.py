"""Radix-2 FFT in FP64, written for the oracle (test infrastructure only).

Sign and scale follow the Fourier matrix of Section 2.1: ``F_n = (exp(-2 pi i
j k / n))``, so ``fft(v) = F_n v`` is unscaled and ``ifft(v) = F_n^* v / n``
(the Matlab convention the paper names in Theorem 2.1).

Only power-of-two lengths are supported: the oracle always embeds at a
power-of-two length L >= d, deliberately a different length and a different
algorithm from the CUDA path's mixed-radix Stockham transform.  The transform
is iterative decimation in time: bit-reversal permutation, then log2(L)
butterfly stages; the stage twiddles are numpy's FP64 ``exp``.
Parity: pinned against ``numpy.fft.fft`` and the O(L^2) Fourier-matrix
product in ``tests/test_oracle.py`` (the FFT tests at its top).
"""

import numpy as np


def next_pow2(n):
    """Smallest power of two >= n (n >= 1)."""
    n = int(n)
    if n < 1:
        raise ValueError("length must be positive")
    return 1 << (n - 1).bit_length()


def _bit_reverse(L):
    bits = L.bit_length() - 1
    idx = np.arange(L)
    rev = np.zeros(L, dtype=np.int64)
    for b in range(bits):
        rev |= ((idx >> b) & 1) << (bits - 1 - b)
    return rev


def fft(a, axis=-1):
    """Unscaled forward DFT ``F_L a`` along ``axis`` (L a power of two)."""
    a = np.asarray(a, dtype=np.complex128)
    a = np.moveaxis(a, axis, -1)
    L = a.shape[-1]
    if L & (L - 1):
        raise ValueError("oracle FFT length must be a power of two, got %d" % L)
    lead = a.shape[:-1]
    a = a[..., _bit_reverse(L)]
    half = 1
    while half < L:
        w = np.exp(-2j * np.pi * np.arange(half) / (2 * half))
        blocks = a.reshape(lead + (L // (2 * half), 2, half))
        even = blocks[..., 0, :]
        odd = blocks[..., 1, :] * w
        a = np.stack((even + odd, even - odd), axis=-2).reshape(lead + (L,))
        half *= 2
    return np.moveaxis(a, -1, axis)


def ifft(a, axis=-1):
    """Scaled inverse DFT ``F_L^* a / L`` along ``axis``."""
    a = np.asarray(a, dtype=np.complex128)
    L = a.shape[axis]
    return np.conj(fft(np.conj(a), axis=axis)) / L


def fft2(A):
    """2D DFT ``F_P A F_Q`` of a P x Q array (both powers of two)."""
    return fft(fft(A, axis=0), axis=1)


def ifft2(A):
    """2D inverse DFT ``conj(F_P) A conj(F_Q) / (P Q)``."""
    return ifft(ifft(A, axis=0), axis=1)


def fftn(A):
    """k-dimensional DFT: ``fft`` along every axis in turn."""
    A = np.asarray(A, dtype=np.complex128)
    for ax in range(A.ndim):
        A = fft(A, axis=ax)
    return A


def ifftn(A):
    """k-dimensional inverse DFT: ``ifft`` along every axis in turn."""
    A = np.asarray(A, dtype=np.complex128)
    for ax in range(A.ndim):
        A = ifft(A, axis=ax)
    return A
