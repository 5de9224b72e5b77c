"""Exponential data fitting on explicit tensors, FP64 CPU oracle.

TEST INFRASTRUCTURE ONLY.

Section 4: a signal x_n = sum_k c_k z_k^n (Section 4.1) gives a Hankel tensor
whose Vandermonde decomposition has factor matrices Z_p with rows z_k^i; the
poles z_k are read off the shift invariance of the column space of the
HOOI factor U (U_up W = U_down, solved by total least squares, eig(W) = poles).
For a 2D signal x_{n1 n2} = sum_k c_k z_{1,k}^{n1} z_{2,k}^{n2} (Section 4.3)
the BHHB tensor's factor columns are Z_2 (.) Z_1 (column-wise Kronecker
product), with two shift invariances: within a block (index i, poles z_1) and
across blocks (index j, poles z_2).

Everything here works on the explicit (dense) tensor with numpy's SVD, so
only small sizes are practical:

* ``reduced_unfolding``    -- Section 4.2: the mode-p unfolding of a Hankel
  tensor with its repeated columns removed, the I_p x (d - I_p + 1) Hankel
  matrix of the same generating vector (and its two-level analogue for a
  BHHB tensor); the initial factors are its leading left singular vectors.
* ``hosvd_init`` / ``hooi``  -- Algorithm 4.1 (HOOI): U_p from the HOSVD,
  then repeatedly U_p <- R leading left singular vectors of
  Unfold_p(A x_q conj(U_q) for q != p); core S = A x_1 conj(U_1) ... .
* ``hotf``                   -- Algorithm 4.2 (square tensors, U_1 = ... = U_m).
* ``tls``                    -- total least squares solution of A W = B.
* ``poles_1d`` / ``poles_2d``-- shift-invariance TLS (Sections 4.1, 4.3).

Readings: the shift ranges printed in Section 4.3 as A_{I,2I-2,:} are read as
the row range A_{I:2I-2,:} (every block but its last row); Algorithm 4.2's
initial Hankel matrix hankel(h_{0:I-1}, h_{I-1:nI-m}) is read with last
index d - 1 (d = mI - m + 1).  Parity: pinned in tests/test_oracle_edf.py.
"""

import numpy as np

from .hankel import mode_product


def unfold(A, p):
    """Mode-p unfolding (p 1-based): rows i_p, columns the other indices."""
    return np.moveaxis(A, p - 1, 0).reshape(A.shape[p - 1], -1)


def leading_left(M, R):
    """R leading left singular vectors and all singular values of M."""
    U, s, _ = np.linalg.svd(M, full_matrices=False)
    return U[:, :R], s


def reduced_unfolding(h, dims, p):
    """Section 4.2: M[i, a] = h[i + a], i < I_p, a <= d - I_p (p 1-based)."""
    h = np.asarray(h)
    I = dims[p - 1]
    return np.array([[h[i + a] for a in range(len(h) - I + 1)] for i in range(I)])


def reduced_block_unfolding(G, n, N, p):
    """Two-level analogue for a BHHB tensor with generating matrix G: rows
    i + n_p j, columns a + (rows(G) - n_p + 1) b, entry G[i + a, j + b]."""
    G = np.asarray(G)
    n_p, N_p = n[p - 1], N[p - 1]
    A, B = G.shape[0] - n_p + 1, G.shape[1] - N_p + 1
    M = np.zeros((n_p * N_p, A * B), dtype=G.dtype)
    for j in range(N_p):
        for i in range(n_p):
            for b in range(B):
                for a in range(A):
                    M[i + n_p * j, a + A * b] = G[i + a, j + b]
    return M


def hosvd_init(A, R):
    """U_p = R leading left singular vectors of each unfolding (HOSVD)."""
    return [leading_left(unfold(A, p), R)[0] for p in range(1, A.ndim + 1)]


def project_all_but(A, Us, p):
    """A x_q conj(U_q) for every mode q != p (the paper's mode product)."""
    B = A
    for q in range(A.ndim, 0, -1):
        if q != p:
            B = mode_product(B, np.conj(Us[q - 1]), q)
    return B


def hooi(A, R, sweeps, Us=None):
    """Algorithm 4.1; returns (Us, core S, singular values of the last sweep)."""
    Us = hosvd_init(A, R) if Us is None else [U.copy() for U in Us]
    svals = []
    for _ in range(sweeps):
        svals = []
        for p in range(1, A.ndim + 1):
            U, s = leading_left(unfold(project_all_but(A, Us, p), p), R)
            Us[p - 1] = U
            svals.append(s)
    S = A
    for q in range(A.ndim, 0, -1):
        S = mode_product(S, np.conj(Us[q - 1]), q)
    return Us, S, svals


def hotf(A, R, sweeps, U=None):
    """Algorithm 4.2 for a square tensor: one factor U in every mode."""
    if U is None:
        U = leading_left(unfold(A, 1), R)[0]
    for _ in range(sweeps):
        U, s = leading_left(unfold(project_all_but(A, [U] * A.ndim, 1), 1), R)
    S = A
    for q in range(A.ndim, 0, -1):
        S = mode_product(S, np.conj(U), q)
    return U, S, s


def tls(A, B):
    """Total least squares W with A W ~ B: from the SVD of [A B],
    W = -V12 V22^{-1} (V's last K columns partitioned in K x K blocks)."""
    K = A.shape[1]
    _, _, Vh = np.linalg.svd(np.hstack([A, B]))
    V = Vh.conj().T
    V12 = V[:K, K:]
    V22 = V[K:, K:]
    return -V12 @ np.linalg.inv(V22)


def poles_1d(U, K):
    """Poles from the shift invariance U[:-1] W = U[1:] (Section 4.1)."""
    W = tls(U[:-1, :K], U[1:, :K])
    return np.linalg.eigvals(W)


def shift_rows_2d(I, J):
    """Row sets of the four shift operators of Section 4.3 on an (I J) x K
    matrix with row index i + I j: within-block up/down, across-block up/down."""
    up1 = [i + I * j for j in range(J) for i in range(I - 1)]
    down1 = [i + 1 + I * j for j in range(J) for i in range(I - 1)]
    up2 = list(range(0, (J - 1) * I))
    down2 = list(range(I, J * I))
    return up1, down1, up2, down2


def poles_2d(U, I, J, K):
    """(z_1 poles, z_2 poles) from the two shift invariances, paired by
    expressing W_2 in the eigenvector basis of W_1."""
    up1, down1, up2, down2 = shift_rows_2d(I, J)
    W1 = tls(U[up1, :K], U[down1, :K])
    W2 = tls(U[up2, :K], U[down2, :K])
    z1, T = np.linalg.eig(W1)
    z2 = np.diag(np.linalg.solve(T, W2 @ T))
    return z1, z2
