"""Pins for the oracle's exponential-data-fitting layer (Section 4) on CPU:
the rank statements of Section 4.3, the printed poles of Example 4.1, exact
recovery of 1D poles from a noiseless signal, TLS on consistent systems, and
the monotone core norm of HOOI."""

import numpy as np
import pytest
from scipy.optimize import linear_sum_assignment

import oracle
from conftest import golden
from oracle import edf
from paper_1401_6238_gb300 import workloads as wl


def match(est, true):
    est, true = np.asarray(est), np.asarray(true)
    C = np.abs(est[:, None] - true[None, :])
    r, c = linear_sum_assignment(C)
    return C[r, c].max()


def example41():
    g = golden("example41_poles.txt")
    z = {(int(d), int(k)): np.exp(a + 2j * np.pi * f) for d, k, a, f in g}
    peaks = [(g[0, 2], g[0, 3], g[2, 2], g[2, 3]), (g[1, 2], g[1, 3], g[3, 2], g[3, 3])]
    return z, peaks


def test_tls_solves_consistent_systems():
    rng = np.random.default_rng(0)
    A = rng.standard_normal((20, 3)) + 1j * rng.standard_normal((20, 3))
    W0 = rng.standard_normal((3, 3)) + 1j * rng.standard_normal((3, 3))
    np.testing.assert_allclose(edf.tls(A, A @ W0), W0, atol=1e-10)


def test_1d_noiseless_rank_and_exact_poles():
    # x_n = sum_k c_k z_k^n, K = 3: the 8 x 8 x 8 Hankel tensor (N = 22) has
    # exactly K nonzero mode singular values and the poles come back exactly
    poles = [0.95 * np.exp(0.4j), 0.9 * np.exp(-1.1j), 0.98 * np.exp(2.0j)]
    x = wl.damped_1d(22, poles, [1.0, 0.7 - 0.2j, 1.3j])
    A = oracle.hankel_tensor(x, [8, 8, 8])
    s = np.linalg.svd(edf.unfold(A, 1), compute_uv=False)
    assert s[3] < 1e-12 * s[0] and s[2] > 1e-3 * s[0]
    U, S, sv = edf.hotf(A, 3, sweeps=2)
    assert match(edf.poles_1d(U, 3), poles) < 1e-9
    Us, S2, _ = edf.hooi(A, 3, sweeps=2)
    assert match(edf.poles_1d(Us[0], 3), poles) < 1e-9


def test_example_41_rank_two_mode_singular_values():
    # Section 4.3: the BHHB tensor of size 6x6x6 with blocks 3x3x3 built from
    # the noiseless 2-peak signal has only two nonzero mode-1 singular values
    z, peaks = example41()
    I, J = 3, 2
    X = wl.damped_2d(3 * I - 2, 3 * J - 2, peaks)
    T = oracle.bhhb_tensor(X, [I] * 3, [J] * 3)
    assert T.shape == (6, 6, 6)
    s = np.linalg.svd(edf.unfold(T, 1), compute_uv=False)
    assert s[1] > 1e-3 * s[0] and np.all(s[2:] < 1e-12 * s[0])


def test_example_41_poles_from_hotf_and_two_tls():
    # Section 4.3: HOTF of the rank-(2,2,2) approximation of the 30x30x30 BHHB
    # tensor with 6x6x6 blocks, then TLS twice, gives the printed poles
    z, peaks = example41()
    I, J = 6, 5
    X = wl.damped_2d(3 * I - 2, 3 * J - 2, peaks)
    T = oracle.bhhb_tensor(X, [I] * 3, [J] * 3)
    assert T.shape == (30, 30, 30)
    U, S, _ = edf.hotf(T, 2, sweeps=2)
    z1, z2 = edf.poles_2d(U, I, J, 2)
    assert match(z1, [z[(1, 1)], z[(1, 2)]]) < 1e-9
    assert match(z2, [z[(2, 1)], z[(2, 2)]]) < 1e-9
    # pairing: peak k has (z1, z2) = (z[(1,k)], z[(2,k)])
    pairs = sorted(zip(np.round(z1, 8), np.round(z2, 8)), key=lambda t: t[0].imag)
    want = sorted([(z[(1, 1)], z[(2, 1)]), (z[(1, 2)], z[(2, 2)])], key=lambda t: t[0].imag)
    for (a, b), (c, d) in zip(pairs, want):
        assert abs(a - c) < 1e-7 and abs(b - d) < 1e-7


def test_hooi_core_norm_does_not_decrease():
    rng = np.random.default_rng(1)
    A = rng.standard_normal((7, 6, 5)) + 1j * rng.standard_normal((7, 6, 5))
    Us = edf.hosvd_init(A, 2)
    norms = []
    for _ in range(5):
        Us, S, _ = edf.hooi(A, 2, sweeps=1, Us=Us)
        norms.append(np.linalg.norm(S))
    assert all(b >= a - 1e-12 for a, b in zip(norms, norms[1:]))


def _column_set(M):
    return {tuple(np.round(c, 12)) for c in M.T}


@pytest.mark.parametrize("dims,p", [([5, 4, 3], 1), ([5, 4, 3], 2), ([4, 4, 4, 2], 4)])
def test_reduced_unfolding_holds_exactly_the_distinct_columns(dims, p):
    # Section 4.2: removing repeated columns of the mode-p unfolding leaves
    # the Hankel matrix of the same generating vector
    rng = np.random.default_rng(p)
    h = rng.standard_normal(sum(dims) - len(dims) + 1) + 1j * rng.standard_normal(sum(dims) - len(dims) + 1)
    full = edf.unfold(oracle.hankel_tensor(h, dims), p)
    red = edf.reduced_unfolding(h, dims, p)
    assert red.shape == (dims[p - 1], len(h) - dims[p - 1] + 1)
    assert _column_set(full) == _column_set(red)
    assert len(_column_set(red)) == red.shape[1]


def test_reduced_block_unfolding_holds_exactly_the_distinct_columns():
    rng = np.random.default_rng(3)
    n, N = [3, 2, 2], [2, 3, 2]
    G = rng.standard_normal((5, 5)) + 1j * rng.standard_normal((5, 5))
    T = oracle.bhhb_tensor(G, n, N)
    for p in (1, 2, 3):
        full = edf.unfold(T, p)
        red = edf.reduced_block_unfolding(G, n, N, p)
        assert red.shape == (n[p - 1] * N[p - 1], (6 - n[p - 1]) * (6 - N[p - 1]))
        assert _column_set(full) == _column_set(red)


def _rel_pole_error(z1, z2, z):
    """Largest relative error of the estimated (z_1, z_2) pairs against the
    exact pairs of Example 4.1, pairs matched on z_1."""
    want = [(z[(1, 1)], z[(2, 1)]), (z[(1, 2)], z[(2, 2)])]
    err = 0.0
    for a, b in zip(z1, z2):
        t1, t2 = min(want, key=lambda w: abs(w[0] - a))
        err = max(err, abs(a - t1) / abs(t1), abs(b - t2) / abs(t2))
    return err


def test_example_41_error_tracks_the_noise():
    # Section 4.3, Example 4.1: with noise, the relative pole errors of the
    # 30x30x30 HOTF + TLS estimate are at the level of the noise, and the
    # mode-1 singular values of the 6x6x6 tensor beyond the second are too
    z, peaks = example41()
    ratios = []
    for sigma in (1e-6, 1e-4, 1e-2):
        for seed in range(3):
            X = wl.damped_2d(16, 13, peaks, noise_std=sigma, seed=seed)
            U, _, _ = edf.hotf(oracle.bhhb_tensor(X, [6] * 3, [5] * 3), 2, sweeps=3)
            ratios.append(_rel_pole_error(*edf.poles_2d(U, 6, 5, 2), z) / sigma)
        X = wl.damped_2d(7, 4, peaks, noise_std=sigma, seed=0)
        s = np.linalg.svd(edf.unfold(oracle.bhhb_tensor(X, [3] * 3, [2] * 3), 1), compute_uv=False)
        assert s[1] > 0.5 * s[0] and 0.1 * sigma < s[2] / s[0] < 10 * sigma
    assert max(ratios) < 1.0 and min(ratios) > 1e-3
    assert max(ratios) / min(ratios) < 5.0  # linear in the noise level
