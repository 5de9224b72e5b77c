"""Exponential data fitting (Section 4) on the GPU against the oracle.

* HOOI (Algorithm 4.1) and HOTF (Algorithm 4.2) driven by the library's
  batched products, started from the same factors as the oracle's dense
  HOOI, give the same subspaces, singular values and low-rank approximation
  (complex128).
* The initial factors from the reduced unfolding (Section 4.2) match the
  SVD of the oracle's explicit reduced unfolding.
* Noiseless signals give the exact poles; Example 4.1 gives its printed
  poles, correctly paired, and its rank-2 statement.
* Full size (complex64): the 1D signal of length 4094 (1366 x 1365 x 1365,
  K = 8, 20 dB) and the 256 x 256 2D signal (BHHB blocks 86^3 x 86^3,
  K = 12, 20 dB): one mode update against products and an SVD computed by
  the oracle, the monotone core norm, and the recovered poles.
"""

import numpy as np
import pytest

import oracle
from conftest import golden
from oracle import edf as oedf
from paper_1401_6238_gb300 import hankel as hk
from paper_1401_6238_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
linear_sum_assignment = pytest.importorskip("scipy.optimize").linear_sum_assignment


@pytest.fixture(scope="module")
def edf():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    hk.load()
    from paper_1401_6238_gb300 import edf as gedf
    return gedf


def np_(t):
    return t.detach().cpu().numpy()


def proj(U):
    return U @ U.conj().T


def match(est, true):
    """Largest distance between estimated and true poles under the best
    one-to-one assignment, and that assignment."""
    C = np.abs(np.asarray(est)[:, None] - np.asarray(true)[None, :])
    r, c = linear_sum_assignment(C)
    return C[r, c].max(), r, c


POLES = [0.95 * np.exp(0.4j), 0.9 * np.exp(-1.1j), 0.98 * np.exp(2.0j)]
AMPS = [1.0, 0.7 - 0.2j, 1.3j]


@pytest.mark.parametrize("symmetric", [True, False])
def test_1d_noiseless_exact_poles(edf, symmetric):
    x = wl.damped_1d(22, POLES, AMPS)
    T = edf.HankelTensor(x, [8, 8, 8], dtype=hk.C128)
    h = edf.HOOI(T, 3, symmetric=symmetric).init()
    h.fit(2)
    err, _, _ = match(np_(edf.poles_1d(h.U[0], 3)), POLES)
    assert err < 1e-9
    h.close()


def recon(S, Us):
    return np.einsum("abc,ia,jb,kc->ijk", S, *Us)


def test_hooi_matches_oracle(edf):
    # Algorithm 4.1 on a non-square noisy tensor, same start as the oracle
    s = wl.damped_1d(94, POLES, AMPS, noise_std=0.05)
    dims = [33, 32, 31]
    A = oracle.hankel_tensor(s, dims)
    U0 = oedf.hosvd_init(A, 4)
    Uo, So, so = oedf.hooi(A, 4, 3, Us=U0)
    T = edf.HankelTensor(s, dims, dtype=hk.C128)
    h = edf.HOOI(T, 4)
    for p in range(3):
        h.set_factor(p, torch.tensor(U0[p]))
    norms = h.fit(3)
    for p in range(3):
        assert np.abs(proj(np_(h.U[p])) - proj(Uo[p])).max() < 1e-10, p
        assert np.abs(np_(h.svals[p])[:8] - so[p][:8]).max() < 1e-11 * so[p][0], p
    S = np_(h.core())
    assert np.abs(recon(S, [np_(U) for U in h.U]) - recon(So, Uo)).max() < 1e-11 * np.abs(A).max()
    assert abs(norms[-1] - np.linalg.norm(So)) < 1e-11 * norms[-1]
    h.close()


def test_hotf_matches_oracle(edf):
    # Algorithm 4.2: one factor, sorted index pairs weighted by multiplicity
    s = wl.damped_1d(46, POLES, AMPS, noise_std=0.05)
    A = oracle.hankel_tensor(s, [16] * 3)
    U0 = oedf.leading_left(oedf.unfold(A, 1), 4)[0]
    Uo, So, so = oedf.hotf(A, 4, 3, U=U0)
    T = edf.HankelTensor(s, [16] * 3, dtype=hk.C128)
    h = edf.HOOI(T, 4, symmetric=True)
    h.set_factor(0, torch.tensor(U0))
    h.fit(3)
    assert np.abs(proj(np_(h.U[0])) - proj(Uo)).max() < 1e-10
    assert np.abs(np_(h.svals[0])[:10] - so[:10]).max() < 1e-11 * so[0]
    U = np_(h.U[0])
    assert np.abs(recon(np_(h.core()), [U] * 3) - recon(So, [Uo] * 3)).max() < 1e-11 * np.abs(A).max()
    h.close()


@pytest.mark.parametrize("noise", [0.0, 0.05])
def test_init_matches_reduced_unfolding_svd(edf, noise):
    # Section 4.2: the initial factor spans the leading left singular
    # vectors of the I_p x (d - I_p + 1) Hankel matrix
    s = wl.damped_1d(94, POLES, AMPS, noise_std=noise)
    dims = [33, 32, 31]
    T = edf.HankelTensor(s, dims, dtype=hk.C128)
    h = edf.HOOI(T, 3).init(power_iters=6)
    for p in range(3):
        Ue = np.linalg.svd(oedf.reduced_unfolding(s, dims, p + 1))[0][:, :3]
        assert np.abs(proj(np_(h.U[p])) - proj(Ue)).max() < (1e-10 if noise == 0 else 1e-6), p
    h.close()


def test_block_init_matches_reduced_unfolding_svd(edf):
    z, peaks = example41()
    X = wl.damped_2d(16, 13, peaks, noise_std=0.02)
    T = edf.HankelTensor(X, [6] * 3, [5] * 3, dtype=hk.C128)
    h = edf.HOOI(T, 2, symmetric=True).init(power_iters=8)
    Ue = np.linalg.svd(oedf.reduced_block_unfolding(X, [6] * 3, [5] * 3, 1))[0][:, :2]
    assert np.abs(proj(np_(h.U[0])) - proj(Ue)).max() < 1e-8
    h.close()


def example41():
    g = golden("example41_poles.txt")
    z = {(int(d), int(k)): np.exp(a + 2j * np.pi * f) for d, k, a, f in g}
    peaks = [(g[0, 2], g[0, 3], g[2, 2], g[2, 3]), (g[1, 2], g[1, 3], g[3, 2], g[3, 3])]
    return z, peaks


@pytest.mark.parametrize("dtype,tol", [(hk.C128, 1e-9), (hk.C64, 1e-4)])
def test_example_41_poles(edf, dtype, tol):
    # Section 4.3: HOTF rank-(2,2,2) of the 30x30x30 BHHB tensor with 6x6x6
    # blocks, then TLS twice: the printed poles, paired by peak
    z, peaks = example41()
    X = wl.damped_2d(16, 13, peaks)
    (z1, z2), norms = edf.fit_2d(X, 6, 5, 2, sweeps=2, dtype=dtype)
    z1, z2 = np_(z1), np_(z2)
    e1, r, c = match(z1, [z[(1, 1)], z[(1, 2)]])
    assert e1 < tol
    # the z_2 estimate that comes with each z_1 belongs to the same peak
    for i, k in zip(r, c):
        assert abs(z2[i] - z[(2, k + 1)]) < tol


def test_example_41_rank_two(edf):
    # Section 4.3: the 6x6x6 BHHB tensor with 3x3x3 blocks of the noiseless
    # signal has exactly two nonzero mode singular values
    z, peaks = example41()
    X = wl.damped_2d(7, 4, peaks)
    T = edf.HankelTensor(X, [3] * 3, [2] * 3, dtype=hk.C128)
    h = edf.HOOI(T, 3, symmetric=True).init()
    h.fit(2)
    s = np_(h.svals[0])
    assert s[1] > 1e-3 * s[0] and s[2] < 1e-12 * s[0]
    h.close()


@pytest.mark.parametrize("sigma", [0.0, 1e-4, 1e-2])
def test_example_41_mode1_singular_values(edf, sigma):
    # Section 4.3, Example 4.1: the mode-1 singular values of the 6x6x6 BHHB
    # tensor (3x3x3 blocks).  With R = 6 the factor is unitary, so one HOTF
    # update's unfolding has exactly the tensor's mode-1 singular values.
    z, peaks = example41()
    X = wl.damped_2d(7, 4, peaks, noise_std=sigma, seed=0)
    want = np.linalg.svd(oedf.unfold(oracle.bhhb_tensor(X, [3] * 3, [2] * 3), 1), compute_uv=False)
    T = edf.HankelTensor(X, [3] * 3, [2] * 3, dtype=hk.C128)
    h = edf.HOOI(T, 6, symmetric=True).init()
    s = np_(h.update(0))
    assert np.abs(s - want).max() < 1e-12 * want[0]
    if sigma == 0:
        assert s[1] > 0.5 * s[0] and s[2] < 1e-12 * s[0]
    h.close()


@pytest.mark.parametrize("sigma", [1e-6, 1e-3])
def test_example_41_noisy_poles_match_oracle(edf, sigma):
    # Example 4.1 with noise: from the same start, the GPU HOTF + TLS gives
    # the oracle's pole estimates, and their error is at the noise level
    z, peaks = example41()
    X = wl.damped_2d(16, 13, peaks, noise_std=sigma, seed=1)
    A = oracle.bhhb_tensor(X, [6] * 3, [5] * 3)
    U0 = oedf.leading_left(oedf.unfold(A, 1), 2)[0]
    Uo, _, _ = oedf.hotf(A, 2, 3, U=U0)
    ao, bo = oedf.poles_2d(Uo, 6, 5, 2)
    T = edf.HankelTensor(X, [6] * 3, [5] * 3, dtype=hk.C128)
    h = edf.HOOI(T, 2, symmetric=True)
    h.set_factor(0, torch.tensor(U0))
    h.fit(3)
    a, b = edf.poles_2d(h.U[0], 6, 5, 2)
    a, b = np_(a), np_(b)
    e, r, c = match(a, ao)
    assert e < 1e-10
    assert np.abs(b[r] - bo[c]).max() < 1e-10
    want = {1: (z[(1, 1)], z[(2, 1)]), 2: (z[(1, 2)], z[(2, 2)])}
    err = max(max(abs(x - w[0]) / abs(w[0]), abs(y - w[1]) / abs(w[1]))
              for x, y in zip(a, b) for w in [min(want.values(), key=lambda w: abs(w[0] - x))])
    assert 1e-3 * sigma < err < sigma


def test_1d_full_size_hooi(edf):
    # 1D signal of length 4094, K = 8, 20 dB: order-3 Hankel 1366x1365x1365,
    # Algorithm 4.1 with R = 8, complex64
    s, z = wl.edf_1d_signal(N=4094, K=8, seed=4, with_poles=True)
    dims = edf.hankel_dims(4094)
    assert dims == [1366, 1365, 1365]
    T = edf.HankelTensor(s, dims, dtype=hk.C64)
    h = edf.HOOI(T, 8).init()
    err0, _, _ = match(np_(edf.poles_1d(h.U[0], 8)), z)
    assert err0 < 1e-2
    norms = h.fit(6)
    assert all(b >= a * (1 - 1e-5) for a, b in zip(norms, norms[1:]))
    for U in h.U:  # Householder QR in complex64: orthonormal to about I_p * eps
        G = np_(U.mH @ U)
        assert np.abs(G - np.eye(8)).max() < 1366 * 6e-8
    # one mode-1 update against the oracle: the 64 products and their SVD
    U2, U3 = np_(h.U[1]).astype(complex), np_(h.U[2]).astype(complex)
    M = np_(h.products(0))
    ref = np.stack([oracle.fast_y(s.astype(np.complex64).astype(complex), [U2[:, i].conj(), U3[:, j].conj()], dims)
                    for i in range(8) for j in range(8)], axis=1)
    assert np.abs(M - ref).max() < 1e-5 * np.abs(ref).max()
    Ur, sr, _ = np.linalg.svd(ref, full_matrices=False)
    sg = np_(h.update(0))
    assert np.abs(sg[:8] - sr[:8]).max() < 1e-5 * sr[0]
    assert np.abs(proj(np_(h.U[0])) - proj(Ur[:, :8])).max() < 1e-3
    h.close()


def test_2d_full_size_hotf(edf):
    # 256 x 256 2D signal, K = 12, 20 dB: order-3 BHHB with blocks
    # (86,86,86) x (86,86,86), Algorithm 4.2 with R = 12, complex64
    S, (z1, z2) = wl.edf_2d_signal(with_poles=True)
    T = edf.HankelTensor(S, [86] * 3, [86] * 3, dtype=hk.C64)
    h = edf.HOOI(T, 12, symmetric=True).init()
    norms = h.fit(3)
    assert all(b >= a * (1 - 1e-5) for a, b in zip(norms, norms[1:]))
    a, b = edf.poles_2d(h.U[0], 86, 86, 12)
    a, b = np_(a), np_(b)
    e1, r, c = match(a, z1)
    assert e1 < 5e-3
    assert np.abs(b[r] - z2[c]).max() < 5e-3
    # one update against the oracle: a sample of the 78 weighted columns
    U = np_(h.U[0]).astype(complex)
    M = np_(h.products(0))
    Sd = S.astype(np.complex64).astype(complex)
    tuples = [(i, j) for i in range(12) for j in range(i, 12)]
    for k in (0, 5, 40, 77):
        i, j = tuples[k]
        Xi = U[:, i].conj().reshape(86, 86, order="F")
        Xj = U[:, j].conj().reshape(86, 86, order="F")
        ref = oracle.fast_block_y(Sd, [Xi, Xj], [86] * 3, [86] * 3).reshape(-1, order="F")
        ref = ref * (1.0 if i == j else np.sqrt(2.0))
        assert np.abs(M[:, k] - ref).max() < 1e-5 * np.abs(ref).max(), k
    h.close()
