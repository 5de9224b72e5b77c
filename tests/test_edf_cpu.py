"""Host-side pieces of the exponential-data-fitting driver (no GPU): the
shift-invariance TLS and pole extraction of Sections 4.1 and 4.3 on exact
Vandermonde factors, the shift row sets, the leading-singular-vector step,
and the Hankel tensor sizes.  (The driver's products run only on the GPU;
tests/test_gpu_edf.py covers them.)"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")
from paper_1401_6238_gb300 import edf  # noqa: E402


def match(est, true):
    est = np.sort_complex(np.asarray(est))
    true = np.sort_complex(np.asarray(true))
    return np.abs(est - true).max()


def test_hankel_dims_sum_to_the_signal_length():
    for N in (22, 94, 4094, 4096):
        for m in (2, 3, 4):
            dims = edf.hankel_dims(N, m)
            assert sum(dims) - m + 1 == N and max(dims) - min(dims) <= 1
    assert edf.hankel_dims(4094) == [1366, 1365, 1365]


def test_tls_recovers_a_consistent_solution():
    rng = np.random.default_rng(0)
    A = torch.tensor(rng.standard_normal((30, 4)) + 1j * rng.standard_normal((30, 4)))
    W = torch.tensor(rng.standard_normal((4, 4)) + 1j * rng.standard_normal((4, 4)))
    assert torch.allclose(edf.tls(A, A @ W), W, atol=1e-10)


def test_poles_1d_from_any_basis_of_the_vandermonde_space():
    # U spans the columns z_k^i (Section 4.1); any basis of that space works
    z = np.array([0.95 * np.exp(0.4j), 0.9 * np.exp(-1.1j), 0.98 * np.exp(2.0j)])
    Z = z[None, :] ** np.arange(12)[:, None]
    T = np.random.default_rng(1).standard_normal((3, 3)) + 1j
    U = torch.tensor(np.linalg.qr(Z @ T)[0])
    assert match(edf.poles_1d(U, 3).numpy(), z) < 1e-10


def test_poles_2d_from_the_column_wise_kronecker_factor():
    # Section 4.3: the factor spans Z_2 (.) Z_1 (row index i + I j); the two
    # shift invariances give z_1 and z_2, paired per peak
    I, J = 6, 5
    z1 = np.array([np.exp(-0.01 + 2j * np.pi * 0.20), np.exp(-0.02 + 2j * np.pi * 0.22)])
    z2 = np.array([np.exp(-0.02 + 2j * np.pi * 0.18), np.exp(-0.01 - 2j * np.pi * 0.20)])
    cols = [np.kron(z2[k] ** np.arange(J), z1[k] ** np.arange(I)) for k in range(2)]
    U = torch.tensor(np.linalg.qr(np.stack(cols, axis=1) @ np.array([[1.0, 0.3], [0.2j, 1.0]]))[0])
    a, b = edf.poles_2d(U, I, J, 2)
    a, b = a.numpy(), b.numpy()
    for k in range(2):
        i = int(np.argmin(np.abs(a - z1[k])))
        assert abs(a[i] - z1[k]) < 1e-10 and abs(b[i] - z2[k]) < 1e-10


def test_shift_rows_2d():
    up1, down1, up2, down2 = (t.tolist() for t in edf.shift_rows_2d(3, 2))
    assert up1 == [0, 1, 3, 4] and down1 == [1, 2, 4, 5]
    assert up2 == [0, 1, 2] and down2 == [3, 4, 5]


@pytest.mark.parametrize("shape", [(40, 9), (300, 256), (20, 60)])
def test_leading_left_matches_the_svd(shape):
    rng = np.random.default_rng(2)
    M = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    U, s = edf.leading_left(torch.tensor(M), 4)
    Ue, se, _ = np.linalg.svd(M, full_matrices=False)
    np.testing.assert_allclose(np.asarray(s)[:min(shape)], se, rtol=1e-10)
    P = U.numpy() @ U.numpy().conj().T
    Pe = Ue[:, :4] @ Ue[:, :4].conj().T
    assert np.abs(P - Pe).max() < 1e-10
