"""Full-size parity of the secondary workloads, sampled against the oracle:

* HOOI tensor-matrix products (Section 4.2): H x_2 u_i x_3 v_j for all
  16 x 16 column pairs of the order-3 Hankel tensor (1366 x 1365 x 1365) of
  a complex 1D exponential signal of length 4094; every product shares h.
* 2D block products (Section 3, BHHB): a 256 x 256 complex 2D exponential
  signal as generating matrix, blocks (86, 86, 86) x (86, 86, 86), 32 vector
  triples, forward y and alpha and the adjoint.
"""

import numpy as np
import pytest

import oracle
from paper_1401_6238_gb300 import hankel as hk
from paper_1401_6238_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    hk.load()
    return torch.device("cuda:0")


def rel(a, b):
    return np.max(np.abs(a - b)) / np.max(np.abs(b))


def hooi_case(R=16, N=4094, seed=4):
    s = wl.edf_1d_signal(N=N, seed=seed)
    dims = [N + 2 - 2 * ((N + 2) // 3), (N + 2) // 3, (N + 2) // 3]
    U = wl.unit_columns(dims[1], R, seed=seed + 1)
    V = wl.unit_columns(dims[2], R, seed=seed + 2)
    x = np.concatenate([U.T.reshape(-1), V.T.reshape(-1)])
    descs = hk.make_descs(R * R)
    for k in range(R * R):
        i, j = divmod(k, R)
        descs[k]["m"] = 3
        descs[k]["n"][:3] = dims
        descs[k]["h_off"] = 0
        descs[k]["x_off"][1] = i * dims[1]
        descs[k]["x_off"][2] = R * dims[1] + j * dims[2]
        descs[k]["y_off"] = k * dims[0]
    return s, x, dims, U, V, descs


def test_hooi_pair_products_full_size(dev):
    R = 16
    s, x, dims, U, V, descs = hooi_case(R)
    assert dims == [1366, 1365, 1365]
    plan = hk.Plan(descs, hk.C64, 0)
    Y = torch.zeros(R * R * dims[0], dtype=torch.complex64, device=dev)
    plan.txv(torch.tensor(s, dtype=torch.complex64, device=dev), torch.tensor(x, dtype=torch.complex64, device=dev), Y)
    torch.cuda.synchronize()
    y = Y.cpu().numpy()
    for k in [0, 1, 17, 100, 255]:
        i, j = divmod(k, R)
        ref = oracle.fast_y(s, [U[:, i], V[:, j]], dims)
        assert rel(y[k * dims[0]:(k + 1) * dims[0]], ref) <= 1e-5, k
    plan.close()


def bhhb_case(count=32, seed=5):
    S = wl.edf_2d_signal(seed=seed)
    n = N = [86, 86, 86]
    Xs = wl.unit_matrices(2 * count + count, 86, 86, seed=seed + 1)  # x_2, x_3 and x_1 per triple
    x = np.concatenate([X.reshape(-1, order="F") for X in Xs])
    descs = hk.make_descs(count)
    for t in range(count):
        descs[t]["m"] = 3
        descs[t]["n"][:3] = n
        descs[t]["N"][:3] = N
        descs[t]["h_off"] = 0
        descs[t]["x_off"][0] = (2 * count + t) * 86 * 86
        descs[t]["x_off"][1] = (2 * t) * 86 * 86
        descs[t]["x_off"][2] = (2 * t + 1) * 86 * 86
        descs[t]["y_off"] = t * 86 * 86
    return S, Xs, x, n, N, descs


def test_bhhb_forward_alpha_full_size(dev):
    count = 32
    S, Xs, x, n, N, descs = bhhb_case(count)
    assert S.shape == (256, 256)
    plan = hk.Plan(descs, hk.C64, hk.BLOCK)
    Y = torch.zeros(count * 86 * 86, dtype=torch.complex64, device=dev)
    A = torch.zeros(count, dtype=torch.complex64, device=dev)
    plan.txv_block(torch.tensor(S.reshape(-1, order="F"), dtype=torch.complex64, device=dev),
                   torch.tensor(x, dtype=torch.complex64, device=dev), Y, A)
    torch.cuda.synchronize()
    y, a = Y.cpu().numpy(), A.cpu().numpy()
    for t in [0, 13, 31]:
        ref = oracle.fast_block_y(S, [Xs[2 * t], Xs[2 * t + 1]], n, N)
        got = y[t * 86 * 86:(t + 1) * 86 * 86].reshape(86, 86, order="F")
        assert rel(got, ref) <= 1e-5, t
        ar = np.sum(oracle.vec(Xs[2 * count + t]) * oracle.vec(ref))
        assert abs(a[t] - ar) <= 1e-5 * np.max(np.abs(ref)) * np.sum(np.abs(Xs[2 * count + t])), t
    plan.close()


def test_bhhb_adjoint_full_size(dev):
    count = 32
    S, Xs, x, n, N, descs = bhhb_case(count)
    plan = hk.Plan(descs, hk.C64, hk.BLOCK)
    rng = np.random.default_rng(12)
    G = (rng.standard_normal((count, 86, 86)) + 1j * rng.standard_normal((count, 86, 86))) / 86
    g = np.concatenate([Gt.reshape(-1, order="F") for Gt in G])
    gh = torch.zeros(S.size, dtype=torch.complex64, device=dev)
    gx = torch.zeros(x.size, dtype=torch.complex64, device=dev)
    plan.backward(torch.tensor(g, dtype=torch.complex64, device=dev),
                  torch.tensor(S.reshape(-1, order="F"), dtype=torch.complex64, device=dev),
                  torch.tensor(x, dtype=torch.complex64, device=dev), gh, gx)
    torch.cuda.synchronize()
    gh, gx = gh.cpu().numpy(), gx.cpu().numpy()
    total = np.zeros((256, 256), complex)
    for t in range(count):
        rH, rXs = oracle.fast_block_grads(S, [Xs[2 * t], Xs[2 * t + 1]], n, N, G[t])
        total += rH
        if t in (0, 31):
            for p in range(2):
                o = (2 * t + p) * 86 * 86
                assert rel(gx[o:o + 86 * 86].reshape(86, 86, order="F"), rXs[p]) <= 2e-5, (t, p)
    # the generating matrix is shared by all 32 triples: its gradient is the sum
    assert rel(gh.reshape(256, 256, order="F"), total) <= 2e-5
    plan.close()
