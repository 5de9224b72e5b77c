"""Tensors longer than one block's shared memory: each length-L transform
runs on a thread-block cluster, two blocks of length L/2 or, where L/2 is
still too long, four of L/4 (radix-2 / radix-4 decimation in frequency,
the spectra passing through the plan workspace across a cluster
barrier).  y, alpha and the gradients against the FP64 oracle, every
element, FP32 and FP64, with and without spectra kept from the forward."""

import numpy as np
import pytest

import oracle
from paper_1401_6238_gb300 import hankel as hk
from paper_1401_6238_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {hk.R32: 1e-5, hk.R64: 1e-12}
# generating lengths past one block's shared memory (FP32: above ~13.6K,
# FP64: above ~6.8K), with ragged sizes and several orders
SHAPES = {hk.R32: [(4, 4096), (3, 5000), (2, 7000), (5, 3000), (4, 3800)],
          hk.R64: [(3, 3000), (2, 4100), (4, 2500), (5, 2000), (4, 4096), (3, 5000)]}
# FP64 at L = 16384 (L/2 beyond one block): the four-block clusters


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    hk.load()
    return torch.device("cuda:0")


def scaled(shapes, seed):
    rng = np.random.default_rng(seed)
    orders, dims, hs, xs = [], [], [], []
    for m, n in shapes:
        d = m * (n - 1) + 1
        x = rng.standard_normal(n)
        orders.append(m)
        dims.append(n)
        hs.append(rng.standard_normal(d) / np.sqrt(d))
        xs.append(x / np.linalg.norm(x))
    return wl.pack_square(orders, dims, hs, xs)


def rel(a, b):
    return np.max(np.abs(a - b)) / np.max(np.abs(b))


@pytest.mark.parametrize("dtype", [hk.R32, hk.R64])
@pytest.mark.parametrize("store", [False, True])
def test_long_forward_and_gradients(dev, dtype, store):
    b = scaled(SHAPES[dtype], seed=50 + dtype)
    flags = hk.SAME_X | (hk.STORE_SPECTRA if store else 0)
    plan = hk.Plan(hk.batch_descs(b), dtype, flags)
    assert plan.info["max_length"] > 8192 if dtype == hk.R32 else plan.info["max_length"] > 6144
    tdt = torch.float32 if dtype == hk.R32 else torch.float64
    T = lambda a: torch.tensor(a, dtype=tdt, device=dev)
    H, X = T(b.h), T(b.x)
    Y = torch.full((b.y_len,), float("nan"), dtype=tdt, device=dev)
    A = torch.full((len(b),), float("nan"), dtype=tdt, device=dev)
    plan.txv(H, X, Y, A)
    g = np.random.default_rng(7).standard_normal(b.y_len)
    gh, gx = torch.zeros_like(H), torch.zeros_like(X)
    plan.backward(T(g), H, X, gh, gx)
    torch.cuda.synchronize()
    y, a, gh, gx = Y.cpu().numpy(), A.cpu().numpy(), gh.cpu().numpy(), gx.cpu().numpy()
    tol = TOL[dtype]
    for i in range(len(b)):
        m, n, h, x = b.tensor(i)
        ref = oracle.fast_y(h, [x] * (m - 1), [n] * m).real
        assert rel(y[b.y_off[i]: b.y_off[i] + n], ref) <= tol, ("y", i, m, n)
        assert abs(a[i] - float(np.dot(x, ref))) <= tol * np.max(np.abs(ref)) * np.sum(np.abs(x)), ("alpha", i)
        rh, rxs = oracle.fast_grads(h, [x] * (m - 1), [n] * m, g[b.y_off[i]: b.y_off[i] + n])
        assert rel(gh[b.h_off[i]: b.h_off[i] + h.size], rh.real) <= tol, ("grad_h", i)
        assert rel(gx[b.x_off[i]: b.x_off[i] + n], sum(r.real for r in rxs)) <= tol, ("grad_x", i)
    plan.close()


def test_long_y_only_alpha_only_and_repeat(dev):
    b = scaled(SHAPES[hk.R32], seed=60)
    plan = hk.Plan(hk.batch_descs(b), hk.R32, hk.SAME_X)
    H = torch.tensor(b.h, dtype=torch.float32, device=dev)
    X = torch.tensor(b.x, dtype=torch.float32, device=dev)
    Y = torch.zeros(b.y_len, dtype=torch.float32, device=dev)
    A = torch.zeros(len(b), dtype=torch.float32, device=dev)
    plan.txv(H, X, Y, None)
    plan.txv(H, X, None, A)
    torch.cuda.synchronize()
    y1, a1 = Y.clone(), A.clone()
    plan.txv(H, X, Y, A)
    torch.cuda.synchronize()
    assert torch.equal(y1, Y) and torch.equal(a1, A)
    plan.close()
    for i in range(len(b)):
        m, n, h, x = b.tensor(i)
        ref = oracle.fast_y(h, [x] * (m - 1), [n] * m).real
        assert rel(y1.cpu().numpy()[b.y_off[i]: b.y_off[i] + n], ref) <= 1e-5
