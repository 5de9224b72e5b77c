"""Real tensors with a different vector in every mode (y = H x_2 ... x_m,
alpha = H x_1 ... x_m; Section 3's m + 1 transform form) on the fused pair
kernel, against the oracle element by element: ragged non-square shapes,
orders 2-5, an odd count (one tensor without a partner), y alone, alpha
alone, FP64 and FP32; the full 8192-tensor batch on sampled tensors; and the
adjoint (general path) of the same plan."""

import numpy as np
import pytest

import oracle
from paper_1401_6238_gb300 import hankel as hk
from paper_1401_6238_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TDT = {hk.R32: torch.float32, hk.R64: torch.float64}


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    hk.load()
    return torch.device("cuda:0")


def ragged_case(count, seed):
    rng = np.random.default_rng(seed)
    tensors, hs, xs = [], [], []
    d = hk.make_descs(count)
    ho = xo = yo = 0
    for i in range(count):
        m = int(rng.integers(2, 6))
        dims = [int(v) for v in rng.integers(3, 400, size=m)]
        dh = sum(dims) - m + 1
        # the benchmark's scaling: h ~ N(0, 1/d), unit-norm vectors
        h = rng.standard_normal(dh) / np.sqrt(dh)
        vs = [v / np.linalg.norm(v) for v in (rng.standard_normal(n) for n in dims)]
        d[i]["m"] = m
        d[i]["n"][:m] = dims
        d[i]["h_off"] = ho
        for p in range(m):
            d[i]["x_off"][p] = xo
            xo += dims[p]
        d[i]["y_off"] = yo
        ho += dh
        yo += dims[0]
        tensors.append((dims, h, vs))
        hs.append(h)
        xs += vs
    return tensors, np.concatenate(hs), np.concatenate(xs), d, yo


@pytest.mark.parametrize("dtype,tol", [(hk.R64, 1e-12), (hk.R32, 1e-5)])
def test_ragged_batch(dev, dtype, tol):
    tensors, h, x, d, ny = ragged_case(301, seed=1)
    plan = hk.Plan(d, dtype, 0)
    assert plan.info["jobs"] < 301  # tensors of equal length share jobs
    H = torch.tensor(h, dtype=TDT[dtype], device=dev)
    X = torch.tensor(x, dtype=TDT[dtype], device=dev)
    Y = torch.zeros(ny, dtype=TDT[dtype], device=dev)
    A = torch.zeros(len(tensors), dtype=TDT[dtype], device=dev)
    plan.txv(H, X, Y, A)
    Y2, A2 = torch.zeros_like(Y), torch.zeros_like(A)
    plan.txv(H, X, Y2, None)
    plan.txv(H, X, None, A2)
    torch.cuda.synchronize()
    y, a = Y.cpu().numpy(), A.cpu().numpy()
    assert torch.equal(Y, Y2) and torch.equal(A, A2)
    for i, (dims, hv, vs) in enumerate(tensors):
        ref = oracle.fast_y(hv, vs[1:], dims).real
        got = y[d[i]["y_off"]: d[i]["y_off"] + dims[0]]
        assert np.abs(got - ref).max() <= tol * np.abs(ref).max(), i
        ar = oracle.fast_alpha(hv, vs, dims).real
        assert abs(a[i] - ar) <= tol * np.abs(ref).max() * np.abs(vs[0]).sum(), i
    plan.close()


def test_full_batch_sampled(dev):
    b, xoffs = wl.batched_distinct(8192)
    d = hk.make_descs(len(b))
    d["m"] = b.orders
    for p in range(8):
        d["n"][:, p] = np.where(p < b.orders, b.dims, 0)
    d["h_off"] = b.h_off
    for i, offs in enumerate(xoffs):
        d["x_off"][i, :len(offs)] = offs
    d["y_off"] = b.y_off
    plan = hk.Plan(d, hk.R32, 0)
    H = torch.tensor(b.h, dtype=torch.float32, device=dev)
    X = torch.tensor(b.x, dtype=torch.float32, device=dev)
    Y = torch.zeros(b.y_len, dtype=torch.float32, device=dev)
    A = torch.zeros(len(b), dtype=torch.float32, device=dev)
    plan.txv(H, X, Y, A)
    torch.cuda.synchronize()
    y, a = Y.cpu().numpy(), A.cpu().numpy()
    for i in np.random.default_rng(0).choice(len(b), 40, replace=False):
        m, n = int(b.orders[i]), int(b.dims[i])
        dh = m * (n - 1) + 1
        hv = b.h[b.h_off[i]: b.h_off[i] + dh]
        vs = [b.x[o: o + n] for o in xoffs[i]]
        ref = oracle.fast_y(hv, vs[1:], [n] * m).real
        assert np.abs(y[b.y_off[i]: b.y_off[i] + n] - ref).max() <= 1e-5 * np.abs(ref).max(), i
        ar = oracle.fast_alpha(hv, vs, [n] * m).real
        assert abs(a[i] - ar) <= 1e-5 * np.abs(ref).max() * np.abs(vs[0]).sum(), i
    plan.close()


def test_adjoint_of_the_same_plan(dev):
    tensors, h, x, d, ny = ragged_case(9, seed=2)
    plan = hk.Plan(d, hk.R64, 0)
    g = np.random.default_rng(3).standard_normal(ny)
    gh = torch.zeros(h.size, dtype=torch.float64, device=dev)
    gx = torch.zeros(x.size, dtype=torch.float64, device=dev)
    plan.backward(torch.tensor(g, device=dev), torch.tensor(h, device=dev), torch.tensor(x, device=dev), gh, gx)
    torch.cuda.synchronize()
    gh, gx = gh.cpu().numpy(), gx.cpu().numpy()
    for i, (dims, hv, vs) in enumerate(tensors):
        rh, rx = oracle.fast_grads(hv, vs[1:], dims, g[d[i]["y_off"]: d[i]["y_off"] + dims[0]])
        assert np.abs(gh[d[i]["h_off"]: d[i]["h_off"] + hv.size] - rh.real).max() <= 1e-12 * np.abs(rh).max(), i
        for p in range(1, len(dims)):
            o = d[i]["x_off"][p]
            assert np.abs(gx[o: o + dims[p]] - rx[p - 1].real).max() <= 1e-12 * np.abs(rx[p - 1]).max(), (i, p)
    plan.close()
