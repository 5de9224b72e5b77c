"""Descriptors that share storage on the fused real path: the forward is
per tensor, and the adjoint must sum each shared region's contributions
(include/hankel.h), which the plan does on the general path."""

import numpy as np
import pytest

import oracle
from paper_1401_6238_gb300 import hankel as hk

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    hk.load()
    return torch.device("cuda:0")


@pytest.mark.parametrize("flags", [hk.SAME_X, hk.SAME_X | hk.STORE_SPECTRA])
def test_shared_h_and_x_gradients_are_summed(dev, flags):
    rng = np.random.default_rng(3)
    m, n = 3, 200
    d = m * (n - 1) + 1
    h = rng.standard_normal(2 * d)
    x = rng.standard_normal(2 * n)
    # tensor 0: (h0, x0); tensor 1: (h0, x1); tensor 2: (h1, x1)
    hs, xs = [0, 0, d], [0, n, n]
    descs = hk.square_descs([m] * 3, [n] * 3, hs, xs, [0, n, 2 * n])
    plan = hk.Plan(descs, hk.R64, flags)
    H, X = torch.tensor(h, device=dev), torch.tensor(x, device=dev)
    Y = torch.zeros(3 * n, dtype=torch.float64, device=dev)
    plan.txv(H, X, Y)
    g = rng.standard_normal(3 * n)
    gh, gx = torch.zeros_like(H), torch.zeros_like(X)
    plan.backward(torch.tensor(g, device=dev), H, X, gh, gx)
    torch.cuda.synchronize()
    y, gh, gx = Y.cpu().numpy(), gh.cpu().numpy(), gx.cpu().numpy()
    want_h, want_x = np.zeros(2 * d), np.zeros(2 * n)
    for t in range(3):
        hv, xv = h[hs[t]: hs[t] + d], x[xs[t]: xs[t] + n]
        ref = oracle.fast_y(hv, [xv, xv], [n] * 3).real
        assert np.abs(y[t * n:(t + 1) * n] - ref).max() <= 1e-12 * np.abs(ref).max()
        rh, rxs = oracle.fast_grads(hv, [xv, xv], [n] * 3, g[t * n:(t + 1) * n])
        want_h[hs[t]: hs[t] + d] += rh.real
        want_x[xs[t]: xs[t] + n] += sum(r.real for r in rxs)
    assert np.abs(gh - want_h).max() <= 1e-12 * np.abs(want_h).max()
    assert np.abs(gx - want_x).max() <= 1e-12 * np.abs(want_x).max()
    plan.close()
