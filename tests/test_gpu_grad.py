"""GPU parity of the adjoint kernels (hankel_txv_backward) and of the
torch.autograd.Function built on them: against the oracle's analytic
gradients and FP64 central finite differences."""

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


def grads(batch, dtype, flags, g, dev, forward_first=False):
    tdt = torch.float32 if dtype == hk.R32 else torch.float64
    plan = hk.Plan(hk.batch_descs(batch), dtype, flags)
    H = torch.tensor(batch.h, dtype=tdt, device=dev)
    X = torch.tensor(batch.x, dtype=tdt, device=dev)
    G = torch.tensor(g, dtype=tdt, device=dev)
    gh = torch.zeros_like(H)
    gx = torch.zeros_like(X)
    if forward_first:
        Y = torch.zeros(batch.y_len, dtype=tdt, device=dev)
        plan.txv(H, X, Y)
    plan.backward(G, H, X, gh, gx)
    torch.cuda.synchronize()
    plan.close()
    return gh.cpu().numpy().astype(np.float64), gx.cpu().numpy().astype(np.float64)


def ref_grads(batch, g, i):
    m, n, h, x = batch.tensor(i)
    gi = g[batch.y_off[i]: batch.y_off[i] + n]
    gh, gxs = oracle.fast_grads(h, [x] * (m - 1), [n] * m, gi)
    return gh.real, sum(v.real for v in gxs)


@pytest.mark.parametrize("dtype,tol", [(hk.R32, 1e-5), (hk.R64, 1e-12)])
@pytest.mark.parametrize("flags", [hk.SAME_X, hk.SAME_X | hk.STORE_SPECTRA])
def test_backward_matches_oracle(dev, dtype, tol, flags):
    b = wl.batched_square(count=24, seed=71, n_lo=16, n_hi=700)
    g = np.random.default_rng(1).standard_normal(b.y_len)
    gh, gx = grads(b, dtype, flags, g, dev, forward_first=bool(flags & hk.STORE_SPECTRA))
    for i in range(len(b)):
        m, n, h, x = b.tensor(i)
        d = len(h)
        rh, rx = ref_grads(b, g, i)
        eh = np.max(np.abs(gh[b.h_off[i]: b.h_off[i] + d] - rh)) / np.max(np.abs(rh))
        ex = np.max(np.abs(gx[b.x_off[i]: b.x_off[i] + n] - rx)) / np.max(np.abs(rx))
        assert eh <= tol and ex <= tol, (i, m, n, eh, ex)


def test_autograd_matches_finite_differences_fp64(dev):
    b = wl.batched_square(count=3, seed=81, n_lo=5, n_hi=9)
    plan = hk.Plan(hk.batch_descs(b), hk.R64, hk.SAME_X)
    H = torch.tensor(b.h, device=dev, requires_grad=True)
    X = torch.tensor(b.x, device=dev, requires_grad=True)
    ny = plan.info["y_elems"]
    t = torch.tensor(np.random.default_rng(2).standard_normal(ny), device=dev)
    y = hk.hankel_txv_autograd(H, X, plan)
    loss = ((y - t) ** 2).sum()
    loss.backward()

    def f(hv, xv):
        y = torch.zeros(ny, dtype=torch.float64, device=dev)
        plan.txv(hv, xv, y)
        return float(((y - t) ** 2).sum())

    eps = 1e-6
    for vec, grad, name in [(H, H.grad, "h"), (X, X.grad, "x")]:
        base = vec.detach().clone()
        rng = np.random.default_rng(3)
        for j in rng.choice(base.numel(), size=min(12, base.numel()), replace=False):
            p, m_ = base.clone(), base.clone()
            p[j] += eps
            m_[j] -= eps
            if name == "h":
                fd = (f(p, X.detach()) - f(m_, X.detach())) / (2 * eps)
            else:
                fd = (f(H.detach(), p) - f(H.detach(), m_)) / (2 * eps)
            assert abs(fd - grad[j].item()) <= 1e-6 * max(1.0, abs(fd)), (name, j, fd, grad[j].item())
    plan.close()


def test_store_spectra_equals_recompute(dev):
    # spectra kept from the forward (per-length adjoint reading them) and
    # recomputed (the persistent adjoint): different kernels and FFT lengths,
    # so not the same bits, but both within the bound of the oracle and of
    # each other
    b = wl.batched_square(count=10, seed=91, n_lo=100, n_hi=900)
    g = np.random.default_rng(4).standard_normal(b.y_len)
    a = grads(b, hk.R32, hk.SAME_X, g, dev)
    c = grads(b, hk.R32, hk.SAME_X | hk.STORE_SPECTRA, g, dev, forward_first=True)
    for i in range(len(b)):
        m, n, h, x = b.tensor(i)
        rh, rxs = oracle.fast_grads(h, [x] * (m - 1), [n] * m, g[b.y_off[i]: b.y_off[i] + n])
        rx = sum(r.real for r in rxs)
        sh, sx = slice(b.h_off[i], b.h_off[i] + h.size), slice(b.x_off[i], b.x_off[i] + n)
        for got in (a, c):
            assert np.max(np.abs(got[0][sh] - rh.real)) <= 1e-5 * np.max(np.abs(rh.real)), ("grad_h", i)
            assert np.max(np.abs(got[1][sx] - rx)) <= 1e-5 * np.max(np.abs(rx)), ("grad_x", i)
        assert np.max(np.abs(a[0][sh] - c[0][sh])) <= 1e-5 * np.max(np.abs(c[0][sh])), ("grad_h a/c", i)
        assert np.max(np.abs(a[1][sx] - c[1][sx])) <= 1e-5 * np.max(np.abs(c[1][sx])), ("grad_x a/c", i)


@pytest.mark.parametrize("dtype,tol", [(hk.R32, 1e-5), (hk.R64, 1e-12)])
@pytest.mark.parametrize("flags", [hk.SAME_X, hk.SAME_X | hk.STORE_SPECTRA])
def test_backward_pairs_of_one_length(dev, dtype, tol, flags):
    """Tensors that share an FFT length run the adjoint in pairs (their
    upstream gradients share one transform): equal sizes, different orders
    with the same generating length (m=3, n=101 and m=4, n=76: d = 301), and
    an odd tensor out; every gradient against the oracle."""
    rng = np.random.default_rng(17)
    shapes = [(3, 101), (4, 76), (3, 101), (5, 40), (5, 40), (4, 76), (3, 300), (3, 300), (4, 300)]
    orders, dims, hs, xs = [], [], [], []
    for m, n in shapes:
        d = m * (n - 1) + 1
        orders.append(m)
        dims.append(n)
        hs.append(rng.standard_normal(d) / np.sqrt(d))
        x = rng.standard_normal(n)
        xs.append(x / np.linalg.norm(x))
    b = wl.pack_square(orders, dims, hs, xs)
    g = rng.standard_normal(b.y_len)
    gh, gx = grads(b, dtype, flags, g, dev, forward_first=bool(flags & hk.STORE_SPECTRA))
    for i in range(len(b)):
        m, n, h, x = b.tensor(i)
        d = len(h)
        rh, rx = ref_grads(b, g, i)
        eh = np.max(np.abs(gh[b.h_off[i]: b.h_off[i] + d] - rh)) / np.max(np.abs(rh))
        ex = np.max(np.abs(gx[b.x_off[i]: b.x_off[i] + n] - rx)) / np.max(np.abs(rx))
        assert eh <= tol and ex <= tol, (i, m, n, eh, ex)
