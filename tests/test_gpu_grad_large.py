"""The gradient workload at full size: order m = 4, n = 4096 (d = 16381,
L = 16384, beyond shared memory, so the transforms run through global
scratch), batch 64, loss ||H(h) x^{m-1} - t||^2 through the
torch.autograd.Function.  FP32 gradients are compared with the oracle's
analytic gradient on a sub-batch; FP64 gradients with FP64 central finite
differences (step 1e-6) on sampled coordinates."""

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


@pytest.fixture(scope="module")
def batch():
    return wl.grad_case(batch=64, m=4, n=4096, seed=3)


def rel(a, b):
    return np.max(np.abs(a - b)) / np.max(np.abs(b))


@pytest.mark.parametrize("flags", [hk.SAME_X | hk.STORE_SPECTRA, hk.SAME_X])
def test_fp32_gradients_match_oracle(dev, batch, flags):
    plan = hk.Plan(hk.batch_descs(batch), hk.R32, flags)
    assert plan.info["max_length"] == 16384
    H = torch.tensor(batch.h, dtype=torch.float32, device=dev, requires_grad=True)
    X = torch.tensor(batch.x, dtype=torch.float32, device=dev, requires_grad=True)
    ny = plan.info["y_elems"]
    t = torch.tensor(batch.extra["target"][:ny], dtype=torch.float32, device=dev)
    y = hk.hankel_txv_autograd(H, X, plan)
    loss = ((y - t) ** 2).sum()
    loss.backward()
    torch.cuda.synchronize()
    yv, gh, gx, tv = y.detach().cpu().numpy(), H.grad.cpu().numpy(), X.grad.cpu().numpy(), t.cpu().numpy()
    for i in (0, 17, 40, 63):
        m, n, h, x = batch.tensor(i)
        yr = oracle.fast_y(h, [x] * (m - 1), [n] * m).real
        o = batch.y_off[i]
        assert rel(yv[o:o + n], yr) <= 1e-5, ("y", i)
        g = 2.0 * (yr - tv[o:o + n])
        rh, rxs = oracle.fast_grads(h, [x] * (m - 1), [n] * m, g)
        rx = sum(v.real for v in rxs)
        eh = rel(gh[batch.h_off[i]: batch.h_off[i] + len(h)], rh.real)
        ex = rel(gx[batch.x_off[i]: batch.x_off[i] + n], rx)
        assert eh <= 1e-5, ("grad_h", i, eh)
        assert ex <= 1e-5, ("grad_x", i, ex)
    plan.close()


def test_fp64_gradients_match_finite_differences(dev, batch):
    sub = batch.subset([5, 6])
    plan = hk.Plan(hk.batch_descs(sub), hk.R64, hk.SAME_X)
    ny = plan.info["y_elems"]
    H = torch.tensor(sub.h, device=dev, requires_grad=True)
    X = torch.tensor(sub.x, device=dev, requires_grad=True)
    t = torch.tensor(np.random.default_rng(9).standard_normal(ny) * 0.01, device=dev)
    loss = ((hk.hankel_txv_autograd(H, X, plan) - t) ** 2).sum()
    loss.backward()

    def f(hv, xv):
        y = torch.zeros(ny, dtype=torch.float64, device=dev)
        plan.txv(hv, xv, y)
        return float(((y - t) ** 2).sum())

    eps = 1e-6
    rng = np.random.default_rng(10)
    for vec, grad, which in [(H, H.grad, "h"), (X, X.grad, "x")]:
        base = vec.detach().clone()
        for j in rng.choice(base.numel(), size=6, replace=False):
            p, m_ = base.clone(), base.clone()
            p[j] += eps
            m_[j] -= eps
            fd = (f(p, X.detach()) - f(m_, X.detach())) / (2 * eps) if which == "h" else \
                 (f(H.detach(), p) - f(H.detach(), m_)) / (2 * eps)
            assert abs(fd - grad[j].item()) <= 1e-6 * max(1.0, abs(fd)) + 1e-9, (which, j, fd, grad[j].item())
    plan.close()
