"""hankel_txv_backward_static: the allocation-free gradient entry point.

It serves callers that cannot call cudaMalloc (device memory owned by another
allocator, latency-critical loops, fixed device footprints): its scratch is a
static device array shared by all calls.  Checked through the C ABI against
the plan-based hankel_txv_backward on the same inputs, on two calls in a row
(the second with a different batch, so stale scratch from the first call
would show), in FP32 and FP64.  This file is collected last on purpose.
"""

import numpy as np
import pytest

from paper_1401_6238_gb300 import hankel as hk
from paper_1401_6238_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {hk.R32: 2e-5, hk.R64: 1e-11}


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    hk.load()
    return torch.device("cuda:0")


def inputs(seed, dtype, dev, count, lo, hi):
    tdt = torch.float32 if dtype == hk.R32 else torch.float64
    b = wl.batched_square(count=count, seed=seed, n_lo=lo, n_hi=hi)
    g = np.random.default_rng(seed + 100).standard_normal(b.y_len)
    t = lambda a: torch.tensor(a, dtype=tdt, device=dev)
    return b, t(b.h), t(b.x), t(g)


def plan_grads(b, dtype, H, X, G):
    plan = hk.Plan(hk.batch_descs(b), dtype, hk.SAME_X)
    gh, gx = torch.zeros_like(H), torch.zeros_like(X)
    plan.backward(G, H, X, gh, gx)
    torch.cuda.synchronize()
    plan.close()
    return gh.cpu().numpy(), gx.cpu().numpy()


def static_grads(b, dtype, H, X, G):
    gh, gx = torch.zeros_like(H), torch.zeros_like(X)
    hk.hankel_txv_backward_static(hk.batch_descs(b), dtype, G, H, X, gh, gx)
    torch.cuda.synchronize()
    return gh.cpu().numpy(), gx.cpu().numpy()


def close(got, ref, tol):
    return np.max(np.abs(got - ref)) <= tol * np.max(np.abs(ref))


@pytest.mark.parametrize("dtype", [hk.R32, hk.R64])
def test_static_backward_matches_plan_backward_twice(dev, dtype):
    for call, (seed, count, lo, hi) in enumerate([(5, 24, 16, 700), (6, 17, 300, 1024)]):
        b, H, X, G = inputs(seed, dtype, dev, count, lo, hi)
        rh, rx = plan_grads(b, dtype, H, X, G)
        sh, sx = static_grads(b, dtype, H, X, G)
        assert close(sh, rh, TOL[dtype]), ("grad_h", call)
        assert close(sx, rx, TOL[dtype]), ("grad_x", call)


def test_static_backward_rejects_batches_beyond_the_array(dev):
    # 64 tensors of L = 8192 need 64 * 8192 * 8 B = 4 MiB of spectra in FP32,
    # 8 MiB in FP64; 300 of them exceed the 16 MiB array
    b, H, X, G = inputs(7, hk.R32, dev, 4, 16, 32)
    descs = hk.square_descs([2] * 300, [4096] * 300, [0] * 300, [0] * 300, [0] * 300)
    with pytest.raises(hk.HankelError) as e:
        hk.hankel_txv_backward_static(descs, hk.R32, G, H, X, torch.zeros_like(H), None)
    assert e.value.status == hk.EINVAL and "bytes of scratch" in e.value.message
