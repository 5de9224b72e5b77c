"""hankel_txv_backward_static: the allocation-free gradient entry point.

It serves callers that cannot call cudaMalloc -- device memory owned by
another allocator, latency-critical loops where cudaMalloc/cudaFree would
synchronise the device, deployments whose device footprint is fixed after
start-up: its scratch is a static device array shared by all calls.

Checked through the C ABI against the FP64 oracle's analytic gradients
(tensor by tensor) and against the plan-based hankel_txv_backward on the same
inputs, on two calls in a row (the second with a different batch, so stale
scratch from the first call would show), in FP32 and FP64, at the bounds the
other parity tests use (inputs scaled as the benchmark's: h ~ N(0, 1/d),
unit-norm x).  Also: order 2, one output at a time with the gaps between
tensors left untouched, the longest FFT length the call accepts, and the
rejections (shared storage, scratch beyond the array).  This file is
collected last on purpose.
"""

import numpy as np
import pytest

import oracle
from paper_1401_6238_gb300 import hankel as hk
from paper_1401_6238_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {hk.R32: 1e-5, hk.R64: 1e-12}
SMEM = 227 * 1024
RED = 512


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    hk.load()
    return torch.device("cuda:0")


def tdtype(dtype):
    return torch.float32 if dtype == hk.R32 else torch.float64


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


def inputs(b, seed, dtype, dev):
    g = np.random.default_rng(seed + 100).standard_normal(b.y_len)
    t = lambda a: torch.tensor(a, dtype=tdtype(dtype), device=dev)
    return t(b.h), t(b.x), t(g), g


def static_grads(b, dtype, H, X, G, want_h=True, want_x=True, fill=0.0):
    gh = torch.full_like(H, fill) if want_h else None
    gx = torch.full_like(X, fill) if want_x else None
    hk.hankel_txv_backward_static(hk.batch_descs(b), dtype, G, H, X, gh, gx)
    torch.cuda.synchronize()
    return (gh.cpu().numpy() if want_h else None), (gx.cpu().numpy() if want_x else None)


def plan_grads(b, dtype, H, X, G):
    plan = hk.Plan(hk.batch_descs(b), dtype, hk.SAME_X)
    gh, gx = torch.zeros_like(H), torch.zeros_like(X)
    plan.backward(G, H, X, gh, gx)
    torch.cuda.synchronize()
    plan.close()
    return gh.cpu().numpy(), gx.cpu().numpy()


def rel(got, ref):
    return np.max(np.abs(got - ref)) / np.max(np.abs(ref))


def check_oracle(b, g, gh, gx, tol):
    """Per tensor: grad_h and grad_x (summed over the modes sharing x) against oracle.fast_grads."""
    for i in range(len(b)):
        m, n, h, x = b.tensor(i)
        rh, rxs = oracle.fast_grads(h, [x] * (m - 1), [n] * m, g[b.y_off[i]: b.y_off[i] + n])
        d = h.size
        if gh is not None:
            e = rel(gh[b.h_off[i]: b.h_off[i] + d], rh.real)
            assert e <= tol, ("grad_h", i, m, n, e)
        if gx is not None:
            e = rel(gx[b.x_off[i]: b.x_off[i] + n], sum(r.real for r in rxs))
            assert e <= tol, ("grad_x", i, m, n, e)


def gaps_untouched(buf, offs, lens, fill):
    covered = np.zeros(buf.size, dtype=bool)
    for o, n in zip(offs, lens):
        covered[o: o + n] = True
    return np.all(buf[~covered] == fill)


@pytest.mark.parametrize("dtype", [hk.R32, hk.R64])
def test_static_backward_matches_oracle_and_plan_twice(dev, dtype):
    for call, (seed, count, lo, hi) in enumerate([(5, 24, 16, 700), (6, 17, 300, 1024)]):
        b = wl.batched_square(count=count, seed=seed, n_lo=lo, n_hi=hi)
        H, X, G, g = inputs(b, seed, dtype, dev)
        sh, sx = static_grads(b, dtype, H, X, G)
        check_oracle(b, g, sh, sx, TOL[dtype])
        rh, rx = plan_grads(b, dtype, H, X, G)
        assert rel(sh, rh) <= TOL[dtype], ("grad_h vs plan", call)
        assert rel(sx, rx) <= TOL[dtype], ("grad_x vs plan", call)


@pytest.mark.parametrize("dtype", [hk.R32, hk.R64])
def test_static_backward_one_output_at_a_time_order_two(dev, dtype):
    shapes = [(2, 9), (2, 200), (3, 40), (2, 1000), (4, 77)]
    b = scaled(shapes, seed=8)
    H, X, G, g = inputs(b, 8, dtype, dev)
    fill = -7.25
    gh, _ = static_grads(b, dtype, H, X, G, want_x=False, fill=fill)
    _, gx = static_grads(b, dtype, H, X, G, want_h=False, fill=fill)
    check_oracle(b, g, gh, None, TOL[dtype])
    check_oracle(b, g, None, gx, TOL[dtype])
    # the padding between segments (16-byte alignment) keeps the fill value
    dl = [m * (n - 1) + 1 for m, n in shapes]
    assert gaps_untouched(gh, b.h_off, dl, fill)
    assert gaps_untouched(gx, b.x_off, [n for _, n in shapes], fill)


def longest_length(dtype):
    """The longest FFT length the entry point accepts: two padded buffers of
    complex values (one pad slot per 16) in one block's shared memory."""
    cs = 8 if dtype == hk.R32 else 16
    L = 2
    while L < 16384 and RED + 2 * ((L + 1) + (L + 1) // 16 + 1) * cs <= SMEM:
        L += 1
    return L


@pytest.mark.parametrize("dtype", [hk.R32, hk.R64])
def test_static_backward_at_the_longest_length(dev, dtype):
    maxL = longest_length(dtype)
    # the longest generating length of order 3 whose planner length fits
    n = (maxL + 2) // 3
    while hk.hankel_fft_length(3 * (n - 1) + 1) > maxL:
        n -= 1
    assert hk.hankel_fft_length(3 * (n - 1) + 1) <= maxL
    # with it, shorter tensors in the same launch (up to 32 jobs per launch)
    shapes = [(3, n), (3, n - 5), (2, 700), (4, 300), (3, 17)]
    b = scaled(shapes, seed=9)
    H, X, G, g = inputs(b, 9, dtype, dev)
    sh, sx = static_grads(b, dtype, H, X, G)
    check_oracle(b, g, sh, sx, TOL[dtype])


def test_static_backward_rejects_shared_storage(dev):
    b = scaled([(3, 50), (3, 50)], seed=10)
    H, X, G, _ = inputs(b, 10, hk.R32, dev)
    descs = hk.batch_descs(b)
    descs["x_off"][1, 0] = descs["x_off"][0, 0]  # both tensors use one vector
    with pytest.raises(hk.HankelError) as e:
        hk.hankel_txv_backward_static(descs, hk.R32, G, H, X, torch.zeros_like(H), torch.zeros_like(X))
    assert e.value.status == hk.EINVAL and "share x storage" in e.value.message


def test_static_backward_rejects_batches_beyond_the_array(dev):
    # 300 tensors of L = 8192 need 300 * 8192 * 8 B = 19.7 MB of spectra in
    # FP32, more than the 16 MiB array
    b = wl.batched_square(count=4, seed=7, n_lo=16, n_hi=32)
    H, X, G, _ = inputs(b, 7, hk.R32, dev)
    descs = hk.square_descs([2] * 300, [4096] * 300, np.arange(300) * 8192, np.arange(300) * 4096, [0] * 300)
    with pytest.raises(hk.HankelError) as e:
        hk.hankel_txv_backward_static(descs, hk.R32, G, H, X, torch.zeros_like(H), None)
    assert e.value.status == hk.EINVAL and "bytes of scratch" in e.value.message
