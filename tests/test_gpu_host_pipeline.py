"""hankel_txv_host on large batches runs as a pipeline of descriptor ranges
(copies in and out overlap the kernels of other ranges).  Its results must
match the device entry point, also when descriptors are stored out of order
(their ranges then overlap) and for the distinct-vector and complex paths."""

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


def per_tensor_close(a, b, offs, lens, tol):
    for o, n in zip(offs, lens):
        ref = b[o:o + n]
        assert np.abs(a[o:o + n] - ref).max() <= tol * max(np.abs(ref).max(), 1e-30)


def test_full_batch_host_matches_device(dev):
    b = wl.batched_square(count=8192, seed=1)
    plan = hk.Plan(hk.batch_descs(b), hk.R32, hk.SAME_X)
    hh = torch.tensor(b.h, dtype=torch.float32).pin_memory()
    xh = torch.tensor(b.x, dtype=torch.float32).pin_memory()
    yh = torch.zeros(b.y_len, dtype=torch.float32).pin_memory()
    ah = torch.zeros(len(b), dtype=torch.float32).pin_memory()
    plan.txv_host(hh, xh, yh, ah)
    Y = torch.zeros(b.y_len, dtype=torch.float32, device=dev)
    A = torch.zeros(len(b), dtype=torch.float32, device=dev)
    plan.txv(hh.to(dev), xh.to(dev), Y, A)
    torch.cuda.synchronize()
    per_tensor_close(yh.numpy(), Y.cpu().numpy(), b.y_off, b.dims, 1e-5)
    assert np.abs(ah.numpy() - A.cpu().numpy()).max() <= 1e-5 * np.abs(A.cpu().numpy()).max()
    # again: other buffers (an eager run), then the same buffers twice (the
    # pipeline replays as a captured graph) with fresh inputs in place
    # (zeros_like is not page-locked: these calls stage through copies, with
    # other job pairings, so they agree to rounding, not bit for bit)
    yh2 = torch.zeros_like(yh)
    plan.txv_host(hh, xh, yh2, None)
    per_tensor_close(yh2.numpy(), yh.numpy(), b.y_off, b.dims, 1e-5)
    # alpha alone
    ah2 = torch.zeros_like(ah)
    plan.txv_host(hh, xh, None, ah2)
    assert np.abs(ah2.numpy() - ah.numpy()).max() <= 1e-5 * np.abs(ah.numpy()).max()
    for scale in (2.0, 0.5):
        hh.mul_(scale)
        yh.zero_()
        ah.zero_()
        plan.txv_host(hh, xh, yh, ah)
        plan.txv(hh.to(dev), xh.to(dev), Y, A)
        torch.cuda.synchronize()
        per_tensor_close(yh.numpy(), Y.cpu().numpy(), b.y_off, b.dims, 1e-5)
        assert np.abs(ah.numpy() - A.cpu().numpy()).max() <= 1e-5 * np.abs(A.cpu().numpy()).max()
    plan.close()


def test_out_of_order_descriptors(dev):
    # 1024 tensors whose descriptors list the stored tensors in a random
    # order: every range of descriptors spans most of the buffers
    rng = np.random.default_rng(5)
    count, m, n = 1024, 3, 1024
    d = 3 * n - 2
    perm = rng.permutation(count)
    h = (rng.standard_normal(count * d) / np.sqrt(d)).astype(np.float32)
    x = (rng.standard_normal(count * n) / np.sqrt(n)).astype(np.float32)
    descs = hk.square_descs([m] * count, [n] * count, perm * d, perm * n, perm * n)
    plan = hk.Plan(descs, hk.R32, hk.SAME_X)
    hh, xh = torch.from_numpy(h).pin_memory(), torch.from_numpy(x).pin_memory()
    yh = torch.zeros(count * n, dtype=torch.float32).pin_memory()
    plan.txv_host(hh, xh, yh, None)
    Y = torch.zeros(count * n, dtype=torch.float32, device=dev)
    plan.txv(hh.to(dev), xh.to(dev), Y)
    torch.cuda.synchronize()
    per_tensor_close(yh.numpy(), Y.cpu().numpy(), perm * n, [n] * count, 1e-5)
    for i in (0, 511, 1023):
        t = perm[i]
        ref = oracle.fast_y(h[t * d:(t + 1) * d].astype(float), [x[t * n:(t + 1) * n].astype(float)] * 2, [n] * 3).real
        assert np.abs(yh.numpy()[t * n:(t + 1) * n] - ref).max() <= 1e-5 * np.abs(ref).max()
    plan.close()


def test_distinct_vectors_host_pipeline(dev):
    bd, xoffs = wl.batched_distinct(2048, seed=3)
    dd = hk.make_descs(len(bd))
    dd["m"] = bd.orders
    for p in range(hk.MAX_ORDER):
        dd["n"][:, p] = np.where(p < bd.orders, bd.dims, 0)
    dd["h_off"] = bd.h_off
    for i, offs in enumerate(xoffs):
        dd["x_off"][i, :len(offs)] = offs
    dd["y_off"] = bd.y_off
    plan = hk.Plan(dd, hk.R32, 0)
    hh = torch.tensor(bd.h, dtype=torch.float32).pin_memory()
    xh = torch.tensor(bd.x, dtype=torch.float32).pin_memory()
    yh = torch.zeros(bd.y_len, dtype=torch.float32).pin_memory()
    ah = torch.zeros(len(bd), dtype=torch.float32).pin_memory()
    plan.txv_host(hh, xh, yh, ah)
    Y = torch.zeros(bd.y_len, dtype=torch.float32, device=dev)
    A = torch.zeros(len(bd), dtype=torch.float32, device=dev)
    plan.txv(hh.to(dev), xh.to(dev), Y, A)
    torch.cuda.synchronize()
    per_tensor_close(yh.numpy(), Y.cpu().numpy(), bd.y_off, bd.dims, 1e-5)
    assert np.abs(ah.numpy() - A.cpu().numpy()).max() <= 1e-5 * np.abs(A.cpu().numpy()).max()
    plan.close()
