"""GPU parity of the real, one-vector-per-tensor path (y = H x^{m-1},
alpha = H x^m) against the FP64 oracle, through the C ABI.

Tolerances: relative infinity-norm error of y, ||y_gpu - y_ref||_inf /
||y_ref||_inf <= 1e-5 for FP32 with m <= 4 (m = 5 is held to the same bound);
1e-12 for FP64.  Integer inputs in FP64 must round to the exact product.
"""

import numpy as np
import pytest

import oracle
from paper_1401_6238_gb300 import hankel as hk
from paper_1401_6238_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL32 = 1e-5
TOL64 = 1e-12


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    hk.load()
    return torch.device("cuda:0")


def run(batch, dtype, flags=hk.SAME_X, want_y=True, want_alpha=False, dev=None):
    tdt = torch.float32 if dtype == hk.R32 else torch.float64
    plan = hk.Plan(hk.batch_descs(batch), dtype, flags)
    H = torch.tensor(batch.h, dtype=tdt, device=dev)
    X = torch.tensor(batch.x, dtype=tdt, device=dev)
    Y = torch.zeros(batch.y_len, dtype=tdt, device=dev) if want_y else None
    A = torch.zeros(len(batch), dtype=tdt, device=dev) if want_alpha else None
    plan.txv(H, X, Y, A)
    torch.cuda.synchronize()
    out = (Y.cpu().numpy().astype(np.float64) if want_y else None,
           A.cpu().numpy().astype(np.float64) if want_alpha else None)
    info = plan.info
    plan.close()
    return out, info


def rel_err(got, ref):
    return np.max(np.abs(got - ref)) / np.max(np.abs(ref))


def check_batch(batch, y, alpha, tol, idx=None):
    worst = 0.0
    for i in (range(len(batch)) if idx is None else idx):
        m, n, h, x = batch.tensor(i)
        ref = oracle.fast_y(h, [x] * (m - 1), [n] * m).real
        if y is not None:
            e = rel_err(y[batch.y_off[i]: batch.y_off[i] + n], ref)
            worst = max(worst, e)
            assert e <= tol, (i, m, n, e)
        if alpha is not None:
            a_ref = float(np.dot(x, ref))
            scale = np.max(np.abs(ref)) * np.sum(np.abs(x))
            assert abs(alpha[i] - a_ref) <= tol * scale, (i, alpha[i], a_ref)
    return worst


def test_plain_fp64_against_brute_force(dev):
    dims, h, x = wl.plain_case(seed=0)
    b = wl.pack_square([3], [64], [h], [x])
    (y, a), info = run(b, hk.R64, want_alpha=True, dev=dev)
    ref = oracle.brute_y(h, [x, x], dims)
    assert rel_err(y[:64], ref) <= TOL64
    assert abs(a[0] - np.dot(x, ref)) <= TOL64 * abs(np.dot(x, ref))
    assert info["count"] == 1


def test_vandermonde_fp64_closed_form(dev):
    m, n, a = 3, 64, 0.97
    d = m * (n - 1) + 1
    h = wl.vandermonde_h(a, d)
    x = np.random.default_rng(2).standard_normal(n)
    b = wl.pack_square([m], [n], [h], [x])
    (y, al), _ = run(b, hk.R64, want_alpha=True, dev=dev)
    s = np.sum(a ** np.arange(n) * x)
    ref = s ** (m - 1) * a ** np.arange(n)
    assert rel_err(y[:n], ref) <= TOL64
    assert abs(al[0] - s ** m) <= TOL64 * abs(s ** m), (al[0], s ** m)


@pytest.mark.parametrize("flags", [hk.SAME_X, hk.SAME_X | hk.ONE_PER_LAUNCH])
def test_small_integers_fp64_bit_exact(dev, flags):
    orders, dims, hs, xs = [], [], [], []
    for k, (m, n) in enumerate([(3, 5), (4, 4), (5, 3), (3, 17), (2, 9), (4, 11)]):
        h, xv = wl.integer_case([n] * m, seed=k)
        orders.append(m)
        dims.append(n)
        hs.append(h)
        xs.append(xv[0])
    b = wl.pack_square(orders, dims, hs, xs)
    (y, a), _ = run(b, hk.R64, flags=flags, want_alpha=True, dev=dev)
    for i in range(len(b)):
        m, n, h, x = b.tensor(i)
        exact = oracle.loop_y(h, [x] * (m - 1), [n] * m)
        np.testing.assert_array_equal(np.rint(y[b.y_off[i]: b.y_off[i] + n]), exact)
        assert np.rint(a[i]) == np.dot(x, exact)


@pytest.mark.parametrize("seed,count,lo,hi", [(21, 96, 16, 300), (22, 64, 280, 1024), (23, 7, 1000, 1024)])
def test_batched_fp32_parity(dev, seed, count, lo, hi):
    b = wl.batched_square(count=count, seed=seed, n_lo=lo, n_hi=hi)
    (y, a), info = run(b, hk.R32, want_alpha=True, dev=dev)
    worst = check_batch(b, y, a, TOL32)
    assert info["jobs"] <= count
    print("worst rel err %.2e over %d tensors" % (worst, count))


def test_fp32_fp64_power_flag(dev):
    b = wl.batched_square(count=24, seed=31, orders=(5,), n_lo=500, n_hi=1024)
    (y, _), _ = run(b, hk.R32, flags=hk.SAME_X | hk.FP64_POWER, dev=dev)
    check_batch(b, y, None, TOL32)


def test_fp64_batched_and_one_per_launch(dev):
    b = wl.batched_square(count=20, seed=41, n_lo=16, n_hi=1024)
    (y1, a1), _ = run(b, hk.R64, want_alpha=True, dev=dev)
    (y2, a2), info = run(b, hk.R64, flags=hk.SAME_X | hk.ONE_PER_LAUNCH, want_alpha=True, dev=dev)
    check_batch(b, y1, a1, TOL64)
    check_batch(b, y2, a2, TOL64)
    assert info["launches"] == len(b)


@pytest.mark.parametrize("case", [
    ([2], [1]),               # d = 1: the smallest transform
    ([2, 3, 2], [1, 2, 1]),   # tiny orders / sizes
    ([8], [3]),               # highest order the ABI allows
    ([3, 3, 3], [16, 17, 16]),  # a ragged pair partner and a leftover single
    ([2], [2048]),            # m = 2: a Hankel matrix-vector product
])
def test_edge_cases(dev, case):
    orders, dims = case
    rng = np.random.default_rng(sum(dims))
    hs = [rng.standard_normal(m * (n - 1) + 1) / np.sqrt(m * (n - 1) + 1) for m, n in zip(orders, dims)]
    xs = [v / np.linalg.norm(v) for v in (rng.standard_normal(n) for n in dims)]
    b = wl.pack_square(orders, dims, hs, xs)
    for dtype, tol in [(hk.R32, TOL32), (hk.R64, TOL64)]:
        (y, a), _ = run(b, dtype, want_alpha=True, dev=dev)
        check_batch(b, y, a, tol)


def test_longest_single_transform_fp32(dev):
    # L = 8192 single tensor, and a pair at L = 8192
    rng = np.random.default_rng(5)
    orders, dims = [2, 2, 3], [4096, 4096, 2731]
    hs = [rng.standard_normal(m * (n - 1) + 1) / 64 for m, n in zip(orders, dims)]
    xs = [rng.standard_normal(n) / 64 for n in dims]
    b = wl.pack_square(orders, dims, hs, xs)
    (y, a), _ = run(b, hk.R32, want_alpha=True, dev=dev)
    check_batch(b, y, a, TOL32)


def test_alpha_only_skips_y(dev):
    b = wl.batched_square(count=10, seed=51, n_lo=16, n_hi=600)
    (y, a), _ = run(b, hk.R32, want_y=False, want_alpha=True, dev=dev)
    assert y is None
    check_batch(b, None, a, TOL32)


def test_host_buffers_entry_point(dev):
    b = wl.batched_square(count=12, seed=61, n_lo=16, n_hi=500)
    plan = hk.Plan(hk.batch_descs(b), hk.R32, hk.SAME_X)
    h = torch.tensor(b.h, dtype=torch.float32).pin_memory()
    x = torch.tensor(b.x, dtype=torch.float32).pin_memory()
    y = torch.zeros(b.y_len, dtype=torch.float32).pin_memory()
    a = torch.zeros(len(b), dtype=torch.float32).pin_memory()
    plan.txv_host(h, x, y, a)
    check_batch(b, y.numpy().astype(np.float64), a.numpy().astype(np.float64), TOL32)
    plan.close()


def test_full_size_batch_every_tensor(dev):
    # the 8192-tensor workload in the launch configuration the benchmark
    # times, every output checked against the oracle (in a process pool)
    from oracle import pool
    b = wl.batched_square(count=8192, seed=1)
    (y, _), info = run(b, hk.R32, dev=dev)
    refs = pool.square_refs(b.tensor(i) for i in range(len(b)))
    err = pool.relative_errors(b, y, refs)
    print("8192 tensors: max rel err %.2e, median %.2e" % (err.max(), np.median(err)))
    assert err.max() <= TOL32, (int(np.argmax(err)), err.max())
    assert info["count"] == 8192
