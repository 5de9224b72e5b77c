"""GPU parity of the persistent FP32 forward kernel (real square tensors with
one vector per tensor, y = H x^{m-1} and alpha = H x^m, Section 3) against
the FP64 oracle, through the C ABI.

The kernel runs every tensor whose generating length d fits one of its FFT
lengths (2^k and 3 * 2^k, 32..4096, and 5120); longer ones run on the
per-length launches in the same call.  Inputs use the benchmark's scaling (h ~ N(0, 1/d),
unit-norm x), at which the FP32 bound is 1e-5 relative in the infinity norm
for every order tested here.
"""

import numpy as np
import pytest

import oracle
from paper_1401_6238_gb300 import hankel as hk
from paper_1401_6238_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL32 = 1e-5
FAST_LENGTHS = [32, 48, 64, 96, 128, 192, 256, 384, 512, 768, 1024, 1536, 2048, 3072, 4096, 5120]


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    hk.load()
    return torch.device("cuda:0")


def scaled_tensors(shapes, seed):
    """Tensors (m, n) with h ~ N(0, 1/d) and unit-norm x, packed."""
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


def run(b, flags=hk.SAME_X, want_y=True, want_alpha=True, dev=None, calls=1):
    plan = hk.Plan(hk.batch_descs(b), hk.R32, flags)
    H = torch.tensor(b.h, dtype=torch.float32, device=dev)
    X = torch.tensor(b.x, dtype=torch.float32, device=dev)
    outs = []
    for _ in range(calls):
        Y = torch.full((b.y_len,), float("nan"), dtype=torch.float32, device=dev) if want_y else None
        A = torch.full((len(b),), float("nan"), dtype=torch.float32, device=dev) if want_alpha else None
        plan.txv(H, X, Y, A)
        torch.cuda.synchronize()
        outs.append((Y.cpu().numpy().astype(np.float64) if want_y else None,
                     A.cpu().numpy().astype(np.float64) if want_alpha else None))
    info = plan.info
    plan.close()
    return outs, info


def check(b, y, a, tol=TOL32):
    worst = 0.0
    for i in range(len(b)):
        m, n, h, x = b.tensor(i)
        ref = oracle.fast_y(h, [x] * (m - 1), [n] * m).real
        if y is not None:
            got = y[b.y_off[i]: b.y_off[i] + n]
            e = np.max(np.abs(got - ref)) / np.max(np.abs(ref))
            worst = max(worst, e)
            assert e <= tol, (i, m, n, e)
        if a is not None:
            a_ref = float(np.dot(x, ref))
            scale = np.max(np.abs(ref)) * np.sum(np.abs(x))
            assert abs(a[i] - a_ref) <= tol * scale, (i, m, n, a[i], a_ref)
    return worst


def shapes_for_length(L, orders):
    """(m, n) pairs whose generating length d = m (n - 1) + 1 lands on FFT
    length L: the smallest d above the previous length, the largest d <= L,
    and one in between, for each order m that reaches L."""
    i = FAST_LENGTHS.index(L)
    lo = FAST_LENGTHS[i - 1] if i > 0 else 0
    out = []
    for m in orders:
        ns = [n for n in range(1, L + 1) if lo < m * (n - 1) + 1 <= L]
        if ns:
            out += [(m, n) for n in sorted({ns[0], ns[len(ns) // 2], ns[-1]})]
    return out


@pytest.mark.parametrize("L", FAST_LENGTHS)
def test_every_length(dev, L):
    shapes = shapes_for_length(L, [2, 3, 4, 5])
    assert shapes
    b = scaled_tensors(shapes, seed=L)
    for i in range(len(b)):
        m, n, _, _ = b.tensor(i)
        assert m * (n - 1) + 1 <= L
    (y, a) = run(b, dev=dev)[0][0]
    worst = check(b, y, a)
    print("L=%d: %d tensors, worst rel err %.2e" % (L, len(b), worst))


@pytest.mark.parametrize("m", [6, 7, 8])
def test_high_orders(dev, m):
    # orders above the benchmark's, FFT lengths of both families
    shapes = [(m, n) for n in (3, 5, 9, 17, 64, 100, 200, 300, 400, 511)]
    b = scaled_tensors(shapes, seed=100 + m)
    (y, a) = run(b, dev=dev)[0][0]
    check(b, y, a)


def test_many_jobs_per_item(dev):
    # 131 tensors of FFT length 64 (64 pair jobs per item): two full items,
    # a partly filled third one and a tensor with no partner
    shapes = [(3, 16 + (i % 6)) for i in range(131)]
    b = scaled_tensors(shapes, seed=7)
    (y, a) = run(b, dev=dev)[0][0]
    check(b, y, a)


def test_fp64_spectrum_products(dev):
    b = wl.batched_square(count=40, seed=33, orders=(4, 5), n_lo=300, n_hi=1024)
    (y, a) = run(b, flags=hk.SAME_X | hk.FP64_POWER, dev=dev)[0][0]
    check(b, y, a)


def test_y_only_and_alpha_only(dev):
    b = wl.batched_square(count=33, seed=34, n_lo=16, n_hi=700)
    (y, a) = run(b, want_alpha=False, dev=dev)[0][0]
    assert a is None
    check(b, y, None)
    (y, a) = run(b, want_y=False, dev=dev)[0][0]
    assert y is None
    check(b, None, a)


def test_mixed_with_longer_lengths(dev):
    # generating lengths above 5120 run on the per-length launches of the
    # same call; both sets must be right, and the plan reports both launches
    shapes = [(5, 1000), (5, 1024), (4, 1300), (3, 2000), (5, 900), (3, 700), (4, 300), (3, 40), (2, 2561)]
    b = scaled_tensors(shapes, seed=9)
    (y, a), info = (lambda o: (o[0][0], o[1]))(run(b, dev=dev))
    assert info["launches"] > 1
    check(b, y, a)


def test_repeat_calls_identical(dev):
    # the work counter re-arms itself: repeated calls give the same bits
    b = wl.batched_square(count=300, seed=35, n_lo=16, n_hi=1024)
    outs, info = run(b, dev=dev, calls=3)
    for y, a in outs[1:]:
        np.testing.assert_array_equal(y, outs[0][0])
        np.testing.assert_array_equal(a, outs[0][1])
    check(b, outs[0][0], outs[0][1])


def test_benchmark_shapes_one_launch(dev):
    # the benchmark's shape mix (orders 3..5, n in [16, 1024], so d <= 5116):
    # a single persistent launch
    b = wl.batched_square(count=512, seed=36, orders=(3, 4, 5), n_lo=16, n_hi=1024)
    assert max(m * (n - 1) + 1 for m, n in zip(b.orders, b.dims)) > 4096  # the longest length is in it
    outs, info = run(b, dev=dev)
    assert info["launches"] == 1
    check(b, outs[0][0], outs[0][1])


def test_longest_length_items_share_the_slab(dev):
    # many tensors of FFT length 5120 (one job per block, the slab in global
    # memory): more jobs than resident blocks, so blocks reuse their slab
    shapes = [(5, 821 + (i * 37) % 204) for i in range(700)]
    b = scaled_tensors(shapes, seed=38)
    outs, info = run(b, dev=dev, calls=2)
    assert info["launches"] == 1
    np.testing.assert_array_equal(outs[0][0], outs[1][0])
    check(b, outs[0][0], outs[0][1])


def test_mixed_orders_same_length(dev):
    # tensors of one FFT length but different orders are never paired (the
    # kernel raises both spectra of a pair to one power): every order must
    # still come out right, including odd counts per (length, order)
    shapes = [(3, 600), (4, 450), (5, 360), (3, 610), (4, 455), (5, 365), (3, 620), (2, 900), (6, 300)]
    b = scaled_tensors(shapes, seed=37)
    (y, a) = run(b, dev=dev)[0][0]
    check(b, y, a)


def test_unaligned_offsets(dev):
    # h and x segments that do not start on 16 bytes: laid out one after
    # another with gaps, starts 1..3 elements past a 16-byte boundary
    b = scaled_tensors([(3, 600), (4, 300), (5, 1000), (3, 17), (2, 40), (5, 200), (4, 700)], seed=39)
    d = hk.batch_descs(b)
    hs, xs, ho, xo = [], [], 0, 0
    for i in range(len(b)):
        m, n, hi, xi = b.tensor(i)
        ho += 1 + i % 3
        xo += 3 - i % 3
        d["h_off"][i], d["x_off"][i, 0] = ho, xo
        hs.append((ho, hi))
        xs.append((xo, xi))
        ho = (ho + hi.size + 7) // 4 * 4
        xo = (xo + n + 7) // 4 * 4
    h, x = np.zeros(ho), np.zeros(xo)
    for o, v in hs:
        h[o: o + v.size] = v
    for o, v in xs:
        x[o: o + v.size] = v
    assert all(int(o) % 4 != 0 for o in d["h_off"]) and all(int(o) % 4 != 0 for o in d["x_off"][:, 0])
    plan = hk.Plan(d, hk.R32, hk.SAME_X)
    assert plan.info["launches"] == 1
    H = torch.tensor(h, dtype=torch.float32, device=dev)
    X = torch.tensor(x, dtype=torch.float32, device=dev)
    Y = torch.full((b.y_len,), float("nan"), dtype=torch.float32, device=dev)
    A = torch.full((len(b),), float("nan"), dtype=torch.float32, device=dev)
    plan.txv(H, X, Y, A)
    torch.cuda.synchronize()
    plan.close()
    check(b, Y.cpu().numpy().astype(np.float64), A.cpu().numpy().astype(np.float64))


@pytest.fixture
def bin_policy():
    """Sets per-bin planner choices for one test and puts the defaults back."""
    yield hk.hankel_set_bin_policy
    hk.hankel_set_bin_policy({})


def test_bin_policy_fp64_powers(dev, bin_policy):
    # orders >= 4 of the 1024 and 4096 bins form their powers in FP64, in the
    # same persistent launch as the FP32 ones; every result stays right
    shapes = [(3, 300), (4, 250), (5, 200), (4, 256), (3, 1300), (4, 1000), (5, 800), (5, 819), (6, 100), (2, 40)]
    b = scaled_tensors(shapes, seed=40)
    bin_policy({1024: (0, 4), 4096: (0, 4)})
    (y, a), info = (lambda o: (o[0][0], o[1]))(run(b, dev=dev))
    lens = [32, 48, 64, 96, 128, 192, 256, 384, 512, 768, 1024, 1536, 2048, 3072, 4096, 5120]
    bins = [next(L for L in lens if L >= m * (n - 1) + 1) for m, n in shapes]
    want = sum(1 for (m, n), L in zip(shapes, bins) if L in (1024, 4096) and m >= 4)
    assert want == 6 and info["fp64_power_tensors"] == want and info["launches"] == 1
    check(b, y, a)
    # the plan flag still forces every tensor
    (y, a), info = (lambda o: (o[0][0], o[1]))(run(b, flags=hk.SAME_X | hk.FP64_POWER, dev=dev))
    assert info["fp64_power_tensors"] == len(b)
    check(b, y, a)


def test_bin_policy_fp64_powers_in_shared_warps(dev, bin_policy):
    # FFT length 96 runs groups of 8 threads, four to a warp: tensors with
    # and without FP64 powers (and padding slots) share warps, which then
    # take one code path (FP64 for all when any group asks)
    shapes = [(3, 30), (4, 22), (5, 18), (2, 45), (3, 29), (4, 21), (5, 17)] * 3
    b = scaled_tensors(shapes, seed=42)
    bin_policy({96: (0, 4)})
    (y, a), info = (lambda o: (o[0][0], o[1]))(run(b, dev=dev))
    assert info["fp64_power_tensors"] == 12 and info["launches"] == 1
    check(b, y, a)
    (y, a), info = (lambda o: (o[0][0], o[1]))(run(b, flags=hk.SAME_X | hk.FP64_POWER, dev=dev))
    check(b, y, a)


def test_bin_policy_routes_a_bin_to_the_per_length_launches(dev, bin_policy):
    b = wl.batched_square(count=200, seed=41, n_lo=16, n_hi=1024)
    (y0, a0), info0 = (lambda o: (o[0][0], o[1]))(run(b, dev=dev))
    assert info0["launches"] == 1
    bin_policy({3072: (1, 99), 256: (1, 99)})
    (y1, a1), info1 = (lambda o: (o[0][0], o[1]))(run(b, dev=dev))
    assert info1["launches"] > 1
    check(b, y0, a0)
    check(b, y1, a1)


# ------------------------------------------------------------- the adjoint

def run_grads(b, g, dev, want_h=True, want_x=True, calls=1, flags=hk.SAME_X, fill=float("nan")):
    plan = hk.Plan(hk.batch_descs(b), hk.R32, flags)
    H = torch.tensor(b.h, dtype=torch.float32, device=dev)
    X = torch.tensor(b.x, dtype=torch.float32, device=dev)
    G = torch.tensor(g, dtype=torch.float32, device=dev)
    outs = []
    for _ in range(calls):
        gh = torch.full_like(H, fill) if want_h else None
        gx = torch.full_like(X, fill) if want_x else None
        plan.backward(G, H, X, gh, gx)
        torch.cuda.synchronize()
        outs.append((gh.cpu().numpy().astype(np.float64) if want_h else None,
                     gx.cpu().numpy().astype(np.float64) if want_x else None))
    plan.close()
    return outs


def check_grads(b, g, gh, gx, tol=TOL32):
    for i in range(len(b)):
        m, n, h, x = b.tensor(i)
        rh, rxs = oracle.fast_grads(h, [x] * (m - 1), [n] * m, g[b.y_off[i]: b.y_off[i] + n])
        if gh is not None:
            got = gh[b.h_off[i]: b.h_off[i] + h.size]
            e = np.max(np.abs(got - rh.real)) / np.max(np.abs(rh.real))
            assert e <= tol, ("grad_h", i, m, n, e)
        if gx is not None:
            ref = sum(r.real for r in rxs)
            e = np.max(np.abs(gx[b.x_off[i]: b.x_off[i] + n] - ref)) / np.max(np.abs(ref))
            assert e <= tol, ("grad_x", i, m, n, e)


def upstream(b, seed):
    return np.random.default_rng(seed).standard_normal(b.y_len)


@pytest.mark.parametrize("L", FAST_LENGTHS)
def test_adjoint_every_length(dev, L):
    shapes = shapes_for_length(L, [2, 3, 4, 5])
    b = scaled_tensors(shapes, seed=200 + L)
    g = upstream(b, L)
    (gh, gx), = run_grads(b, g, dev)
    check_grads(b, g, gh, gx)


def test_adjoint_high_orders_and_odd_counts(dev):
    # orders 6..8 and an odd number of tensors per length (a tensor without a
    # partner, padding slots in the warps of short lengths)
    shapes = [(6, 50), (7, 40), (8, 30), (6, 300), (7, 250), (8, 200), (3, 17), (4, 800)]
    b = scaled_tensors(shapes, seed=210)
    g = upstream(b, 11)
    (gh, gx), = run_grads(b, g, dev)
    check_grads(b, g, gh, gx)


def test_adjoint_one_gradient_at_a_time(dev):
    # one output only; the other buffer is not passed, and the gaps between
    # segments keep their fill
    b = wl.batched_square(count=65, seed=212, n_lo=16, n_hi=1024)
    g = upstream(b, 12)
    fill = -3.5
    (gh, _), = run_grads(b, g, dev, want_x=False, fill=fill)
    (_, gx), = run_grads(b, g, dev, want_h=False, fill=fill)
    check_grads(b, g, gh, None)
    check_grads(b, g, None, gx)
    covered = np.zeros(gh.size, bool)
    for i in range(len(b)):
        covered[b.h_off[i]: b.h_off[i] + b.orders[i] * (b.dims[i] - 1) + 1] = True
    assert np.all(gh[~covered] == fill)


def test_adjoint_mixed_with_longer_lengths_and_repeat(dev):
    # generating lengths above 5120 take the per-length adjoint in the same
    # call; repeated calls give the same bits (the counter re-arms)
    shapes = [(5, 1000), (4, 1300), (3, 2000), (3, 700), (4, 300), (3, 40), (2, 2561), (5, 1024)]
    b = scaled_tensors(shapes, seed=213)
    g = upstream(b, 13)
    outs = run_grads(b, g, dev, calls=3)
    for gh, gx in outs[1:]:
        np.testing.assert_array_equal(gh, outs[0][0])
        np.testing.assert_array_equal(gx, outs[0][1])
    check_grads(b, g, outs[0][0], outs[0][1])


def test_adjoint_benchmark_shapes(dev):
    b = wl.batched_square(count=400, seed=214, orders=(3, 4, 5), n_lo=16, n_hi=1024)
    plan = hk.Plan(hk.batch_descs(b), hk.R32, hk.SAME_X)
    assert plan.info["backward_launches"] == 1  # the persistent adjoint alone
    plan.close()
    g = upstream(b, 14)
    (gh, gx), = run_grads(b, g, dev)
    check_grads(b, g, gh, gx)
