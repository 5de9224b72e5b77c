"""Anti-circulant tensor-vector products (Section 2.1, Theorem 2.1, the
procedures opening Section 3) on the GPU: FFTs of length exactly n, no
padding.  References take the other road: the anti-circulant tensor is the
Hankel tensor of the periodic generating vector h_k = c[k mod n], whose
products the oracle computes by zero-padded embedding at a power-of-two
length (and, for the block case, the level-2 oracle on the periodic
generating matrix).  Also Corollary 2.2's eigenpairs, the adjoint, and
block anti-circulant (BAAB) tensors."""

import numpy as np
import pytest

import oracle
from oracle import level as lv
from paper_1401_6238_gb300 import hankel as hk

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TDT = {hk.R32: torch.float32, hk.C64: torch.complex64, hk.R64: torch.float64, hk.C128: torch.complex128}


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    hk.load()
    return torch.device("cuda:0")


def t_(a, dtype, dev):
    return torch.tensor(np.ascontiguousarray(a), dtype=TDT[dtype], device=dev)


def rel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


def periodic(c, m):
    return oracle.anticirculant_generating_vector(np.asarray(c), m)


@pytest.mark.parametrize("dtype,tol", [(hk.R64, 1e-12), (hk.R32, 1e-5)])
def test_real_same_x(dev, dtype, tol):
    rng = np.random.default_rng(1)
    cases = [(2, 64), (3, 60), (4, 210), (3, 2048), (5, 7), (3, 60)]
    cs = [rng.standard_normal(n) for m, n in cases]
    xs = [rng.standard_normal(n) for m, n in cases]
    ho = np.cumsum([0] + [n for m, n in cases])[:-1]
    d = hk.square_descs([m for m, n in cases], [n for m, n in cases], ho, ho, ho)
    plan = hk.Plan(d, dtype, hk.SAME_X | hk.ANTICIRCULANT)
    H, X = t_(np.concatenate(cs), dtype, dev), t_(np.concatenate(xs), dtype, dev)
    Y = torch.zeros(int(ho[-1] + cases[-1][1]), dtype=TDT[dtype], device=dev)
    A = torch.zeros(len(cases), dtype=TDT[dtype], device=dev)
    plan.txv(H, X, Y, A)
    torch.cuda.synchronize()
    y, a = Y.cpu().numpy(), A.cpu().numpy()
    for i, (m, n) in enumerate(cases):
        ref = oracle.fast_y(periodic(cs[i], m), [xs[i]] * (m - 1), [n] * m).real
        assert rel(y[ho[i]: ho[i] + n], ref) <= tol, (m, n)
        ar = oracle.fast_alpha(periodic(cs[i], m), [xs[i]] * m, [n] * m).real
        assert abs(a[i] - ar) <= tol * np.abs(ref).max() * np.abs(xs[i]).sum(), (m, n)
    plan.close()


@pytest.mark.parametrize("dtype,tol", [(hk.C128, 1e-12), (hk.C64, 1e-5)])
def test_complex_distinct_vectors(dev, dtype, tol):
    rng = np.random.default_rng(2)
    cr = lambda n: rng.standard_normal(n) + 1j * rng.standard_normal(n)
    cases = [(3, 48), (4, 30), (2, 96)]
    hs, xs, d = [], [], hk.make_descs(len(cases))
    xo = yo = ho = 0
    for i, (m, n) in enumerate(cases):
        c = cr(n)
        vs = [cr(n) for _ in range(m)]
        d[i]["m"] = m
        d[i]["n"][:m] = n
        d[i]["h_off"] = ho
        for p in range(m):
            d[i]["x_off"][p] = xo
            xo += n
        d[i]["y_off"] = yo
        ho += n
        yo += n
        hs.append(c)
        xs.append(vs)
    plan = hk.Plan(d, dtype, hk.ANTICIRCULANT)
    Y = torch.zeros(yo, dtype=TDT[dtype], device=dev)
    A = torch.zeros(len(cases), dtype=TDT[dtype], device=dev)
    plan.txv(t_(np.concatenate(hs), dtype, dev), t_(np.concatenate([v for vs in xs for v in vs]), dtype, dev), Y, A)
    torch.cuda.synchronize()
    y, a = Y.cpu().numpy(), A.cpu().numpy()
    for i, (m, n) in enumerate(cases):
        ref = oracle.fast_y(periodic(hs[i], m), xs[i][1:], [n] * m)
        assert rel(y[d[i]["y_off"]: d[i]["y_off"] + n], ref) <= tol, (m, n)
        ar = oracle.fast_alpha(periodic(hs[i], m), xs[i], [n] * m)
        assert abs(a[i] - ar) <= tol * np.abs(ref).max() * np.abs(xs[i][0]).sum(), (m, n)
    plan.close()


@pytest.mark.parametrize("m", [3, 4])
def test_corollary_2_2_eigenpairs(dev, m):
    # C 1^{m-1} = n^{m-2} (1^T c) 1, and for even n C 1~^{m-1} = n^{m-2} (1~^T c) 1~
    n = 60
    rng = np.random.default_rng(3)
    c = rng.standard_normal(n)
    one, alt = np.ones(n), (-1.0) ** np.arange(n)
    d = hk.square_descs([m, m], [n, n], [0, 0], [0, n], [0, n])
    plan = hk.Plan(d, hk.R64, hk.SAME_X | hk.ANTICIRCULANT)
    Y = torch.zeros(2 * n, dtype=torch.float64, device=dev)
    plan.txv(t_(c, hk.R64, dev), t_(np.concatenate([one, alt]), hk.R64, dev), Y)
    torch.cuda.synchronize()
    y = Y.cpu().numpy()
    lam1, lam2 = n ** (m - 2) * c.sum(), n ** (m - 2) * (alt @ c)
    assert np.abs(y[:n] - lam1 * one).max() <= 1e-12 * abs(lam1)
    assert np.abs(y[n:] - lam2 * alt).max() <= 1e-12 * abs(lam2)
    plan.close()


def test_real_backward(dev):
    # the adjoint of the circular product: the oracle's gradients of the
    # periodic Hankel tensor, folded back onto c (h_k = c[k mod n])
    rng = np.random.default_rng(4)
    m, n = 3, 60
    c, x, g = rng.standard_normal(n), rng.standard_normal(n), rng.standard_normal(n)
    d = hk.square_descs([m], [n], [0], [0], [0])
    plan = hk.Plan(d, hk.R64, hk.SAME_X | hk.ANTICIRCULANT)
    gh = torch.zeros(n, dtype=torch.float64, device=dev)
    gx = torch.zeros(n, dtype=torch.float64, device=dev)
    plan.backward(t_(g, hk.R64, dev), t_(c, hk.R64, dev), t_(x, hk.R64, dev), gh, gx)
    torch.cuda.synchronize()
    rh, rxs = oracle.fast_grads(periodic(c, m), [x] * (m - 1), [n] * m, g)
    fold = np.zeros(n)
    np.add.at(fold, np.arange(rh.shape[0]) % n, rh.real)
    assert rel(gh.cpu().numpy(), fold) <= 1e-12
    assert rel(gx.cpu().numpy(), sum(r.real for r in rxs)) <= 1e-12
    plan.close()


def test_complex_backward(dev):
    rng = np.random.default_rng(5)
    cr = lambda n: rng.standard_normal(n) + 1j * rng.standard_normal(n)
    m, n = 3, 48
    c, vs, g = cr(n), [cr(n) for _ in range(m)], cr(n)
    d = hk.make_descs(1)
    d[0]["m"] = m
    d[0]["n"][:m] = n
    d[0]["x_off"][:m] = [0, n, 2 * n]
    plan = hk.Plan(d, hk.C128, hk.ANTICIRCULANT)
    gh = torch.zeros(n, dtype=torch.complex128, device=dev)
    gx = torch.zeros(3 * n, dtype=torch.complex128, device=dev)
    plan.backward(t_(g, hk.C128, dev), t_(c, hk.C128, dev), t_(np.concatenate(vs), hk.C128, dev), gh, gx)
    torch.cuda.synchronize()
    rh, rxs = oracle.fast_grads(periodic(c, m), vs[1:], [n] * m, g)
    fold = np.zeros(n, complex)
    np.add.at(fold, np.arange(rh.shape[0]) % n, rh)
    assert rel(gh.cpu().numpy(), fold) <= 1e-12
    gx = gx.cpu().numpy()
    for p in (1, 2):
        assert rel(gx[p * n:(p + 1) * n], rxs[p - 1]) <= 1e-12, p
    plan.close()


def test_block_anticirculant(dev):
    # BAAB (Section 2.2): diagonalised by F_N (x) F_n; equal to the BHHB
    # tensor of the periodic generating matrix G[a, b] = C[a mod n, b mod N]
    rng = np.random.default_rng(6)
    cr = lambda s: rng.standard_normal(s) + 1j * rng.standard_normal(s)
    m, n, N = 3, 6, 4
    C = cr((n, N))
    Xs = [cr((n, N)) for _ in range(m)]
    G = C[np.arange(m * (n - 1) + 1)[:, None] % n, np.arange(m * (N - 1) + 1)[None, :] % N]
    sizes = [[n] * m, [N] * m]
    d = hk.make_descs(1)
    d[0]["m"] = m
    d[0]["n"][:m] = n
    d[0]["N"][:m] = N
    d[0]["x_off"][:m] = [0, n * N, 2 * n * N]
    plan = hk.Plan(d, hk.C128, hk.BLOCK | hk.ANTICIRCULANT)
    Y = torch.zeros(n * N, dtype=torch.complex128, device=dev)
    A = torch.zeros(1, dtype=torch.complex128, device=dev)
    plan.txv_block(t_(lv.vec(C), hk.C128, dev), t_(np.concatenate([lv.vec(X) for X in Xs]), hk.C128, dev), Y, A)
    torch.cuda.synchronize()
    ref = lv.fast_level_y(G, Xs[1:], sizes)
    assert rel(lv.unvec(Y.cpu().numpy(), (n, N)), ref) <= 1e-12
    ar = lv.fast_level_alpha(G, Xs, sizes)
    assert abs(A.cpu().numpy()[0] - ar) <= 1e-12 * abs(ar), (A.cpu().numpy()[0], ar)
    # the same through a level-3 multilevel plan with a trivial third level
    md = hk.level_descs([[n] * m, [N] * m, [1] * m], [0], [[0, n * N, 2 * n * N]], [0])
    plan3 = hk.Plan(md, hk.C128, hk.ANTICIRCULANT)
    Y3 = torch.zeros_like(Y)
    plan3.txv_block(t_(lv.vec(C), hk.C128, dev), t_(np.concatenate([lv.vec(X) for X in Xs]), hk.C128, dev), Y3)
    torch.cuda.synchronize()
    assert torch.equal(Y3, Y)
    plan.close()
    plan3.close()


@pytest.mark.parametrize("dtype,tol", [(hk.R64, 1e-12), (hk.R32, 1e-5)])
def test_dimensions_without_a_transform_length(dev, dtype, tol):
    # n prime (or with a factor above 7): the library runs the Hankel tensor
    # of the periodic generating vector instead; forward, alpha and adjoint
    rng = np.random.default_rng(7)
    cases = [(3, 11), (2, 97), (4, 1021), (3, 13)]
    cs = [rng.standard_normal(n) / np.sqrt(n) for m, n in cases]
    xs = [rng.standard_normal(n) / np.sqrt(n) for m, n in cases]
    offs = np.cumsum([0] + [n for m, n in cases])[:-1]
    d = hk.square_descs([m for m, n in cases], [n for m, n in cases], offs, offs, offs)
    plan = hk.Plan(d, dtype, hk.SAME_X | hk.ANTICIRCULANT)
    total = int(offs[-1] + cases[-1][1])
    H, X = t_(np.concatenate(cs), dtype, dev), t_(np.concatenate(xs), dtype, dev)
    Y = torch.zeros(total, dtype=TDT[dtype], device=dev)
    A = torch.zeros(len(cases), dtype=TDT[dtype], device=dev)
    plan.txv(H, X, Y, A)
    g = rng.standard_normal(total)
    gh, gx = torch.zeros_like(H), torch.zeros_like(X)
    plan.backward(t_(g, dtype, dev), H, X, gh, gx)
    torch.cuda.synchronize()
    y, a, gh, gx = Y.cpu().numpy(), A.cpu().numpy(), gh.cpu().numpy(), gx.cpu().numpy()
    for i, (m, n) in enumerate(cases):
        o = offs[i]
        ref = oracle.fast_y(periodic(cs[i], m), [xs[i]] * (m - 1), [n] * m).real
        assert rel(y[o:o + n], ref) <= tol, (m, n)
        ar = oracle.fast_alpha(periodic(cs[i], m), [xs[i]] * m, [n] * m).real
        assert abs(a[i] - ar) <= tol * np.abs(ref).max() * np.abs(xs[i]).sum(), (m, n)
        rh, rxs = oracle.fast_grads(periodic(cs[i], m), [xs[i]] * (m - 1), [n] * m, g[o:o + n])
        fold = np.zeros(n)
        np.add.at(fold, np.arange(rh.shape[0]) % n, rh.real)
        assert rel(gh[o:o + n], fold) <= 10 * tol, (m, n)
        assert rel(gx[o:o + n], sum(r.real for r in rxs)) <= 10 * tol, (m, n)
    plan.close()


def test_shared_compressed_vector_gradients_are_summed(dev):
    # two complex products of one c (n = 11) with distinct vectors: the
    # gradient with respect to c is the sum of both folds
    rng = np.random.default_rng(8)
    cr = lambda n: rng.standard_normal(n) + 1j * rng.standard_normal(n)
    m, n = 3, 11
    c = cr(n)
    vs = [cr(n) for _ in range(6)]
    d = hk.make_descs(2)
    for t in range(2):
        d[t]["m"] = m
        d[t]["n"][:m] = n
        d[t]["h_off"] = 0
        d[t]["x_off"][:m] = [(3 * t + p) * n for p in range(m)]
        d[t]["y_off"] = t * n
    plan = hk.Plan(d, hk.C128, hk.ANTICIRCULANT)
    g = cr(2 * n)
    gh = torch.zeros(n, dtype=torch.complex128, device=dev)
    gx = torch.zeros(6 * n, dtype=torch.complex128, device=dev)
    Y = torch.zeros(2 * n, dtype=torch.complex128, device=dev)
    plan.txv(t_(c, hk.C128, dev), t_(np.concatenate(vs), hk.C128, dev), Y)
    plan.backward(t_(g, hk.C128, dev), t_(c, hk.C128, dev), t_(np.concatenate(vs), hk.C128, dev), gh, gx)
    torch.cuda.synchronize()
    fold = np.zeros(n, complex)
    y = Y.cpu().numpy()
    for t in range(2):
        ref = oracle.fast_y(periodic(c, m), vs[3 * t + 1: 3 * t + 3], [n] * m)
        assert rel(y[t * n:(t + 1) * n], ref) <= 1e-12
        rh, rxs = oracle.fast_grads(periodic(c, m), vs[3 * t + 1: 3 * t + 3], [n] * m, g[t * n:(t + 1) * n])
        np.add.at(fold, np.arange(rh.shape[0]) % n, rh)
        for p in (1, 2):
            o = (3 * t + p) * n
            assert rel(gx.cpu().numpy()[o:o + n], rxs[p - 1]) <= 1e-12, (t, p)
    assert rel(gh.cpu().numpy(), fold) <= 1e-12
    plan.close()


def test_corollary_2_2_for_odd_n(dev):
    # odd n: the all-ones eigenpair, through the periodic embedding
    n, m = 11, 4
    c = np.random.default_rng(9).standard_normal(n)
    d = hk.square_descs([m], [n], [0], [0], [0])
    plan = hk.Plan(d, hk.R64, hk.SAME_X | hk.ANTICIRCULANT)
    Y = torch.zeros(n, dtype=torch.float64, device=dev)
    plan.txv(t_(c, hk.R64, dev), t_(np.ones(n), hk.R64, dev), Y)
    torch.cuda.synchronize()
    lam = n ** (m - 2) * c.sum()
    assert np.abs(Y.cpu().numpy() - lam).max() <= 1e-12 * abs(lam)
    plan.close()
