"""GPU parity of the general path against the FP64 oracle: complex data, a
different vector in every mode, alpha with its own x_1, operands shared by
many descriptors (the HOOI tensor-matrix products of Section 4.2), BHHB
tensors (Section 3 block procedures) and their adjoints."""

import numpy as np
import pytest

import oracle
from paper_1401_6238_gb300 import hankel as hk
from paper_1401_6238_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TDT = {hk.R32: "float32", hk.C64: "complex64", hk.R64: "float64", hk.C128: "complex128"}
TOL = {hk.R32: 1e-5, hk.C64: 1e-5, hk.R64: 1e-12, hk.C128: 1e-12}


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    hk.load()
    return torch.device("cuda:0")


class Packer:
    """Flat h / x buffers with offsets (shared operands reuse an offset)."""

    def __init__(self, cplx):
        self.cplx = cplx
        self.h, self.x = [], []
        self.hp = self.xp = 0

    def add_h(self, v):
        off = self.hp
        self.h.append(np.asarray(v).reshape(-1, order="F"))
        self.hp += self.h[-1].size
        return off

    def add_x(self, v):
        off = self.xp
        self.x.append(np.asarray(v).reshape(-1, order="F"))
        self.xp += self.x[-1].size
        return off

    def arrays(self):
        dt = np.complex128 if self.cplx else np.float64
        return np.concatenate(self.h).astype(dt), np.concatenate(self.x).astype(dt)


def to_dev(a, dtype, dev):
    return torch.tensor(a, dtype=getattr(torch, TDT[dtype]), device=dev)


def rnd(rng, shape, cplx):
    v = rng.standard_normal(shape)
    return v + 1j * rng.standard_normal(shape) if cplx else v


def rel(got, ref):
    return np.max(np.abs(got - ref)) / max(np.max(np.abs(ref)), 1e-300)


@pytest.mark.parametrize("dtype", [hk.C64, hk.C128, hk.R32, hk.R64])
def test_distinct_vectors_and_alpha(dev, dtype):
    cplx = dtype in (hk.C64, hk.C128)
    rng = np.random.default_rng(3)
    cases = [[5, 3, 4], [16, 9, 30, 7], [64, 64], [2, 2, 2, 2, 2], [100, 37, 250], [1, 1, 1]]
    pk = Packer(cplx)
    descs = hk.make_descs(len(cases))
    refs, yoff = [], 0
    for i, dims in enumerate(cases):
        m = len(dims)
        h = rnd(rng, oracle.d_of(dims), cplx)
        xs = [rnd(rng, n, cplx) for n in dims]
        descs[i]["m"] = m
        descs[i]["n"][:m] = dims
        descs[i]["h_off"] = pk.add_h(h)
        for p in range(m):
            descs[i]["x_off"][p] = pk.add_x(xs[p])
        descs[i]["y_off"] = yoff
        yoff += dims[0]
        refs.append((oracle.fast_y(h, xs[1:], dims), oracle.fast_alpha(h, xs, dims), h, xs, dims))
    H, X = pk.arrays()
    plan = hk.Plan(descs, dtype, 0)
    Y = torch.zeros(yoff, dtype=getattr(torch, TDT[dtype]), device=dev)
    A = torch.zeros(len(cases), dtype=getattr(torch, TDT[dtype]), device=dev)
    plan.txv(to_dev(H, dtype, dev), to_dev(X, dtype, dev), Y, A)
    torch.cuda.synchronize()
    y, a = Y.cpu().numpy(), A.cpu().numpy()
    off = 0
    for i, (yr, ar, h, xs, dims) in enumerate(refs):
        if not cplx:
            yr, ar = yr.real, ar.real
        assert rel(y[off:off + dims[0]], yr) <= TOL[dtype], (i, dims)
        scale = np.max(np.abs(yr)) * np.sum(np.abs(xs[0]))
        assert abs(a[i] - ar) <= TOL[dtype] * scale, (i, a[i], ar)
        off += dims[0]
    plan.close()


def hooi_products(N=4094, R=8, seed=4, dtype=hk.C64, dev=None, check=True):
    """H x_2 u_i x_3 u_j for all column pairs, H the order-3 Hankel tensor of
    a 1D exponential signal (Section 4.2); every descriptor shares h."""
    s = wl.edf_1d_signal(N=N, seed=seed)
    # order-3 tensor as close to square as the length allows (1366 x 1365 x 1365 for N = 4094)
    dims = [N + 2 - 2 * ((N + 2) // 3), (N + 2) // 3, (N + 2) // 3]
    assert oracle.d_of(dims) == N
    U = wl.unit_columns(dims[1], R, seed=seed + 1)
    V = wl.unit_columns(dims[2], R, seed=seed + 2)
    pk = Packer(True)
    h_off = pk.add_h(s)
    uo = [pk.add_x(U[:, i]) for i in range(R)]
    vo = [pk.add_x(V[:, j]) for j in range(R)]
    descs = hk.make_descs(R * R)
    for k in range(R * R):
        i, j = divmod(k, R)
        descs[k]["m"] = 3
        descs[k]["n"][:3] = dims
        descs[k]["h_off"] = h_off
        descs[k]["x_off"][1] = uo[i]
        descs[k]["x_off"][2] = vo[j]
        descs[k]["y_off"] = k * dims[0]
    return s, dims, U, V, descs, pk


def test_hooi_pair_products_share_h(dev):
    R = 6
    s, dims, U, V, descs, pk = hooi_products(N=302, R=R)
    H, X = pk.arrays()
    plan = hk.Plan(descs, hk.C64, 0)
    info = plan.info
    Y = torch.zeros(R * R * dims[0], dtype=torch.complex64, device=dev)
    plan.txv(to_dev(H, hk.C64, dev), to_dev(X, hk.C64, dev), Y)
    torch.cuda.synchronize()
    y = Y.cpu().numpy()
    for k in range(R * R):
        i, j = divmod(k, R)
        ref = oracle.fast_y(s, [U[:, i], V[:, j]], dims)
        assert rel(y[k * dims[0]:(k + 1) * dims[0]], ref) <= 1e-5, k
    # one spectrum for h and one per distinct column
    assert info["workspace_bytes"] > 0


def block_case(n, N, cplx, rng, count=1, share_H=True):
    m = len(n)
    pk = Packer(cplx)
    d1, d2 = sum(n) - m + 1, sum(N) - m + 1
    Hs = [rnd(rng, (d1, d2), cplx) for _ in range(1 if share_H else count)]
    hoffs = [pk.add_h(Hm) for Hm in Hs]
    descs = hk.make_descs(count)
    Xs_all = []
    for t in range(count):
        Xs = [rnd(rng, (n[p], N[p]), cplx) for p in range(m)]
        Xs_all.append(Xs)
        descs[t]["m"] = m
        descs[t]["n"][:m] = n
        descs[t]["N"][:m] = N
        descs[t]["h_off"] = hoffs[0 if share_H else t]
        for p in range(m):
            descs[t]["x_off"][p] = pk.add_x(Xs[p])
        descs[t]["y_off"] = t * n[0] * N[0]
    return Hs, Xs_all, descs, pk


@pytest.mark.parametrize("dtype", [hk.C64, hk.C128])
@pytest.mark.parametrize("n,N", [([3, 2, 4], [2, 5, 3]), ([6, 6, 6], [5, 5, 5]), ([2, 3], [4, 4])])
def test_block_forward_and_alpha(dev, dtype, n, N):
    rng = np.random.default_rng(sum(n) + sum(N))
    Hs, Xs_all, descs, pk = block_case(n, N, True, rng, count=3)
    H, X = pk.arrays()
    plan = hk.Plan(descs, dtype, hk.BLOCK)
    Y = torch.zeros(3 * n[0] * N[0], dtype=getattr(torch, TDT[dtype]), device=dev)
    A = torch.zeros(3, dtype=getattr(torch, TDT[dtype]), device=dev)
    plan.txv_block(to_dev(H, dtype, dev), to_dev(X, dtype, dev), Y, A)
    torch.cuda.synchronize()
    y, a = Y.cpu().numpy(), A.cpu().numpy()
    for t in range(3):
        Xs = Xs_all[t]
        ref = oracle.brute_block_y(Hs[0], Xs[1:], n, N)
        got = y[t * n[0] * N[0]:(t + 1) * n[0] * N[0]].reshape(N[0], n[0]).T
        assert rel(got, ref) <= TOL[dtype], t
        ar = oracle.brute_block_alpha(Hs[0], Xs, n, N)
        assert abs(a[t] - ar) <= TOL[dtype] * np.max(np.abs(ref)) * np.sum(np.abs(Xs[0])), t
    plan.close()


@pytest.mark.parametrize("dtype,tol", [(hk.C64, 1e-5), (hk.C128, 1e-12), (hk.R64, 1e-12)])
def test_general_backward_1d(dev, dtype, tol):
    cplx = dtype in (hk.C64, hk.C128)
    rng = np.random.default_rng(8)
    cases = [[5, 3, 4], [40, 9, 30], [7, 7]]
    pk = Packer(cplx)
    descs = hk.make_descs(len(cases))
    data, yoff = [], 0
    for i, dims in enumerate(cases):
        m = len(dims)
        h = rnd(rng, oracle.d_of(dims), cplx)
        xs = [rnd(rng, n, cplx) for n in dims]
        descs[i]["m"] = m
        descs[i]["n"][:m] = dims
        descs[i]["h_off"] = pk.add_h(h)
        for p in range(m):
            descs[i]["x_off"][p] = pk.add_x(xs[p])
        descs[i]["y_off"] = yoff
        g = rnd(rng, dims[0], cplx)
        data.append((h, xs, dims, g, descs[i]["h_off"], list(descs[i]["x_off"][:m])))
        yoff += dims[0]
    H, X = pk.arrays()
    G = np.concatenate([d[3] for d in data])
    plan = hk.Plan(descs, dtype, 0)
    gh = torch.zeros(H.size, dtype=getattr(torch, TDT[dtype]), device=dev)
    gx = torch.zeros(X.size, dtype=getattr(torch, TDT[dtype]), device=dev)
    plan.backward(to_dev(G, dtype, dev), to_dev(H, dtype, dev), to_dev(X, dtype, dev), gh, gx)
    torch.cuda.synchronize()
    gh, gx = gh.cpu().numpy(), gx.cpu().numpy()
    for h, xs, dims, g, ho, xo in data:
        rh, rxs = oracle.fast_grads(h, xs[1:], dims, g)
        if not cplx:
            rh, rxs = rh.real, [v.real for v in rxs]
        assert rel(gh[ho:ho + len(h)], rh) <= tol
        for p in range(1, len(dims)):
            assert rel(gx[xo[p]:xo[p] + dims[p]], rxs[p - 1]) <= tol, p
        # x_1 is not an input of y: its gradient region stays zero
        assert np.all(gx[xo[0]:xo[0] + dims[0]] == 0)
    plan.close()


@pytest.mark.parametrize("share_H", [True, False])
def test_block_backward_shared_generator(dev, share_H):
    rng = np.random.default_rng(11)
    n, N, count = [3, 4, 3], [4, 2, 3], 4
    Hs, Xs_all, descs, pk = block_case(n, N, True, rng, count=count, share_H=share_H)
    H, X = pk.arrays()
    Gs = [rnd(rng, (n[0], N[0]), True) for _ in range(count)]
    G = np.concatenate([g.reshape(-1, order="F") for g in Gs])
    plan = hk.Plan(descs, hk.C128, hk.BLOCK)
    gh = torch.zeros(H.size, dtype=torch.complex128, device=dev)
    gx = torch.zeros(X.size, dtype=torch.complex128, device=dev)
    plan.backward(to_dev(G, hk.C128, dev), to_dev(H, hk.C128, dev), to_dev(X, hk.C128, dev), gh, gx)
    torch.cuda.synchronize()
    gh, gx = gh.cpu().numpy(), gx.cpu().numpy()
    d1, d2 = sum(n) - 2, sum(N) - 2
    total = np.zeros((d1, d2), complex)
    for t in range(count):
        Hm = Hs[0 if share_H else t]
        rH, rXs = oracle.brute_block_grads(Hm, Xs_all[t][1:], n, N, Gs[t])
        if share_H:
            total += rH
        else:
            ho = descs[t]["h_off"]
            got = gh[ho:ho + d1 * d2].reshape(d2, d1).T
            assert rel(got, rH) <= 1e-12, (t, rel(got, rH))
        for p in range(1, 3):
            xo = descs[t]["x_off"][p]
            got = gx[xo:xo + n[p] * N[p]].reshape(N[p], n[p]).T
            assert rel(got, rXs[p - 1]) <= 1e-12, (t, p, rel(got, rXs[p - 1]))
    if share_H:
        got = gh[:d1 * d2].reshape(d2, d1).T
        assert rel(got, total) <= 1e-12, rel(got, total)
    plan.close()


@pytest.mark.parametrize("block", [False, True])
def test_backward_one_gradient_only(dev, block):
    """An adjoint call that asks for grad_h alone, or grad_x alone, gives the
    same values as the call that asks for both (the gradient lines of both
    kinds share launches; a line whose buffer is absent stores nothing)."""
    rng = np.random.default_rng(21)
    if block:
        n, N = [3, 4, 3], [4, 2, 3]
        Hs, Xs_all, descs, pk = block_case(n, N, True, rng, count=3, share_H=False)
        G = np.concatenate([rnd(rng, (n[0], N[0]), True).reshape(-1, order="F") for _ in range(3)])
        flags = hk.BLOCK
    else:
        cases = [[5, 3, 4], [40, 9, 30], [7, 7]]
        pk = Packer(True)
        descs = hk.make_descs(len(cases))
        yoff = 0
        for i, dims in enumerate(cases):
            m = len(dims)
            descs[i]["m"] = m
            descs[i]["n"][:m] = dims
            descs[i]["h_off"] = pk.add_h(rnd(rng, oracle.d_of(dims), True))
            for p in range(m):
                descs[i]["x_off"][p] = pk.add_x(rnd(rng, dims[p], True))
            descs[i]["y_off"] = yoff
            yoff += dims[0]
        G = rnd(rng, yoff, True)
        flags = 0
    H, X = pk.arrays()
    plan = hk.Plan(descs, hk.C128, flags)
    args = (to_dev(G, hk.C128, dev), to_dev(H, hk.C128, dev), to_dev(X, hk.C128, dev))
    both_h = torch.zeros(H.size, dtype=torch.complex128, device=dev)
    both_x = torch.zeros(X.size, dtype=torch.complex128, device=dev)
    plan.backward(*args, both_h, both_x)
    only_h = torch.zeros_like(both_h)
    plan.backward(*args, only_h, None)
    only_x = torch.zeros_like(both_x)
    plan.backward(*args, None, only_x)
    torch.cuda.synchronize()
    assert torch.count_nonzero(both_h).item() > 0 and torch.count_nonzero(both_x).item() > 0
    assert torch.equal(only_h, both_h)
    assert torch.equal(only_x, both_x)
    plan.close()
