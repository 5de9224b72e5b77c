"""Level-k block Hankel products (Section 2.2 and the close of Section 3) on
the GPU against the oracle's k-dimensional FFT products, element by element:
forward y and alpha for levels 1-4 (ragged sizes, an inactive level) in all
four dtypes, the adjoint, shared operands, level 1 and 2 against the
one-level and BHHB plans, and a full-size level-3 workload (64^3 signal,
sizes (22,22,22) per level, 32 vector triples) on sampled outputs."""

import numpy as np
import pytest

from oracle import level as lv
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


def T(a, dtype, dev):
    return torch.tensor(np.ascontiguousarray(a), dtype=getattr(torch, TDT[dtype]), device=dev)


def pack(sizes, count, seed, cplx):
    """``count`` tensors of one shape with their own G and x_1..x_m."""
    rng = np.random.default_rng(seed)
    m = len(sizes[0])
    draw = (lambda s: rng.standard_normal(s) + 1j * rng.standard_normal(s)) if cplx else rng.standard_normal
    Gs = [draw(lv.gen_shape(sizes)) for _ in range(count)]
    Xss = [[draw(lv.mode_shape(sizes, p)) for p in range(m)] for _ in range(count)]
    hs, xs, xoffs, hoffs, yoffs = [], [], [], [], []
    ho = xo = yo = 0
    ny = int(np.prod(lv.mode_shape(sizes, 0)))
    for G, Xs in zip(Gs, Xss):
        hoffs.append(ho)
        hs.append(lv.vec(G))
        ho += G.size
        offs = []
        for X in Xs:
            offs.append(xo)
            xs.append(lv.vec(X))
            xo += X.size
        xoffs.append(offs)
        yoffs.append(yo)
        yo += ny
    d = hk.level_descs(sizes, hoffs, xoffs, yoffs)
    return Gs, Xss, np.concatenate(hs), np.concatenate(xs), d, yo


def rel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


SIZES = [
    [[20, 17, 13], [6, 5, 4], [3, 4, 2]],      # level 3, ragged
    [[5, 4], [3, 3], [2, 2], [4, 2]],          # level 4, order 2
    [[30, 20, 10], [1, 1, 1], [4, 3, 5]],      # level 3 with an inactive middle level
    [[9, 7, 5, 3]],                            # level 1, order 4
]


@pytest.mark.parametrize("dtype", [hk.C128, hk.C64, hk.R64, hk.R32])
@pytest.mark.parametrize("sizes", SIZES)
def test_level_forward(dev, dtype, sizes):
    cplx = dtype in (hk.C64, hk.C128)
    Gs, Xss, h, x, d, ny = pack(sizes, 3, seed=len(sizes) + dtype, cplx=cplx)
    plan = hk.Plan(d, dtype, 0)
    Y = torch.zeros(ny, dtype=getattr(torch, TDT[dtype]), device=dev)
    A = torch.zeros(3, dtype=getattr(torch, TDT[dtype]), device=dev)
    plan.txv_block(T(h, dtype, dev), T(x, dtype, dev), Y, A)
    torch.cuda.synchronize()
    y, a = Y.cpu().numpy(), A.cpu().numpy()
    shape = lv.mode_shape(sizes, 0)
    for t in range(3):
        ref = lv.fast_level_y(Gs[t], Xss[t][1:], sizes)
        got = lv.unvec(y[d["y_off"][t]: d["y_off"][t] + ref.size], shape)
        assert rel(got, ref) <= TOL[dtype], t
        ar = lv.fast_level_alpha(Gs[t], Xss[t], sizes)
        scale = np.abs(ref).max() * np.abs(Xss[t][0]).sum()
        assert abs(a[t] - ar) <= TOL[dtype] * scale, t
    # alpha alone (no product transforms) gives the same alpha
    A2 = torch.zeros_like(A)
    plan.txv_block(T(h, dtype, dev), T(x, dtype, dev), None, A2)
    torch.cuda.synchronize()
    assert np.abs(A2.cpu().numpy() - a).max() <= 1e-6 * np.abs(a).max()
    plan.close()


@pytest.mark.parametrize("dtype", [hk.C128, hk.C64, hk.R32])
@pytest.mark.parametrize("sizes", SIZES[:3])
def test_level_backward(dev, dtype, sizes):
    cplx = dtype in (hk.C64, hk.C128)
    Gs, Xss, h, x, d, ny = pack(sizes, 2, seed=7 + dtype, cplx=cplx)
    rng = np.random.default_rng(9)
    shape = lv.mode_shape(sizes, 0)
    Gy = [rng.standard_normal(shape) + (1j * rng.standard_normal(shape) if cplx else 0) for _ in range(2)]
    gy = np.concatenate([lv.vec(g) for g in Gy])
    plan = hk.Plan(d, dtype, 0)
    gh = torch.zeros(h.size, dtype=getattr(torch, TDT[dtype]), device=dev)
    gx = torch.zeros(x.size, dtype=getattr(torch, TDT[dtype]), device=dev)
    plan.backward(T(gy, dtype, dev), T(h, dtype, dev), T(x, dtype, dev), gh, gx)
    torch.cuda.synchronize()
    gh, gx = gh.cpu().numpy(), gx.cpu().numpy()
    tol = 10 * TOL[dtype]
    for t in range(2):
        rG, rX = lv.fast_level_grads(Gs[t], Xss[t][1:], sizes, Gy[t])
        got = lv.unvec(gh[d["h_off"][t]: d["h_off"][t] + rG.size], rG.shape)
        assert rel(got, rG) <= tol, t
        for p in range(1, len(sizes[0])):
            o = d["x_off"][t][p]
            got = lv.unvec(gx[o: o + rX[p - 1].size], rX[p - 1].shape)
            assert rel(got, rX[p - 1]) <= tol, (t, p)
    plan.close()


def test_level_shared_operands_sum_gradients(dev):
    # one generating tensor, vector columns shared between products (the
    # tensor-matrix product pattern of Section 4.2 on a level-3 tensor)
    sizes = [[6, 5, 5], [4, 3, 3], [2, 3, 3]]
    rng = np.random.default_rng(3)
    cr = lambda s: rng.standard_normal(s) + 1j * rng.standard_normal(s)
    G = cr(lv.gen_shape(sizes))
    cols = [cr(lv.mode_shape(sizes, 1)) for _ in range(3)]
    n0 = int(np.prod(lv.mode_shape(sizes, 0)))
    nc = cols[0].size
    x = np.concatenate([np.zeros(n0)] + [lv.vec(c) for c in cols])
    pairs = [(0, 1), (1, 2), (2, 2), (0, 0), (2, 1)]
    d = hk.level_descs(sizes, [0] * len(pairs), [[0, n0 + i * nc, n0 + j * nc] for i, j in pairs],
                       [t * n0 for t in range(len(pairs))])
    plan = hk.Plan(d, hk.C128, 0)
    Y = torch.zeros(len(pairs) * n0, dtype=torch.complex128, device=dev)
    plan.txv_block(T(lv.vec(G), hk.C128, dev), T(x, hk.C128, dev), Y)
    gyv = cr(len(pairs) * n0)
    gh = torch.zeros(G.size, dtype=torch.complex128, device=dev)
    gx = torch.zeros(x.size, dtype=torch.complex128, device=dev)
    plan.backward(T(gyv, hk.C128, dev), T(lv.vec(G), hk.C128, dev), T(x, hk.C128, dev), gh, gx)
    torch.cuda.synchronize()
    y, gh, gx = Y.cpu().numpy(), gh.cpu().numpy(), gx.cpu().numpy()
    shape0 = lv.mode_shape(sizes, 0)
    tG = np.zeros(G.shape, complex)
    tc = [np.zeros(cols[0].shape, complex) for _ in range(3)]
    for t, (i, j) in enumerate(pairs):
        ref = lv.fast_level_y(G, [cols[i], cols[j]], sizes)
        assert rel(lv.unvec(y[t * n0:(t + 1) * n0], shape0), ref) <= 1e-12
        rG, rX = lv.fast_level_grads(G, [cols[i], cols[j]], sizes, lv.unvec(gyv[t * n0:(t + 1) * n0], shape0))
        tG += rG
        tc[i] += rX[0]
        tc[j] += rX[1]
    assert rel(lv.unvec(gh, G.shape), tG) <= 1e-12
    for c in range(3):
        got = lv.unvec(gx[n0 + c * nc: n0 + (c + 1) * nc], cols[0].shape)
        assert rel(got, tc[c]) <= 1e-12, c
    plan.close()


def test_level2_equals_bhhb_plan_and_level1_equals_general_plan(dev):
    sizes = [[7, 5, 6], [4, 3, 2]]
    Gs, Xss, h, x, d, ny = pack(sizes, 2, seed=4, cplx=True)
    bd = hk.make_descs(2)
    bd["m"] = 3
    bd["n"][:, :3] = sizes[0]
    bd["N"][:, :3] = sizes[1]
    bd["h_off"] = d["h_off"]
    bd["x_off"][:, :3] = d["x_off"][:, :3]
    bd["y_off"] = d["y_off"]
    outs = []
    for descs in (d, bd):
        plan = hk.Plan(descs, hk.C64, hk.BLOCK if descs.dtype == hk.DESC_DTYPE else 0)
        Y = torch.zeros(ny, dtype=torch.complex64, device=dev)
        plan.txv_block(T(h, hk.C64, dev), T(x, hk.C64, dev), Y)
        torch.cuda.synchronize()
        outs.append(Y.cpu().numpy())
        plan.close()
    assert np.array_equal(outs[0], outs[1])
    sizes1 = [[9, 7, 5]]
    Gs, Xss, h, x, d1, ny = pack(sizes1, 2, seed=5, cplx=True)
    gd = hk.make_descs(2)
    gd["m"] = 3
    gd["n"][:, :3] = sizes1[0]
    gd["h_off"] = d1["h_off"]
    gd["x_off"][:, :3] = d1["x_off"][:, :3]
    gd["y_off"] = d1["y_off"]
    p1, p2 = hk.Plan(d1, hk.C128, 0), hk.Plan(gd, hk.C128, 0)
    Y1 = torch.zeros(ny, dtype=torch.complex128, device=dev)
    Y2 = torch.zeros_like(Y1)
    p1.txv_block(T(h, hk.C128, dev), T(x, hk.C128, dev), Y1)
    p2.txv(T(h, hk.C128, dev), T(x, hk.C128, dev), Y2)
    torch.cuda.synchronize()
    assert torch.equal(Y1, Y2)
    p1.close()
    p2.close()


def level3_case(count=32, seed=10):
    S = wl.edf_3d_signal(seed=seed)
    sizes = [[22, 22, 22]] * 3
    Xs = wl.random_arrays(2 * count, (22, 22, 22), seed=seed + 1)
    n = 22 ** 3
    x = np.concatenate([lv.vec(X) for X in Xs])
    d = hk.level_descs(sizes, [0] * count, [[0, 2 * t * n, (2 * t + 1) * n] for t in range(count)],
                       [t * n for t in range(count)])
    return S, sizes, Xs, x, d


def test_level3_full_size(dev):
    count = 32
    S, sizes, Xs, x, d = level3_case(count)
    assert lv.gen_shape(sizes) == S.shape == (64, 64, 64)
    plan = hk.Plan(d, hk.C64, 0)
    n = 22 ** 3
    Y = torch.zeros(count * n, dtype=torch.complex64, device=dev)
    plan.txv_block(T(lv.vec(S), hk.C64, dev), T(x, hk.C64, dev), Y)
    torch.cuda.synchronize()
    y = Y.cpu().numpy()
    for t in (0, 17, 31):
        ref = lv.fast_level_y(S, [Xs[2 * t], Xs[2 * t + 1]], sizes)
        assert rel(lv.unvec(y[t * n:(t + 1) * n], (22, 22, 22)), ref) <= 1e-5, t
    plan.close()


def test_autograd_through_a_level3_plan(dev):
    # torch.autograd through HankelTxV on a level-k plan: the gradients of a
    # real loss equal the oracle's adjoint (complex128)
    sizes = [[5, 4, 3], [3, 2, 2], [2, 3, 2]]
    Gs, Xss, h, x, d, ny = pack(sizes, 1, seed=11, cplx=True)
    plan = hk.Plan(d, hk.C128, 0)
    H = torch.tensor(h, dtype=torch.complex128, device=dev, requires_grad=True)
    X = torch.tensor(x, dtype=torch.complex128, device=dev, requires_grad=True)
    rng = np.random.default_rng(4)
    w = torch.tensor(rng.standard_normal(ny) + 1j * rng.standard_normal(ny), device=dev)
    y = hk.hankel_txv_autograd(H, X, plan)
    loss = (w.conj() * y).real.sum()  # dL/dy (PyTorch convention) is w
    loss.backward()
    torch.cuda.synchronize()
    shape = lv.mode_shape(sizes, 0)
    rG, rX = lv.fast_level_grads(Gs[0], Xss[0][1:], sizes, lv.unvec(w.cpu().numpy(), shape))
    assert rel(lv.unvec(H.grad.cpu().numpy(), rG.shape), rG) <= 1e-12
    for p in range(1, 3):
        o = d["x_off"][0][p]
        got = lv.unvec(X.grad.cpu().numpy()[o: o + rX[p - 1].size], rX[p - 1].shape)
        assert rel(got, rX[p - 1]) <= 1e-12, p
    plan.close()
