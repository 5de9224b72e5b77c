"""Randomised differential test: many small plans drawn from a fixed seed --
every dtype, one-level (square and not, one vector or one per mode),
anti-circulant, BHHB and level-3 tensors, with and without stored spectra,
FP64 spectrum products or one tensor per launch, shared operands -- each checked against the oracle for y, alpha and the
adjoint.  A failure names the case's index for reproduction."""

import numpy as np
import pytest

import oracle
from oracle import level as lv
from paper_1401_6238_gb300 import hankel as hk

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TDT = {hk.R32: torch.float32, hk.C64: torch.complex64, hk.R64: torch.float64, hk.C128: torch.complex128}
TOL = {hk.R32: 1e-5, hk.C64: 1e-5, hk.R64: 1e-12, hk.C128: 1e-12}


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    hk.load()
    return torch.device("cuda:0")


def rel(a, b):
    s = np.abs(b).max()
    return np.abs(a - b).max() / (s if s > 0 else 1.0)


def draw_case(rng):
    dtype = int(rng.choice([hk.R32, hk.C64, hk.R64, hk.C128]))
    cplx = dtype in (hk.C64, hk.C128)
    kind = str(rng.choice(["square", "distinct", "anti", "block", "level3"]))
    m = int(rng.integers(2, 5))
    count = int(rng.integers(1, 6))
    store = bool(rng.integers(0, 2))
    shared_h = bool(rng.integers(0, 2)) and count > 1
    if kind == "square":
        sizes = [[int(rng.integers(2, 300))] * m]
    elif kind == "anti":
        sizes = [[int(rng.choice([7, 11, 12, 30, 64, 97, 120]))] * m]
    elif kind == "distinct":
        sizes = [[int(v) for v in rng.integers(2, 200, size=m)]]
    elif kind == "block":
        sizes = [[int(v) for v in rng.integers(1, 12, size=m)], [int(v) for v in rng.integers(1, 8, size=m)]]
    else:
        sizes = [[int(v) for v in rng.integers(1, 6, size=m)] for _ in range(3)]
    same_x = kind in ("square", "anti") and bool(rng.integers(0, 2))
    extra = int(rng.choice([0, 0, 0, hk.FP64_POWER, hk.ONE_PER_LAUNCH]))
    return dict(dtype=dtype, cplx=cplx, kind=kind, m=m, count=count, store=store, shared_h=shared_h, sizes=sizes,
                same_x=same_x, extra=extra)


def draw(rng, shape, cplx):
    v = rng.standard_normal(shape)
    return v + 1j * rng.standard_normal(shape) if cplx else v


CASES = 150


@pytest.mark.parametrize("idx", range(CASES))
def test_fuzz_case(dev, idx):
    rng = np.random.default_rng(1000 + idx)
    c = draw_case(rng)
    m, count, sizes, cplx, dtype = c["m"], c["count"], c["sizes"], c["cplx"], c["dtype"]
    anti = c["kind"] == "anti"
    levels = len(sizes)
    gshape = tuple(s[0] for s in sizes) if anti else lv.gen_shape(sizes)
    mshape = [lv.mode_shape(sizes, p) for p in range(m)]
    G = [draw(rng, gshape, cplx) / np.sqrt(np.prod(gshape)) for _ in range(count)]
    if c["shared_h"]:
        G = [G[0]] * count
    nx = 1 if c["same_x"] else m
    X = [[draw(rng, mshape[p], cplx) / np.sqrt(np.prod(mshape[p])) for p in range(nx)] for _ in range(count)]
    # pack
    hsz = int(np.prod(gshape))
    h_off = [0 if c["shared_h"] else t * hsz for t in range(count)]
    hbuf = np.concatenate([lv.vec(G[t]) for t in range(1 if c["shared_h"] else count)])
    xs, x_offs, xo = [], [], 0
    for t in range(count):
        offs = []
        for p in range(nx):
            offs.append(xo)
            xs.append(lv.vec(X[t][p]))
            xo += X[t][p].size
        x_offs.append(offs)
    xbuf = np.concatenate(xs)
    ny = int(np.prod(mshape[0]))
    y_offs = [t * ny for t in range(count)]
    flags = (hk.SAME_X if c["same_x"] else 0) | (hk.STORE_SPECTRA if c["store"] else 0) | (hk.ANTICIRCULANT if anti else 0)
    if levels < 3:
        flags |= c["extra"]
    if levels == 1:
        d = hk.make_descs(count)
        d["m"] = m
        d["n"][:, :m] = sizes[0]
        d["h_off"] = h_off
        for t in range(count):
            d["x_off"][t, :nx] = x_offs[t]
        d["y_off"] = y_offs
    elif levels == 2:
        d = hk.make_descs(count)
        d["m"] = m
        d["n"][:, :m] = sizes[0]
        d["N"][:, :m] = sizes[1]
        d["h_off"] = h_off
        for t in range(count):
            d["x_off"][t, :nx] = x_offs[t]
        d["y_off"] = y_offs
        flags |= hk.BLOCK
    else:
        d = hk.level_descs(sizes, h_off, x_offs, y_offs)
    plan = hk.Plan(d, dtype, flags)
    T = lambda a: torch.tensor(np.ascontiguousarray(a if cplx else np.real(a)), dtype=TDT[dtype], device=dev)
    H, Xt = T(hbuf), T(xbuf)
    Y = torch.zeros(count * ny, dtype=TDT[dtype], device=dev)
    A = torch.zeros(count, dtype=TDT[dtype], device=dev)
    run = plan.txv_block if plan.flags & hk.BLOCK else plan.txv
    run(H, Xt, Y, A)
    gy = draw(rng, count * ny, cplx)
    gh, gx = torch.zeros_like(H), torch.zeros_like(Xt)
    plan.backward(T(gy), H, Xt, gh, gx)
    torch.cuda.synchronize()
    y, a, gh, gx = Y.cpu().numpy(), A.cpu().numpy(), gh.cpu().numpy(), gx.cpu().numpy()
    tol = TOL[dtype]
    want_h = np.zeros(hbuf.shape, complex)
    want_x = np.zeros(xbuf.shape, complex)
    for t in range(count):
        vecs = [X[t][0 if c["same_x"] else p] for p in range(m)]
        if anti:
            hp = oracle.anticirculant_generating_vector(np.asarray(G[t]).reshape(-1), m) if levels == 1 else None
            ref = oracle.fast_y(hp, vecs[1:], [sizes[0][0]] * m)
            ar = oracle.fast_alpha(hp, vecs, [sizes[0][0]] * m)
            rh, rx = oracle.fast_grads(hp, vecs[1:], [sizes[0][0]] * m, gy[y_offs[t]: y_offs[t] + ny])
            fold = np.zeros(gshape[0], complex)
            np.add.at(fold, np.arange(rh.shape[0]) % gshape[0], rh)
            rh = fold
        else:
            ref = lv.vec(lv.fast_level_y(G[t], vecs[1:], sizes))
            ar = lv.fast_level_alpha(G[t], vecs, sizes)
            rG, rx = lv.fast_level_grads(G[t], vecs[1:], sizes, lv.unvec(gy[y_offs[t]: y_offs[t] + ny], mshape[0]))
            rh = lv.vec(rG)
            rx = [lv.vec(r) for r in rx]
        if not cplx:
            ref, ar = ref.real, ar.real
        ey = rel(y[y_offs[t]: y_offs[t] + ny], ref)
        assert ey <= tol, (idx, c, "y", t, ey)
        scale = np.abs(ref).max() * np.abs(vecs[0]).sum()
        ea = abs(a[t] - ar) / max(scale, 1e-30)
        assert ea <= tol, (idx, c, "alpha", t, ea)
        want_h[h_off[t]: h_off[t] + hsz] += rh
        for p in range(1, m):
            o = x_offs[t][0 if c["same_x"] else p]
            want_x[o: o + rx[p - 1].size] += rx[p - 1]
    if not cplx:
        want_h, want_x = want_h.real, want_x.real
    eh = rel(gh, want_h)
    assert eh <= tol, (idx, c, "grad_h", eh)
    # x_1 receives no gradient from y (it enters only alpha)
    ex = rel(gx, want_x)
    assert ex <= tol, (idx, c, "grad_x", ex)
    plan.close()
