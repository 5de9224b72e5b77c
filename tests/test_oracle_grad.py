"""Pins for the oracle's gradients: FP64 central finite differences, the
adjoint (dot-product) identity and Euler's identity for homogeneous maps."""

import numpy as np
import pytest

import oracle


def loss_and_g(y, t):
    r = y - t
    return float(np.sum(np.abs(r) ** 2)), 2.0 * r


def fd_grad(f, v, eps=1e-6):
    """Central differences; complex v gives dL/dRe + i dL/dIm."""
    v = np.array(v, dtype=complex if np.iscomplexobj(v) else float)
    g = np.zeros_like(v)
    for k in range(v.size):
        for unit in ([1.0, 1j] if np.iscomplexobj(v) else [1.0]):
            vp, vm = v.copy(), v.copy()
            vp.flat[k] += eps * unit
            vm.flat[k] -= eps * unit
            g.flat[k] += unit * (f(vp) - f(vm)) / (2 * eps)
    return g


@pytest.mark.parametrize("dims,cplx", [([4, 3, 5], False), ([3, 4, 2, 3], False), ([4, 3, 3], True), ([5, 2], True)])
def test_grads_match_finite_differences(dims, cplx):
    rng = np.random.default_rng(len(dims) * 11 + sum(dims))
    d = oracle.d_of(dims)

    def r(shape):
        v = rng.standard_normal(shape)
        return v + 1j * rng.standard_normal(shape) if cplx else v

    h = r(d)
    xs = [r(n) for n in dims[1:]]
    t = r(dims[0])
    y = oracle.brute_y(h, xs, dims)
    _, g = loss_and_g(y, t)
    gh, gxs = oracle.brute_grads(h, xs, dims, g)
    fh = fd_grad(lambda hv: loss_and_g(oracle.brute_y(hv, xs, dims), t)[0], h)
    np.testing.assert_allclose(gh if cplx else gh.real, fh, rtol=1e-6, atol=1e-6)
    for p in range(len(xs)):
        def f(xv, p=p):
            xx = list(xs)
            xx[p] = xv
            return loss_and_g(oracle.brute_y(h, xx, dims), t)[0]
        np.testing.assert_allclose(gxs[p] if cplx else gxs[p].real, fd_grad(f, xs[p]), rtol=1e-6, atol=1e-6)
    # FFT form agrees with the explicit-tensor form
    fgh, fgxs = oracle.fast_grads(h, xs, dims, g)
    np.testing.assert_allclose(fgh, gh, atol=1e-11)
    for a, b in zip(fgxs, gxs):
        np.testing.assert_allclose(a, b, atol=1e-11)


def test_same_x_grad_and_euler_identity():
    # one x in all modes: grad_x = sum_p grad_x_p; y is homogeneous of
    # degree m-1 in x, so <grad_x(r), x> = (m-1) <r, y>
    rng = np.random.default_rng(3)
    m, n = 4, 6
    dims = [n] * m
    h = rng.standard_normal(oracle.d_of(dims))
    x = rng.standard_normal(n)
    r = rng.standard_normal(n)
    y = oracle.fast_y(h, [x] * (m - 1), dims).real
    _, gxs = oracle.fast_grads(h, [x] * (m - 1), dims, r)
    gx = sum(g.real for g in gxs)
    np.testing.assert_allclose(gx @ x, (m - 1) * (r @ y), rtol=1e-11)
    f = lambda xv: r @ oracle.fast_y(h, [xv] * (m - 1), dims).real
    np.testing.assert_allclose(gx, fd_grad(f, x), rtol=1e-6, atol=1e-7)


def test_adjoint_identity_in_h():
    # y is linear in h: <r, y(dh)> = <grad_h(r), dh>
    rng = np.random.default_rng(4)
    dims = [7, 5, 6]
    d = oracle.d_of(dims)
    xs = [rng.standard_normal(n) for n in dims[1:]]
    r = rng.standard_normal(dims[0])
    dh = rng.standard_normal(d)
    gh, _ = oracle.fast_grads(rng.standard_normal(d), xs, dims, r)
    np.testing.assert_allclose(r @ oracle.fast_y(dh, xs, dims).real, gh.real @ dh, rtol=1e-11)


@pytest.mark.parametrize("n,N", [([2, 3, 2], [3, 2, 2]), ([2, 2], [3, 3])])
def test_block_grads_match_finite_differences(n, N):
    rng = np.random.default_rng(sum(n) * 5 + sum(N))
    m = len(n)

    def r(shape):
        return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)

    Hgen = r((sum(n) - m + 1, sum(N) - m + 1))
    Xs = [r((n[p], N[p])) for p in range(1, m)]
    T = r((n[0], N[0]))
    _, G = loss_and_g(oracle.brute_block_y(Hgen, Xs, n, N), T)
    gH, gXs = oracle.brute_block_grads(Hgen, Xs, n, N, G)
    fH = fd_grad(lambda Hv: loss_and_g(oracle.brute_block_y(Hv, Xs, n, N), T)[0], Hgen)
    np.testing.assert_allclose(gH, fH, rtol=1e-6, atol=1e-6)
    for p in range(m - 1):
        def f(Xv, p=p):
            XX = list(Xs)
            XX[p] = Xv
            return loss_and_g(oracle.brute_block_y(Hgen, XX, n, N), T)[0]
        np.testing.assert_allclose(gXs[p], fd_grad(f, Xs[p]), rtol=1e-6, atol=1e-6)
    fgH, fgXs = oracle.fast_block_grads(Hgen, Xs, n, N, G)
    np.testing.assert_allclose(fgH, gH, atol=1e-10)
    for a, b in zip(fgXs, gXs):
        np.testing.assert_allclose(a, b, atol=1e-10)
