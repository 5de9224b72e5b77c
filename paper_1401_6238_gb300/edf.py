"""Exponential data fitting on the GPU (Section 4), driven by the library's
batched Hankel tensor-vector products.

A signal x_n = sum_k c_k z_k^n (Section 4.1) or x_{n1 n2} = sum_k c_k
z_{1,k}^{n1} z_{2,k}^{n2} (Section 4.3) is arranged as an order-m Hankel
tensor (generating vector x) or a two-level block Hankel tensor (BHHB,
generating matrix x).  Its best rank-(R_1..R_m) approximation by HOOI
(Algorithm 4.1; Algorithm 4.2 for square tensors, one factor U in every
mode) gives factor columns whose shift invariance yields the poles.

What runs where:

* The tensor-matrix products of each mode update,
  (A x_q conj(U_q) for q != p)_{:, i..} = A x_q conj(u_{q,i}) ...  (Section
  4.2), are one batch of Hankel (or BHHB) tensor-vector products in
  libhankel.so.  One plan per mode is made once; every sweep rewrites the
  conjugated factor columns in place and replays it.
* The initial factors come from the mode-p unfolding reduced to its
  distinct columns, the I_p x (d - I_p + 1) Hankel matrix of Section 4.2
  (for a BHHB tensor the analogous two-level Hankel matrix).  That matrix is
  itself an order-2 Hankel (BHHB) tensor, so a randomized range finder with
  power iterations applies it and its adjoint through the same library.
* The small dense linear algebra -- leading left singular vectors of the
  I_p x (R^{m-1}) unfolding (QR on the device, then the SVD of the small
  triangular factor), the core tensor, the total-least-squares shift
  equations -- runs in torch.linalg; the small SVDs and the K x K
  eigenproblems that give the poles run on the host.

For a square tensor with one factor (Algorithm 4.2) the unfolding's columns
for index tuples that are permutations of one another are equal (the tensor
is symmetric), so only sorted tuples are computed and each column is scaled
by the square root of its multiplicity: the scaled matrix has the same
Gram matrix M M^H, hence the same left singular vectors and values.
"""

import itertools
import math

import numpy as np
import torch

from . import hankel as hk

_CDTYPE = {hk.C64: torch.complex64, hk.C128: torch.complex128}


def hankel_dims(N, m=3):
    """Mode sizes I_1 >= ... >= I_m, as equal as possible, of the order-m
    Hankel tensor of an N-sample signal (sum I_p - m + 1 = N)."""
    total = N + m - 1
    base, extra = divmod(total, m)
    return [base + 1] * extra + [base] * (m - extra)


def _batch_plan(n, N, xoffs, ylen, dtype, block):
    """A plan of len(xoffs) products of one order-len(n) tensor shape: product
    k reads x_q at xoffs[k][q-2] (q = 2..m) and writes y at k * ylen."""
    T, m = len(xoffs), len(n)
    d = hk.make_descs(T)
    d["m"] = m
    d["n"][:, :m] = n
    d["N"][:, :m] = N if block else 1
    d["h_off"] = 0
    d["x_off"][:, 1:m] = np.asarray(xoffs, dtype=np.int64).reshape(T, m - 1)
    d["y_off"] = np.arange(T, dtype=np.int64) * ylen
    return hk.Plan(d, dtype, hk.BLOCK if block else 0)


HOST_SVD_MAX = 256  # triangular factors up to this order are decomposed on the host


def leading_left(M, R):
    """R leading left singular vectors and the singular values of M.

    A tall M is reduced by a Householder QR on the device; the small
    triangular factor's SVD runs in complex128 LAPACK on the host when its
    order is at most HOST_SVD_MAX (on the device it costs milliseconds for
    the strongly graded factors HOOI produces), on the device otherwise."""
    rows, cols = M.shape
    if cols <= rows:
        Q, T = torch.linalg.qr(M)
        if cols <= HOST_SVD_MAX:
            W, s, _ = np.linalg.svd(T.to(torch.complex128).cpu().numpy())
            return Q @ torch.from_numpy(W[:, :R]).to(device=M.device, dtype=M.dtype), torch.from_numpy(s)
        W, s, _ = torch.linalg.svd(T)
        return Q @ W[:, :R], s
    U, s, _ = torch.linalg.svd(M, full_matrices=False)
    return U[:, :R], s


class HankelTensor:
    """An order-m Hankel tensor (``blocks`` None) or BHHB tensor on the device.

    ``gen`` is the generating vector (length d = sum I_p - m + 1) or the
    generating matrix (sum n_p - m + 1) x (sum N_p - m + 1); ``dims`` are
    I_p, or for a BHHB tensor the block sizes n_p, with ``blocks`` the block
    counts N_p.  Mode p has size I_p, or n_p N_p with index i + n_p j.
    """

    def __init__(self, gen, dims, blocks=None, dtype=hk.C64, device=None):
        self.dtype = int(dtype)
        self.tdtype = _CDTYPE[self.dtype]
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.dims = [int(v) for v in dims]
        self.m = len(self.dims)
        self.block = blocks is not None
        self.blocks = [int(v) for v in blocks] if self.block else [1] * self.m
        self.d = sum(self.dims) - self.m + 1
        self.D = sum(self.blocks) - self.m + 1
        g = torch.as_tensor(gen)
        if self.block:
            if tuple(g.shape) != (self.d, self.D):
                raise ValueError("generating matrix must be %d x %d" % (self.d, self.D))
            g = g.T.reshape(-1)  # column-major
        elif tuple(g.shape) != (self.d,):
            raise ValueError("generating vector must have length %d" % self.d)
        self.h = g.to(device=self.device, dtype=self.tdtype).contiguous()
        self.sizes = [n * N for n, N in zip(self.dims, self.blocks)]

    def plan(self, n, N, xoffs, ylen):
        return _batch_plan(n, N, xoffs, ylen, self.dtype, self.block)

    def run(self, plan, X, Y):
        if self.block:
            plan.txv_block(self.h, X, Y)
        else:
            plan.txv(self.h, X, Y)

    def reduced_columns(self, p):
        """(d - I_p + 1, D - N_p + 1): the reduced mode-p unfolding (Section
        4.2) has their product as its number of columns."""
        return self.d - self.dims[p] + 1, self.D - self.blocks[p] + 1

    def unfolding_matrix_ops(self, p, cols):
        """Plans applying the reduced mode-p unfolding M (Section 4.2) and its
        transpose to ``cols`` columns: M is the order-2 Hankel (BHHB) tensor
        with the same generating data and sizes (I_p, d - I_p + 1)."""
        n2, N2 = self.reduced_columns(p)
        inner = n2 * N2
        fwd = self.plan([self.dims[p], n2], [self.blocks[p], N2], [[c * inner] for c in range(cols)], self.sizes[p])
        adj = self.plan([n2, self.dims[p]], [N2, self.blocks[p]], [[c * self.sizes[p]] for c in range(cols)], inner)
        return fwd, adj


def _cols(buf, count, length):
    """Columns stored one after another in a flat buffer, as a length x count view."""
    return buf[: count * length].view(count, length).T


def range_finder(T, p, R, oversample=8, power_iters=2, seed=0):
    """R leading left singular vectors of the reduced mode-p unfolding of T
    (Section 4.2) by a randomized range finder with power iterations; every
    product with the Hankel matrix or its adjoint is a library call."""
    size = T.sizes[p]
    n2, N2 = T.reduced_columns(p)
    inner = n2 * N2
    k = min(R + oversample, size, inner)
    fwd, adj = T.unfolding_matrix_ops(p, k)
    dev, dt = T.device, T.tdtype
    rng = np.random.default_rng(seed)
    om = (rng.standard_normal((k, inner)) + 1j * rng.standard_normal((k, inner))) / math.sqrt(2.0)
    Xin = torch.zeros(k * max(inner, size), dtype=dt, device=dev)
    Xin[: k * inner].copy_(torch.as_tensor(om.reshape(-1), dtype=dt))
    Yout = torch.zeros(k * max(inner, size), dtype=dt, device=dev)

    def apply_M(Z):  # Z: inner x k  ->  size x k
        Xin[: k * inner].view(k, inner).copy_(Z.T)
        T.run(fwd, Xin, Yout)
        return _cols(Yout, k, size).clone()

    def apply_MH(Qm):  # Qm: size x k  ->  inner x k, M^H q = conj(M^T conj(q))
        Xin[: k * size].view(k, size).copy_(Qm.T.conj())
        T.run(adj, Xin, Yout)
        return _cols(Yout, k, inner).conj()

    Q = torch.linalg.qr(apply_M(_cols(Xin, k, inner).clone()))[0]
    for _ in range(power_iters):
        Z = torch.linalg.qr(apply_MH(Q))[0]
        Q = torch.linalg.qr(apply_M(Z))[0]
    # B = Q^H M; with B^H = Q2 T2 and T2 = W S V^H, B = V S (Q2 W)^H, so the
    # left singular vectors of M ~ Q B are Q V
    _, T2 = torch.linalg.qr(apply_MH(Q))
    _, s, Vh = np.linalg.svd(T2.to(torch.complex128).cpu().numpy())
    fwd.close()
    adj.close()
    return Q @ torch.from_numpy(Vh.conj().T[:, :R]).to(device=dev, dtype=dt), torch.from_numpy(s)


class HOOI:
    """Best rank-(R_1..R_m) approximation of a Hankel / BHHB tensor by HOOI.

    ``symmetric=False``: Algorithm 4.1, one factor per mode, modes updated in
    turn.  ``symmetric=True``: Algorithm 4.2 for a square tensor, one factor
    U shared by all modes.  ``U[p]`` holds the current factors (I_p x R_p,
    orthonormal columns); ``svals[p]`` the singular values of the last
    unfolding of mode p.
    """

    def __init__(self, T, ranks, symmetric=False):
        self.T = T
        m = T.m
        self.ranks = [int(ranks)] * m if np.isscalar(ranks) else [int(r) for r in ranks]
        self.symmetric = bool(symmetric)
        if self.symmetric and (len(set(T.dims)) != 1 or len(set(T.blocks)) != 1 or len(set(self.ranks)) != 1):
            raise ValueError("Algorithm 4.2 needs a square tensor and one rank")
        nf = 1 if self.symmetric else m
        # conjugated factor columns, mode after mode: conj(U_q)^T, flat
        self.base = [0] * nf
        for q in range(1, nf):
            self.base[q] = self.base[q - 1] + self.ranks[q - 1] * T.sizes[q - 1]
        total = self.base[-1] + self.ranks[nf - 1] * T.sizes[nf - 1]
        self.X = torch.zeros(total, dtype=T.tdtype, device=T.device)
        self.U = [None] * m
        self.svals = [None] * m
        self.plans, self.Y, self.weights = {}, {}, {}
        for p in range(nf):
            self._make_mode_plan(p)
        self._core_plan = None

    def _factor(self, q):
        return 0 if self.symmetric else q

    def _tuples(self, p, full=False):
        others = [q for q in range(self.T.m) if q != p]
        if self.symmetric and not full:
            tups = list(itertools.combinations_with_replacement(range(self.ranks[0]), self.T.m - 1))
            w = []
            for t in tups:
                c = math.factorial(len(t))
                for v in set(t):
                    c //= math.factorial(t.count(v))
                w.append(math.sqrt(c))
            return others, tups, w
        tups = list(itertools.product(*[range(self.ranks[q]) for q in others]))
        return others, tups, None

    def _offsets(self, others, tups):
        T = self.T
        return [[self.base[self._factor(q)] + i * T.sizes[q] for q, i in zip(others, t)] for t in tups]

    def _mode_plan(self, p, full=False):
        T = self.T
        others, tups, w = self._tuples(p, full)
        plan = T.plan([T.dims[p]] + [T.dims[q] for q in others], [T.blocks[p]] + [T.blocks[q] for q in others],
                      self._offsets(others, tups), T.sizes[p])
        Y = torch.zeros(len(tups) * T.sizes[p], dtype=T.tdtype, device=T.device)
        wt = None if w is None else torch.tensor(w, dtype=T.tdtype, device=T.device)
        return plan, Y, wt, tups

    def _make_mode_plan(self, p):
        self.plans[p], self.Y[p], self.weights[p], _ = self._mode_plan(p)

    def set_factor(self, p, U):
        """Install U (I_p x R_p) as the factor of mode p."""
        T, q = self.T, self._factor(p)
        U = U.to(device=T.device, dtype=T.tdtype)
        r = self.ranks[p]
        self.X[self.base[q]: self.base[q] + r * T.sizes[p]].view(r, T.sizes[p]).copy_(U[:, :r].T.conj())
        for pp in range(T.m):
            if self._factor(pp) == q:
                self.U[pp] = U[:, :r]

    def init(self, oversample=8, power_iters=2, seed=0):
        """Initial factors from the reduced unfoldings (Section 4.2)."""
        T = self.T
        done = {}
        for p in range(1 if self.symmetric else T.m):
            key = (T.dims[p], T.blocks[p], self.ranks[p])
            if key not in done:
                done[key] = range_finder(T, p, self.ranks[p], oversample, power_iters, seed + p)[0]
            self.set_factor(p, done[key])
        return self

    def products(self, p):
        """Unfold_p(A x_q conj(U_q), q != p), scaled columns for Algorithm 4.2."""
        T = self.T
        plan, Y = self.plans[p], self.Y[p]
        T.run(plan, self.X, Y)
        M = _cols(Y, Y.numel() // T.sizes[p], T.sizes[p])
        if self.weights[p] is not None:
            M = M * self.weights[p][None, :]
        return M

    def update(self, p):
        """One mode update of Algorithm 4.1 (or the update of Algorithm 4.2)."""
        U, s = leading_left(self.products(p), self.ranks[p])
        self.set_factor(p, U)
        self.svals[p] = s
        if self.symmetric:
            self.svals = [s] * self.T.m
        return s

    def sweep(self):
        """One pass over the modes; returns ||S||_F of the resulting core,
        the norm of the R_p leading singular values of the last unfolding."""
        s = None
        for p in range(1 if self.symmetric else self.T.m):
            s = self.update(p)
        last = 0 if self.symmetric else self.T.m - 1
        return float(torch.linalg.vector_norm(s[: self.ranks[last]]))

    def fit(self, sweeps, tol=None):
        """Up to ``sweeps`` sweeps; with ``tol`` stop once the core norm
        changes by less than tol (relative).  Returns the core norms."""
        norms = []
        for _ in range(sweeps):
            norms.append(self.sweep())
            if tol is not None and len(norms) > 1 and abs(norms[-1] - norms[-2]) <= tol * norms[-1]:
                break
        return norms

    def core(self):
        """S = A x_1 conj(U_1) ... x_m conj(U_m), shape (R_1, ..., R_m)."""
        if self._core_plan is None:
            self._core_plan = self._mode_plan(0, full=True)
        plan, Y, _, tups = self._core_plan
        self.T.run(plan, self.X, Y)
        M = _cols(Y, len(tups), self.T.sizes[0])
        return (self.U[0].mH @ M).reshape(self.ranks)

    def close(self):
        for plan in self.plans.values():
            plan.close()
        if self._core_plan is not None:
            self._core_plan[0].close()


# ------------------------------------------------------------- poles

def tls(A, B):
    """Total least squares W with A W ~ B: with [A B] = P S V^H and V split
    in K x K blocks, W = -V_12 V_22^{-1}."""
    K = A.shape[1]
    _, _, Vh = torch.linalg.svd(torch.cat([A, B], dim=1), full_matrices=False)
    V = Vh.mH
    return -V[:K, K:] @ torch.linalg.inv(V[K:, K:])


def poles_1d(U, K):
    """Poles z_k of Section 4.1: U's first K columns satisfy U_up W = U_down
    (rows 0..I-2 and 1..I-1); eig(W) are the poles."""
    U = U[:, :K].to(torch.complex128)
    W = tls(U[:-1], U[1:])
    return torch.linalg.eigvals(W.cpu())


def shift_rows_2d(I, J, device=None):
    """Row sets of the shift operators of Section 4.3 on a factor whose row
    index is i + I j: within a block (i -> i+1) and across blocks (j -> j+1)."""
    i = torch.arange(I - 1, device=device)
    j = torch.arange(J, device=device)
    up1 = (i[None, :] + I * j[:, None]).reshape(-1)
    up2 = torch.arange((J - 1) * I, device=device)
    return up1, up1 + 1, up2, up2 + I


def poles_2d(U, I, J, K):
    """(z_1, z_2) pole pairs of Section 4.3 from the two shift invariances,
    each solved by total least squares; z_2 is paired with z_1 by expressing
    W_2 in the eigenvector basis of W_1."""
    U = U[:, :K].to(torch.complex128)
    up1, down1, up2, down2 = shift_rows_2d(I, J, U.device)
    W1 = tls(U[up1], U[down1]).cpu()
    W2 = tls(U[up2], U[down2]).cpu()
    z1, E = torch.linalg.eig(W1)
    z2 = torch.diagonal(torch.linalg.solve(E, W2 @ E))
    return z1, z2


def fit_1d(signal, K, R=None, m=3, sweeps=10, dtype=hk.C64, symmetric=None, tol=None, **init):
    """Poles of a 1D signal (Section 4.1): order-m Hankel tensor, HOOI
    (Algorithm 4.2 when the tensor is square), TLS on the mode-1 factor."""
    dims = hankel_dims(len(signal), m)
    T = HankelTensor(np.asarray(signal), dims, dtype=dtype)
    if symmetric is None:
        symmetric = len(set(dims)) == 1
    h = HOOI(T, R or K, symmetric=symmetric).init(**init)
    norms = h.fit(sweeps, tol)
    z = poles_1d(h.U[0], K)
    h.close()
    return z, norms


def fit_2d(signal, I, J, K, R=None, sweeps=10, dtype=hk.C64, tol=None, **init):
    """Pole pairs of a 2D signal of size (3I-2) x (3J-2) (Section 4.3):
    order-3 BHHB tensor with blocks I x I x I, J blocks per mode, Algorithm
    4.2, then the two shift-invariance TLS problems."""
    T = HankelTensor(np.asarray(signal), [I] * 3, [J] * 3, dtype=dtype)
    h = HOOI(T, R or K, symmetric=True).init(**init)
    norms = h.fit(sweeps, tol)
    z = poles_2d(h.U[0], I, J, K)
    h.close()
    return z, norms
