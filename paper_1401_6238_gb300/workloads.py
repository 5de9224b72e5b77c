"""Seeded synthetic inputs shaped like the paper's workloads.

This module holds random draws and buffer layout only -- none of the
product's arithmetic -- so that the CUDA path and the FP64 oracle can be fed
identical inputs.  Every generator takes an explicit seed and uses
``numpy.random.default_rng``.

Workloads (the paper publishes no dataset; these stand in for its Example 3.1
products and its Section 4 exponential-data-fitting signals):

* ``plain_case``     -- one square real tensor, m=3, n=64, h and x ~ N(0,1)
  (a Section 3 product of the Example 3.1 kind), plus the Vandermonde
  generator h_k = a^k of the Section 4.1 decomposition.
* ``batched_square`` -- thousands of square real tensors, order m uniform in
  {3,4,5}, dimension n uniform in [16,1024], h ~ N(0, 1/d_H), x a unit-norm
  Gaussian vector; packed into flat buffers with 16-byte aligned segments.
* ``batched_distinct`` -- the same batch shape with a different vector in
  every mode (the y = H x_2 ... x_m and alpha = H x_1 ... x_m products).
* ``grad_case``      -- m=4, n=4096 batch for the gradient checks.
* ``edf_1d_signal`` / ``edf_2d_signal`` -- sums of damped complex
  exponentials plus complex Gaussian noise at a given SNR (Sections 4.1, 4.3).
* ``damped_1d`` / ``damped_2d`` -- noiseless (or lightly noisy) damped
  exponentials with given poles, e.g. the 2-peak signal of Example 4.1.
* ``unit_columns``   -- random complex unit-norm columns standing in for the
  HOOI factor columns of Section 4.2.
* ``edf_3d_signal`` / ``random_arrays`` -- a 3D damped-exponential signal
  (generating tensor of a level-3 block Hankel tensor) and random arrays.
"""

from dataclasses import dataclass, field

import numpy as np

ALIGN = 4  # elements; segment starts are 16-byte aligned for 4-byte reals


def _align(n, a=ALIGN):
    return (n + a - 1) // a * a


def generating_length(dims):
    """Length of the generating vector for mode sizes ``dims`` (Section 1)."""
    return int(sum(dims)) - len(dims) + 1


def plain_case(seed=0, m=3, n=64):
    rng = np.random.default_rng(seed)
    dims = [n] * m
    d = generating_length(dims)
    h = rng.standard_normal(d)
    x = rng.standard_normal(n)
    return dims, h, x


def vandermonde_h(a, d):
    return np.asarray(a, dtype=np.float64) ** np.arange(d)


def integer_case(dims, seed=0, lo=-3, hi=3):
    rng = np.random.default_rng(seed)
    d = generating_length(dims)
    h = rng.integers(lo, hi + 1, size=d).astype(np.float64)
    xs = [rng.integers(lo, hi + 1, size=n).astype(np.float64) for n in dims]
    return h, xs


@dataclass
class Batch:
    """Square real tensors packed in three flat buffers.

    ``orders[i]``, ``dims[i]`` give tensor i; its generating vector is
    ``h[h_off[i] : h_off[i] + d_i]``, its vector ``x[x_off[i] : + n_i]`` and
    its output ``y[y_off[i] : + n_i]``.
    """
    orders: np.ndarray
    dims: np.ndarray
    h: np.ndarray
    x: np.ndarray
    h_off: np.ndarray
    x_off: np.ndarray
    y_off: np.ndarray
    y_len: int
    extra: dict = field(default_factory=dict)

    def __len__(self):
        return int(self.orders.shape[0])

    def tensor(self, i):
        m, n = int(self.orders[i]), int(self.dims[i])
        d = generating_length([n] * m)
        h = self.h[self.h_off[i]: self.h_off[i] + d]
        x = self.x[self.x_off[i]: self.x_off[i] + n]
        return m, n, h, x

    def subset(self, idx):
        """A new Batch holding tensors ``idx`` (re-packed)."""
        parts = [self.tensor(int(i)) for i in idx]
        return pack_square([p[0] for p in parts], [p[1] for p in parts],
                           [p[2] for p in parts], [p[3] for p in parts])


def pack_square(orders, dims, hs, xs, dtype=np.float64):
    h_off, x_off, y_off = [], [], []
    hp = xp = yp = 0
    for m, n, h, x in zip(orders, dims, hs, xs):
        h_off.append(hp)
        x_off.append(xp)
        y_off.append(yp)
        hp += _align(len(h))
        xp += _align(len(x))
        yp += _align(n)
    H = np.zeros(max(hp, 1), dtype=dtype)
    X = np.zeros(max(xp, 1), dtype=dtype)
    for o, h in zip(h_off, hs):
        H[o: o + len(h)] = h
    for o, x in zip(x_off, xs):
        X[o: o + len(x)] = x
    return Batch(np.asarray(orders, np.int32), np.asarray(dims, np.int32), H, X,
                 np.asarray(h_off, np.int64), np.asarray(x_off, np.int64),
                 np.asarray(y_off, np.int64), max(yp, 1))


def batched_square(count=8192, seed=1, orders=(3, 4, 5), n_lo=16, n_hi=1024):
    """``count`` square real tensors: m ~ U(orders), n ~ U[n_lo, n_hi],
    h ~ N(0, 1/d_H), x ~ Gaussian scaled to unit 2-norm."""
    rng = np.random.default_rng(seed)
    ms = rng.choice(np.asarray(orders), size=count)
    ns = rng.integers(n_lo, n_hi + 1, size=count)
    hs, xs = [], []
    for m, n in zip(ms, ns):
        d = generating_length([n] * m)
        hs.append(rng.standard_normal(d) / np.sqrt(d))
        x = rng.standard_normal(n)
        xs.append(x / np.linalg.norm(x))
    return pack_square(ms, ns, hs, xs)


def batched_distinct(count=8192, seed=12, orders=(3, 4, 5), n_lo=16, n_hi=1024):
    """``count`` square real tensors with a different unit-norm vector in
    every mode (x_1 .. x_m; x_1 enters only alpha): m ~ U(orders),
    n ~ U[n_lo, n_hi], h ~ N(0, 1/d).  Returns (Batch, x_offsets) where
    x_offsets[i] lists the m vector offsets of tensor i in ``Batch.x``."""
    rng = np.random.default_rng(seed)
    ms = rng.choice(np.asarray(orders), size=count)
    ns = rng.integers(n_lo, n_hi + 1, size=count)
    hs, xs, xoffs = [], [], []
    xo = 0
    for m, n in zip(ms, ns):
        d = generating_length([n] * m)
        hs.append(rng.standard_normal(d) / np.sqrt(d))
        offs = []
        for _ in range(m):
            x = rng.standard_normal(n)
            xs.append(x / np.linalg.norm(x))
            offs.append(xo)
            xo += _align(n)
        xoffs.append(offs)
    b = pack_square(ms, ns, hs, [np.zeros(1)] * count)
    X = np.zeros(max(xo, 1))
    k = 0
    for offs, n in zip(xoffs, ns):
        for o in offs:
            X[o: o + n] = xs[k]
            k += 1
    b.x = X
    return b, xoffs


def grad_case(batch=64, m=4, n=4096, seed=3, target_scale=0.01):
    """Batch for the gradient checks: square real tensors and targets t."""
    rng = np.random.default_rng(seed)
    d = generating_length([n] * m)
    hs = [rng.standard_normal(d) / np.sqrt(d) for _ in range(batch)]
    xs = []
    for _ in range(batch):
        x = rng.standard_normal(n)
        xs.append(x / np.linalg.norm(x))
    b = pack_square([m] * batch, [n] * batch, hs, xs)
    b.extra["target"] = rng.standard_normal(b.y_len) * target_scale
    return b


def _noise(rng, shape, signal, snr_db):
    p_sig = np.mean(np.abs(signal) ** 2)
    p_noise = p_sig / (10.0 ** (snr_db / 10.0))
    return np.sqrt(p_noise / 2.0) * (rng.standard_normal(shape) + 1j * rng.standard_normal(shape))


def edf_1d_signal(N=4094, K=8, snr_db=20.0, seed=4, with_poles=False):
    """s_t = sum_k a_k e^{i phi_k} exp((-alpha_k + i omega_k) t) + noise
    (the model of Section 4.1 with unit sampling interval); with
    ``with_poles`` also the true poles exp(-alpha_k + i omega_k)."""
    rng = np.random.default_rng(seed)
    alpha = rng.uniform(0.001, 0.05, K)
    omega = rng.uniform(-np.pi, np.pi, K)
    amp = rng.uniform(0.5, 2.0, K)
    phase = rng.uniform(-np.pi, np.pi, K)
    t = np.arange(N)
    s = np.zeros(N, dtype=np.complex128)
    for k in range(K):
        s += amp[k] * np.exp(1j * phase[k]) * np.exp((-alpha[k] + 1j * omega[k]) * t)
    noisy = s + _noise(rng, N, s, snr_db)
    if with_poles:
        return noisy, np.exp(-alpha + 1j * omega)
    return noisy


def edf_2d_signal(N1=256, N2=256, K=12, snr_db=20.0, seed=5, with_poles=False):
    """x_{n1 n2} = sum_k c_k z_{1,k}^{n1} z_{2,k}^{n2} + noise (Section 4.3);
    with ``with_poles`` also the true pole pairs (z_1, z_2)."""
    rng = np.random.default_rng(seed)
    a1 = rng.uniform(0.002, 0.03, K)
    a2 = rng.uniform(0.002, 0.03, K)
    w1 = rng.uniform(-np.pi, np.pi, K)
    w2 = rng.uniform(-np.pi, np.pi, K)
    c = rng.uniform(0.5, 2.0, K) * np.exp(1j * rng.uniform(-np.pi, np.pi, K))
    n1 = np.arange(N1)[:, None]
    n2 = np.arange(N2)[None, :]
    s = np.zeros((N1, N2), dtype=np.complex128)
    for k in range(K):
        s += c[k] * np.exp((-a1[k] + 1j * w1[k]) * n1) * np.exp((-a2[k] + 1j * w2[k]) * n2)
    noisy = s + _noise(rng, (N1, N2), s, snr_db)
    if with_poles:
        return noisy, (np.exp(-a1 + 1j * w1), np.exp(-a2 + 1j * w2))
    return noisy


def damped_2d(N1, N2, peaks, noise_std=0.0, seed=8):
    """x_{n1 n2} = sum_k exp((a_k + 2 pi i f_k) n1) exp((b_k + 2 pi i g_k) n2)
    plus complex Gaussian noise of the given standard deviation; ``peaks`` is
    a list of (a_k, f_k, b_k, g_k) (the 2-peak signal of Section 4.3,
    Example 4.1, takes its parameters from the paper)."""
    n1 = np.arange(N1)[:, None]
    n2 = np.arange(N2)[None, :]
    x = np.zeros((N1, N2), dtype=np.complex128)
    for a, f, b, g in peaks:
        x += np.exp((a + 2j * np.pi * f) * n1) * np.exp((b + 2j * np.pi * g) * n2)
    if noise_std > 0:
        rng = np.random.default_rng(seed)
        x += noise_std * (rng.standard_normal(x.shape) + 1j * rng.standard_normal(x.shape)) / np.sqrt(2)
    return x


def damped_1d(N, poles, amps, noise_std=0.0, seed=9):
    """x_n = sum_k c_k z_k^n plus complex Gaussian noise (Section 4.1)."""
    n = np.arange(N)
    x = np.zeros(N, dtype=np.complex128)
    for z, c in zip(poles, amps):
        x += c * np.asarray(z, dtype=np.complex128) ** n
    if noise_std > 0:
        rng = np.random.default_rng(seed)
        x += noise_std * (rng.standard_normal(N) + 1j * rng.standard_normal(N)) / np.sqrt(2)
    return x


def unit_columns(n, R, seed=6):
    """R random complex columns of length n, each of unit 2-norm."""
    rng = np.random.default_rng(seed)
    U = rng.standard_normal((n, R)) + 1j * rng.standard_normal((n, R))
    return U / np.linalg.norm(U, axis=0, keepdims=True)


def unit_matrices(count, n, N, seed=7):
    """``count`` random complex n x N matrices of unit Frobenius norm."""
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((count, n, N)) + 1j * rng.standard_normal((count, n, N))
    return X / np.linalg.norm(X.reshape(count, -1), axis=1)[:, None, None]


def edf_3d_signal(shape=(64, 64, 64), K=6, snr_db=20.0, seed=10):
    """x_{n1 n2 n3} = sum_k c_k z_{1,k}^{n1} z_{2,k}^{n2} z_{3,k}^{n3} + noise:
    the three-dimensional analogue of the Section 4.3 signal, generating
    tensor of a level-3 block Hankel tensor (Section 2.2)."""
    rng = np.random.default_rng(seed)
    s = np.zeros(shape, dtype=np.complex128)
    axes = [np.arange(n) for n in shape]
    for _ in range(K):
        c = rng.uniform(0.5, 2.0) * np.exp(1j * rng.uniform(-np.pi, np.pi))
        term = np.asarray(c, dtype=np.complex128)
        for ax, t in enumerate(axes):
            z = np.exp(-rng.uniform(0.002, 0.03) + 1j * rng.uniform(-np.pi, np.pi))
            sh = [1] * len(shape)
            sh[ax] = shape[ax]
            term = term * (z ** t).reshape(sh)
        s += term
    return s + _noise(rng, shape, s, snr_db)


def random_arrays(count, shape, seed=11, complex_=True):
    """``count`` random arrays of the given shape with unit Frobenius norm."""
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((count,) + tuple(shape))
    if complex_:
        X = X + 1j * rng.standard_normal((count,) + tuple(shape))
    return X / np.linalg.norm(X.reshape(count, -1), axis=1).reshape((count,) + (1,) * len(shape))
