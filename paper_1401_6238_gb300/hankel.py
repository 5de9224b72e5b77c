"""Thin Python binding of the C ABI in include/hankel.h (libhankel.so).

Argument marshalling only: every step of the products runs in the library's
CUDA kernels.  The functions ``hankel_plan``, ``hankel_txv``,
``hankel_txv_host``, ``hankel_txv_block``, ``hankel_txv_backward``,
``hankel_plan_multilevel``,
``hankel_plan_query``, ``hankel_plan_destroy`` and ``hankel_last_error``
mirror the C entry points one to one; ``Plan`` and ``HankelTxV`` (a
``torch.autograd.Function``) are conveniences built on them.

Buffers are torch tensors (device memory for the compute calls, host memory
for ``hankel_txv_host``) or raw integer addresses.  The library is loaded on
first use and a missing or unloadable library raises ``HankelError``: there
is no fallback implementation.
"""

import ctypes
import os

import numpy as np

MAX_ORDER = 8

OK, EINVAL, ENOMEM, ECUDA, EUNSUPPORTED, ETIMEOUT = range(6)
R32, C64, R64, C128 = range(4)
SAME_X, FP64_POWER, STORE_SPECTRA, BLOCK, ONE_PER_LAUNCH, ANTICIRCULANT = 1, 2, 4, 8, 16, 32

STATUS_NAMES = {OK: "HANKEL_OK", EINVAL: "HANKEL_EINVAL", ENOMEM: "HANKEL_ENOMEM", ECUDA: "HANKEL_ECUDA",
                EUNSUPPORTED: "HANKEL_EUNSUPPORTED", ETIMEOUT: "HANKEL_ETIMEOUT"}

# Mirror of struct hankel_desc (natural C alignment).
DESC_DTYPE = np.dtype([("m", np.int32), ("n", np.int32, (MAX_ORDER,)), ("N", np.int32, (MAX_ORDER,)),
                       ("h_off", np.int64), ("x_off", np.int64, (MAX_ORDER,)), ("y_off", np.int64)], align=True)
# Mirror of struct hankel_mdesc (level-k block Hankel tensors).
MAX_LEVELS = 4
MDESC_DTYPE = np.dtype([("m", np.int32), ("levels", np.int32), ("n", np.int32, (MAX_LEVELS, MAX_ORDER)),
                        ("h_off", np.int64), ("x_off", np.int64, (MAX_ORDER,)), ("y_off", np.int64)], align=True)


class PlanInfo(ctypes.Structure):
    _fields_ = [(name, ctypes.c_int64) for name in
                ("count", "jobs", "launches", "distinct_lengths", "max_length", "sum_length", "workspace_bytes",
                 "h_elems", "x_elems", "y_elems", "fp64_power_tensors", "backward_launches")]

    def as_dict(self):
        return {f[0]: getattr(self, f[0]) for f in self._fields_}


class HankelError(RuntimeError):
    def __init__(self, status, message):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), message))
        self.status = status
        self.message = message


LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libhankel.so")
_lib = None

_SIGS = {
    "hankel_plan": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.c_void_p, ctypes.c_int64, ctypes.c_int,
                                   ctypes.c_uint32]),
    "hankel_plan_multilevel": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.c_void_p, ctypes.c_int64,
                                              ctypes.c_int, ctypes.c_uint32]),
    "hankel_txv": (ctypes.c_int, [ctypes.c_void_p] * 6),
    "hankel_txv_host": (ctypes.c_int, [ctypes.c_void_p] * 6),
    "hankel_txv_block": (ctypes.c_int, [ctypes.c_void_p] * 6),
    "hankel_txv_backward": (ctypes.c_int, [ctypes.c_void_p] * 7),
    "hankel_txv_backward_static": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int] +
                                   [ctypes.c_void_p] * 6),
    "hankel_plan_query": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(PlanInfo)]),
    "hankel_fft_length": (ctypes.c_int64, [ctypes.c_int64]),
    "hankel_set_tuning": (ctypes.c_int, [ctypes.c_double, ctypes.c_int]),
    "hankel_get_tuning": (ctypes.c_int, [ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int)]),
    "hankel_set_bin_policy": (ctypes.c_int, [ctypes.c_int32] + [ctypes.POINTER(ctypes.c_int32)] * 3),
    "hankel_get_bin_policy": (ctypes.c_int, [ctypes.c_int32] + [ctypes.POINTER(ctypes.c_int32)] * 2),
    "hankel_plan_destroy": (None, [ctypes.c_void_p]),
    "hankel_last_error": (ctypes.c_char_p, []),
    "hankel_version": (ctypes.c_char_p, []),
}


def load():
    """Load libhankel.so (after torch, so both share one CUDA runtime)."""
    global _lib
    if _lib is None:
        import torch  # noqa: F401  (loads the CUDA runtime first)
        if not os.path.exists(LIB_PATH):
            raise HankelError(EUNSUPPORTED, "libhankel.so is not built (run __graft_entry__.build())")
        try:
            lib = ctypes.CDLL(LIB_PATH)
        except OSError as e:
            raise HankelError(EUNSUPPORTED, "cannot load %s: %s" % (LIB_PATH, e))
        for name, (res, args) in _SIGS.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        _apply_cached_tuning()
    return _lib


TUNING_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "autotune.json")


def _apply_cached_tuning():
    """Apply the autotuner's cached choice for this device, if there is one."""
    try:
        import json
        import torch
        if not os.path.exists(TUNING_PATH) or not torch.cuda.is_available():
            return
        rec = json.load(open(TUNING_PATH))
        if rec.get("device") == torch.cuda.get_device_name():
            best = rec["best"]
            _lib.hankel_set_tuning(float(best["pass_cost"]), int(best["points_per_thread"]))
            bins = {int(b["L"]): (int(b["path"]), int(b["fp64_from_m"])) for b in rec.get("bins", [])}
            if bins:
                hankel_set_bin_policy(bins)
    except Exception:
        pass


def _check(status):
    if status != OK:
        raise HankelError(status, load().hankel_last_error().decode())


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, int):
        return t
    if isinstance(t, np.ndarray):
        return t.ctypes.data
    return t.data_ptr()


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


# ------------------------------------------------------------- C ABI mirror

def hankel_plan(descs, dtype, flags=0):
    """Make a plan from a DESC_DTYPE array; returns the opaque handle."""
    descs = np.ascontiguousarray(descs, dtype=DESC_DTYPE)
    h = ctypes.c_void_p()
    _check(load().hankel_plan(ctypes.byref(h), descs.ctypes.data, descs.shape[0], int(dtype), int(flags)))
    return h.value


def hankel_plan_multilevel(descs, dtype, flags=0):
    """Make a plan for level-k block Hankel tensors from an MDESC_DTYPE array."""
    descs = np.ascontiguousarray(descs, dtype=MDESC_DTYPE)
    h = ctypes.c_void_p()
    _check(load().hankel_plan_multilevel(ctypes.byref(h), descs.ctypes.data, descs.shape[0], int(dtype), int(flags)))
    return h.value


def hankel_txv(plan, h, x, y, alpha, stream=None):
    _check(load().hankel_txv(plan, _ptr(h), _ptr(x), _ptr(y), _ptr(alpha), _stream(stream)))


def hankel_txv_host(plan, h, x, y, alpha, stream=None):
    _check(load().hankel_txv_host(plan, _ptr(h), _ptr(x), _ptr(y), _ptr(alpha), _stream(stream)))


def hankel_txv_block(plan, H, X, Y, alpha, stream=None):
    _check(load().hankel_txv_block(plan, _ptr(H), _ptr(X), _ptr(Y), _ptr(alpha), _stream(stream)))


def hankel_txv_backward(plan, grad_y, h, x, grad_h, grad_x, stream=None):
    _check(load().hankel_txv_backward(plan, _ptr(grad_y), _ptr(h), _ptr(x), _ptr(grad_h), _ptr(grad_x),
                                      _stream(stream)))


STATIC_SCRATCH_BYTES = 16 << 20


def hankel_txv_backward_static(descs, dtype, grad_y, h, x, grad_h, grad_x, stream=None):
    """Gradients of the real one-vector product without any device
    allocation: the scratch is a static device array of STATIC_SCRATCH_BYTES
    shared by every call (see include/hankel.h)."""
    descs = np.ascontiguousarray(descs, dtype=DESC_DTYPE)
    _check(load().hankel_txv_backward_static(descs.ctypes.data, descs.shape[0], int(dtype), _ptr(grad_y), _ptr(h),
                                             _ptr(x), _ptr(grad_h), _ptr(grad_x), _stream(stream)))


def hankel_plan_query(plan):
    info = PlanInfo()
    _check(load().hankel_plan_query(plan, ctypes.byref(info)))
    return info.as_dict()


def hankel_fft_length(d):
    return int(load().hankel_fft_length(int(d)))


def hankel_set_tuning(pass_cost, points_per_thread):
    _check(load().hankel_set_tuning(float(pass_cost), int(points_per_thread)))


def hankel_get_tuning():
    c, p = ctypes.c_double(), ctypes.c_int()
    _check(load().hankel_get_tuning(ctypes.byref(c), ctypes.byref(p)))
    return c.value, p.value


def hankel_set_bin_policy(bins):
    """bins: {L: (path, fp64_from_m)} for the persistent kernel's length
    bins; an empty mapping puts every bin back to its default."""
    n = len(bins)
    arr = lambda vals: (ctypes.c_int32 * max(n, 1))(*vals)
    Ls = sorted(bins)
    _check(load().hankel_set_bin_policy(n, arr(Ls), arr([int(bins[L][0]) for L in Ls]),
                                        arr([int(bins[L][1]) for L in Ls])))


def hankel_get_bin_policy(L):
    """(path, fp64_from_m) of length bin L."""
    p, f = ctypes.c_int32(), ctypes.c_int32()
    _check(load().hankel_get_bin_policy(int(L), ctypes.byref(p), ctypes.byref(f)))
    return p.value, f.value


def hankel_plan_destroy(plan):
    if plan:
        load().hankel_plan_destroy(plan)


def hankel_last_error():
    return load().hankel_last_error().decode()


def hankel_version():
    return load().hankel_version().decode()


# ------------------------------------------------------------- conveniences

def make_descs(count):
    return np.zeros(count, dtype=DESC_DTYPE)


def make_mdescs(count):
    return np.zeros(count, dtype=MDESC_DTYPE)


def level_descs(sizes, h_offs, x_offs, y_offs):
    """Level-k descriptors of tensors sharing one shape: ``sizes[l][p]`` is
    the size of mode p+1 at level l+1; ``x_offs[t]`` lists the offsets of
    x_1..x_m of tensor t."""
    k, m = len(sizes), len(sizes[0])
    count = len(h_offs)
    d = make_mdescs(count)
    d["m"] = m
    d["levels"] = k
    for l in range(k):
        d["n"][:, l, :m] = sizes[l]
    d["h_off"] = h_offs
    for t in range(count):
        d["x_off"][t, : len(x_offs[t])] = x_offs[t]
    d["y_off"] = y_offs
    return d


def square_descs(orders, dims, h_off, x_off, y_off):
    """Descriptors of square tensors with one vector each (HANKEL_SAME_X)."""
    orders = np.asarray(orders)
    dims = np.asarray(dims)
    d = make_descs(orders.shape[0])
    d["m"] = orders
    for p in range(MAX_ORDER):
        d["n"][:, p] = np.where(p < orders, dims, 0)
        d["N"][:, p] = np.where(p < orders, 1, 0)
    d["h_off"] = h_off
    d["x_off"][:, 0] = x_off
    d["y_off"] = y_off
    return d


def batch_descs(batch):
    """Descriptors for a ``workloads.Batch``."""
    return square_descs(batch.orders, batch.dims, batch.h_off, batch.x_off, batch.y_off)


_TORCH_DTYPE = {R32: "float32", C64: "complex64", R64: "float64", C128: "complex128"}


class Plan:
    """Owns one library plan; methods take torch tensors."""

    def __init__(self, descs, dtype, flags=0):
        self.dtype = int(dtype)
        self.flags = int(flags)
        if np.asarray(descs).dtype == MDESC_DTYPE:
            self.handle = hankel_plan_multilevel(descs, dtype, flags)
            self.flags |= BLOCK  # level-k plans compute through txv_block
        else:
            self.handle = hankel_plan(descs, dtype, flags)
        self.info = hankel_plan_query(self.handle)

    def torch_dtype(self):
        import torch
        return getattr(torch, _TORCH_DTYPE[self.dtype])

    def _checkt(self, *ts):
        for t in ts:
            if t is None:
                continue
            if t.dtype != self.torch_dtype():
                raise HankelError(EINVAL, "tensor dtype %s does not match the plan (%s)" % (t.dtype, self.torch_dtype()))
            if not t.is_contiguous():
                raise HankelError(EINVAL, "tensors must be contiguous")

    def txv(self, h, x, y=None, alpha=None, stream=None):
        self._checkt(h, x, y, alpha)
        hankel_txv(self.handle, h, x, y, alpha, stream)

    def txv_block(self, H, X, Y=None, alpha=None, stream=None):
        self._checkt(H, X, Y, alpha)
        hankel_txv_block(self.handle, H, X, Y, alpha, stream)

    def txv_host(self, h, x, y=None, alpha=None, stream=None):
        hankel_txv_host(self.handle, h, x, y, alpha, stream)

    def backward(self, grad_y, h, x, grad_h=None, grad_x=None, stream=None):
        self._checkt(grad_y, h, x, grad_h, grad_x)
        hankel_txv_backward(self.handle, grad_y, h, x, grad_h, grad_x, stream)

    def close(self):
        if getattr(self, "handle", None):
            hankel_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _autograd():
    import torch

    class HankelTxV(torch.autograd.Function):
        """y = H x^{m-1} per descriptor, differentiable in h and x.

        forward(h, x, plan) -> y (flat buffer of plan.info['y_elems']); block
        and level-k plans run through txv_block.  The backward runs the
        library's adjoint kernels; with a plan made with STORE_SPECTRA it
        reuses the spectra of the forward call.
        """

        @staticmethod
        def forward(ctx, h, x, plan):
            y = torch.zeros(plan.info["y_elems"], dtype=h.dtype, device=h.device)
            if plan.flags & BLOCK:  # BHHB and level-k plans
                plan.txv_block(h.contiguous(), x.contiguous(), y)
            else:
                plan.txv(h.contiguous(), x.contiguous(), y)
            ctx.save_for_backward(h, x)
            ctx.plan = plan
            return y

        @staticmethod
        def backward(ctx, gy):
            h, x = ctx.saved_tensors
            gh = torch.zeros_like(h) if ctx.needs_input_grad[0] else None
            gx = torch.zeros_like(x) if ctx.needs_input_grad[1] else None
            if gh is not None or gx is not None:
                ctx.plan.backward(gy.contiguous(), h.contiguous(), x.contiguous(), gh, gx)
            return gh, gx, None

    return HankelTxV


_HankelTxV = None


def hankel_txv_autograd(h, x, plan):
    """Differentiable y = H x^{m-1} through ``HankelTxV``."""
    global _HankelTxV
    if _HankelTxV is None:
        _HankelTxV = _autograd()
    return _HankelTxV.apply(h, x, plan)
