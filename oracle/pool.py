"""The oracle's fast products over a whole batch of square tensors, spread
over worker processes.  TEST INFRASTRUCTURE ONLY (see the package header):
used by the parity tests and by the CPU-baseline leg of the benchmark.

Each worker computes y = H x^{m-1} by ``hankel.fast_y`` (Section 3, the
product for y) for a slice of the batch.  The pool is started with the
``spawn`` method, so that it is safe to use after the parent process has
initialised a GPU.
"""

import multiprocessing as mp
import os

import numpy as np

from .hankel import fast_y


def _square_refs(task):
    """y (real part) for each (m, n, h, x) of one slice."""
    return [fast_y(h, [x] * (m - 1), [n] * m).real for m, n, h, x in task]


def square_refs(tensors, procs=None):
    """Oracle outputs for a list of (m, n, h, x) tuples, in order.

    procs: worker processes (default: the host's CPU count); 1 runs in this
    process.
    """
    tensors = list(tensors)
    procs = procs or os.cpu_count() or 1
    if procs <= 1 or len(tensors) < 2:
        return _square_refs(tensors)
    chunk = max(1, (len(tensors) + 4 * procs - 1) // (4 * procs))
    tasks = [tensors[i: i + chunk] for i in range(0, len(tensors), chunk)]
    with mp.get_context("spawn").Pool(processes=min(procs, len(tasks))) as pool:
        parts = pool.map(_square_refs, tasks)
    return [y for part in parts for y in part]


def relative_errors(batch, y, refs):
    """Per-tensor ||y_i - ref_i||_inf / ||ref_i||_inf for a workloads.Batch."""
    out = np.empty(len(batch))
    for i, ref in enumerate(refs):
        n = int(batch.dims[i])
        got = np.asarray(y[batch.y_off[i]: batch.y_off[i] + n], dtype=np.float64)
        out[i] = np.max(np.abs(got - ref)) / np.max(np.abs(ref))
    return out
