"""hankel_txv inside a CUDA graph, captured once and replayed: the benchmark's
shape mix as its one persistent launch (whose work counter re-arms itself
at the end of every launch), and a batch with tensors longer than the
persistent kernel's lengths, whose extra launches fork over the plan's
streams and join back with events.  Replays on new inputs give the same
bits as direct calls."""

import numpy as np
import pytest

from paper_1401_6238_gb300 import hankel as hk
from paper_1401_6238_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    hk.load()
    return torch.device("cuda:0")


@pytest.mark.parametrize("n_hi,launches", [(1024, 1), (2000, 2)])
def test_capture_and_replay(dev, n_hi, launches):
    # n <= 1024, m <= 5: d <= 5116, one persistent launch; n up to 2000
    # reaches d > 5120, which adds the per-length launches
    b = wl.batched_square(count=300, seed=17, n_lo=16, n_hi=n_hi)
    plan = hk.Plan(hk.batch_descs(b), hk.R32, hk.SAME_X)
    assert (plan.info["launches"] == 1) if launches == 1 else (plan.info["launches"] > 1)
    H = torch.tensor(b.h, dtype=torch.float32, device=dev)
    X = torch.tensor(b.x, dtype=torch.float32, device=dev)
    Y = torch.zeros(b.y_len, dtype=torch.float32, device=dev)
    A = torch.zeros(len(b), dtype=torch.float32, device=dev)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        plan.txv(H, X, Y, A, s)  # warm-up outside capture (sets kernel attributes)
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        plan.txv(H, X, Y, A)
    for seed in (18, 19):
        b2 = wl.batched_square(count=300, seed=17, n_lo=16, n_hi=n_hi)
        rng = np.random.default_rng(seed)
        H.copy_(torch.tensor(b2.h * rng.uniform(0.5, 2.0), dtype=torch.float32))
        X.copy_(torch.tensor(b2.x, dtype=torch.float32))
        Y.zero_()
        g.replay()
        torch.cuda.synchronize()
        y_graph, a_graph = Y.clone(), A.clone()
        plan.txv(H, X, Y, A)
        torch.cuda.synchronize()
        assert torch.equal(y_graph, Y) and torch.equal(a_graph, A)
    plan.close()
