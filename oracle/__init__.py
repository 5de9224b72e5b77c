"""FP64 CPU oracle for the fast Hankel tensor-vector product (Ding, Qi, Wei).

TEST INFRASTRUCTURE ONLY.  Nothing on the product path imports, calls or links
anything in this package: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may use it.  It
shares no code, table or helper with the CUDA library under
``paper_1401_6238_gb300/``; the only thing both sides see is the seeded input
generator ``paper_1401_6238_gb300.workloads``, which holds none of the
method's arithmetic.

Contents (each function cites the passage it restates):

* ``hankel``  -- definitions of Section 1 and Section 2.1 (Hankel tensor,
  generating vector, mode-p product), direct summation by loops and by the
  explicit tensor, and the fast procedures of Section 3 (anti-circulant
  embedding, y = H x_2 ... x_m and alpha = H x_1 ... x_m).
* ``fft``     -- an independently written radix-2 FFT (power-of-two lengths)
  that the fast procedures use; Section 2.1 fixes its sign and scale.
* ``block``   -- BHHB tensors (Section 2.2) and the block fast products of
  Section 3 via 2D FFTs.
* ``grad``    -- gradients of the products (the paper is silent on them; they
  are derived from the definition, see the module header).
* ``level``   -- level-k block Hankel tensors (Section 2.2) and their fast
  products by k-dimensional FFTs (end of Section 3), with gradients.
* ``edf``     -- HOOI / HOTF (Algorithms 4.1, 4.2) on explicit tensors and the
  total-least-squares pole estimates of Sections 4.1 and 4.3.

Parity status: every function here is pinned by ``tests/test_oracle*.py``
against something other than itself (loops over index tuples, closed forms,
library routines, finite differences, printed examples).
"""

from .fft import fft, ifft, fft2, ifft2, fftn, ifftn, next_pow2
from .hankel import (
    d_of,
    hankel_tensor,
    mode_product,
    loop_y,
    loop_alpha,
    brute_y,
    brute_alpha,
    fast_y,
    fast_alpha,
    anticirculant_generating_vector,
    anticirculant_y,
    anticirculant_alpha,
)
from .block import (
    bhhb_tensor,
    vec,
    unvec,
    brute_block_y,
    brute_block_alpha,
    fast_block_y,
    fast_block_alpha,
)
from . import edf  # noqa: F401
from . import level  # noqa: F401
from .grad import (
    brute_grads,
    fast_grads,
    brute_block_grads,
    fast_block_grads,
)

__all__ = [
    "fft", "ifft", "fft2", "ifft2", "fftn", "ifftn", "next_pow2",
    "d_of", "hankel_tensor", "mode_product", "loop_y", "loop_alpha",
    "brute_y", "brute_alpha", "fast_y", "fast_alpha",
    "anticirculant_generating_vector", "anticirculant_y", "anticirculant_alpha",
    "bhhb_tensor", "vec", "unvec", "brute_block_y", "brute_block_alpha",
    "fast_block_y", "fast_block_alpha",
    "brute_grads", "fast_grads", "brute_block_grads", "fast_block_grads",
]
