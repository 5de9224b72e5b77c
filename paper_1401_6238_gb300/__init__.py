"""GB300-native (sm_103a) fast Hankel tensor-vector products.

Ding, Qi, Wei, "Fast Hankel Tensor-Vector Products and Application to
Exponential Data Fitting": y = H x_2 ... x_m and alpha = H x_1 ... x_m for
Hankel and BHHB tensors by anti-circulant embedding and FFTs (Section 3),
plus their adjoints.  The compute path is the C-ABI library libhankel.so
(include/hankel.h) with hand-written CUDA kernels; ``hankel`` is its thin
Python binding and ``workloads`` the seeded synthetic inputs.
"""

from . import workloads  # noqa: F401
from .hankel import (  # noqa: F401
    ANTICIRCULANT, BLOCK, C64, C128, FP64_POWER, ONE_PER_LAUNCH, R32, R64, SAME_X, STORE_SPECTRA,
    HankelError, Plan, batch_descs, hankel_fft_length, hankel_last_error, hankel_plan, hankel_plan_destroy,
    hankel_plan_query, hankel_txv, hankel_txv_autograd, hankel_txv_backward, hankel_txv_block, hankel_txv_host,
    hankel_version, load, make_descs, square_descs, MDESC_DTYPE, hankel_plan_multilevel, level_descs, make_mdescs,
)
