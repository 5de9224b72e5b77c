// jobs.h -- work descriptors shared by the host planner and the kernels.
#pragma once

#include <stdint.h>

#include "hankel.h"

namespace hk {

// Plan of one length-L forward transform: L = radix[0] * ... * radix[npass-1],
// twiddles at tw_off in the plan's twiddle array; magic[p] = ceil(2^32 / Ns_p)
// with Ns_p = radix[0] * ... * radix[p-1], so that b mod Ns_p is a
// multiply-high (exact for b * Ns_p < 2^32).
struct FftPlan {
    int32_t L, npass, tw_off;
    uint8_t radix[8];
    uint32_t magic[8];
};

inline void fill_magic(FftPlan& P) {
    uint64_t Ns = 1;
    for (int p = 0; p < 8; ++p) {
        P.magic[p] = (p < P.npass) ? (uint32_t)((0x100000000ull + Ns - 1) / Ns) : 0u;
        if (p < P.npass) Ns *= P.radix[p];
    }
}

// Real square tensors with one vector per tensor (y = H x^{m-1}).  A job is
// either a pair (A, B) of tensors with the same L -- two real problems share
// every complex transform -- or a single tensor, whose h and x share one
// transform as h + i x.
// A single job may also be `split`: its length L exceeds what one block's
// shared memory holds, so each length-L transform runs on a thread-block
// cluster of s = 2 or 4 blocks, block c computing the bins s k + c by one
// length-M transform, M = L/s (decimation in frequency); P is then the
// length-M plan and twL the offset of the length-L twiddle table.
struct RealJob {
    FftPlan P;
    int32_t single;
    int32_t mA, nA, dA, iA;
    int32_t mB, nB, dB, iB;
    int32_t split, twL;  // split: 2 / 3 a cluster of four / two blocks (P: length L/4 / L/2)
    int64_t hA, xA, yA, hB, xB, yB;
    int64_t wsA, wsB;  // element offsets of each tensor's spectrum in the workspace
};

// Real tensors with a different vector in every mode (y = H x_2 ... x_m,
// alpha = H x_1 ... x_m): a pair (A, B) of tensors with the same FFT length
// shares every complex transform -- h_A + i h_B, then x_{A,p} + i x_{B,p}
// mode by mode -- so a pair costs m + 1 transforms (Section 3's count for one
// product).  iB < 0: tensor A alone.
struct MultiJob {
    FftPlan P;
    int32_t mA, mB, iA, iB;
    int32_t dA, dB;
    int32_t nA[HANKEL_MAX_ORDER], nB[HANKEL_MAX_ORDER];
    int64_t hA, hB, yA, yB;
    int64_t xA[HANKEL_MAX_ORDER], xB[HANKEL_MAX_ORDER];
};

// Anti-circulant tensor whose dimension n the transforms do not cover, run as
// the Hankel tensor of its periodic generating vector h_k = c[k mod n],
// k < d = m (n - 1) + 1, expanded from c (at c_off) into a workspace (at
// ws_off).  Gradients fold back: grad_c[j] = sum over k = j mod n of grad_h[k],
// summed over every entry of one fold group (entries that share c).
struct ExpandEntry {
    int64_t c_off, ws_off;
    int32_t n, d;
};
struct FoldGroup {
    int64_t c_off;
    int32_t n, first, count;  // entries [first, first + count) of the expansion table
};

// Launch of one group of jobs that share a block size.
struct RealLaunch {
    int32_t first, count;  // range in the job table
    int32_t nthr, split, Lmax, arrays;  // split: the jobs' split (RealJob::split)
    int32_t fp64;  // nonzero: spectrum powers in FP64 (some tensor of the launch asks for them)
};

// Persistent forward kernel (fast_path.cu): a pair job of two real square
// one-vector tensors A and B with one FFT length; iA < 0 marks an empty slot
// and iB < 0 a missing partner (both then read and write nothing).
struct FastJob {
    int32_t mA, nA, dA, iA;
    int32_t mB, nB, dB, iB;
    int32_t fA, fB;  // nonzero: the tensor's spectrum power in FP64
    int64_t hA, xA, yA, hB, xB, yB;
};
// One work item of the persistent kernel: the jobs [first, first + G) of FFT
// length L, G = jobs per item of that length (one per thread group of a block).
struct FastItem {
    int32_t L, first;
};

}  // namespace hk
