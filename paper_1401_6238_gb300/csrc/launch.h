// launch.h -- host-side launchers of the kernels (implemented in the .cu files).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>

#include <string>

#include "jobs.h"

namespace hk {

// bytes at the start of dynamic shared memory reserved for block reductions
constexpr int RED_BYTES = 512;
// shared-memory elements of one padded length-L buffer (one pad slot per 16)
constexpr size_t smem_elems_host(int L) { return (size_t)L + (size_t)(L >> 4) + 1; }
// shared-memory slots of the real-path kernels' twiddle table (L <= 16384)
constexpr int TW_SMEM_HOST = (16384 + 63) / 64 + 64;

cudaError_t launch_real_forward(bool dbl, const RealLaunch& lc, const RealJob* jobs, const void* h, const void* x,
                                void* y, void* alpha, const void* tw, void* ws, int flags, cudaStream_t st);
cudaError_t launch_real_backward(bool dbl, const RealLaunch& lc, const RealJob* jobs, const void* gy, const void* h,
                                 const void* x, void* gh, void* gx, const void* tw, void* ws, int flags, int stored,
                                 cudaStream_t st);
cudaError_t launch_real_multi(bool dbl, const RealLaunch& lc, const MultiJob* jobs, const void* h, const void* x,
                              void* y, void* alpha, const void* tw, cudaStream_t st);
cudaError_t launch_twiddles(bool dbl, void* out, int L, cudaStream_t st);
// periodic expansion of anti-circulant generating vectors and the fold of
// their gradients (elem: bytes per element of the plan's dtype; cplx: complex)
cudaError_t launch_expand(int elem, const ExpandEntry* e, int count, int max_d, const void* c, void* h, cudaStream_t st);
cudaError_t launch_fold(bool dbl, bool cplx, const ExpandEntry* e, const FoldGroup* g, int ngroups, int max_n,
                        const void* gh, void* gc, cudaStream_t st);
// per-pass twiddle layout of fft_stage.cuh (real-data kernels)
cudaError_t launch_stage_twiddles(bool dbl, void* out, const FftPlan& P, cudaStream_t st);
int stage_twiddle_count(const FftPlan& P);
// persistent forward kernel of fast_path.cu: its FFT lengths, jobs per item
// and launch (t2, t3, t5 = the w_4096^e, w_3072^e, w_5120^e tables; slab =
// grid x fast_slab_bytes(L) bytes for the longest length L of the items;
// ctr = four zeroed ints (the forward's two, the adjoint's two); flags:
// HANKEL_FP64_POWER when some job's fA or fB
// asks for FP64 spectrum powers)
bool fast_length_ok(int L);
int fast_length(int64_t d);
int fast_jobs_per_item(int L);
int fast_blocks_per_sm();
size_t fast_smem_bytes();
size_t fast_slab_bytes(int L);
cudaError_t launch_fast_forward(const FastItem* items, int nitems, int grid, const FastJob* jobs, const void* h,
                                const void* x, void* y, void* alpha, const void* t2, const void* t3, const void* t5,
                                void* slab, int* ctr, int flags, cudaStream_t st);
// the persistent adjoint over the same items and jobs (gradients of a real
// loss through y; gy laid out as y, gh / gx as h / x, either may be null)
cudaError_t launch_fast_backward(const FastItem* items, int nitems, int grid, const FastJob* jobs, const void* gy,
                                 const void* h, const void* x, void* gh, void* gx, const void* t2, const void* t3,
                                 const void* t5, void* slab, int* ctr, cudaStream_t st);
size_t real_launch_smem(bool dbl, const RealLaunch& lc);
bool fft_factor(int L, FftPlan* P);
void set_last_error(const std::string& msg);

}  // namespace hk
