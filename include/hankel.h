/*
 * hankel.h -- C ABI of the GB300 (sm_103a) fast Hankel tensor-vector product
 * library (libhankel.so).
 *
 * Method: Ding, Qi, Wei, "Fast Hankel Tensor-Vector Products and Application
 * to Exponential Data Fitting".  An order-m Hankel tensor H of size
 * n_1 x ... x n_m has entries H[i_1..i_m] = h[i_1 + ... + i_m] (0-based,
 * Section 1) and is stored only through its generating vector h of length
 * d = n_1 + ... + n_m - m + 1.  The library computes the two products of
 * Section 3,
 *
 *     y     = H x_2 x_3 ... x_m      (length n_1)
 *     alpha = H x_1 x_2 ... x_m      (scalar)
 *
 * with the mode product of Section 2.1 (no conjugation anywhere), by
 * embedding H in an anti-circulant tensor (Theorem 2.1) of FFT length
 * L >= d:  y = fft(ifft(h~) .* fft(x~_2) .* ... .* fft(x~_m))[0:n_1],
 * alpha = ifft(h~)^T (fft(x~_1) .* ... .* fft(x~_m)).  The two-level block
 * (BHHB) products of Section 3 use 2D FFTs of the zero-padded generating
 * matrix.  Gradients (not in the paper) are the adjoint correlations.
 *
 * Conventions shared by every call:
 *   - Element: one value of the plan's dtype (a real, or an interleaved
 *     (re, im) pair for the complex dtypes).  Offsets count elements.
 *   - Ownership: the caller owns every input and output buffer (device
 *     memory unless the call says host).  A plan owns only its descriptor
 *     tables, twiddle tables and workspace, all allocated in hankel_plan()
 *     and freed in hankel_plan_destroy().
 *   - Streams: compute calls are asynchronous on `stream` (a cudaStream_t;
 *     NULL = legacy default stream).  They return once the work is queued.
 *     One plan must not run on two streams at the same time (its workspace
 *     is shared).
 *   - Errors: every call returns a status; no exception or abort crosses
 *     the ABI.  hankel_last_error() gives a message for the calling thread's
 *     last failure.  Descriptor validation happens in hankel_plan(); compute
 *     calls validate pointers only.
 *   - Threads: distinct plans may be used from distinct host threads.
 */
#ifndef HANKEL_H
#define HANKEL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define HANKEL_MAX_ORDER 8

typedef enum {
    HANKEL_OK = 0,
    HANKEL_EINVAL = 1,        /* bad argument or descriptor (message says which) */
    HANKEL_ENOMEM = 2,        /* a device or host allocation failed */
    HANKEL_ECUDA = 3,         /* a CUDA runtime call failed (message has its string) */
    HANKEL_EUNSUPPORTED = 4,  /* valid request this build does not implement */
    HANKEL_ETIMEOUT = 5       /* a bounded device-side wait gave up */
} hankel_status;

typedef enum {
    HANKEL_R32 = 0,   /* float                       */
    HANKEL_C64 = 1,   /* complex float  (re, im)     */
    HANKEL_R64 = 2,   /* double                      */
    HANKEL_C128 = 3   /* complex double (re, im)     */
} hankel_dtype;

/* Plan flags (bitwise OR). */
enum {
    /* One vector per tensor, x_off[0], used in every mode (the y = H x^{m-1}
     * and alpha = H x^m products of Section 2.1).  Otherwise x_p is at
     * x_off[p-1]. */
    HANKEL_SAME_X = 1u << 0,
    /* Form the spectrum power / product and the pointwise product with the
     * h spectrum in FP64 even for the FP32 dtypes, for every tensor of the
     * plan.  Without it the planner does so only where the bin policy
     * (hankel_set_bin_policy) asks. */
    HANKEL_FP64_POWER = 1u << 1,
    /* hankel_txv() keeps the spectra it computes in plan workspace so that
     * the next hankel_txv_backward() reuses them instead of recomputing. */
    HANKEL_STORE_SPECTRA = 1u << 2,
    /* Descriptors describe BHHB tensors (use N[]); calls go through
     * hankel_txv_block(). */
    HANKEL_BLOCK = 1u << 3,
    /* Plain path: one tensor per kernel launch, no pairing or batching
     * (the comparison baseline; meant for the FP64 dtypes). */
    HANKEL_ONE_PER_LAUNCH = 1u << 4,
    /* Descriptors describe anti-circulant tensors (Section 2.1:
     * C[i_1..i_m] = c[(i_1 + ... + i_m) mod n]), square with every mode of
     * size n (for BHHB and level-k plans: per level, the block anti-circulant
     * tensors of Section 2.2).  h holds the compressed generating vector c
     * (length n; block plans: the compressed generating array, column-major)
     * and the products of Section 3 run at FFT length exactly n (Theorem
     * 2.1) when n is one of this build's FFT lengths (hankel_fft_length(n)
     * == n, a 2,3,5,7-smooth length).  For other n (one-level plans) the
     * tensor runs as the Hankel tensor of its periodic generating vector
     * c[k mod n], k < m (n - 1) + 1, expanded in plan workspace;
     * HANKEL_EUNSUPPORTED when that embedding exceeds the longest transform
     * (block and level-k plans: whenever a dimension is not a transform
     * length).  y has n entries per level. */
    HANKEL_ANTICIRCULANT = 1u << 5
};

/*
 * One tensor of a batch.
 *   m      order, 2 <= m <= HANKEL_MAX_ORDER.
 *   n[p]   n_{p+1}: mode sizes (for BHHB: the block's mode sizes).
 *   N[p]   N_{p+1}: number of blocks along mode p+1 (BHHB only; ignored and
 *          treated as 1 otherwise).
 *   h_off  offset of h (length d) in the h buffer; for BHHB the generating
 *          matrix, (sum n - m + 1) x (sum N - m + 1), column-major
 *          (Section 2.2).
 *   x_off  offsets of x_1..x_m in the x buffer (only x_off[0] with
 *          HANKEL_SAME_X).  x_1 is read only when alpha is requested.
 *          BHHB: x_p = vec(X_p), X_p of size n_p x N_p column-major.
 *   y_off  offset of y (n_1 elements; BHHB: n_1 x N_1 column-major).
 * Descriptors may share h or x storage (the same offset); output regions
 * must not overlap.
 */
typedef struct hankel_desc {
    int32_t m;
    int32_t n[HANKEL_MAX_ORDER];
    int32_t N[HANKEL_MAX_ORDER];
    int64_t h_off;
    int64_t x_off[HANKEL_MAX_ORDER];
    int64_t y_off;
} hankel_desc;

/*
 * One level-k block Hankel tensor (Section 2.2: a block Hankel tensor whose
 * blocks are level-(k-1) block Hankel tensors; level 1 is a Hankel tensor,
 * level 2 a BHHB tensor).
 *   m       order, 2 <= m <= HANKEL_MAX_ORDER.
 *   levels  k, 1 <= k <= HANKEL_MAX_LEVELS.
 *   n[l][p] size of mode p+1 at level l+1 (level 1 innermost).  Mode p+1
 *           has prod_l n[l][p] entries; its index in mixed radix, level 1
 *           fastest, is I = a_1 + n[0][p] (a_2 + n[1][p] (a_3 + ...)), and
 *           the tensor entry is G[sum_p a_1, ..., sum_p a_k].
 *   h_off   offset of the generating tensor G, an order-k array of size
 *           D_l = sum_p n[l][p] - m + 1 along level l, stored column-major
 *           (level 1 fastest).
 *   x_off   offsets of x_1..x_m: x_p is an array of size n[0][p] x ... x
 *           n[k-1][p], column-major (only x_off[0] with HANKEL_SAME_X).
 *   y_off   offset of y, laid out like x_1.
 * A level whose sizes are all 1 adds nothing (its D_l is 1).
 */
#define HANKEL_MAX_LEVELS 4
typedef struct hankel_mdesc {
    int32_t m;
    int32_t levels;
    int32_t n[HANKEL_MAX_LEVELS][HANKEL_MAX_ORDER];
    int64_t h_off;
    int64_t x_off[HANKEL_MAX_ORDER];
    int64_t y_off;
} hankel_mdesc;

typedef struct hankel_plan_s* hankel_plan_t;
typedef struct CUstream_st* hankel_stream_t; /* same type as cudaStream_t */

/* Read-only facts about a plan (for logging and tests). */
typedef struct hankel_plan_info {
    int64_t count;            /* descriptors */
    int64_t jobs;             /* kernel work units (a unit holds 1 or 2 tensors) */
    int64_t launches;         /* kernel launches per hankel_txv() */
    int64_t distinct_lengths; /* distinct FFT lengths L (bins) */
    int64_t max_length;       /* largest L */
    int64_t sum_length;       /* sum over descriptors of L */
    int64_t workspace_bytes;  /* device workspace owned by the plan */
    int64_t h_elems;          /* minimum h/x/y buffer sizes implied by the offsets */
    int64_t x_elems;
    int64_t y_elems;
    int64_t fp64_power_tensors; /* tensors whose spectrum power is formed in FP64 */
    int64_t backward_launches;  /* kernel launches per hankel_txv_backward() (real path; else 0) */
} hankel_plan_info;

/*
 * hankel_plan -- validate `count` descriptors and build a reusable plan.
 * Section 3 (problem statement of the products and the embedding length).
 *   out     receives the plan (set to NULL on failure).
 *   descs   host array of `count` descriptors (copied; may be freed after).
 *   dtype   element type of every buffer used with the plan.
 *   flags   HANKEL_* flags above.
 * Chooses per tensor the FFT length L >= d (a 2,3,5,7-smooth length chosen
 * by a cost model, the same for every call), groups tensors into jobs and
 * kernel launches, builds FP64-generated twiddle tables on the current device
 * and allocates workspace.  Synchronous.
 * FP32 real tensors with one vector (HANKEL_SAME_X, square) and d <= 5120,
 * without HANKEL_STORE_SPECTRA, HANKEL_ONE_PER_LAUNCH or
 * HANKEL_ANTICIRCULANT, run instead in one persistent launch per
 * hankel_txv (and per hankel_txv_backward, unless their h or x regions
 * overlap or some of them form FP64 powers) at the shortest length >= d of
 * 16 2^k and 12 2^k (32 .. 4096) and 5120; hankel_set_bin_policy can move a
 * length bin back to the per-length launches.  Longer tensors that exceed
 * one block's shared memory run each transform on a thread-block cluster.
 * Errors: EINVAL for m out of range, a non-positive size, negative offsets,
 * a length beyond the supported maximum; ENOMEM; ECUDA.
 */
hankel_status hankel_plan(hankel_plan_t* out, const hankel_desc* descs, int64_t count,
                          hankel_dtype dtype, uint32_t flags);

/*
 * hankel_plan_multilevel -- a plan for level-k block Hankel tensors
 * (Section 2.2; the fast products of Section 3 with k-dimensional FFTs, as
 * the end of Section 3 states):
 *   Y = fftn(ifftn(G~) .* fftn(X~_2) .* ... .* fftn(X~_m))[0:n[0][0], ..., 0:n[k-1][0]],
 *   alpha = <ifftn(G~), fftn(X~_1) .* ... .* fftn(X~_m)>,
 * every array zero-padded to L_1 x ... x L_k with L_l >= D_l.
 *   descs, count, dtype  as hankel_plan (descriptors copied).
 *   flags   HANKEL_SAME_X, HANKEL_STORE_SPECTRA and HANKEL_ANTICIRCULANT;
 *           other bits are EINVAL.
 * The plan computes through hankel_txv_block (forward), hankel_txv_host and
 * hankel_txv_backward (adjoint, the k-dimensional analogue of the BHHB
 * gradients); hankel_txv refuses it.  Synchronous.
 * Errors: EINVAL for m or levels out of range, a non-positive size,
 * negative offsets, unknown flags; EUNSUPPORTED for an L_l beyond the
 * supported maximum; ENOMEM; ECUDA.
 */
hankel_status hankel_plan_multilevel(hankel_plan_t* out, const hankel_mdesc* descs, int64_t count,
                                     hankel_dtype dtype, uint32_t flags);

/*
 * hankel_txv -- y = H x_2 ... x_m and/or alpha = H x_1 ... x_m for every
 * descriptor (Section 3, the fast procedures for y and alpha).
 *   h, x   device buffers of generating vectors and mode vectors.
 *   y      device buffer receiving each y at y_off (NULL: y not computed).
 *   alpha  device array of `count` elements receiving alpha per descriptor
 *          (NULL: not computed).  For real dtypes alpha is real.
 * At least one of y and alpha must be non-NULL.  Real dtypes return real y
 * (the imaginary part of the final transform is not an output).
 * Errors: EINVAL (NULL plan, both outputs NULL, plan made with
 * HANKEL_BLOCK), ECUDA (launch failure).
 */
hankel_status hankel_txv(hankel_plan_t plan, const void* h, const void* x, void* y, void* alpha,
                         hankel_stream_t stream);

/*
 * hankel_txv_host -- hankel_txv on HOST buffers; returns after `stream` has
 * finished (the host buffers are ready).  When every buffer is page-locked
 * memory mapped into the device address space (cudaHostAlloc /
 * cudaHostRegister, as cudaPointerGetAttributes reports), the kernels read
 * and write the host buffers directly across the host link.  Otherwise h and
 * x are copied to plan-owned device staging buffers and y / alpha back, all
 * queued on `stream`; large batches are pipelined over descriptor ranges
 * (sub-plans whose copies overlap each other's kernels).  The first staged
 * call allocates the staging buffers (they live until hankel_plan_destroy).
 * Errors: as hankel_txv, plus ENOMEM.
 */
hankel_status hankel_txv_host(hankel_plan_t plan, const void* h, const void* x, void* y, void* alpha,
                              hankel_stream_t stream);

/*
 * hankel_txv_block -- BHHB products (Section 3, the block procedures):
 *   Y = vec^{-1}( H x_2 ... x_m ) = fft2(ifft2(H~) .* fft2(X~_2) ... )[0:n_1, 0:N_1],
 *   alpha = <ifft2(H~), fft2(X~_1) .* ... .* fft2(X~_m)>.
 * Buffers as hankel_txv, with column-major matrices (Section 3's vec).
 * The plan must have been made with HANKEL_BLOCK or by
 * hankel_plan_multilevel (then the level-k products above).
 */
hankel_status hankel_txv_block(hankel_plan_t plan, const void* H, const void* X, void* Y, void* alpha,
                               hankel_stream_t stream);

/*
 * hankel_txv_backward -- gradients of a real loss through y (not in the
 * paper; the adjoints of the Section 3 products).  With z = x_2 * ... * x_m
 * (linear convolution) and g = dLoss/dy:
 *   grad_h[j]   = sum_i g_i conj(z[j - i]),                 j < d
 *   grad_x_p    = conj(H x_1 conj(g) x_q ... x_q), mode p free (q != 1, p),
 *   with HANKEL_SAME_X: grad_x = sum_p grad_x_p = (m-1) conj(H x_1 conj(g) x_3 x ... x_m x).
 * For complex dtypes g and the gradients follow PyTorch's convention
 * (dL/dRe + i dL/dIm), i.e. the adjoint of the map is applied.  BHHB plans use
 * the 2D analogue.
 *   grad_y  device buffer laid out like y.
 *   grad_h  device buffer laid out like h (NULL: not computed).
 *   grad_x  device buffer laid out like x (NULL: not computed).
 * Gradients are WRITTEN, not accumulated; where several descriptors share one
 * h or x region the contributions are summed into it.
 * With HANKEL_STORE_SPECTRA the spectra saved by the last hankel_txv() on
 * this plan are reused (they must come from the same h and x).
 */
hankel_status hankel_txv_backward(hankel_plan_t plan, const void* grad_y, const void* h, const void* x,
                                  void* grad_h, void* grad_x, hankel_stream_t stream);

/*
 * hankel_txv_backward_static -- the gradients hankel_txv_backward computes, for
 * real square tensors with one vector per tensor (the HANKEL_SAME_X case:
 * x_off[0] in every mode), WITHOUT allocating any device memory.  The paper
 * has no counterpart to this call.
 *
 * Some callers cannot call cudaMalloc: a process whose device memory is
 * already owned by another allocator (a framework's caching allocator that
 * has reserved the GPU), a latency-critical loop that cannot pay for
 * cudaMalloc/cudaFree (they synchronise the device), or a deployment whose
 * device footprint must stay fixed after start-up.  This call needs no plan:
 * it takes the descriptors directly (host array, as for hankel_plan), passes
 * its job table as kernel arguments, and keeps its scratch -- the twiddle
 * tables and one spectrum of L complex values per tensor -- in a single
 * static device array of HANKEL_STATIC_SCRATCH_BYTES, which every GPU that
 * loads the library holds until the process exits.
 *   descs, count  as hankel_plan (copied during the call).
 *   dtype         HANKEL_R32 or HANKEL_R64.
 *   grad_y, h, x  device buffers laid out as for hankel_txv_backward.
 *   grad_h/grad_x device outputs (either may be NULL), written, not accumulated.
 * A batch whose scratch would exceed the array (the sum over tensors of
 * L * 2 * sizeof(real), plus one twiddle table per distinct L, each rounded
 * up to 256 bytes) is rejected with HANKEL_EINVAL and a message giving the
 * bytes it needs; so are non-square tensors, FFT lengths beyond the
 * shared-memory limit, and descriptors whose h regions or x regions overlap
 * (each tensor's gradients are written, not summed as hankel_txv_backward
 * does for shared storage).  Spectrum products are formed in the data
 * precision: there is no HANKEL_FP64_POWER option here.  No cudaMalloc, cudaFree or allocating library call is
 * made.  The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current: make that first call
 * before any stream capture.  Every call shares the array and overwrites the
 * parts it uses (nothing in it needs to start at zero), so calls that overlap
 * on the GPU -- on two streams, or from two host threads -- race; the caller
 * must serialise them.
 */
#define HANKEL_STATIC_SCRATCH_BYTES (16u << 20)
hankel_status hankel_txv_backward_static(const hankel_desc* descs, int64_t count, hankel_dtype dtype,
                                         const void* grad_y, const void* h, const void* x, void* grad_h,
                                         void* grad_x, hankel_stream_t stream);

/* hankel_plan_query -- copy the plan's facts into *info. */
hankel_status hankel_plan_query(hankel_plan_t plan, hankel_plan_info* info);

/*
 * hankel_set_tuning -- planner knobs for plans made after the call
 * (process-wide; existing plans keep their choices).
 *   pass_cost          fixed cost of one radix pass in the planner's cost
 *                      model (FP32 operations per point, default 10): larger
 *                      values favour FFT lengths with fewer passes.
 *   points_per_thread  transform points each thread owns, 8, 16 (default),
 *                      32 or 64: sets the threads per job.
 * The project's autotuner (paper_1401_6238_gb300/autotune.py) times
 * candidate settings on the device and caches the fastest in a JSON file
 * that the Python binding applies when it loads the library.
 * Errors: EINVAL for values outside the ranges above.
 */
hankel_status hankel_set_tuning(double pass_cost, int points_per_thread);

/* hankel_get_tuning -- the current planner knobs. */
hankel_status hankel_get_tuning(double* pass_cost, int* points_per_thread);

/*
 * hankel_set_bin_policy -- per-length-bin planner choices for FP32 plans
 * of real square tensors with one vector (Section 3 products), made after
 * the call (process-wide; existing plans keep theirs).  A bin is one FFT
 * length of the persistent forward kernel (32 .. 5120: 2^k, 3 2^k, 5120);
 * a tensor belongs to the bin of the shortest such length >= its d.
 *   nbins         entries in the arrays (0: every bin back to the default)
 *   L[i]          the bin's length
 *   path[i]       0: the persistent launch (default); 1: the per-length
 *                 launches of the general real path
 *   fp64_from_m[i] the bin's tensors of order m >= fp64_from_m[i] form
 *                 their spectrum power (Section 3, X^{m-1}) in FP64; 9 or
 *                 more (the default 99): never.  HANKEL_FP64_POWER still
 *                 forces FP64 powers for every tensor of a plan.
 * Bins not listed keep their current choices.  The project's autotuner
 * (paper_1401_6238_gb300/autotune.py) times both paths and measures the
 * FP32 error with and without FP64 powers per bin against the oracle, and
 * the Python binding applies its cached table when it loads the library.
 * Errors: EINVAL for a NULL array with nbins > 0, a length that is not a
 * bin, path not 0 or 1, fp64_from_m outside [2, 99].
 */
hankel_status hankel_set_bin_policy(int32_t nbins, const int32_t* L, const int32_t* path, const int32_t* fp64_from_m);

/* hankel_get_bin_policy -- the current choices of bin L (EINVAL if L is not
 * a bin or an output is NULL). */
hankel_status hankel_get_bin_policy(int32_t L, int32_t* path, int32_t* fp64_from_m);

/* hankel_fft_length -- the FFT length the planner picks for generating
 * length d (d >= 1), or -1 when d is beyond the supported maximum. */
int64_t hankel_fft_length(int64_t d);

/* hankel_plan_destroy -- free the plan and everything it owns (synchronises
 * the device first).  NULL is ignored. */
void hankel_plan_destroy(hankel_plan_t plan);

/* hankel_last_error -- message for the calling thread's last failed call
 * ("" if none).  The pointer stays valid until the thread's next call. */
const char* hankel_last_error(void);

/* hankel_version -- library version string. */
const char* hankel_version(void);

#ifdef __cplusplus
}
#endif

#endif /* HANKEL_H */
