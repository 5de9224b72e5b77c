// fast_path.cu -- one persistent launch for batches of real square tensors
// with one vector per tensor: y = H x^{m-1} and alpha = H x^m (Section 2.1
// notation), by the embedding of Section 3 at FFT lengths L = R 2T with
// R in {16, 12} (powers of two and three times powers of two, 32..4096) and
// L = 5120 (R = 20, T = 256).
//
// Work unit: a pair job, two tensors A and B with one FFT length L, run by a
// group of T = L / R threads.  Per tensor the generating vector and the
// vector share one complex transform, S = fft(h~ + i x~) (zero-padded on
// load); bins k and L-k of S give
//     H_k = (S_k + conj S_{L-k}) / 2,  X_k = -i (S_k - conj S_{L-k}) / 2,
// the Section 3 spectral product P_k = ifft(h~)_k X_k^{m-1} with
// ifft(h~)_k = conj(H_k) / L, and alpha = sum_k ifft(h~)_k X_k^m.  P_A and
// P_B are Hermitian, so y~ = fft(P_A + i P_B) returns y_A in its real part
// and y_B in its imaginary part (truncated to n on store).  Three length-L
// transforms per two tensors.
//
// Transforms are Stockham passes (fft_core.cuh conventions): pass radix R,
// Ns = product of the earlier radices, butterfly b takes inputs b + r L/R,
// multiplies input r by w_{Ns R}^{r (b mod Ns)}, and writes output r to
// (b - b mod Ns) R + b mod Ns + r Ns.  Forward passes: the power-of-two part
// of L first, radix R last; the final transform of the product starts with
// radix R.
//
// Register-resident mirror pass.  In the last pass (Ns = L/R, NB = L/R
// butterflies) thread u of a group holds butterflies u and NB - u (u >= 1),
// or 0 and NB/2 (u = 0).  Their bins are mirror images: bin u + s NB pairs
// with bin (NB - u) + (R-1-s) NB, so the unpacking, the spectrum power and
// the packing of P_A + i P_B need no data from other threads, and the first
// pass of the final transform (radix R, the same butterflies, no twiddles)
// starts from these registers.
//
// All other passes go through two shared-memory buffers written alternately
// (one barrier per pass).  Twiddles come from three FP32 tables rounded from
// FP64 (w_4096^e, w_3072^e and w_5120^e) held in shared memory.  P_A waits
// in a thread-private shared-memory slab while tensor B is transformed; at
// L = 5120 the two exchange buffers take that room and the slab is a
// per-block slice of global memory (written and read back by the same
// thread, so it stays in L2).
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>

#include "fft_core.cuh"
#include "launch.h"

namespace hk {
namespace fp {

#ifndef HK_FAST_MIN_BLOCKS
#define HK_FAST_MIN_BLOCKS 2  // resident blocks per SM the register budget is sized for
#endif
constexpr int BLOCK = 256;                  // threads per block
constexpr int PTS = 4096;                   // complex points a block's groups hold together
constexpr int BUF = PTS + PTS / 16;         // padded elements of one exchange buffer
constexpr int RED = 8;                      // doubles of reduction scratch
constexpr int STASH = 16;                   // complex slots per thread of the thread-private slab
// two-level twiddle tables in shared memory: w_4096^e = A2[e >> 6] B2[e & 63],
// w_3072^e = A3[e >> 6] B3[e & 63] (the stage_twiddle_kernel layout: A then B)
constexpr int TW2 = 4096 / 64 + 64;
constexpr int TW3 = 3072 / 64 + 64;
constexpr int TW5 = 5120 / 64 + 64;
constexpr int LONG = 5120;  // the one length whose slab lives in global memory

// padded shared-memory index: one slot every 16 elements (bank spread)
__device__ __forceinline__ int pad(int i) { return i + (i >> 4); }

__host__ __device__ constexpr bool pow2(int v) { return (v & (v - 1)) == 0; }
// radix of the last pass; the thread group of a job has one thread per
// last-pass butterfly
__host__ __device__ constexpr int rlast(int L) { return pow2(L) ? 16 : (L % 5 == 0 ? 20 : 12); }
__host__ __device__ constexpr int nthr(int L) { return L / rlast(L); }
// radix of the power-of-two passes for Q = L / R: 16 first, then the rest
__host__ __device__ constexpr int q0(int Q) { return Q >= 16 ? 16 : Q; }
__host__ __device__ constexpr int q1(int Q) { return Q > 16 ? Q / 16 : 1; }

// Dynamic shared memory of the kernel: reduction scratch, the two-level
// twiddle tables, the two exchange buffers (fixed offsets, so device
// functions address it without pointers in registers).
extern __shared__ __align__(16) unsigned char fp_smem[];
__device__ __forceinline__ double* sm_red() { return reinterpret_cast<double*>(fp_smem); }
__device__ __forceinline__ cx<float>* sm_t2() { return reinterpret_cast<cx<float>*>(fp_smem + RED * sizeof(double)); }
__device__ __forceinline__ cx<float>* sm_t3() { return sm_t2() + TW2; }
__device__ __forceinline__ cx<float>* sm_t5() { return sm_t3() + TW3; }
__device__ __forceinline__ cx<float>* sm_buf(int i) { return sm_t5() + TW5 + i * BUF; }
// complex slots of one group's exchange buffer: the padded length, rounded
// up to an even count (every group's buffer starts on 16 bytes)
__host__ __device__ constexpr int gslots(int L) { return ((L + L / 16) + 1) & ~1; }
// exchange buffer i of length L: BUF apart, or the padded lengths of the
// block's groups apart when that is longer (L = 5120, whose two buffers then
// cover the slab's room)
__host__ __device__ constexpr int sm_bufL_stride(int L) {
    return (BLOCK / (L / rlast(L))) * gslots(L) > BUF ? (BLOCK / (L / rlast(L))) * gslots(L) : BUF;
}
__host__ __device__ constexpr int sm_bufL_span(int L) {
    return sm_bufL_stride(L) + (BLOCK / (L / rlast(L))) * gslots(L);
}
template <int L>
__device__ __forceinline__ cx<float>* sm_bufL(int i) {
    return sm_buf(0) + i * sm_bufL_stride(L);
}
// thread-private slab: slot s of thread i at sm_stash()[s * BLOCK + i]
__device__ __forceinline__ cx<float>* sm_stash() { return sm_buf(2); }

struct Tw {
    // w_M^e for M dividing 4096 (a power of two), 5120 (a multiple of 5) or 3072
    template <int M>
    __device__ __forceinline__ cx<float> get(int e) const {
        if constexpr (pow2(M)) {
            const int f = e * (4096 / M);
            return cmul(sm_t2()[f >> 6], sm_t2()[64 + (f & 63)]);
        } else if constexpr (M % 5 == 0) {
            const int f = e * (5120 / M);
            return cmul(sm_t5()[f >> 6], sm_t5()[80 + (f & 63)]);
        } else {
            const int f = e * (3072 / M);
            return cmul(sm_t3()[f >> 6], sm_t3()[48 + (f & 63)]);
        }
    }
};

template <int R>
__device__ __forceinline__ void dft(cx<float>* a) { DFT<float, R>::run(a); }

// p[r] = w^r for r = 1 .. R-1 by a multiplication tree of depth <= 4
// (w^2 = w w, w^4 = w^2 w^2, w^8 = w^4 w^4; any other power one product of
// those), so each power carries at most four roundings.
template <int R>
__device__ __forceinline__ void powers(cx<float> w, cx<float>* p) {
    p[1] = w;
    if (R > 2) p[2] = cmul(w, w);
#pragma unroll
    for (int r = 3; r < R; ++r) {
        const int hi = (r >= 8) ? 8 : (r >= 4) ? 4 : 2;
        p[r] = (r == hi) ? cmul(p[hi / 2], p[hi / 2]) : cmul(p[hi], p[r - hi]);
    }
}

// x + i y for complex x, y
__device__ __forceinline__ cx<float> plus_i(cx<float> a, cx<float> b) { return mk<float>(a.x - b.y, a.y + b.x); }
__device__ __forceinline__ cx<float> sel(bool c, cx<float> a, cx<float> b) { return c ? a : b; }

// -------------------------------------------------------------- pass pieces

// Asynchronous zero-padded copy of h~ and x~ (length L each) into a buffer
// as two planes of floats, h~ at [0, L) and x~ at [L, 2L): 4-byte cp.async
// copies whose source size 0 zero-fills (the source address then stays a
// valid one, the array's start).  (16-byte copies, which the planes allow
// for segments starting on 16 bytes, issued fewer instructions but made
// the whole benchmark batch slower.)  Completion: stage_wait() and a barrier.
template <int L, int T>
__device__ __forceinline__ void stage(cx<float>* buf, const float* h, int d, const float* x, int n, int t) {
    float* hs = reinterpret_cast<float*>(buf);
    float* xs = hs + L;
#pragma unroll 4
    for (int i = t; i < L; i += T) {
        const unsigned dh = (unsigned)__cvta_generic_to_shared(hs + i), dx = (unsigned)__cvta_generic_to_shared(xs + i);
        const int sa = i < d ? 4 : 0, sb = i < n ? 4 : 0;
        const float* pa = i < d ? h + i : h;
        const float* pb = i < n ? x + i : x;
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(dh), "l"(pa), "r"(sa) : "memory");
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(dx), "l"(pb), "r"(sb) : "memory");
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
}
__device__ __forceinline__ void stage_wait() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// R elements b + r S (r < R) of a padded buffer; when S is a multiple of 16
// the padded index is linear in r.
template <int R, int S>
__device__ __forceinline__ void sload(cx<float>* v, const cx<float>* buf, int b) {
    if constexpr (S % 16 == 0) {
        const cx<float>* p = buf + pad(b);
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = p[r * (S + S / 16)];
    } else {
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = buf[pad(b + r * S)];
    }
}
template <int R, int S>
__device__ __forceinline__ void sstore(cx<float>* buf, int base, const cx<float>* v) {
    if constexpr (S % 16 == 0) {
        cx<float>* p = buf + pad(base);
#pragma unroll
        for (int r = 0; r < R; ++r) p[r * (S + S / 16)] = v[r];
    } else if constexpr (S == 1 && R == 16) {
        cx<float>* p = buf + pad(base);  // base is a multiple of 16: no pad slot inside
#pragma unroll
        for (int r = 0; r < R; ++r) p[r] = v[r];
    } else {
#pragma unroll
        for (int r = 0; r < R; ++r) buf[pad(base + r * S)] = v[r];
    }
}

// One pass, shared memory to shared memory, with butterflies b = t + T j
// (j = 0, 1, ...), each loaded, twiddled, transformed and stored before the
// next.  The twiddles of butterfly b are the powers of w_{NS R}^{b mod NS};
// when NS divides T every butterfly of the thread has the same ones.
template <int L, int R, int NS, int T>
__device__ __forceinline__ void seq_pass(const cx<float>* src, cx<float>* dst, int t, const Tw& tw) {
    constexpr int NB = L / R;
    constexpr int IT = (NB + T - 1) / T;
    constexpr bool shared_k = (T % NS) == 0;
    cx<float> p[R];
    if constexpr (NS > 1 && shared_k) powers<R>(tw.get<NS * R>(t % NS), p);
#pragma unroll 1
    for (int j = 0; j < IT; ++j) {
        const int b = t + T * j;
        if (IT * T == NB || b < NB) {
            cx<float> v[R];
            sload<R, NB>(v, src, b);
            const int k = (NS > 1) ? b % NS : 0;
            if constexpr (NS > 1) {
                if constexpr (!shared_k) powers<R>(tw.get<NS * R>(k), p);
#pragma unroll
                for (int r = 1; r < R; ++r) v[r] = cmul(v[r], p[r]);
            }
            dft<R>(v);
            sstore<R, NS>(dst, (b - k) * R + k, v);
        }
    }
}

// First forward pass (Ns = 1, no twiddles) reading the staged planes:
// butterfly b takes h~ and x~ at b + r L/R as one complex value each.
template <int L, int R, int T>
__device__ __forceinline__ void first_pass(const cx<float>* src, cx<float>* dst, int t) {
    constexpr int NB = L / R;
    constexpr int IT = (NB + T - 1) / T;
    const float* hs = reinterpret_cast<const float*>(src);
    const float* xs = hs + L;
#pragma unroll 1
    for (int j = 0; j < IT; ++j) {
        const int b = t + T * j;
        if (IT * T == NB || b < NB) {
            cx<float> v[R];
#pragma unroll
            for (int r = 0; r < R; ++r) v[r] = mk<float>(hs[b + r * NB], xs[b + r * NB]);
            dft<R>(v);
            sstore<R, 1>(dst, b * R, v);
        }
    }
}

// Last-pass butterfly of thread t in a group of T threads (one butterfly per
// thread, NB = T).  Within each aligned run of 2H lanes (H = min(T, 32) / 2)
// lane j of the first half takes butterfly j' and lane j of the second half
// its mirror NB - j' (j' = (t / 2H) H + j), so that mirror partners are
// lanes t and t ^ H of one warp; j' = 0 pairs the two self-mirrored
// butterflies 0 and NB/2.
template <int T>
__device__ __forceinline__ int last_b(int t) {
    constexpr int H = (T < 32 ? T : 32) / 2;
    const int j = (t / (2 * H)) * H + t % H;
    return ((t / H) & 1) == 0 ? j : (j == 0 ? T / 2 : T - j);
}

// Last pass (Ns = L/R): butterfly b, loaded from `src`, twiddled by the
// powers of w_L^b, transformed; v[s] is bin b + s L/R.
template <int L, int R>
__device__ __forceinline__ void last_pass(cx<float>* v, const cx<float>* src, int b, const Tw& tw) {
    constexpr int NB = L / R;
    cx<float> p[R];
    powers<R>(tw.get<L>(b), p);
    sload<R, NB>(v, src, b);
#pragma unroll
    for (int r = 1; r < R; ++r) v[r] = cmul(v[r], p[r]);
    dft<R>(v);
}

// ------------------------------------------------------------ the product

// X^E for E = 1 .. 4 with the fewest dependent products; E = 0 takes the
// exponent e (1 .. 7) at run time.
template <int E, typename C>
__device__ __forceinline__ C times_pow(C p, C X, int e) {
    if constexpr (E == 1) {
        return cmul(p, X);
    } else if constexpr (E == 2) {
        return cmul(p, cmul(X, X));
    } else if constexpr (E == 3) {
        return cmul(cmul(p, X), cmul(X, X));
    } else if constexpr (E == 4) {
        const C X2 = cmul(X, X);
        return cmul(p, cmul(X2, X2));
    } else {
        if (e & 1) p = cmul(p, X);
        if (e & 6) {
            const C X2 = cmul(X, X);
            if (e & 2) p = cmul(p, X2);
            if (e & 4) p = cmul(p, cmul(X2, X2));
        }
        return p;
    }
}

// Spectral product at bin k without its scale: S_k = a, S_{L-k} = c;
// returns conj(2 H_k) (2 X_k)^e with H, X unpacked from S (e = m - 1), which
// is 2^m L P_k for P_k = conj(H_k)/L X_k^{m-1}; the power-of-two factor
// 2^-m / L is applied, exactly, to y and alpha on store.  When alpha is
// wanted (WA), adds Re(2^m L P_k 2 X_k) / 2 to acc.  The FP32 path sums alpha
// in FP32 throughout (its terms carry FP32 rounding already): an FP64
// instruction holds this GPU's narrow FP64 pipe for many cycles.
template <bool F64, bool WA, int E, typename A>
__device__ __forceinline__ cx<float> product(cx<float> a, cx<float> c, int e, A& acc) {
    if constexpr (F64) {
        const cx<double> X = mk<double>((double)a.y + c.y, (double)c.x - a.x);
        const cx<double> p = times_pow<E>(mk<double>((double)a.x + c.x, (double)c.y - a.y), X, e);
        if constexpr (WA) acc += 0.5 * (p.x * X.x - p.y * X.y);
        return mk<float>((float)p.x, (float)p.y);
    } else {
        const cx<float> X = mk<float>(a.y + c.y, c.x - a.x);
        const cx<float> p = times_pow<E>(mk<float>(a.x + c.x, c.y - a.y), X, e);
        if constexpr (WA) acc += 0.5f * (p.x * X.x - p.y * X.y);
        return p;
    }
}

// The spectral products of one tensor on the thread's bins b + s NB, s < R
// (v: the spectrum S on those bins).  Bin b + s NB pairs with bin
// L - (b + s NB): slot R-1-s of the mirror-partner lane (lane ^ H); the
// lane of butterfly NB/2 is its own partner (it reads its own slot R-1-s by
// shuffling from itself) and the lane of butterfly 0 pairs slot s with its
// own slot (R-s) mod R, which is the previous step's slot R-1-s.
// B == false: P_A into the slab; B == true: Q = P_A + i P_B into the slab.
template <int R, bool F64, bool WA, int E, typename A>
__device__ __forceinline__ void products(const cx<float>* v, cx<float>* st, bool B, int src, bool self0, int e, A& acc) {
    cx<float> prev = v[0];
#pragma unroll
    for (int s = 0; s < R; ++s) {
        const cx<float> o = v[R - 1 - s];
        cx<float> cpart = mk<float>(__shfl_sync(0xffffffffu, o.x, src), __shfl_sync(0xffffffffu, o.y, src));
        cpart = sel(self0, prev, cpart);
        prev = o;
        const cx<float> p = product<F64, WA, E>(v[s], cpart, e, acc);
        st[s * BLOCK] = B ? plus_i(st[s * BLOCK], p) : p;
    }
}

// Barrier of one group: named barrier for multi-warp groups, the warp's for
// groups within a warp (every lane runs the same code, padded with empty
// jobs, so the whole warp always arrives).
template <int T>
__device__ __forceinline__ void gsync(int g) {
    if constexpr (T >= 64) {
        asm volatile("bar.sync %0, %1;" ::"r"(1 + g), "n"(T) : "memory");
    } else {
        __syncwarp();
    }
}

// Sum of one value over the T threads of a group (valid in thread 0 of the
// group); the partial sums of the warps meet in the group's slots of the
// reduction scratch (one double-sized slot per warp, whatever the type, so
// that groups summing floats and doubles never share bytes).
template <int T, typename A>
__device__ __forceinline__ A group_sum(A v, double* red, int g, int t) {
#pragma unroll
    for (int o = (T < 32 ? T : 32) / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if constexpr (T > 32) {
        double* r = red + g * (T / 32);
        if ((t & 31) == 0) *reinterpret_cast<A*>(r + (t >> 5)) = v;
        gsync<T>(g);
        A s = 0;
        if (t == 0)
            for (int i = 0; i < T / 32; ++i) s += *reinterpret_cast<const A*>(r + i);
        gsync<T>(g);
        return s;
    }
    return v;
}

// Kernel arguments, kept in shared memory for the item functions.
struct Params {
    const FastItem* items;
    const FastJob* jobs;
    const float* h;
    const float* x;
    float* y;
    float* alpha;
    int* ctr;
    cx<float>* slab;  // L = 5120: R BLOCK complex values per block
    const float* gy;  // adjoint: upstream gradients (laid out as y) and outputs
    float* gh;
    float* gx;
    int nitems;
    int after;  // the item after the next one (claimed during the current item)
};
__shared__ Params fp_par;

// One item: every group of the block runs one pair job of length L.
// `staged`: the buffer (0/1) into which the previous item already copied
// this job's first input, or -1.  `next`: the index of the block's next
// item; when it has the same length its first input is staged here, into
// the buffer returned (-1 otherwise).
template <int L, bool WA, bool MIX>
__device__ __noinline__ int run_item(int first, int staged, int next) {
    constexpr int R = rlast(L), T = nthr(L), Q = L / R, GS = gslots(L);
    constexpr int QA = q0(Q), QB = q1(Q);  // power-of-two passes (QB == 1: none)
    constexpr int H = (T < 32 ? T : 32) / 2;  // mirror partner: lane ^ H
    static_assert(BLOCK % T == 0, "a block holds whole groups");
    static_assert(L == LONG ? (sm_bufL_span(L) <= 2 * BUF + STASH * BLOCK)
                            : (sm_bufL_span(L) <= 2 * BUF && R <= STASH),
                  "the exchange buffers (and the shared-memory slab) fit the dynamic shared memory");
    const Params& c = fp_par;
    const Tw tw;
    const int g = threadIdx.x / T, t = threadIdx.x % T;
    const FastJob& J = c.jobs[first + g];
    auto buf = [&](int i) { return sm_bufL<L>(i) + g * GS; };
    const int b = last_b<T>(t);
    const bool self0 = b == 0;  // self-mirrored butterflies 0 and T/2
    const int lane = threadIdx.x & 31, src = (b == T / 2) ? lane : (lane ^ H);
    cx<float> v[R];
    // P_A, slot s at st[s * BLOCK]
    cx<float>* const st = (L == LONG ? c.slab + (size_t)blockIdx.x * R * BLOCK : sm_stash()) + threadIdx.x;
    // FP64 spectrum powers per tensor.  A group narrower than a warp shares
    // its warp with other groups, whose lanes must reach the same shuffles:
    // there the warp takes FP64 powers when any of its groups asks for them.
    // (MIX: the plan has such tensors; without them no FP64 code is compiled in)
    bool f64A = MIX && J.fA != 0, f64B = MIX && J.fB != 0;
    if constexpr (MIX && T < 32) {
        f64A = __any_sync(0xffffffffu, f64A);
        f64B = __any_sync(0xffffffffu, f64B);
    }
    // alpha: FP32 sums, FP64 ones for a tensor with its power in FP64
    float aA = 0, aB = 0;
    double a64A = 0, a64B = 0;
    int after = 0;
    if (threadIdx.x == 0) after = atomicAdd(c.ctr, 1) + (int)gridDim.x;  // stored at the end

    int cur = staged;
    if (cur < 0) {
        cur = 1;
        stage<L, T>(buf(cur), c.h + J.hA, J.dA, c.x + J.xA, J.nA, t);
        stage_wait();
        gsync<T>(g);
    }
    // forward transforms of h~ + i x~ (tensor A, then B) and their spectral
    // products; after B, the thread's stash slots hold Q = P_A + i P_B on its bins
#pragma unroll 1
    for (int tensor = 0; tensor < 2; ++tensor) {
        const bool B = tensor == 1;
        const int m = B ? J.mB : J.mA;
        first_pass<L, QA, T>(buf(cur), buf(cur ^ 1), t);
        gsync<T>(g);
        cur ^= 1;
        if constexpr (QB > 1) {
            seq_pass<L, QB, QA, T>(buf(cur), buf(cur ^ 1), t, tw);
            gsync<T>(g);
            cur ^= 1;
        }
        // the other buffer is free: tensor B's input streams in meanwhile
        if (!B) stage<L, T>(buf(cur ^ 1), c.h + J.hB, J.dB, c.x + J.xB, J.nB, t);
        last_pass<L, R>(v, buf(cur), b, tw);
        const int e = m - 1;
        float a = 0;
        double ad = 0;
        if (MIX && (B ? f64B : f64A)) {
            if constexpr (MIX) products<R, true, WA, 0>(v, st, B, src, self0, e, ad);
        } else if constexpr (T >= 32) {
            // the power with a compile-time exponent for the common orders
            switch (e) {
                case 2: products<R, false, WA, 2>(v, st, B, src, self0, e, a); break;
                case 3: products<R, false, WA, 3>(v, st, B, src, self0, e, a); break;
                case 4: products<R, false, WA, 4>(v, st, B, src, self0, e, a); break;
                default: products<R, false, WA, 0>(v, st, B, src, self0, e, a); break;
            }
        } else {
            products<R, false, WA, 0>(v, st, B, src, self0, e, a);
        }
        if (!B) {
            aA = a;
            a64A = ad;
            stage_wait();
            gsync<T>(g);
            cur ^= 1;
        } else {
            aB = a;
            a64B = ad;
        }
    }

    int staged_next = -1;
    // y~ = fft(P_A + i P_B): first pass (radix R, butterfly b) from
    // registers, then the power-of-two passes, the last one storing y.
    if (c.y != nullptr) {
#pragma unroll
        for (int s = 0; s < R; ++s) v[s] = st[s * BLOCK];
        dft<R>(v);
        sstore<R, 1>(buf(cur ^ 1), b * R, v);
        gsync<T>(g);
        cur ^= 1;
        if constexpr (QB > 1) {
            seq_pass<L, QB, R, T>(buf(cur), buf(cur ^ 1), t, tw);
            gsync<T>(g);
            cur ^= 1;
        }
    }
    // the next item's first input, when it has this length, into the free buffer
    if (next < c.nitems) {
        const FastItem N = c.items[next];
        if (N.L == L) {
            const FastJob& K = c.jobs[N.first + g];
            staged_next = cur ^ 1;
            stage<L, T>(buf(staged_next), c.h + K.hA, K.dA, c.x + K.xA, K.nA, t);
        }
    }
    if (c.y != nullptr) {
        // last pass (radix QA, Ns = L/QA, butterflies b = t + T j); output
        // bin b + s Ns, stored when below n
        constexpr int NBL = L / QA;
        constexpr int IT = (NBL + T - 1) / T;
        const int nA = J.nA, nB = J.nB, nmax = max(nA, nB);
        float* yA = c.y + J.yA;
        float* yB = c.y + J.yB;
        const float scA = ldexpf(1.0f / (float)L, -J.mA), scB = ldexpf(1.0f / (float)L, -J.mB);
#pragma unroll 1
        for (int j = 0; j < IT; ++j) {
            const int bl = t + T * j;
            if ((IT * T == NBL || bl < NBL) && bl < nmax) {
                cx<float> w[QA];
                last_pass<L, QA>(w, buf(cur), bl, tw);
#pragma unroll
                for (int s = 0; s < QA; ++s) {
                    const int i0 = bl + s * NBL;
                    if (i0 < nA) yA[i0] = w[s].x * scA;
                    if (i0 < nB) yB[i0] = w[s].y * scB;
                }
            }
        }
    }
    if constexpr (WA) {
        // (the FP64 choices are uniform over the group, and over the warp for
        // groups narrower than one: the sums' shuffles and barriers agree)
        float sA = 0, sB = 0;
        double sA64 = 0, sB64 = 0;
        if constexpr (MIX) {
            if (f64A) sA64 = group_sum<T>(a64A, sm_red(), g, t); else sA = group_sum<T>(aA, sm_red(), g, t);
            if (f64B) sB64 = group_sum<T>(a64B, sm_red(), g, t); else sB = group_sum<T>(aB, sm_red(), g, t);
        } else {
            sA = group_sum<T>(aA, sm_red(), g, t);
            sB = group_sum<T>(aB, sm_red(), g, t);
        }
        if (t == 0) {
            // the same power-of-two scale as y
            const float scA = ldexpf(1.0f / (float)L, -J.mA), scB = ldexpf(1.0f / (float)L, -J.mB);
            if (J.iA >= 0) c.alpha[J.iA] = f64A ? (float)(sA64 * (double)scA) : sA * scA;
            if (J.iB >= 0) c.alpha[J.iB] = f64B ? (float)(sB64 * (double)scB) : sB * scB;
        }
    }
    if (threadIdx.x == 0) fp_par.after = after;
    return staged_next;
}

template <bool WA, bool MIX>
__global__ void __launch_bounds__(BLOCK, HK_FAST_MIN_BLOCKS)
    fast_fwd_kernel(const FastItem* __restrict__ items, int nitems, const FastJob* __restrict__ jobs,
                    const float* __restrict__ h, const float* __restrict__ x, float* __restrict__ y,
                    float* __restrict__ alpha, const cx<float>* __restrict__ tw2, const cx<float>* __restrict__ tw3,
                    const cx<float>* __restrict__ tw5, cx<float>* slab, int* ctr) {
    cx<float>* t2 = sm_t2();
    cx<float>* t3 = sm_t3();
    cx<float>* t5 = sm_t5();
    for (int i = threadIdx.x; i < TW2; i += BLOCK) t2[i] = ldg_cx(tw2 + i);
    for (int i = threadIdx.x; i < TW3; i += BLOCK) t3[i] = ldg_cx(tw3 + i);
    for (int i = threadIdx.x; i < TW5; i += BLOCK) t5[i] = ldg_cx(tw5 + i);
    if (threadIdx.x == 0) {
        fp_par.items = items;
        fp_par.jobs = jobs;
        fp_par.h = h;
        fp_par.x = x;
        fp_par.y = y;
        fp_par.alpha = alpha;
        fp_par.ctr = ctr;
        fp_par.slab = slab;
        fp_par.nitems = nitems;
        // items: blockIdx.x first, then claimed from the counter; the claim
        // of the item after the next one overlaps the current item
        fp_par.after = atomicAdd(ctr, 1) + (int)gridDim.x;
    }
    __syncthreads();
    int it = blockIdx.x, next = fp_par.after;
    int staged = -1;
    __syncthreads();
    while (it < nitems) {
        const FastItem I = items[it];
        switch (I.L) {
            case 5120: staged = run_item<5120, WA, MIX>(I.first, staged, next); break;
            case 4096: staged = run_item<4096, WA, MIX>(I.first, staged, next); break;
            case 3072: staged = run_item<3072, WA, MIX>(I.first, staged, next); break;
            case 2048: staged = run_item<2048, WA, MIX>(I.first, staged, next); break;
            case 1536: staged = run_item<1536, WA, MIX>(I.first, staged, next); break;
            case 1024: staged = run_item<1024, WA, MIX>(I.first, staged, next); break;
            case 768: staged = run_item<768, WA, MIX>(I.first, staged, next); break;
            case 512: staged = run_item<512, WA, MIX>(I.first, staged, next); break;
            case 384: staged = run_item<384, WA, MIX>(I.first, staged, next); break;
            case 256: staged = run_item<256, WA, MIX>(I.first, staged, next); break;
            case 192: staged = run_item<192, WA, MIX>(I.first, staged, next); break;
            case 128: staged = run_item<128, WA, MIX>(I.first, staged, next); break;
            case 96: staged = run_item<96, WA, MIX>(I.first, staged, next); break;
            case 64: staged = run_item<64, WA, MIX>(I.first, staged, next); break;
            case 48: staged = run_item<48, WA, MIX>(I.first, staged, next); break;
            case 32: staged = run_item<32, WA, MIX>(I.first, staged, next); break;
            default: staged = -1; break;
        }
        // the staged copies must land before the next item reads them
        if (staged >= 0) stage_wait();
        __syncthreads();
        it = next;
        next = fp_par.after;
        __syncthreads();
    }
    // copies staged for an item that does not exist are never issued
    // (run_item stages only for next < nitems)
    // the last block to finish re-arms the counter for the next launch
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(ctr + 1, 1) == (int)gridDim.x - 1) {
            ctr[0] = 0;
            ctr[1] = 0;
            __threadfence();
        }
    }
}

// ------------------------------------------------------------ the adjoint

// Gradients of a real loss through y = H x^{m-1} (the adjoint of the
// product: with G = fft(g~), Q_k = G_k X_k^{m-1} / L + i (m-1) ifft(h~)_k
// G_k X_k^{m-2}, and fft(Q) holds grad_h, index reversed, in its real part
// and grad_x in its imaginary part).  Pair job (A, B) of one length: G =
// fft(g~_A + i g~_B) once, its bins kept in the thread-private slab; then per
// tensor U = fft(h~ + i x~), whose last pass leaves U on the thread's bins in
// registers and the mirror bins with the partner lane as in the forward
// kernel, G_A / G_B unpacked from the slab (the mirror bins' slots are read
// from the partner thread's slab), Q formed in registers and transformed,
// its first pass (radix R, no twiddles) from the same registers.  Five
// transforms per pair, spectra never leave the block.
// The adjoint spectrum on the thread's bins b + s NB, times 2^m L:
// q_s = 2G X'^{m-1} + i (m-1) conj(2H) 2G X'^{m-2} with 2H, X' = 2X from U
// (v: U on the bins; U_{L-k} from the mirror lane as in the forward product)
// and 2G_A or 2G_B from the slab (own slot s, the mirror bin's slot of the
// partner thread, gp); every factor 2 and the 1/L are one power-of-two scale
// 2^-m / L on the stored gradients.  E: the exponent m - 2 at compile time
// (1 .. 3), 0 for the run-time one.
template <int R, int E>
__device__ __forceinline__ void adj_bins(const cx<float>* v, cx<float>* q, const cx<float>* gs, const cx<float>* gp,
                                         int src, bool self0, bool B, int m, int e) {
    const float fm = (float)(m - 1);
    cx<float> prev = v[0];
#pragma unroll
    for (int s = 0; s < R; ++s) {
        const cx<float> o = v[R - 1 - s];
        cx<float> uc = mk<float>(__shfl_sync(0xffffffffu, o.x, src), __shfl_sync(0xffffffffu, o.y, src));
        uc = sel(self0, prev, uc);  // U_{L-k}
        prev = o;
        const cx<float> a = v[s];
        // conj(2H) = conj(U_k + conj U_{L-k}), 2X = -i (U_k - conj U_{L-k})
        const cx<float> H2c = mk<float>(a.x + uc.x, uc.y - a.y);
        const cx<float> X2 = mk<float>(a.y + uc.y, uc.x - a.x);
        const cx<float> Gk = gs[s * BLOCK];
        const cx<float> Gc = gp[(self0 ? (R - s) % R : R - 1 - s) * BLOCK];  // G_{L-k}
        // 2G_A = G_k + conj G_{L-k}, 2G_B = -i (G_k - conj G_{L-k})
        const cx<float> G2 = B ? mk<float>(Gk.y + Gc.y, Gc.x - Gk.x) : mk<float>(Gk.x + Gc.x, Gk.y - Gc.y);
        const cx<float> gx2 = E == 0 ? times_pow<0>(G2, X2, e) : times_pow<E>(G2, X2, E);  // 2G X'^{m-2}
        const cx<float> qh = cmul(gx2, X2);
        const cx<float> qx = cmul(H2c, gx2);
        q[s] = mk<float>(qh.x - fm * qx.y, qh.y + fm * qx.x);
    }
}

template <int L>
__device__ __noinline__ int run_adj_item(int first, int staged, int next) {
    constexpr int R = rlast(L), T = nthr(L), Q = L / R, GS = gslots(L);
    constexpr int QA = q0(Q), QB = q1(Q);
    constexpr int H = (T < 32 ? T : 32) / 2;
    constexpr int NBL = L / QA;
    constexpr int IT = (NBL + T - 1) / T;
    static_assert(BLOCK % T == 0, "a block holds whole groups");
    const Params& c = fp_par;
    const Tw tw;
    const int g = threadIdx.x / T, t = threadIdx.x % T;
    const FastJob& J = c.jobs[first + g];
    auto buf = [&](int i) { return sm_bufL<L>(i) + g * GS; };
    const int b = last_b<T>(t);
    const bool self0 = b == 0, selfh = b == T / 2;
    const int lane = threadIdx.x & 31, src = selfh ? lane : (lane ^ H);
    // the slab: G on the thread's bins, slot s at gs[s * BLOCK]; the mirror
    // bin of slot s is slot R-1-s of the partner thread (slot (R-s) mod R of
    // this thread for butterfly 0, slot R-1-s of this thread for NB/2)
    cx<float>* const slab = (L == LONG ? c.slab + (size_t)blockIdx.x * R * BLOCK : sm_stash());
    cx<float>* const gs = slab + threadIdx.x;
    const cx<float>* const gp = slab + ((self0 || selfh) ? threadIdx.x : (threadIdx.x ^ H));
    int after = 0;
    if (threadIdx.x == 0) after = atomicAdd(c.ctr + 2, 1) + (int)gridDim.x;  // stored at the end
    const float invL = 1.0f / (float)L;
    cx<float> v[R], q[R];

    int cur = staged;
    if (cur < 0) {
        cur = 1;
        stage<L, T>(buf(cur), c.gy + J.yA, J.nA, c.gy + J.yB, J.nB, t);
        stage_wait();
        gsync<T>(g);
    }
    // G = fft(g~_A + i g~_B) into the slab; A's inputs stream in meanwhile
    first_pass<L, QA, T>(buf(cur), buf(cur ^ 1), t);
    gsync<T>(g);
    cur ^= 1;
    if constexpr (QB > 1) {
        seq_pass<L, QB, QA, T>(buf(cur), buf(cur ^ 1), t, tw);
        gsync<T>(g);
        cur ^= 1;
    }
    stage<L, T>(buf(cur ^ 1), c.h + J.hA, J.dA, c.x + J.xA, J.nA, t);
    last_pass<L, R>(v, buf(cur), b, tw);
#pragma unroll
    for (int s = 0; s < R; ++s) gs[s * BLOCK] = v[s];
    stage_wait();
    gsync<T>(g);  // the slab and A's inputs are complete
    cur ^= 1;

    int staged_next = -1;
#pragma unroll 1
    for (int tensor = 0; tensor < 2; ++tensor) {
        // (a missing partner or a padding slot runs on zeros and stores
        // nothing: groups narrower than a warp share it, and every lane of a
        // warp must reach the same shuffles)
        const bool B = tensor == 1;
        const int m = B ? J.mB : J.mA;
        // U = fft(h~ + i x~)
        first_pass<L, QA, T>(buf(cur), buf(cur ^ 1), t);
        gsync<T>(g);
        cur ^= 1;
        if constexpr (QB > 1) {
            seq_pass<L, QB, QA, T>(buf(cur), buf(cur ^ 1), t, tw);
            gsync<T>(g);
            cur ^= 1;
        }
        last_pass<L, R>(v, buf(cur), b, tw);
        // Q on the thread's bins, times 2^m L (the scale is applied on store)
        const int e = m - 2;
        if constexpr (T >= 32) {
            switch (e) {
                case 1: adj_bins<R, 1>(v, q, gs, gp, src, self0, B, m, e); break;
                case 2: adj_bins<R, 2>(v, q, gs, gp, src, self0, B, m, e); break;
                case 3: adj_bins<R, 3>(v, q, gs, gp, src, self0, B, m, e); break;
                default: adj_bins<R, 0>(v, q, gs, gp, src, self0, B, m, e); break;
            }
        } else {
            adj_bins<R, 0>(v, q, gs, gp, src, self0, B, m, e);
        }
        // fft(Q): first pass from registers, the power-of-two passes, the last
        // one storing the gradients
        dft<R>(q);
        sstore<R, 1>(buf(cur ^ 1), b * R, q);
        gsync<T>(g);
        cur ^= 1;
        if constexpr (QB > 1) {
            seq_pass<L, QB, R, T>(buf(cur), buf(cur ^ 1), t, tw);
            gsync<T>(g);
            cur ^= 1;
        }
        // the free buffer takes B's inputs, or after B the block's next item's
        // upstream gradients when it has this length
        if (!B) {
            stage<L, T>(buf(cur ^ 1), c.h + J.hB, J.dB, c.x + J.xB, J.nB, t);
        } else if (next < c.nitems) {
            const FastItem N = c.items[next];
            if (N.L == L) {
                const FastJob& K = c.jobs[N.first + g];
                staged_next = cur ^ 1;
                stage<L, T>(buf(staged_next), c.gy + K.yA, K.nA, c.gy + K.yB, K.nB, t);
            }
        }
        const int n = B ? J.nB : J.nA, d = B ? J.dB : J.dA;
        float* gh = c.gh ? c.gh + (B ? J.hB : J.hA) : nullptr;
        float* gx = c.gx ? c.gx + (B ? J.xB : J.xA) : nullptr;
        const float sc = ldexpf(invL, -m);
#pragma unroll 1
        for (int j = 0; j < IT; ++j) {
            const int bl = t + T * j;
            if (IT * T == NBL || bl < NBL) {
                cx<float> w[QA];
                last_pass<L, QA>(w, buf(cur), bl, tw);
#pragma unroll
                for (int s = 0; s < QA; ++s) {
                    const int i0 = bl + s * NBL;
                    const int jh = i0 == 0 ? 0 : L - i0;
                    if (gh != nullptr && jh < d) gh[jh] = w[s].x * sc;
                    if (gx != nullptr && i0 < n) gx[i0] = w[s].y * sc;
                }
            }
        }
        if (!B) {
            stage_wait();
            gsync<T>(g);  // B's inputs are complete; the buffers are free
            cur ^= 1;
        }
    }
    if (threadIdx.x == 0) fp_par.after = after;
    return staged_next;
}

__global__ void __launch_bounds__(BLOCK, HK_FAST_MIN_BLOCKS)
    fast_bwd_kernel(const FastItem* __restrict__ items, int nitems, const FastJob* __restrict__ jobs,
                    const float* __restrict__ gy, const float* __restrict__ h, const float* __restrict__ x,
                    float* __restrict__ gh, float* __restrict__ gx, const cx<float>* __restrict__ tw2,
                    const cx<float>* __restrict__ tw3, const cx<float>* __restrict__ tw5, cx<float>* slab,
                    int* ctr) {
    cx<float>* t2 = sm_t2();
    cx<float>* t3 = sm_t3();
    cx<float>* t5 = sm_t5();
    for (int i = threadIdx.x; i < TW2; i += BLOCK) t2[i] = ldg_cx(tw2 + i);
    for (int i = threadIdx.x; i < TW3; i += BLOCK) t3[i] = ldg_cx(tw3 + i);
    for (int i = threadIdx.x; i < TW5; i += BLOCK) t5[i] = ldg_cx(tw5 + i);
    if (threadIdx.x == 0) {
        fp_par.items = items;
        fp_par.jobs = jobs;
        fp_par.h = h;
        fp_par.x = x;
        fp_par.y = nullptr;
        fp_par.alpha = nullptr;
        fp_par.ctr = ctr;
        fp_par.slab = slab;
        fp_par.gy = gy;
        fp_par.gh = gh;
        fp_par.gx = gx;
        fp_par.nitems = nitems;
        // items: blockIdx.x first, then claimed from the adjoint's counter
        // (ctr[2], ctr[3]); the claim of the item after the next one
        // overlaps the current item
        fp_par.after = atomicAdd(ctr + 2, 1) + (int)gridDim.x;
    }
    __syncthreads();
    int it = blockIdx.x, next = fp_par.after;
    int staged = -1;
    __syncthreads();
    while (it < nitems) {
        const FastItem I = items[it];
        switch (I.L) {
            case 5120: staged = run_adj_item<5120>(I.first, staged, next); break;
            case 4096: staged = run_adj_item<4096>(I.first, staged, next); break;
            case 3072: staged = run_adj_item<3072>(I.first, staged, next); break;
            case 2048: staged = run_adj_item<2048>(I.first, staged, next); break;
            case 1536: staged = run_adj_item<1536>(I.first, staged, next); break;
            case 1024: staged = run_adj_item<1024>(I.first, staged, next); break;
            case 768: staged = run_adj_item<768>(I.first, staged, next); break;
            case 512: staged = run_adj_item<512>(I.first, staged, next); break;
            case 384: staged = run_adj_item<384>(I.first, staged, next); break;
            case 256: staged = run_adj_item<256>(I.first, staged, next); break;
            case 192: staged = run_adj_item<192>(I.first, staged, next); break;
            case 128: staged = run_adj_item<128>(I.first, staged, next); break;
            case 96: staged = run_adj_item<96>(I.first, staged, next); break;
            case 64: staged = run_adj_item<64>(I.first, staged, next); break;
            case 48: staged = run_adj_item<48>(I.first, staged, next); break;
            case 32: staged = run_adj_item<32>(I.first, staged, next); break;
            default: staged = -1; break;
        }
        if (staged >= 0) stage_wait();
        __syncthreads();
        it = next;
        next = fp_par.after;
        __syncthreads();
    }
    // the last block to finish re-arms the adjoint's counter
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(ctr + 3, 1) == (int)gridDim.x - 1) {
            ctr[2] = 0;
            ctr[3] = 0;
            __threadfence();
        }
    }
}

}  // namespace fp

bool fast_length_ok(int L) {
    switch (L) {
        case 5120: case 4096: case 3072: case 2048: case 1536: case 1024: case 768: case 512: case 384:
        case 256: case 192: case 128: case 96: case 64: case 48: case 32: return true;
        default: return false;
    }
}

int fast_length(int64_t d) {
    static const int lens[] = {32, 48, 64, 96, 128, 192, 256, 384, 512, 768, 1024, 1536, 2048, 3072, 4096, 5120};
    for (int L : lens)
        if (L >= d) return L;
    return 0;
}

int fast_jobs_per_item(int L) { return fp::BLOCK / fp::nthr(L); }

size_t fast_slab_bytes(int L) { return L == fp::LONG ? (size_t)fp::rlast(L) * fp::BLOCK * sizeof(cx<float>) : 0; }

size_t fast_smem_bytes() {
    return fp::RED * sizeof(double) +
           ((size_t)fp::TW2 + fp::TW3 + fp::TW5 + 2 * (size_t)fp::BUF + (size_t)fp::STASH * fp::BLOCK) *
               sizeof(cx<float>);
}

cudaError_t launch_fast_forward(const FastItem* items, int nitems, int grid, const FastJob* jobs, const void* h,
                                const void* x, void* y, void* alpha, const void* t2, const void* t3, const void* t5,
                                void* slab, int* ctr, int flags, cudaStream_t st) {
    const size_t smem = fast_smem_bytes();
    // HANKEL_FP64_POWER here: some job asks for FP64 spectrum powers (the
    // job table says which tensors), so the kernel variant holding that
    // code runs
    const bool wa = alpha != nullptr, mix = (flags & HANKEL_FP64_POWER) != 0;
    auto k = wa ? (mix ? fp::fast_fwd_kernel<true, true> : fp::fast_fwd_kernel<true, false>)
                : (mix ? fp::fast_fwd_kernel<false, true> : fp::fast_fwd_kernel<false, false>);
    const int variant = 2 * mix + wa;
    static std::mutex mu;
    static bool done[4][64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    {
        std::lock_guard<std::mutex> lk(mu);
        if (dev < 64 && !done[variant][dev]) {
            e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            // shared memory for the resident blocks only; the rest stays L1
            // (spill slots, descriptors)
            int maxsm = 0;
            if (e == cudaSuccess) e = cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
            if (e == cudaSuccess && maxsm > 0) {
                const size_t want = (size_t)HK_FAST_MIN_BLOCKS * (smem + 1024);
                const int pct = (int)std::min<size_t>(100, (want * 100 + maxsm - 1) / maxsm);
                e = cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, pct);
            }
            if (e != cudaSuccess) return e;
            done[variant][dev] = true;
        }
    }
    k<<<grid, fp::BLOCK, smem, st>>>(items, nitems, jobs, (const float*)h, (const float*)x, (float*)y, (float*)alpha,
                                     (const cx<float>*)t2, (const cx<float>*)t3, (const cx<float>*)t5,
                                     (cx<float>*)slab, ctr);
    return cudaGetLastError();
}

int fast_blocks_per_sm() { return HK_FAST_MIN_BLOCKS; }

cudaError_t launch_fast_backward(const FastItem* items, int nitems, int grid, const FastJob* jobs, const void* gy,
                                 const void* h, const void* x, void* gh, void* gx, const void* t2, const void* t3,
                                 const void* t5, void* slab, int* ctr, cudaStream_t st) {
    const size_t smem = fast_smem_bytes();
    auto k = fp::fast_bwd_kernel;
    static std::mutex mu;
    static bool done[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    {
        std::lock_guard<std::mutex> lk(mu);
        if (dev < 64 && !done[dev]) {
            e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            int maxsm = 0;
            if (e == cudaSuccess) e = cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
            if (e == cudaSuccess && maxsm > 0) {
                const size_t want = (size_t)HK_FAST_MIN_BLOCKS * (smem + 1024);
                const int pct = (int)std::min<size_t>(100, (want * 100 + maxsm - 1) / maxsm);
                e = cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, pct);
            }
            if (e != cudaSuccess) return e;
            done[dev] = true;
        }
    }
    k<<<grid, fp::BLOCK, smem, st>>>(items, nitems, jobs, (const float*)gy, (const float*)h, (const float*)x,
                                     (float*)gh, (float*)gx, (const cx<float>*)t2, (const cx<float>*)t3,
                                     (const cx<float>*)t5, (cx<float>*)slab, ctr);
    return cudaGetLastError();
}

}  // namespace hk
