// fft_stage.cuh -- compact Stockham transform for the real-data kernels.
//
// Same radix-R Stockham passes as fft_core.cuh (natural order in and out,
// out of place, ping-pong between two shared buffers), arranged to keep the
// kernels small and the hot loops branch-free: the transform is one
// non-inlined function per (type, final store), each pass is one of four
// variants (global->shared, shared->shared, shared->store, global->store),
// and k = b mod Ns uses a multiply-high instead of a division.
//
// Twiddles come from a small two-level table copied into shared memory once
// per block (see TwTab), so the passes issue no global loads for them.
#pragma once

#include "fft_core.cuh"

namespace hk {

// Zero-padded read of two real global arrays as one complex signal a + i b.
template <typename T>
struct GLd {
    const T* a;
    int na;
    const T* b;
    int nb;
    __device__ __forceinline__ cx<T> operator()(int i) const {
        return mk<T>(i < na ? __ldg(a + i) : T(0), i < nb ? __ldg(b + i) : T(0));
    }
};

template <typename T>
struct SLd {
    const cx<T>* s;
    __device__ __forceinline__ cx<T> operator()(int i) const { return s[sp(i)]; }
};

template <typename T>
struct SSt {
    cx<T>* s;
    __device__ __forceinline__ void operator()(int i, cx<T> v) const { s[sp(i)] = v; }
};

// Truncated store of two real results: Re -> a[i] (i < na), Im -> b[i] (i < nb).
template <typename T>
struct PairSt {
    T* a;
    int na;
    T* b;
    int nb;
    __device__ __forceinline__ void operator()(int i, cx<T> v) const {
        if (i < na) a[i] = v.x;
        if (i < nb) b[i] = v.y;
    }
};

// Adjoint store: Re -> a[(L - i) mod L] (< na), Im -> b[i] (i < nb); either may be null.
template <typename T>
struct AdjSt {
    T* a;
    int na;
    T* b;
    int nb;
    int L;
    __device__ __forceinline__ void operator()(int i, cx<T> v) const {
        const int j = (i == 0) ? 0 : L - i;
        if (a != nullptr && j < na) a[j] = v.x;
        if (b != nullptr && i < nb) b[i] = v.y;
    }
};

// Plain complex global store.
template <typename T>
struct GSt {
    cx<T>* p;
    __device__ __forceinline__ void operator()(int i, cx<T> v) const { p[i] = v; }
};

// Asynchronous zero-padded copy of two real global arrays into a shared
// buffer as one complex signal: buf[i] = (a[i] if i < na else 0) + i (b[i]
// if i < nb else 0), i < L.  4-byte cp.async copies; a source size of 0
// zero-fills.  Completion: cp_wait_all() and then a barrier.
template <typename T>
__device__ __forceinline__ void cp_async_pair(cx<T>* buf, const T* a, int na, const T* b, int nb, int L,
                                              const Group& g) {
    static_assert(sizeof(T) == 4 || sizeof(T) == 8, "real type");
    for (int i = g.tid; i < L; i += g.nthr) {
        T* d = reinterpret_cast<T*>(&buf[sp(i)]);
        const unsigned da = (unsigned)__cvta_generic_to_shared(d);
        const unsigned db = (unsigned)__cvta_generic_to_shared(d + 1);
        const int sa = (i < na) ? (int)sizeof(T) : 0;
        const int sb = (i < nb) ? (int)sizeof(T) : 0;
        const T* pa = (i < na) ? a + i : a;  // a is always a valid address; with
        const T* pb = (i < nb) ? b + i : a;  // source size 0 nothing is read
        if (sizeof(T) == 4) {
            asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(da), "l"(pa), "r"(sa) : "memory");
            asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(db), "l"(pb), "r"(sb) : "memory");
        } else {
            asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(da), "l"(pa), "r"(sa) : "memory");
            asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(db), "l"(pb), "r"(sb) : "memory");
        }
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
}

// Wait until at most `n` of this thread's committed copy groups are pending.
template <int n>
__device__ __forceinline__ void cp_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(n) : "memory");
}

// k = b mod Ns by a multiply-high with m = ceil(2^32 / Ns) (exact for b * Ns < 2^32).
__device__ __forceinline__ int mod_magic(int b, int Ns, unsigned m) {
    return b - Ns * (int)__umulhi((unsigned)b, m);
}

// Twiddles from a two-level table in shared memory: w_L^e = A[e >> 6] B[e & 63]
// with A[j] = w_L^{64 j} (ceil(L/64) entries) and B[j] = w_L^j (64 entries),
// both FP64-generated and rounded.  The powers w^r of a butterfly's base
// twiddle come from a multiplication tree of depth <= 4 (w^2 = w w,
// w^4 = w^2 w^2, w^8 = w^4 w^4, every other power one more product).
constexpr int TW_LO = 64;
__host__ __device__ constexpr int tw_table_elems(int L) { return (L + TW_LO - 1) / TW_LO + TW_LO; }

template <typename T>
struct TwTab {
    const cx<T>* A;
    const cx<T>* B;
    __device__ __forceinline__ cx<T> operator()(int e) const { return cmul(A[e >> 6], B[e & (TW_LO - 1)]); }
};

template <typename T, int R>
__device__ __forceinline__ void apply_twiddles(cx<T>* v, cx<T> w) {
    cx<T> p[R];
    p[1] = w;
    if (R > 2) p[2] = cmul(w, w);
#pragma unroll
    for (int r = 3; r < R; ++r) {
        // largest power of two below r times the rest
        const int hi = (r >= 8) ? 8 : (r >= 4) ? 4 : 2;
        p[r] = (r == hi) ? cmul(p[hi / 2], p[hi / 2]) : cmul(p[hi], p[r - hi]);
    }
#pragma unroll
    for (int r = 1; r < R; ++r) v[r] = cmul(v[r], p[r]);
}

template <typename T, int R, class Src, class Dst>
__device__ __forceinline__ void pass_st(const Src& src, const Dst& dst, int L, int Ns, unsigned magic,
                                        const TwTab<T>& tw, const Group& g) {
    const int nb = L / R;  // compile-time divisor
    const int twstride = (Ns > 1) ? (int)__umulhi((unsigned)nb, magic) : nb;  // L / (Ns R), exact as Ns | nb
    for (int b = g.tid; b < nb; b += g.nthr) {
        cx<T> v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = src(b + r * nb);
        const int k = (Ns > 1) ? mod_magic(b, Ns, magic) : 0;
        if (Ns > 1) apply_twiddles<T, R>(v, tw(k * twstride));
        DFT<T, R>::run(v);
        const int base = (b - k) * R + k;
#pragma unroll
        for (int r = 0; r < R; ++r) dst(base + r * Ns, v[r]);
    }
}

// Shared -> shared pass when nb = L/R and Ns are multiples of 16: the padded
// index is then linear in r (sp(i + r s) = sp(i) + r (s + s/16)), so each
// butterfly computes one address per side.
template <typename T, int R>
__device__ __forceinline__ void pass_lin(const cx<T>* __restrict__ s, cx<T>* __restrict__ d, int L, int Ns,
                                         unsigned magic, const TwTab<T>& tw, const Group& g) {
    const int nb = L / R;
    const int twstride = (int)__umulhi((unsigned)nb, magic);  // L / (Ns R), Ns >= 16 here
    const int rs = nb + (nb >> 4), ws = Ns + (Ns >> 4);
    for (int b = g.tid; b < nb; b += g.nthr) {
        cx<T> v[R];
        const cx<T>* sb = s + sp(b);
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = sb[r * rs];
        const int k = mod_magic(b, Ns, magic);
        apply_twiddles<T, R>(v, tw(k * twstride));
        DFT<T, R>::run(v);
        cx<T>* db = d + sp((b - k) * R + k);
#pragma unroll
        for (int r = 0; r < R; ++r) db[r * ws] = v[r];
    }
}

template <typename T>
__device__ __forceinline__ void pass_lin_sel(int R, const cx<T>* s, cx<T>* d, int L, int Ns, unsigned magic,
                                             const TwTab<T>& tw, const Group& g) {
    switch (R) {
        case 16: pass_lin<T, 16>(s, d, L, Ns, magic, tw, g); break;
        case 8: pass_lin<T, 8>(s, d, L, Ns, magic, tw, g); break;
        case 4: pass_lin<T, 4>(s, d, L, Ns, magic, tw, g); break;
        case 2: pass_lin<T, 2>(s, d, L, Ns, magic, tw, g); break;
        case 3: pass_lin<T, 3>(s, d, L, Ns, magic, tw, g); break;
        case 5: pass_lin<T, 5>(s, d, L, Ns, magic, tw, g); break;
        case 7: pass_lin<T, 7>(s, d, L, Ns, magic, tw, g); break;
        default: break;
    }
}

template <typename T, class Src, class Dst>
__device__ __forceinline__ void pass_sel(int R, const Src& src, const Dst& dst, int L, int Ns, unsigned magic,
                                         const TwTab<T>& tw, const Group& g) {
    switch (R) {
        case 16: pass_st<T, 16>(src, dst, L, Ns, magic, tw, g); break;
        case 8: pass_st<T, 8>(src, dst, L, Ns, magic, tw, g); break;
        case 4: pass_st<T, 4>(src, dst, L, Ns, magic, tw, g); break;
        case 2: pass_st<T, 2>(src, dst, L, Ns, magic, tw, g); break;
        case 3: pass_st<T, 3>(src, dst, L, Ns, magic, tw, g); break;
        case 5: pass_st<T, 5>(src, dst, L, Ns, magic, tw, g); break;
        case 7: pass_st<T, 7>(src, dst, L, Ns, magic, tw, g); break;
        default: break;
    }
}

// Full transform.  Pass 0 reads the global pair `gfirst`, or the shared
// buffer `sfirst` when that is not null (which must then not be b0); the
// passes ping-pong between b0 (written by pass 0) and b1; the last pass
// writes `last` unless `keep`, in which case the result stays in shared
// memory and its buffer is returned.  Every pass ends with a barrier.
// Each pass is one of four branch-free variants: global->shared,
// shared->shared, shared->last, global->last.
template <typename T, class Last>
__device__ __noinline__ cx<T>* fft_stage(FftPlan P, GLd<T> gfirst, const cx<T>* sfirst, cx<T>* b0, cx<T>* b1,
                                         Last last, bool keep, TwTab<T> twp, Group g) {
    cx<T>* buf[2] = {b0, b1};
    int Ns = 1;
    for (int p = 0; p < P.npass; ++p) {
        const int R = P.radix[p];
        const unsigned magic = P.magic[p];
        const bool to_last = (p == P.npass - 1) && !keep;
        const cx<T>* sp_src = (p == 0) ? sfirst : buf[(p - 1) & 1];
        if (sp_src == nullptr) {
            if (to_last)
                pass_sel<T>(R, gfirst, last, P.L, Ns, magic, twp, g);
            else
                pass_sel<T>(R, gfirst, SSt<T>{buf[p & 1]}, P.L, Ns, magic, twp, g);
        } else {
            if (to_last)
                pass_sel<T>(R, SLd<T>{sp_src}, last, P.L, Ns, magic, twp, g);
            else if ((((P.L / R) | Ns) & 15) == 0)
                pass_lin_sel<T>(R, sp_src, buf[p & 1], P.L, Ns, magic, twp, g);
            else
                pass_sel<T>(R, SLd<T>{sp_src}, SSt<T>{buf[p & 1]}, P.L, Ns, magic, twp, g);
        }
        g.sync();
        Ns *= R;
    }
    return keep ? buf[(P.npass - 1) & 1] : nullptr;
}

// Complex global buffer used as transform scratch (lengths beyond shared memory).
template <typename T>
struct CLd {
    const cx<T>* p;
    __device__ __forceinline__ cx<T> operator()(int i) const { return p[i]; }
};

// Transform through two global scratch buffers w0, w1 (L complex each):
// pass 0 reads `gfirst` (zero-padded real pair) or `cfirst` when not null;
// passes ping-pong between w0 (written by pass 0) and w1; the last pass
// writes `last` unless `keep`, in which case the buffer holding the result
// is returned.  Barriers between passes make each block's global writes
// visible to its own threads.
template <typename T, class Last>
__device__ __noinline__ cx<T>* fft_global(FftPlan P, GLd<T> gfirst, const cx<T>* cfirst, cx<T>* w0, cx<T>* w1,
                                          Last last, bool keep, TwTab<T> twp, Group g) {
    cx<T>* buf[2] = {w0, w1};
    int Ns = 1;
    for (int p = 0; p < P.npass; ++p) {
        const int R = P.radix[p];
        const unsigned magic = P.magic[p];
        const bool to_last = (p == P.npass - 1) && !keep;
        const cx<T>* src = (p == 0) ? cfirst : buf[(p - 1) & 1];
        if (src == nullptr) {
            if (to_last)
                pass_sel<T>(R, gfirst, last, P.L, Ns, magic, twp, g);
            else
                pass_sel<T>(R, gfirst, GSt<T>{buf[p & 1]}, P.L, Ns, magic, twp, g);
        } else {
            if (to_last)
                pass_sel<T>(R, CLd<T>{src}, last, P.L, Ns, magic, twp, g);
            else
                pass_sel<T>(R, CLd<T>{src}, GSt<T>{buf[p & 1]}, P.L, Ns, magic, twp, g);
        }
        __threadfence_block();
        g.sync();
        Ns *= R;
    }
    return keep ? buf[(P.npass - 1) & 1] : nullptr;
}

// Copy the two-level twiddle table of length L from global memory into `dst`
// (shared memory); returns the table view.  Caller synchronises.
template <typename T>
__device__ __forceinline__ TwTab<T> load_twiddles(cx<T>* dst, const cx<T>* __restrict__ src, int L, const Group& g) {
    const int n = tw_table_elems(L);
    for (int i = g.tid; i < n; i += g.nthr) dst[i] = ldg_cx(src + i);
    return TwTab<T>{dst, dst + (L + TW_LO - 1) / TW_LO};
}

}  // namespace hk
