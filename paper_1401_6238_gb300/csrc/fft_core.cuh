// fft_core.cuh -- shared-memory mixed-radix FFT building blocks (sm_103a).
//
// Every transform here is the unscaled forward DFT of Section 2.1,
// X_k = sum_j x_j exp(-2 pi i j k / L); the scaled inverse the paper calls
// ifft is obtained by the callers as conj(fft(conj(.)))/L, so only one
// direction is compiled.
//
// A length-L transform is a sequence of Stockham radix-R passes
// (L = R_0 R_1 ... R_{P-1}, Ns = R_0 ... R_{p-1} before pass p).  In pass p
// butterfly b in [0, L/R) takes the R inputs b + r L/R, multiplies input r by
// w_{Ns R}^{r k} with k = b mod Ns, applies the radix-R DFT and writes output
// r to (b - k) R + k + r Ns.  After the last pass the data are in natural
// order, so no digit reversal is ever needed.  Each thread keeps its
// butterflies' inputs in registers, which makes the pass in-place in shared
// memory (all reads, one barrier, all writes); the first pass may read global
// memory directly (zero-padding fused into the load) and the last pass may
// write global memory directly (truncation fused into the store).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "jobs.h"

namespace hk {

template <typename T>
struct __align__(2 * sizeof(T)) cx {
    T x, y;
};

template <typename T>
__device__ __forceinline__ cx<T> mk(T a, T b) {
    cx<T> r;
    r.x = a;
    r.y = b;
    return r;
}
template <typename T>
__device__ __forceinline__ cx<T> operator+(cx<T> a, cx<T> b) { return mk<T>(a.x + b.x, a.y + b.y); }
template <typename T>
__device__ __forceinline__ cx<T> operator-(cx<T> a, cx<T> b) { return mk<T>(a.x - b.x, a.y - b.y); }
// FP32 complex add / subtract as one packed f32x2 operation each
// (sm_100 family); FP64 stays scalar.
__device__ __forceinline__ cx<float> operator+(cx<float> a, cx<float> b) {
    const float2 r = __fadd2_rn(make_float2(a.x, a.y), make_float2(b.x, b.y));
    return mk<float>(r.x, r.y);
}
__device__ __forceinline__ cx<float> operator-(cx<float> a, cx<float> b) {
    const float2 r = __ffma2_rn(make_float2(b.x, b.y), make_float2(-1.f, -1.f), make_float2(a.x, a.y));
    return mk<float>(r.x, r.y);
}

template <typename T>
__device__ __forceinline__ cx<T> cmul(cx<T> a, cx<T> b) {
    return mk<T>(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
template <typename T>
__device__ __forceinline__ cx<T> conjg(cx<T> a) { return mk<T>(a.x, -a.y); }
template <typename T>
__device__ __forceinline__ cx<T> scal(cx<T> a, T s) { return mk<T>(a.x * s, a.y * s); }
// read-only cached load of a complex value
__device__ __forceinline__ cx<float> ldg_cx(const cx<float>* p) {
    const float2 v = __ldg(reinterpret_cast<const float2*>(p));
    return mk<float>(v.x, v.y);
}
__device__ __forceinline__ cx<double> ldg_cx(const cx<double>* p) {
    const double2 v = __ldg(reinterpret_cast<const double2*>(p));
    return mk<double>(v.x, v.y);
}
// multiply by -i and by +i
template <typename T>
__device__ __forceinline__ cx<T> mul_ni(cx<T> a) { return mk<T>(a.y, -a.x); }
template <typename T>
__device__ __forceinline__ cx<T> mul_pi(cx<T> a) { return mk<T>(-a.y, a.x); }

// ---------------------------------------------------------------- radices
// Constants of the small DFTs: cos and sin of 2 pi q / R.
struct K {
    static constexpr double SQRT1_2 = 0.70710678118654752440;
    static constexpr double C8 = 0.92387953251128675613;  // cos(pi/8)
    static constexpr double S8 = 0.38268343236508977173;  // sin(pi/8)
};

__host__ __device__ constexpr double cos_2pi(int R, int q) {
    // cos(2 pi q / R) for R in {3, 5, 7}, any q (reduced mod R)
    return (q % R == 0) ? 1.0
         : R == 3 ? -0.5
         : R == 5 ? (((q % 5) == 1 || (q % 5) == 4) ? 0.30901699437494742410 : -0.80901699437494742410)
         : ((q % 7) == 1 || (q % 7) == 6) ? 0.62348980185873353053
         : ((q % 7) == 2 || (q % 7) == 5) ? -0.22252093395631440429
         : -0.90096886790241912624;
}
__host__ __device__ constexpr double sin_2pi(int R, int q) {
    // sin(2 pi q / R) for R in {3, 5, 7}
    return (q % R == 0) ? 0.0
         : R == 3 ? ((q % 3) == 1 ? 0.86602540378443864676 : -0.86602540378443864676)
         : R == 5 ? ((q % 5) == 1 ? 0.95105651629515357212
                   : (q % 5) == 2 ? 0.58778525229247312917
                   : (q % 5) == 3 ? -0.58778525229247312917
                   : -0.95105651629515357212)
         : (q % 7) == 1 ? 0.78183148246802980871
         : (q % 7) == 2 ? 0.97492791218182360702
         : (q % 7) == 3 ? 0.43388373911755812048
         : (q % 7) == 4 ? -0.43388373911755812048
         : (q % 7) == 5 ? -0.97492791218182360702
         : -0.78183148246802980871;
}

template <typename T, int R>
struct DFT;

template <typename T>
struct DFT<T, 2> {
    static __device__ __forceinline__ void run(cx<T>* a) {
        cx<T> t = a[0] - a[1];
        a[0] = a[0] + a[1];
        a[1] = t;
    }
};

template <typename T>
struct DFT<T, 4> {
    static __device__ __forceinline__ void run(cx<T>* a) {
        cx<T> t0 = a[0] + a[2], t1 = a[0] - a[2];
        cx<T> t2 = a[1] + a[3], t3 = mul_ni(a[1] - a[3]);
        a[0] = t0 + t2;
        a[2] = t0 - t2;
        a[1] = t1 + t3;
        a[3] = t1 - t3;
    }
};

template <typename T>
struct DFT<T, 8> {
    static __device__ __forceinline__ void run(cx<T>* a) {
        cx<T> e[4] = {a[0], a[2], a[4], a[6]};
        cx<T> o[4] = {a[1], a[3], a[5], a[7]};
        DFT<T, 4>::run(e);
        DFT<T, 4>::run(o);
        const T c = (T)K::SQRT1_2;
        // o_k *= w8^k, w8 = exp(-i pi / 4)
        o[1] = mk<T>((o[1].x + o[1].y) * c, (o[1].y - o[1].x) * c);
        o[2] = mul_ni(o[2]);
        o[3] = mk<T>((o[3].y - o[3].x) * c, -(o[3].x + o[3].y) * c);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            a[k] = e[k] + o[k];
            a[k + 4] = e[k] - o[k];
        }
    }
};

template <typename T>
struct DFT<T, 16> {
    static __device__ __forceinline__ void run(cx<T>* a) {
        cx<T> e[8], o[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            e[k] = a[2 * k];
            o[k] = a[2 * k + 1];
        }
        DFT<T, 8>::run(e);
        DFT<T, 8>::run(o);
        const T c1 = (T)K::C8, s1 = (T)K::S8, h = (T)K::SQRT1_2;
        // o_k *= w16^k, w16 = exp(-i pi / 8)
        o[1] = cmul(o[1], mk<T>(c1, -s1));
        o[2] = mk<T>((o[2].x + o[2].y) * h, (o[2].y - o[2].x) * h);
        o[3] = cmul(o[3], mk<T>(s1, -c1));
        o[4] = mul_ni(o[4]);
        o[5] = cmul(o[5], mk<T>(-s1, -c1));
        o[6] = mk<T>((o[6].y - o[6].x) * h, -(o[6].x + o[6].y) * h);
        o[7] = cmul(o[7], mk<T>(-c1, -s1));
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            a[k] = e[k] + o[k];
            a[k + 8] = e[k] - o[k];
        }
    }
};

// Odd prime radix: with s_j = a_j + a_{R-j}, d_j = a_j - a_{R-j},
// X_k = A_k - i B_k and X_{R-k} = A_k + i B_k where
// A_k = a_0 + sum_j s_j cos(2 pi j k / R), B_k = sum_j d_j sin(2 pi j k / R).
template <typename T, int R>
struct DFTodd {
    static __device__ __forceinline__ void run(cx<T>* a) {
        constexpr int H = (R - 1) / 2;
        cx<T> s[H], d[H];
#pragma unroll
        for (int j = 1; j <= H; ++j) {
            s[j - 1] = a[j] + a[R - j];
            d[j - 1] = a[j] - a[R - j];
        }
        cx<T> out[R];
        cx<T> x0 = a[0];
#pragma unroll
        for (int j = 0; j < H; ++j) x0 = x0 + s[j];
        out[0] = x0;
#pragma unroll
        for (int k = 1; k <= H; ++k) {
            cx<T> A = a[0];
            cx<T> B = mk<T>(0, 0);
#pragma unroll
            for (int j = 1; j <= H; ++j) {
                const T c = (T)cos_2pi(R, j * k);
                const T sn = (T)sin_2pi(R, j * k);
                A = mk<T>(fma(c, s[j - 1].x, A.x), fma(c, s[j - 1].y, A.y));
                B = mk<T>(fma(sn, d[j - 1].x, B.x), fma(sn, d[j - 1].y, B.y));
            }
            out[k] = A + mul_ni(B);
            out[R - k] = A + mul_pi(B);
        }
#pragma unroll
        for (int k = 0; k < R; ++k) a[k] = out[k];
    }
};
template <typename T>
struct DFT<T, 3> : DFTodd<T, 3> {};
template <typename T>
struct DFT<T, 5> : DFTodd<T, 5> {};
template <typename T>
struct DFT<T, 7> : DFTodd<T, 7> {};

// Composite radix N = N1 N2 with coprime factors by the prime-factor
// (Good-Thomas) map: input n = (N2 n1 + N1 n2) mod N, output
// k = (N2 e1 k1 + N1 e2 k2) mod N with e1 = N2^-1 mod N1, e2 = N1^-1 mod N2,
// so that w_N^{nk} = w_N1^{n1 k1} w_N2^{n2 k2}: N2 transforms of size N1,
// then N1 of size N2, with no twiddle factors between them.
__host__ __device__ constexpr int inv_mod(int a, int m) {
    int r = 1;
    while ((a * r) % m != 1) ++r;
    return r;
}
template <typename T, int N1, int N2>
struct DFTpfa {
    static __device__ __forceinline__ void run(cx<T>* a) {
        constexpr int N = N1 * N2;
        constexpr int e1 = inv_mod(N2 % N1, N1), e2 = inv_mod(N1 % N2, N2);
        cx<T> A[N2][N1];
#pragma unroll
        for (int n2 = 0; n2 < N2; ++n2) {
#pragma unroll
            for (int n1 = 0; n1 < N1; ++n1) A[n2][n1] = a[(N2 * n1 + N1 * n2) % N];
            DFT<T, N1>::run(A[n2]);
        }
#pragma unroll
        for (int k1 = 0; k1 < N1; ++k1) {
            cx<T> B[N2];
#pragma unroll
            for (int n2 = 0; n2 < N2; ++n2) B[n2] = A[n2][k1];
            DFT<T, N2>::run(B);
#pragma unroll
            for (int k2 = 0; k2 < N2; ++k2) a[(N2 * e1 * k1 + N1 * e2 * k2) % N] = B[k2];
        }
    }
};
template <typename T>
struct DFT<T, 12> : DFTpfa<T, 4, 3> {};
template <typename T>
struct DFT<T, 20> : DFTpfa<T, 4, 5> {};

// ------------------------------------------------------------- shared memory
// One padding slot every 16 elements spreads strided butterfly accesses over
// the banks.
__device__ __forceinline__ int sp(int i) { return i + (i >> 4); }
__host__ __device__ constexpr int smem_elems(int L) { return L + (L >> 4) + 1; }

struct Group {
    int tid, nthr, bar;  // bar 0: the whole block; > 0: named barrier; < 0: lanes `mask` of one warp
    unsigned mask = 0xffffffffu;
    __device__ __forceinline__ void sync() const {
        if (bar == 0) {
            __syncthreads();
        } else if (bar > 0) {
            asm volatile("bar.sync %0, %1;" ::"r"(bar), "r"(nthr) : "memory");
        } else {
            __syncwarp(mask);
        }
    }
};

template <typename T>
struct Smem {
    cx<T>* p;
    __device__ __forceinline__ cx<T> operator()(int i) const { return p[sp(i)]; }
    __device__ __forceinline__ void operator()(int i, cx<T> v) const { p[sp(i)] = v; }
};

// One Stockham pass, out of place: `src` and `dst` never alias.  Each loop
// iteration is one butterfly, so a thread holds only R values.  Callers put a
// barrier after the pass whenever its output is read by other threads.
template <typename T, int R, class Src, class Dst>
__device__ __forceinline__ void pass_r(const Src& src, const Dst& dst, int L, int Ns,
                                       const cx<T>* __restrict__ tw, const Group& g) {
    const int nb = L / R;
    const int twstride = L / (Ns * R);
    for (int b = g.tid; b < nb; b += g.nthr) {
        cx<T> v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = src(b + r * nb);
        const int k = b % Ns;
        if (Ns > 1) {
            const int kk = k * twstride;
#pragma unroll
            for (int r = 1; r < R; ++r) v[r] = cmul(v[r], ldg_cx(&tw[r * kk]));
        }
        DFT<T, R>::run(v);
        const int base = (b - k) * R + k;
#pragma unroll
        for (int r = 0; r < R; ++r) dst(base + r * Ns, v[r]);
    }
}

template <typename T, class Src, class Dst>
__device__ __forceinline__ void pass_any(int R, const Src& src, const Dst& dst, int L, int Ns,
                                         const cx<T>* __restrict__ tw, const Group& g) {
    switch (R) {
        case 16: pass_r<T, 16>(src, dst, L, Ns, tw, g); break;
        case 8: pass_r<T, 8>(src, dst, L, Ns, tw, g); break;
        case 4: pass_r<T, 4>(src, dst, L, Ns, tw, g); break;
        case 2: pass_r<T, 2>(src, dst, L, Ns, tw, g); break;
        case 3: pass_r<T, 3>(src, dst, L, Ns, tw, g); break;
        case 5: pass_r<T, 5>(src, dst, L, Ns, tw, g); break;
        case 7: pass_r<T, 7>(src, dst, L, Ns, tw, g); break;
        default: break;  // the planner only emits the radices above
    }
}

// Transform whose result stays in shared memory.  Pass 0 reads `first`
// (a global loader or a combining functor); the passes ping-pong between
// b0 and b1, which must both be free on entry.  Returns the buffer holding
// the result, after a barrier.
template <typename T, class Src>
__device__ __forceinline__ cx<T>* fft_smem(const FftPlan& P, const Src& first, cx<T>* b0, cx<T>* b1,
                                           const cx<T>* __restrict__ tw, const Group& g) {
    cx<T>* buf[2] = {b0, b1};
    int Ns = 1;
    pass_any<T>(P.radix[0], first, Smem<T>{b0}, P.L, Ns, tw, g);
    g.sync();
    Ns *= P.radix[0];
    for (int p = 1; p < P.npass; ++p) {
        pass_any<T>(P.radix[p], Smem<T>{buf[(p - 1) & 1]}, Smem<T>{buf[p & 1]}, P.L, Ns, tw, g);
        g.sync();
        Ns *= P.radix[p];
    }
    return buf[(P.npass - 1) & 1];
}

// Transform whose last pass writes through `last` (a global sink): pass 0
// reads `first`, intermediate passes ping-pong between b0 and b1.
template <typename T, class Src, class Dst>
__device__ __forceinline__ void fft_out(const FftPlan& P, const Src& first, cx<T>* b0, cx<T>* b1, const Dst& last,
                                        const cx<T>* __restrict__ tw, const Group& g) {
    if (P.npass == 1) {
        pass_any<T>(P.radix[0], first, last, P.L, 1, tw, g);
        return;
    }
    cx<T>* buf[2] = {b0, b1};
    int Ns = 1;
    pass_any<T>(P.radix[0], first, Smem<T>{b0}, P.L, Ns, tw, g);
    g.sync();
    Ns *= P.radix[0];
    for (int p = 1; p < P.npass - 1; ++p) {
        pass_any<T>(P.radix[p], Smem<T>{buf[(p - 1) & 1]}, Smem<T>{buf[p & 1]}, P.L, Ns, tw, g);
        g.sync();
        Ns *= P.radix[p];
    }
    pass_any<T>(P.radix[P.npass - 1], Smem<T>{buf[(P.npass - 2) & 1]}, last, P.L, Ns, tw, g);
}

// Block-wide sum of one double per thread (result valid in thread 0).
__device__ __forceinline__ double group_sum(double v, double* red, const Group& g) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int w = g.tid >> 5, nw = (g.nthr + 31) >> 5;
    if ((g.tid & 31) == 0) red[w] = v;
    g.sync();
    double s = 0.0;
    if (g.tid == 0)
        for (int i = 0; i < nw; ++i) s += red[i];
    g.sync();
    return s;
}

}  // namespace hk
