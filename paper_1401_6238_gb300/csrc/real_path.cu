// real_path.cu -- fused kernels for real Hankel tensors: square tensors with
// one vector per tensor, y = H x^{m-1} and alpha = H x^m (Section 2.1
// notation, Section 3 procedures) and their adjoints, and tensors with a
// different vector in every mode (real_multi_kernel, the m + 1 transform
// form of Section 3).
//
// Forward, pair job (tensors A, B with the same FFT length L):
//   S1 = fft(h~_A + i h~_B), S2 = fft(x~_A + i x~_B)      (zero-pad on load)
//   H_A = (S1_k + conj S1_{L-k})/2, H_B = -i (S1_k - conj S1_{L-k})/2, same for X
//   ifft(h~) = conj(H)/L for real h, P = ifft(h~) .* X^{m-1}   (Section 3)
//   y~ = fft(P_A + i P_B): y_A = Re y~[0:n_A], y_B = Im y~[0:n_B] (truncate on store)
// P_A, P_B are Hermitian, so their transforms are real and one complex
// transform returns both.  alpha = sum_k ifft(h~)_k X_k^m needs no final
// transform.  A single job packs h + i x into one transform instead.
//
// Backward (single jobs): with g = dLoss/dy and U = fft(h~ + i x~), G = fft(g~),
//   grad_h = ifft(G .* X^{m-1})[0:d]            (linear convolution g * z)
//   grad_x = (m-1) fft(ifft(h~) .* G .* X^{m-2})[0:n]
// Both spectra are Hermitian; ifft(Q)[j] = fft(Q)[(L-j) mod L]/L, so one
// forward transform of Q_h/L + i Q_x returns grad_h (real part, index
// reversed) and grad_x (imaginary part).
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <utility>

#include "fft_stage.cuh"
#include "launch.h"

namespace cg = cooperative_groups;

namespace hk {

// shared-memory slots reserved for the twiddle table (largest L = 16384)
constexpr int TW_SMEM = tw_table_elems(16384);

template <typename T>
struct PairLoad {
    const T* a;
    int na;
    const T* b;
    int nb;
    __device__ __forceinline__ cx<T> operator()(int i) const {
        return mk<T>(i < na ? __ldg(a + i) : T(0), i < nb ? __ldg(b + i) : T(0));
    }
};

template <typename T>
struct PairStore {
    T* a;
    int na;
    T* b;
    int nb;
    __device__ __forceinline__ void operator()(int i, cx<T> v) const {
        if (i < na) a[i] = v.x;
        if (i < nb) b[i] = v.y;
    }
};

template <typename T>
struct AdjStore {
    T* gh;
    int d;
    T* gx;
    int n;
    int L;
    __device__ __forceinline__ void operator()(int i, cx<T> v) const {
        const int j = (i == 0) ? 0 : L - i;
        if (gh != nullptr && j < d) gh[j] = v.x;
        if (gx != nullptr && i < n) gx[i] = v.y;
    }
};

template <typename A, typename T>
__device__ __forceinline__ cx<A> up(cx<T> v) { return mk<A>((A)v.x, (A)v.y); }

// p X^e for 0 <= e <= 7 by binary powering (straight-line, depth <= 3).
template <typename A>
__device__ __forceinline__ cx<A> times_pow(cx<A> p, cx<A> X, int e) {
    if (e & 1) p = cmul(p, X);
    if (e & 6) {
        const cx<A> X2 = cmul(X, X);
        if (e & 2) p = cmul(p, X2);
        if (e & 4) p = cmul(p, cmul(X2, X2));
    }
    return p;
}

// k-th and (L-k)-th bins of two real signals packed as a + i b.
template <typename T>
__device__ __forceinline__ void unpack(cx<T> u, cx<T> w_conj, cx<T>& a, cx<T>& b) {
    a = scal(u + w_conj, T(0.5));
    b = scal(mul_ni(u - w_conj), T(0.5));
}

// Spectral product of one tensor at bin k: P = ifft(h~)_k X_k^{m-1}, plus the
// alpha term ifft(h~)_k X_k^m; formed in A precision, the alpha term rounded
// to the data type T (summed in T per thread: FP64 instructions hold this
// GPU's narrow FP64 pipe for many cycles, and FP32 data carry FP32 rounding
// already).
template <typename A, typename T>
__device__ __forceinline__ cx<T> product(cx<T> Hk, cx<T> Xk, int m, T invL, T& aterm, bool want_alpha = true) {
    const cx<A> hh = scal(up<A>(conjg(Hk)), (A)invL);
    const cx<A> X = up<A>(Xk);
    const cx<A> p = times_pow(hh, X, m - 1);
    if (want_alpha) aterm = (T)cmul(p, X).x;
    return mk<T>((T)p.x, (T)p.y);
}

// Alpha contribution of bins k and L-k (their terms are complex conjugates).
template <typename T>
__device__ __forceinline__ T alpha_term(cx<T> Hk, cx<T> Xk, int m, T invL, bool fp64, int k, int kc) {
    T at = T(0);
    if (fp64)
        product<double>(Hk, Xk, m, invL, at);
    else
        product<T>(Hk, Xk, m, invL, at);
    return (k == kc) ? at : T(2) * at;
}

template <typename T>
__global__ void __launch_bounds__(512) real_fwd_kernel(const RealJob* __restrict__ jobs, int first,
                                                        const T* __restrict__ h, const T* __restrict__ x,
                                                        T* __restrict__ y, T* __restrict__ alpha,
                                                        const cx<T>* __restrict__ tw_all, cx<T>* __restrict__ ws,
                                                        int Lmax, int flags) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double* red = reinterpret_cast<double*>(smem_raw);
    cx<T>* tws = reinterpret_cast<cx<T>*>(smem_raw + RED_BYTES);
    cx<T>* bA = tws + TW_SMEM;
    cx<T>* bB = bA + smem_elems(Lmax);
    cx<T>* bC = bB + smem_elems(Lmax);
    const RealJob J = jobs[first + blockIdx.x];
    const Group g{(int)threadIdx.x, (int)blockDim.x, 0};
    const FftPlan P = J.P;
    const int L = P.L;
    const TwTab<T> tw = load_twiddles(tws, tw_all + P.tw_off, L, g);
    const bool fp64 = (flags & HANKEL_FP64_POWER) != 0;
    const T invL = T(1) / T(L);
    const PairSt<T> store{y + J.yA, J.nA, y + J.yB, J.single ? 0 : J.nB};
    T aA = T(0), aB = T(0);
    cx<T>*S1, *F, *O;

    g.sync();
    if (J.single) {
        // S = fft(h~ + i x~); Q_k = ifft(h~)_k X_k^{m-1}
        S1 = fft_stage<T>(P, GLd<T>{h + J.hA, J.dA, x + J.xA, J.nA}, nullptr, bA, bB, store, true, tw, g);
        F = (S1 == bA) ? bB : bA;
        if (flags & HANKEL_STORE_SPECTRA)
            for (int k = g.tid; k < L; k += g.nthr) ws[J.wsA + k] = S1[sp(k)];
        for (int k = g.tid; k <= L / 2; k += g.nthr) {
            const int kc = (k == 0) ? 0 : L - k;
            cx<T> Hk, Xk;
            unpack(S1[sp(k)], conjg(S1[sp(kc)]), Hk, Xk);
            T at = T(0);
            const bool wa = alpha != nullptr;
            const cx<T> Pk =
                fp64 ? product<double>(Hk, Xk, J.mA, invL, at, wa) : product<T>(Hk, Xk, J.mA, invL, at, wa);
            if (wa) aA += (k == kc) ? at : T(2) * at;
            F[sp(k)] = Pk;
            if (kc != k) F[sp(kc)] = conjg(Pk);
        }
        O = S1;
    } else {
        // S1 = fft(h~_A + i h~_B), S2 = fft(x~_A + i x~_B); Q_k = P_A,k + i P_B,k
        // both inputs stream into shared memory asynchronously; the x pair
        // arrives while the h pair is being transformed
        cp_async_pair(bA, h + J.hA, J.dA, h + J.hB, J.dB, L, g);
        cp_async_pair(bC, x + J.xA, J.nA, x + J.xB, J.nB, L, g);
        cp_wait<1>();
        g.sync();
        const GLd<T> none{nullptr, 0, nullptr, 0};
        S1 = fft_stage<T>(P, none, bA, bB, bA, store, true, tw, g);
        cx<T>* other = (S1 == bA) ? bB : bA;
        cp_wait<0>();
        g.sync();
        cx<T>* S2 = fft_stage<T>(P, none, bC, other, bC, store, true, tw, g);
        F = (S2 == bC) ? other : bC;
        for (int k = g.tid; k <= L / 2; k += g.nthr) {
            const int kc = (k == 0) ? 0 : L - k;
            cx<T> HA, HB, XA, XB;
            unpack(S1[sp(k)], conjg(S1[sp(kc)]), HA, HB);
            unpack(S2[sp(k)], conjg(S2[sp(kc)]), XA, XB);
            T atA = T(0), atB = T(0);
            cx<T> PA, PB;
            const bool wa = alpha != nullptr;
            if (fp64) {
                PA = product<double>(HA, XA, J.mA, invL, atA, wa);
                PB = product<double>(HB, XB, J.mB, invL, atB, wa);
            } else {
                PA = product<T>(HA, XA, J.mA, invL, atA, wa);
                PB = product<T>(HB, XB, J.mB, invL, atB, wa);
            }
            if (wa) {
                aA += (k == kc) ? atA : T(2) * atA;
                aB += (k == kc) ? atB : T(2) * atB;
            }
            F[sp(k)] = PA + mul_pi(PB);
            if (kc != k) F[sp(kc)] = conjg(PA) + mul_pi(conjg(PB));
        }
        O = S1;
    }
    g.sync();
    if (y != nullptr) fft_stage<T>(P, GLd<T>{nullptr, 0, nullptr, 0}, F, O, F, store, false, tw, g);
    if (alpha != nullptr) {
        const double sA = group_sum((double)aA, red, g);
        const double sB = J.single ? 0.0 : group_sum((double)aB, red, g);
        if (g.tid == 0) {
            alpha[J.iA] = (T)sA;
            if (!J.single && J.iB >= 0) alpha[J.iB] = (T)sB;
        }
    }
}

// Pair of real tensors with distinct mode vectors (MultiJob).  acc holds the
// running spectral products P_A = ifft(h~_A) X_{A,2} ... and P_B for the
// bins k = 0..L/2 (the rest follow by Hermitian symmetry): P_A at slot k,
// P_B at slot L - k; at the self-paired bins 0 and L/2 both are real and
// share one slot (real part A, imaginary part B).
template <typename T>
__global__ void __launch_bounds__(512) real_multi_kernel(const MultiJob* __restrict__ jobs, int first,
                                                          const T* __restrict__ h, const T* __restrict__ x,
                                                          T* __restrict__ y, T* __restrict__ alpha,
                                                          const cx<T>* __restrict__ tw_all, int Lmax) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double* red = reinterpret_cast<double*>(smem_raw);
    cx<T>* tws = reinterpret_cast<cx<T>*>(smem_raw + RED_BYTES);
    cx<T>* bA = tws + TW_SMEM;
    cx<T>* bB = bA + smem_elems(Lmax);
    cx<T>* acc = bB + smem_elems(Lmax);
    const MultiJob& J = jobs[first + blockIdx.x];
    const Group g{(int)threadIdx.x, (int)blockDim.x, 0};
    const FftPlan P = J.P;
    const int L = P.L;
    const TwTab<T> tw = load_twiddles(tws, tw_all + P.tw_off, L, g);
    const bool two = J.iB >= 0;
    const int mA = J.mA, mB = two ? J.mB : 0;
    const T invL = T(1) / T(L);
    const PairSt<T> keep_st{nullptr, 0, nullptr, 0};
    g.sync();
    // ifft(h~) = conj(fft(h~)) / L for both tensors
    cx<T>* S = fft_stage<T>(P, GLd<T>{h + J.hA, J.dA, two ? h + J.hB : nullptr, two ? J.dB : 0}, nullptr, bA, bB,
                            keep_st, true, tw, g);
    for (int k = g.tid; k <= L / 2; k += g.nthr) {
        const int kc = (k == 0) ? 0 : L - k;
        cx<T> HA, HB;
        unpack(S[sp(k)], conjg(S[sp(kc)]), HA, HB);
        if (kc == k) {
            acc[sp(k)] = mk<T>(HA.x * invL, HB.x * invL);
        } else {
            acc[sp(k)] = scal(conjg(HA), invL);
            acc[sp(kc)] = scal(conjg(HB), invL);
        }
    }
    g.sync();
    // modes 2..m: one transform of x_{A,p} + i x_{B,p} each, multiplied in
    const int mmax = max(mA, mB);
    for (int p = 1; p < mmax; ++p) {
        const bool inA = p < mA, inB = p < mB;
        S = fft_stage<T>(P, GLd<T>{inA ? x + J.xA[p] : nullptr, inA ? J.nA[p] : 0, inB ? x + J.xB[p] : nullptr,
                                   inB ? J.nB[p] : 0},
                         nullptr, bA, bB, keep_st, true, tw, g);
        for (int k = g.tid; k <= L / 2; k += g.nthr) {
            const int kc = (k == 0) ? 0 : L - k;
            cx<T> XA, XB;
            unpack(S[sp(k)], conjg(S[sp(kc)]), XA, XB);
            if (kc == k) {
                const cx<T> v = acc[sp(k)];
                acc[sp(k)] = mk<T>(inA ? v.x * XA.x : v.x, inB ? v.y * XB.x : v.y);
            } else {
                if (inA) acc[sp(k)] = cmul(acc[sp(k)], XA);
                if (inB) acc[sp(kc)] = cmul(acc[sp(kc)], XB);
            }
        }
        g.sync();
    }
    if (y != nullptr) {
        // Q = P_A + i P_B on all L bins; fft(Q) = y_A + i y_B (both real)
        for (int k = g.tid; k <= L / 2; k += g.nthr) {
            const int kc = (k == 0) ? 0 : L - k;
            if (kc == k) {
                bA[sp(k)] = acc[sp(k)];
            } else {
                const cx<T> PA = acc[sp(k)], PB = acc[sp(kc)];
                bA[sp(k)] = PA + mul_pi(PB);
                bA[sp(kc)] = conjg(PA) + mul_pi(conjg(PB));
            }
        }
        g.sync();
        fft_stage<T>(P, GLd<T>{nullptr, 0, nullptr, 0}, bA, bB, bA,
                     PairSt<T>{y + J.yA, J.nA[0], two ? y + J.yB : nullptr, two ? J.nB[0] : 0}, false, tw, g);
    }
    if (alpha != nullptr) {
        // alpha = sum_k P_k X_{1,k}: bins k and L - k contribute complex conjugates
        S = fft_stage<T>(P, GLd<T>{x + J.xA[0], J.nA[0], two ? x + J.xB[0] : nullptr, two ? J.nB[0] : 0}, nullptr,
                         bA, bB, keep_st, true, tw, g);
        T aA = T(0), aB = T(0);
        for (int k = g.tid; k <= L / 2; k += g.nthr) {
            const int kc = (k == 0) ? 0 : L - k;
            cx<T> XA, XB;
            unpack(S[sp(k)], conjg(S[sp(kc)]), XA, XB);
            // terms and each thread's sums in T precision; FP64 only for the
            // sum over the block (FP64 arithmetic is slow on this part)
            T tA, tB;
            if (kc == k) {
                const cx<T> v = acc[sp(k)];
                tA = v.x * XA.x;
                tB = v.y * XB.x;
            } else {
                const cx<T> PA = acc[sp(k)], PB = acc[sp(kc)];
                tA = T(2) * (PA.x * XA.x - PA.y * XA.y);
                tB = T(2) * (PB.x * XB.x - PB.y * XB.y);
            }
            aA += tA;
            aB += tB;
        }
        const double sA = group_sum((double)aA, red, g);
        const double sB = two ? group_sum((double)aB, red, g) : 0.0;
        if (g.tid == 0) {
            alpha[J.iA] = (T)sA;
            if (two) alpha[J.iB] = (T)sB;
        }
    }
}

template <typename A, typename T>
__device__ __forceinline__ cx<T> adjoint_bin(cx<T> U, cx<T> Wc, cx<T> G, int m, T invL) {
    cx<T> Hk, Xk;
    unpack(U, Wc, Hk, Xk);
    const cx<A> X = up<A>(Xk);
    const cx<A> Gk = up<A>(G);
    const cx<A> hh = scal(up<A>(conjg(Hk)), (A)invL);
    const cx<A> gxm2 = times_pow(Gk, X, m - 2);        // G X^{m-2}
    const cx<A> qh = scal(cmul(gxm2, X), (A)invL);      // G X^{m-1} / L
    const cx<A> qx = scal(cmul(hh, gxm2), (A)(m - 1));  // (m-1) ifft(h~) G X^{m-2}
    return mk<T>((T)(qh.x - qx.y), (T)(qh.y + qx.x));   // qh + i qx
}

template <typename T>
__global__ void __launch_bounds__(512) real_bwd_kernel(const RealJob* __restrict__ jobs, int first,
                                                        const T* __restrict__ gy, const T* __restrict__ h,
                                                        const T* __restrict__ x, T* __restrict__ gh,
                                                        T* __restrict__ gx, const cx<T>* __restrict__ tw_all,
                                                        cx<T>* ws, int Lmax, int flags, int stored) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cx<T>* tws = reinterpret_cast<cx<T>*>(smem_raw + RED_BYTES);
    cx<T>* bA = tws + TW_SMEM;
    cx<T>* bB = bA + smem_elems(Lmax);
    const RealJob J = jobs[first + blockIdx.x];
    const Group g{(int)threadIdx.x, (int)blockDim.x, 0};
    const FftPlan P = J.P;
    const int L = P.L;
    const TwTab<T> tw = load_twiddles(tws, tw_all + P.tw_off, L, g);
    g.sync();
    const bool fp64 = (flags & HANKEL_FP64_POWER) != 0;
    const T invL = T(1) / T(L);
    cx<T>* U = ws + J.wsA;

    // U = fft(h~ + i x~) straight to workspace (or kept from the forward call)
    if (!stored) fft_stage<T>(P, GLd<T>{h + J.hA, J.dA, x + J.xA, J.nA}, nullptr, bA, bB, GSt<T>{U}, false, tw, g);
    const AdjSt<T> store{gh ? gh + J.hA : nullptr, J.dA, gx ? gx + J.xA : nullptr, J.nA, L};
    cx<T>* G = fft_stage<T>(P, GLd<T>{gy + J.yA, J.nA, nullptr, 0}, nullptr, bA, bB, store, true, tw, g);
    cx<T>* F = (G == bA) ? bB : bA;
    for (int k = g.tid; k < L; k += g.nthr) {
        const int kc = (k == 0) ? 0 : L - k;
        const cx<T> Uk = U[k], Uc = conjg(U[kc]), Gk = G[sp(k)];
        F[sp(k)] = fp64 ? adjoint_bin<double>(Uk, Uc, Gk, J.mA, invL) : adjoint_bin<T>(Uk, Uc, Gk, J.mA, invL);
    }
    g.sync();
    fft_stage<T>(P, GLd<T>{nullptr, 0, nullptr, 0}, F, G, F, store, false, tw, g);
}

// Pair jobs of the adjoint: tensors A and B with one FFT length share the
// transform of their upstream gradients, G = fft(g~_A + i g~_B), unpacked per
// bin (G_A = (G_k + conj G_{L-k})/2, G_B = -i (G_k - conj G_{L-k})/2); U_A
// and U_B = fft(h~ + i x~) go to (or come from) workspace as in the single
// job, and each tensor's Q then takes one transform: five transforms per pair
// instead of six.  G stays in buffer bC while A's and B's transforms use bA
// and bB.  iB < 0: tensor A alone.
template <typename T>
__global__ void __launch_bounds__(512) real_bwd_pair_kernel(const RealJob* __restrict__ jobs, int first,
                                                             const T* __restrict__ gy, const T* __restrict__ h,
                                                             const T* __restrict__ x, T* __restrict__ gh,
                                                             T* __restrict__ gx, const cx<T>* __restrict__ tw_all,
                                                             cx<T>* ws, int Lmax, int flags, int stored) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cx<T>* tws = reinterpret_cast<cx<T>*>(smem_raw + RED_BYTES);
    cx<T>* bA = tws + TW_SMEM;
    cx<T>* bB = bA + smem_elems(Lmax);
    cx<T>* bC = bB + smem_elems(Lmax);
    const RealJob J = jobs[first + blockIdx.x];
    const Group g{(int)threadIdx.x, (int)blockDim.x, 0};
    const FftPlan P = J.P;
    const int L = P.L;
    const TwTab<T> tw = load_twiddles(tws, tw_all + P.tw_off, L, g);
    g.sync();
    const bool two = J.iB >= 0;
    const bool fp64 = (flags & HANKEL_FP64_POWER) != 0;
    const T invL = T(1) / T(L);
    cx<T>* UA = ws + J.wsA;
    cx<T>* UB = ws + J.wsB;
    const GLd<T> none{nullptr, 0, nullptr, 0};
    const AdjSt<T> stA{gh ? gh + J.hA : nullptr, J.dA, gx ? gx + J.xA : nullptr, J.nA, L};
    const AdjSt<T> stB{gh && two ? gh + J.hB : nullptr, J.dB, gx && two ? gx + J.xB : nullptr, J.nB, L};
    // U_A, U_B = fft(h~ + i x~) straight to workspace (or kept from the forward call)
    if (!stored) {
        fft_stage<T>(P, GLd<T>{h + J.hA, J.dA, x + J.xA, J.nA}, nullptr, bA, bB, GSt<T>{UA}, false, tw, g);
        if (two) fft_stage<T>(P, GLd<T>{h + J.hB, J.dB, x + J.xB, J.nB}, nullptr, bA, bB, GSt<T>{UB}, false, tw, g);
    }
    // G = fft(g~_A + i g~_B), ping-ponged so that it ends in bC (the last of
    // npass passes writes the first buffer when npass is odd): both tensors'
    // transforms then have bA and bB
    fft_stage<T>(P, GLd<T>{gy + J.yA, J.nA, two ? gy + J.yB : nullptr, two ? J.nB : 0}, nullptr,
                 (P.npass & 1) ? bC : bA, (P.npass & 1) ? bA : bC, stA, true, tw, g);
    for (int t = 0; t < (two ? 2 : 1); ++t) {
        const cx<T>* U = (t == 0) ? UA : UB;
        const int m = (t == 0) ? J.mA : J.mB;
        for (int k = g.tid; k < L; k += g.nthr) {
            const int kc = (k == 0) ? 0 : L - k;
            const cx<T> Gk = bC[sp(k)], Gc = conjg(bC[sp(kc)]);
            // G_A = (G_k + conj G_{L-k}) / 2, G_B = -i (G_k - conj G_{L-k}) / 2
            const cx<T> Gt = (t == 0) ? scal(Gk + Gc, T(0.5)) : scal(mul_ni(Gk - Gc), T(0.5));
            const cx<T> Uk = U[k], Uc = conjg(U[kc]);
            bA[sp(k)] = fp64 ? adjoint_bin<double>(Uk, Uc, Gt, m, invL) : adjoint_bin<T>(Uk, Uc, Gt, m, invL);
        }
        g.sync();
        fft_stage<T>(P, none, bA, bB, bA, (t == 0) ? stA : stB, false, tw, g);
    }
}

// Single jobs whose transforms exceed shared memory: the same steps with
// the transform scratch in global workspace (two L-buffers per job at wsB,
// L2-resident in practice); shared memory holds only the twiddle table.
template <typename T>
__global__ void __launch_bounds__(512) real_fwd_global_kernel(const RealJob* __restrict__ jobs, int first,
                                                               const T* __restrict__ h, const T* __restrict__ x,
                                                               T* __restrict__ y, T* __restrict__ alpha,
                                                               const cx<T>* __restrict__ tw_all, cx<T>* ws,
                                                               int flags) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double* red = reinterpret_cast<double*>(smem_raw);
    cx<T>* tws = reinterpret_cast<cx<T>*>(smem_raw + RED_BYTES);
    const RealJob J = jobs[first + blockIdx.x];
    const Group g{(int)threadIdx.x, (int)blockDim.x, 0};
    const FftPlan P = J.P;
    const int L = P.L;
    const TwTab<T> tw = load_twiddles(tws, tw_all + P.tw_off, L, g);
    g.sync();
    const bool fp64 = (flags & HANKEL_FP64_POWER) != 0;
    const T invL = T(1) / T(L);
    cx<T>* W0 = ws + J.wsB;
    cx<T>* W1 = W0 + L;
    const PairSt<T> store{y + J.yA, J.nA, nullptr, 0};
    cx<T>* S = fft_global<T>(P, GLd<T>{h + J.hA, J.dA, x + J.xA, J.nA}, nullptr, W0, W1, store, true, tw, g);
    cx<T>* F = (S == W0) ? W1 : W0;
    if (flags & HANKEL_STORE_SPECTRA)
        for (int k = g.tid; k < L; k += g.nthr) ws[J.wsA + k] = S[k];
    T aA = T(0);
    const bool wa = alpha != nullptr;
    for (int k = g.tid; k <= L / 2; k += g.nthr) {
        const int kc = (k == 0) ? 0 : L - k;
        cx<T> Hk, Xk;
        unpack(S[k], conjg(S[kc]), Hk, Xk);
        T at = T(0);
        const cx<T> Pk = fp64 ? product<double>(Hk, Xk, J.mA, invL, at, wa) : product<T>(Hk, Xk, J.mA, invL, at, wa);
        if (wa) aA += (k == kc) ? at : T(2) * at;
        F[k] = Pk;
        if (kc != k) F[kc] = conjg(Pk);
    }
    __threadfence_block();
    g.sync();
    if (y != nullptr) fft_global<T>(P, GLd<T>{nullptr, 0, nullptr, 0}, F, S, F, store, false, tw, g);
    if (wa) {
        const double sA = group_sum((double)aA, red, g);
        if (g.tid == 0) alpha[J.iA] = (T)sA;
    }
}

template <typename T>
__global__ void __launch_bounds__(512) real_bwd_global_kernel(const RealJob* __restrict__ jobs, int first,
                                                               const T* __restrict__ gy, const T* __restrict__ h,
                                                               const T* __restrict__ x, T* __restrict__ gh,
                                                               T* __restrict__ gx, const cx<T>* __restrict__ tw_all,
                                                               cx<T>* ws, int flags, int stored) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cx<T>* tws = reinterpret_cast<cx<T>*>(smem_raw + RED_BYTES);
    const RealJob J = jobs[first + blockIdx.x];
    const Group g{(int)threadIdx.x, (int)blockDim.x, 0};
    const FftPlan P = J.P;
    const int L = P.L;
    const TwTab<T> tw = load_twiddles(tws, tw_all + P.tw_off, L, g);
    g.sync();
    const bool fp64 = (flags & HANKEL_FP64_POWER) != 0;
    const T invL = T(1) / T(L);
    cx<T>* U = ws + J.wsA;
    cx<T>* W0 = ws + J.wsB;
    cx<T>* W1 = W0 + L;
    if (!stored) fft_global<T>(P, GLd<T>{h + J.hA, J.dA, x + J.xA, J.nA}, nullptr, W0, W1, GSt<T>{U}, false, tw, g);
    const AdjSt<T> store{gh ? gh + J.hA : nullptr, J.dA, gx ? gx + J.xA : nullptr, J.nA, L};
    cx<T>* G = fft_global<T>(P, GLd<T>{gy + J.yA, J.nA, nullptr, 0}, nullptr, W0, W1, store, true, tw, g);
    cx<T>* F = (G == W0) ? W1 : W0;
    for (int k = g.tid; k < L; k += g.nthr) {
        const int kc = (k == 0) ? 0 : L - k;
        const cx<T> Uk = U[k], Uc = conjg(U[kc]), Gk = G[k];
        F[k] = fp64 ? adjoint_bin<double>(Uk, Uc, Gk, J.mA, invL) : adjoint_bin<T>(Uk, Uc, Gk, J.mA, invL);
    }
    __threadfence_block();
    g.sync();
    fft_global<T>(P, GLd<T>{nullptr, 0, nullptr, 0}, F, G, F, store, false, tw, g);
}

// ---------------------------------------------------------------- split jobs
// A length L = 2M transform as two length-M transforms (decimation in
// frequency): with u the input, X[2k + c] = sum_n v_c[n] w_M^{nk} where
// v_0[n] = u[n] + u[n + M] and v_1[n] = (u[n] - u[n + M]) w_L^n.  Block c of a
// job stages v_c in shared memory, transforms it and stores the bins 2k + c,
// so a job's two blocks run on two SMs and every pass stays in shared memory.

// Real signals a + i b, zero-padded (the same reading as GLd).
template <typename T>
struct PairSrc {
    const T* a;
    int na;
    const T* b;
    int nb;
    __device__ __forceinline__ cx<T> operator()(int i) const {
        return mk<T>(i < na ? a[i] : T(0), i < nb ? b[i] : T(0));
    }
};

// Forward spectral product P_k = ifft(h~)_k X_k^{m-1} from the stored
// spectrum S = fft(h~ + i x~).
template <typename T>
struct ProductSrc {
    const cx<T>* S;
    int L, m;
    T invL;
    bool fp64;
    __device__ __forceinline__ cx<T> operator()(int k) const {
        const int kc = (k == 0) ? 0 : L - k;
        cx<T> Hk, Xk;
        unpack(S[k], conjg(S[kc]), Hk, Xk);
        T at;
        return fp64 ? product<double>(Hk, Xk, m, invL, at, false) : product<T>(Hk, Xk, m, invL, at, false);
    }
};

// Adjoint spectrum Q_k from U = fft(h~ + i x~) and G = fft(g~).
template <typename T>
struct AdjointSrc {
    const cx<T>* U;
    const cx<T>* G;
    int L, m;
    T invL;
    bool fp64;
    __device__ __forceinline__ cx<T> operator()(int k) const {
        const int kc = (k == 0) ? 0 : L - k;
        return fp64 ? adjoint_bin<double>(U[k], conjg(U[kc]), G[k], m, invL)
                    : adjoint_bin<T>(U[k], conjg(U[kc]), G[k], m, invL);
    }
};

// v_c[n] into shared memory (padded layout), n < M.
template <typename T, class Src>
__device__ __forceinline__ void dif_stage(cx<T>* buf, const Src& u, int M, int c, const TwTab<T>& twL,
                                          const Group& g) {
    for (int n = g.tid; n < M; n += g.nthr) {
        const cx<T> a = u(n), b = u(n + M);
        buf[sp(n)] = (c == 0) ? a + b : cmul(a - b, twL(n));
    }
}

// v_c[n] = w_L^{c n} sum_j u[n + j M] (-i)^{j c} (j, c < 4) into shared
// memory, n < M = L/4: block c of a four-way split, whose length-M
// transform gives the bins 4k + c of the length-L one.
template <typename T, class Src>
__device__ __forceinline__ void dif4_stage(cx<T>* buf, const Src& u, int M, int c, const TwTab<T>& twL,
                                           const Group& g) {
    // unrolled: the loads of several n in flight at once (they come from L2)
#pragma unroll 4
    for (int n = g.tid; n < M; n += g.nthr) {
        const cx<T> a0 = u(n), a1 = u(n + M), a2 = u(n + 2 * M), a3 = u(n + 3 * M);
        cx<T> v;
        if (c == 0) {
            v = (a0 + a2) + (a1 + a3);
        } else if (c == 2) {
            v = (a0 + a2) - (a1 + a3);
        } else {
            const cx<T> e = a0 - a2, o = a1 - a3;  // c = 1: e - i o; c = 3: e + i o
            v = (c == 1) ? e + mul_ni(o) : e + mul_pi(o);
        }
        buf[sp(n)] = (c == 0) ? v : cmul(v, twL(c * n));
    }
}

// Stores of a split job's block c: bin s k + c of the whole spectrum (s = 2
// or 4 blocks per transform).
template <typename T>
struct SplitSt {  // complex bins s k + c
    cx<T>* p;
    int c, s;
    __device__ __forceinline__ void operator()(int k, cx<T> v) const { p[s * k + c] = v; }
};

template <typename T>
struct SplitRealSt {  // real part of the bins s k + c, truncated to n
    T* y;
    int n, c, s;
    __device__ __forceinline__ void operator()(int k, cx<T> v) const {
        const int i = s * k + c;
        if (i < n) y[i] = v.x;
    }
};

template <typename T>
struct SplitAdjSt {  // AdjSt at the bins s k + c
    AdjSt<T> st;
    int c, s;
    __device__ __forceinline__ void operator()(int k, cx<T> v) const { st(s * k + c, v); }
};

// Shared-memory layout of the split kernels: twiddle tables of lengths M and
// L = 2M, then two padded buffers of Mmax.
template <typename T>
struct SplitSmem {
    TwTab<T> twM, twL;
    cx<T>*b0, *b1;
};

template <typename T>
__device__ __forceinline__ SplitSmem<T> split_smem(unsigned char* raw, const RealJob& J, const cx<T>* tw_all,
                                                  int Mmax, const Group& g, int ways = 2) {
    cx<T>* t0 = reinterpret_cast<cx<T>*>(raw + RED_BYTES);
    cx<T>* t1 = t0 + TW_SMEM;
    SplitSmem<T> s;
    s.twM = load_twiddles(t0, tw_all + J.P.tw_off, J.P.L, g);
    s.twL = load_twiddles(t1, tw_all + J.twL, ways * J.P.L, g);
    s.b0 = t1 + TW_SMEM;
    s.b1 = s.b0 + smem_elems(Mmax);
    return s;
}

// Split jobs on thread-block clusters: the W = 2 or 4 blocks of one tensor
// form a cluster (block c = rank in the cluster), each running a length-L/W
// transform after a radix-W decimation-in-frequency stage, so that one
// tensor occupies W SMs and the whole of a forward or adjoint product is one
// launch.  The spectra pass between the two transforms
// through the plan workspace (L2-resident): a cluster barrier (release /
// acquire at cluster scope) makes each block's quarter of the spectrum
// visible to the other three.  The blocks of a cluster run together, so the
// barrier never waits on a block that has not started.

template <int W, typename T, class Src>
__device__ __forceinline__ void difw_stage(cx<T>* buf, const Src& u, int M, int c, const TwTab<T>& twL,
                                           const Group& g) {
    if constexpr (W == 4)
        dif4_stage(buf, u, M, c, twL, g);
    else
        dif_stage(buf, u, M, c, twL, g);
}

// y = fft(P)[0:n] and alpha: S = fft(h~ + i x~) into wsA, barrier, then the
// product's transform.
template <typename T, int W>
__global__ void __cluster_dims__(W, 1, 1) __launch_bounds__(512)
    cluster_forward_kernel(const RealJob* __restrict__ jobs, int first, const T* __restrict__ h,
                           const T* __restrict__ x, T* __restrict__ y, T* __restrict__ alpha, cx<T>* ws,
                           const cx<T>* __restrict__ tw_all, int Mmax, int flags) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double* red = reinterpret_cast<double*>(smem_raw);
    cg::cluster_group cl = cg::this_cluster();
    const int c = (int)cl.block_rank();
    const RealJob J = jobs[first + (int)blockIdx.x / W];
    const Group g{(int)threadIdx.x, (int)blockDim.x, 0};
    const SplitSmem<T> sm = split_smem(smem_raw, J, tw_all, Mmax, g, W);
    const int M = J.P.L, L = W * M;
    const bool fp64 = (flags & HANKEL_FP64_POWER) != 0;
    const T invL = T(1) / T(L);
    cx<T>* S = ws + J.wsA;
    g.sync();
    difw_stage<W>(sm.b0, PairSrc<T>{h + J.hA, J.dA, x + J.xA, J.nA}, M, c, sm.twL, g);
    g.sync();
    fft_stage<T>(J.P, GLd<T>{nullptr, 0, nullptr, 0}, sm.b0, sm.b1, sm.b0, SplitSt<T>{S, c, W}, false, sm.twM, g);
    cl.sync();
    if (y != nullptr) {
        difw_stage<W>(sm.b0, ProductSrc<T>{S, L, J.mA, invL, fp64}, M, c, sm.twL, g);
        g.sync();
        fft_stage<T>(J.P, GLd<T>{nullptr, 0, nullptr, 0}, sm.b0, sm.b1, sm.b0, SplitRealSt<T>{y + J.yA, J.nA, c, W},
                     false, sm.twM, g);
    }
    if (alpha != nullptr) {
        // each block sums 1/W of the bins 0 .. L/2; block 0 adds the other
        // blocks' partial sums after a second barrier
        T aA = T(0);
        for (int k = c * g.nthr + g.tid; k <= L / 2; k += W * g.nthr) {
            const int kc = (k == 0) ? 0 : L - k;
            cx<T> Hk, Xk;
            unpack(S[k], conjg(S[kc]), Hk, Xk);
            aA += alpha_term(Hk, Xk, J.mA, invL, fp64, k, kc);
        }
        const double sA = group_sum((double)aA, red, g);
        // slots 33 .. 32 + W - 1 of block 0's reduction scratch (past group_sum's)
        double* part = cl.map_shared_rank(red, 0);
        if (g.tid == 0 && c != 0) part[32 + c] = sA;
        cl.sync();
        if (g.tid == 0 && c == 0) {
            double t = sA;
            for (int r = 1; r < W; ++r) t += red[32 + r];
            alpha[J.iA] = (T)t;
        }
    }
}

// Gradients: G = fft(g~) into wsB (and U = fft(h~ + i x~) into wsA unless
// kept from the forward), barrier, then the adjoint's transform.
template <typename T, int W>
__global__ void __cluster_dims__(W, 1, 1) __launch_bounds__(512)
    cluster_backward_kernel(const RealJob* __restrict__ jobs, int first, const T* __restrict__ gy,
                            const T* __restrict__ h, const T* __restrict__ x, T* __restrict__ gh, T* __restrict__ gx,
                            cx<T>* ws, const cx<T>* __restrict__ tw_all, int Mmax, int flags, int stored) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cg::cluster_group cl = cg::this_cluster();
    const int c = (int)cl.block_rank();
    const RealJob J = jobs[first + (int)blockIdx.x / W];
    const Group g{(int)threadIdx.x, (int)blockDim.x, 0};
    const SplitSmem<T> sm = split_smem(smem_raw, J, tw_all, Mmax, g, W);
    const int M = J.P.L, L = W * M;
    const bool fp64 = (flags & HANKEL_FP64_POWER) != 0;
    const T invL = T(1) / T(L);
    g.sync();
    if (!stored) {
        difw_stage<W>(sm.b0, PairSrc<T>{h + J.hA, J.dA, x + J.xA, J.nA}, M, c, sm.twL, g);
        g.sync();
        fft_stage<T>(J.P, GLd<T>{nullptr, 0, nullptr, 0}, sm.b0, sm.b1, sm.b0, SplitSt<T>{ws + J.wsA, c, W}, false,
                     sm.twM, g);
        g.sync();
    }
    difw_stage<W>(sm.b0, PairSrc<T>{gy + J.yA, J.nA, nullptr, 0}, M, c, sm.twL, g);
    g.sync();
    fft_stage<T>(J.P, GLd<T>{nullptr, 0, nullptr, 0}, sm.b0, sm.b1, sm.b0, SplitSt<T>{ws + J.wsB, c, W}, false,
                 sm.twM, g);
    cl.sync();
    difw_stage<W>(sm.b0, AdjointSrc<T>{ws + J.wsA, ws + J.wsB, L, J.mA, invL, fp64}, M, c, sm.twL, g);
    g.sync();
    const AdjSt<T> st{gh ? gh + J.hA : nullptr, J.dA, gx ? gx + J.xA : nullptr, J.nA, L};
    fft_stage<T>(J.P, GLd<T>{nullptr, 0, nullptr, 0}, sm.b0, sm.b1, sm.b0, SplitAdjSt<T>{st, c, W}, false, sm.twM, g);
}

// ------------------------------------------------ anti-circulant expansion

struct alignas(16) Bytes16 {
    unsigned long long a, b;
};

template <typename E>
__global__ void expand_kernel(const ExpandEntry* __restrict__ e, int count, const E* __restrict__ c, E* h) {
    for (int t = blockIdx.y; t < count; t += gridDim.y) {
        const ExpandEntry x = e[t];
        for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < x.d; k += gridDim.x * blockDim.x)
            h[x.ws_off + k] = c[x.c_off + (k % x.n)];
    }
}

template <typename V>
__global__ void fold_kernel(const ExpandEntry* __restrict__ e, const FoldGroup* __restrict__ groups, int ngroups,
                            const V* __restrict__ gh, V* gc) {
    for (int gi = blockIdx.y; gi < ngroups; gi += gridDim.y) {
        const FoldGroup G = groups[gi];
        for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < G.n; j += gridDim.x * blockDim.x) {
            V acc = gh[e[G.first].ws_off + j];
            bool first = true;
            for (int t = G.first; t < G.first + G.count; ++t) {
                const ExpandEntry x = e[t];
                for (int k = j; k < x.d; k += G.n) {
                    if (first) {
                        first = false;
                        continue;  // the first term initialised acc
                    }
                    acc = acc + gh[x.ws_off + k];
                }
            }
            gc[G.c_off + j] = acc;
        }
    }
}

cudaError_t launch_expand(int elem, const ExpandEntry* e, int count, int max_d, const void* c, void* h,
                          cudaStream_t st) {
    const dim3 grid((unsigned)std::min(64, (max_d + 255) / 256), (unsigned)std::min(count, 65535));
    switch (elem) {
        case 4: expand_kernel<float><<<grid, 256, 0, st>>>(e, count, (const float*)c, (float*)h); break;
        case 8: expand_kernel<double><<<grid, 256, 0, st>>>(e, count, (const double*)c, (double*)h); break;
        default: expand_kernel<Bytes16><<<grid, 256, 0, st>>>(e, count, (const Bytes16*)c, (Bytes16*)h); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_fold(bool dbl, bool cplx, const ExpandEntry* e, const FoldGroup* g, int ngroups, int max_n,
                        const void* gh, void* gc, cudaStream_t st) {
    const dim3 grid((unsigned)std::min(64, (max_n + 255) / 256), (unsigned)std::min(ngroups, 65535));
    if (cplx && dbl)
        fold_kernel<cx<double>><<<grid, 256, 0, st>>>(e, g, ngroups, (const cx<double>*)gh, (cx<double>*)gc);
    else if (cplx)
        fold_kernel<cx<float>><<<grid, 256, 0, st>>>(e, g, ngroups, (const cx<float>*)gh, (cx<float>*)gc);
    else if (dbl)
        fold_kernel<double><<<grid, 256, 0, st>>>(e, g, ngroups, (const double*)gh, (double*)gc);
    else
        fold_kernel<float><<<grid, 256, 0, st>>>(e, g, ngroups, (const float*)gh, (float*)gc);
    return cudaGetLastError();
}

// Two-level twiddle table of length L (fft_stage.cuh): A[j] = w_L^{64 j},
// B[j] = w_L^j, from FP64 sincospi rounded to T.
template <typename T>
__global__ void stage_twiddle_kernel(cx<T>* out, int L) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    const int nA = (L + TW_LO - 1) / TW_LO;
    if (e >= nA + TW_LO) return;
    const long long j = (e < nA) ? (long long)e * TW_LO : (long long)(e - nA);
    double s, c;
    sincospi(-2.0 * (double)(j % L) / (double)L, &s, &c);
    out[e] = mk<T>((T)c, (T)s);
}

template <typename T>
__global__ void twiddle_kernel(cx<T>* out, int L) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < L) {
        double s, c;
        sincospi(-2.0 * (double)j / (double)L, &s, &c);
        out[j] = mk<T>((T)c, (T)s);
    }
}

// ------------------------------------------------------------------ host side

// Raise a kernel's dynamic shared-memory limit only when a launch needs more
// than already granted (no attribute calls in steady state, so launches can
// be captured into CUDA graphs).  Grants are kept per device and per kernel
// (kernels of one signature are distinct entries).
static cudaError_t ensure_smem_fn(const void* fn, size_t bytes) {
    static std::mutex mu;
    static std::map<std::pair<int, const void*>, size_t> granted;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lk(mu);
    size_t& g = granted[std::make_pair(dev, fn)];
    if (bytes <= g) return cudaSuccess;
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess) g = bytes;
    return e;
}

template <class K>
static cudaError_t ensure_smem(K kernel, size_t bytes) {
    return ensure_smem_fn(reinterpret_cast<const void*>(kernel), bytes);
}

template <typename T>
static size_t real_smem_bytes(const RealLaunch& lc) {
    return RED_BYTES + ((size_t)TW_SMEM + (size_t)lc.arrays * smem_elems(lc.Lmax)) * sizeof(cx<T>);
}

template <typename T>
static size_t split_smem_bytes(const RealLaunch& lc) {
    return RED_BYTES + ((size_t)2 * TW_SMEM + (size_t)2 * smem_elems(lc.Lmax)) * sizeof(cx<T>);
}

template <typename T>
static cudaError_t launch_fwd_t(const RealLaunch& lc, const RealJob* jobs, const void* h, const void* x, void* y,
                                void* alpha, const void* tw, void* ws, int flags, cudaStream_t st) {
    if (lc.split >= 2) {  // a cluster of W blocks per job
        const int W = lc.split == 2 ? 4 : 2;
        const size_t smem = split_smem_bytes<T>(lc);
        auto k = W == 4 ? cluster_forward_kernel<T, 4> : cluster_forward_kernel<T, 2>;
        cudaError_t e = ensure_smem(k, smem);
        if (e != cudaSuccess) return e;
        k<<<lc.count * W, lc.nthr, smem, st>>>(jobs, lc.first, (const T*)h, (const T*)x, (T*)y, (T*)alpha, (cx<T>*)ws,
                                                (const cx<T>*)tw, lc.Lmax, flags);
        return cudaGetLastError();
    }
    const size_t smem = real_smem_bytes<T>(lc);
    if (lc.arrays == 0) {
        real_fwd_global_kernel<T><<<lc.count, lc.nthr, smem, st>>>(jobs, lc.first, (const T*)h, (const T*)x, (T*)y,
                                                                   (T*)alpha, (const cx<T>*)tw, (cx<T>*)ws, flags);
        return cudaGetLastError();
    }
    auto k = real_fwd_kernel<T>;
    cudaError_t e = ensure_smem(k, smem);
    if (e != cudaSuccess) return e;
    k<<<lc.count, lc.nthr, smem, st>>>(jobs, lc.first, (const T*)h, (const T*)x, (T*)y, (T*)alpha,
                                       (const cx<T>*)tw, (cx<T>*)ws, lc.Lmax, flags);
    return cudaGetLastError();
}

template <typename T>
static cudaError_t launch_bwd_t(const RealLaunch& lc, const RealJob* jobs, const void* gy, const void* h,
                                const void* x, void* gh, void* gx, const void* tw, void* ws, int flags, int stored,
                                cudaStream_t st) {
    if (lc.split >= 2) {  // a cluster of W blocks per job
        const int W = lc.split == 2 ? 4 : 2;
        const size_t smem = split_smem_bytes<T>(lc);
        auto k = W == 4 ? cluster_backward_kernel<T, 4> : cluster_backward_kernel<T, 2>;
        cudaError_t e = ensure_smem(k, smem);
        if (e != cudaSuccess) return e;
        k<<<lc.count * W, lc.nthr, smem, st>>>(jobs, lc.first, (const T*)gy, (const T*)h, (const T*)x, (T*)gh, (T*)gx,
                                                (cx<T>*)ws, (const cx<T>*)tw, lc.Lmax, flags, stored);
        return cudaGetLastError();
    }
    const size_t smem = real_smem_bytes<T>(lc);
    if (lc.arrays == 3) {  // pair jobs
        auto k = real_bwd_pair_kernel<T>;
        cudaError_t e = ensure_smem(k, smem);
        if (e != cudaSuccess) return e;
        k<<<lc.count, lc.nthr, smem, st>>>(jobs, lc.first, (const T*)gy, (const T*)h, (const T*)x, (T*)gh, (T*)gx,
                                           (const cx<T>*)tw, (cx<T>*)ws, lc.Lmax, flags, stored);
        return cudaGetLastError();
    }
    if (lc.arrays == 0) {
        real_bwd_global_kernel<T><<<lc.count, lc.nthr, smem, st>>>(jobs, lc.first, (const T*)gy, (const T*)h,
                                                                   (const T*)x, (T*)gh, (T*)gx, (const cx<T>*)tw,
                                                                   (cx<T>*)ws, flags, stored);
        return cudaGetLastError();
    }
    auto k = real_bwd_kernel<T>;
    cudaError_t e = ensure_smem(k, smem);
    if (e != cudaSuccess) return e;
    k<<<lc.count, lc.nthr, smem, st>>>(jobs, lc.first, (const T*)gy, (const T*)h, (const T*)x, (T*)gh, (T*)gx,
                                       (const cx<T>*)tw, (cx<T>*)ws, lc.Lmax, flags, stored);
    return cudaGetLastError();
}

template <typename T>
static cudaError_t launch_multi_t(const RealLaunch& lc, const MultiJob* jobs, const void* h, const void* x, void* y,
                                  void* alpha, const void* tw, cudaStream_t st) {
    const size_t smem = real_smem_bytes<T>(lc);
    auto k = real_multi_kernel<T>;
    cudaError_t e = ensure_smem(k, smem);
    if (e != cudaSuccess) return e;
    k<<<lc.count, lc.nthr, smem, st>>>(jobs, lc.first, (const T*)h, (const T*)x, (T*)y, (T*)alpha,
                                       (const cx<T>*)tw, lc.Lmax);
    return cudaGetLastError();
}

cudaError_t launch_real_multi(bool dbl, const RealLaunch& lc, const MultiJob* jobs, const void* h, const void* x,
                              void* y, void* alpha, const void* tw, cudaStream_t st) {
    return dbl ? launch_multi_t<double>(lc, jobs, h, x, y, alpha, tw, st)
               : launch_multi_t<float>(lc, jobs, h, x, y, alpha, tw, st);
}

cudaError_t launch_real_forward(bool dbl, const RealLaunch& lc, const RealJob* jobs, const void* h, const void* x,
                                void* y, void* alpha, const void* tw, void* ws, int flags, cudaStream_t st) {
    return dbl ? launch_fwd_t<double>(lc, jobs, h, x, y, alpha, tw, ws, flags, st)
               : launch_fwd_t<float>(lc, jobs, h, x, y, alpha, tw, ws, flags, st);
}

cudaError_t launch_real_backward(bool dbl, const RealLaunch& lc, const RealJob* jobs, const void* gy, const void* h,
                                 const void* x, void* gh, void* gx, const void* tw, void* ws, int flags, int stored,
                                 cudaStream_t st) {
    return dbl ? launch_bwd_t<double>(lc, jobs, gy, h, x, gh, gx, tw, ws, flags, stored, st)
               : launch_bwd_t<float>(lc, jobs, gy, h, x, gh, gx, tw, ws, flags, stored, st);
}

cudaError_t launch_twiddles(bool dbl, void* out, int L, cudaStream_t st) {
    const int nb = (L + 255) / 256;
    if (dbl)
        twiddle_kernel<double><<<nb, 256, 0, st>>>((cx<double>*)out, L);
    else
        twiddle_kernel<float><<<nb, 256, 0, st>>>((cx<float>*)out, L);
    return cudaGetLastError();
}

cudaError_t launch_stage_twiddles(bool dbl, void* out, const FftPlan& P, cudaStream_t st) {
    const int total = tw_table_elems(P.L);
    const int nb = (total + 255) / 256;
    if (dbl)
        stage_twiddle_kernel<double><<<nb, 256, 0, st>>>((cx<double>*)out, P.L);
    else
        stage_twiddle_kernel<float><<<nb, 256, 0, st>>>((cx<float>*)out, P.L);
    return cudaGetLastError();
}

int stage_twiddle_count(const FftPlan& P) { return tw_table_elems(P.L); }

size_t real_launch_smem(bool dbl, const RealLaunch& lc) {
    if (lc.split) return dbl ? split_smem_bytes<double>(lc) : split_smem_bytes<float>(lc);
    return dbl ? real_smem_bytes<double>(lc) : real_smem_bytes<float>(lc);
}

}  // namespace hk
