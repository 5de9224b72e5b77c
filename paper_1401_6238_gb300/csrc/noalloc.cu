// noalloc.cu -- hankel_txv_backward_static: the adjoint of the real
// one-vector product (grad_h, grad_x of y = H x^{m-1}) for callers that
// cannot allocate device memory.  The paper has no counterpart; it is the
// same computation as the plan-based backward kernel in real_path.cu, with
// its scratch (the spectra U = fft(h~ + i x~) and the twiddle tables) placed
// in one file-scope device array instead of plan workspace, and its job
// table passed as kernel parameters.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <utility>
#include <vector>

#include "fft_core.cuh"
#include "hankel.h"
#include "launch.h"

namespace hk {
namespace {

constexpr int kJobsPerLaunch = 32;
constexpr int kMaxDevices = 64;

// The scratch every call shares.  Each device that loads the library holds it
// until the process exits.
__device__ __align__(256) unsigned char g_static_scratch[HANKEL_STATIC_SCRATCH_BYTES];

std::mutex g_mu;
void* g_scratch_addr[kMaxDevices] = {nullptr};

struct StaticJobs {
    RealJob job[kJobsPerLaunch];
};

template <typename T>
struct SLoad {
    const T* a;
    int na;
    const T* b;
    int nb;
    __device__ __forceinline__ cx<T> operator()(int i) const {
        return mk<T>(i < na ? a[i] : T(0), (b != nullptr && i < nb) ? b[i] : T(0));
    }
};

template <typename T>
struct SAdjStore {
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

// bin k of Q = G X^{m-1} / L + i (m-1) ifft(h~) G X^{m-2}, from U = fft(h~ + i x~)
template <typename T>
struct SAdjCombine {
    const cx<T>* U;
    const cx<T>* G;
    int m, L;
    T invL;
    __device__ __forceinline__ cx<T> operator()(int k) const {
        const int kc = (k == 0) ? 0 : L - k;
        const cx<T> u = U[k], w = conjg(U[kc]);
        const cx<T> Hk = scal(u + w, T(0.5)), Xk = scal(mul_ni(u - w), T(0.5));
        const cx<T> hh = scal(conjg(Hk), invL);
        cx<T> gxm2 = G[sp(k)];
        for (int i = 0; i < m - 2; ++i) gxm2 = cmul(gxm2, Xk);
        const cx<T> qh = scal(cmul(gxm2, Xk), invL);
        const cx<T> qx = scal(cmul(hh, gxm2), T(m - 1));
        return mk<T>(qh.x - qx.y, qh.y + qx.x);
    }
};

template <typename T>
__global__ void __launch_bounds__(512) static_bwd_kernel(StaticJobs jobs, const T* __restrict__ gy,
                                                          const T* __restrict__ h, const T* __restrict__ x,
                                                          T* __restrict__ gh, T* __restrict__ gx, int Lmax) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cx<T>* bA = reinterpret_cast<cx<T>*>(smem_raw + RED_BYTES);
    cx<T>* bB = bA + smem_elems(Lmax);
    const RealJob& J = jobs.job[blockIdx.x];
    const Group g{(int)threadIdx.x, (int)blockDim.x, 0};
    const FftPlan P = J.P;
    const int L = P.L;
    // twiddles and spectra live in the static array (byte offsets in tw_off / wsA)
    const cx<T>* tw = reinterpret_cast<const cx<T>*>(g_static_scratch + (size_t)P.tw_off);
    cx<T>* U = reinterpret_cast<cx<T>*>(g_static_scratch + (size_t)J.wsA);
    const T invL = T(1) / T(L);
    cx<T>* S = fft_smem<T>(P, SLoad<T>{h + J.hA, J.dA, x + J.xA, J.nA}, bA, bB, tw, g);
    for (int k = g.tid; k < L; k += g.nthr) U[k] = S[sp(k)];
    g.sync();
    cx<T>* G = fft_smem<T>(P, SLoad<T>{gy + J.yA, J.nA, nullptr, 0}, bA, bB, tw, g);
    cx<T>* F = (G == bA) ? bB : bA;
    fft_out<T>(P, SAdjCombine<T>{U, G, J.mA, L, invL}, F, G,
               SAdjStore<T>{gh ? gh + J.hA : nullptr, J.dA, gx ? gx + J.xA : nullptr, J.nA, L}, tw, g);
}

// Device address of the static array on the current device, looked up once
// per device.
hankel_status scratch_base(void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        set_last_error(std::string("cudaGetDevice: ") + cudaGetErrorString(e));
        return HANKEL_ECUDA;
    }
    if (dev < 0 || dev >= kMaxDevices) {
        set_last_error("device ordinal beyond the supported range");
        return HANKEL_EUNSUPPORTED;
    }
    std::lock_guard<std::mutex> lk(g_mu);
    if (g_scratch_addr[dev] == nullptr) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess || p == nullptr) {
            set_last_error(std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e));
            return HANKEL_ECUDA;
        }
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return HANKEL_OK;
}

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

// Raise the kernel's dynamic shared-memory limit only when a launch needs
// more than already granted on this device.
template <typename T>
cudaError_t grant_smem(size_t bytes) {
    static size_t granted[kMaxDevices] = {0};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_mu);
    if (bytes <= granted[dev]) return cudaSuccess;
    e = cudaFuncSetAttribute(static_bwd_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess) granted[dev] = bytes;
    return e;
}

template <typename T>
hankel_status run_static(const hankel_desc* descs, int64_t count, const void* gy, const void* h, const void* x,
                         void* gh, void* gx, cudaStream_t st) {
    const size_t cs = sizeof(cx<T>);
    // largest L whose two ping-pong buffers fit one block's shared memory
    int maxL = 2;
    while (maxL < 16384 && RED_BYTES + 2 * smem_elems_host(maxL + 1) * cs <= 227 * 1024) ++maxL;
    std::vector<RealJob> jobs;
    std::map<int, size_t> tw_at;
    size_t used = 0;
    for (int64_t i = 0; i < count; ++i) {
        const hankel_desc& d = descs[i];
        if (d.m < 2 || d.m > HANKEL_MAX_ORDER) {
            set_last_error("descriptor " + std::to_string(i) + ": order outside [2, 8]");
            return HANKEL_EINVAL;
        }
        for (int p = 0; p < d.m; ++p)
            if (d.n[p] != d.n[0] || d.n[p] < 1) {
                set_last_error("descriptor " + std::to_string(i) + ": needs a square tensor with n >= 1");
                return HANKEL_EINVAL;
            }
        if (d.h_off < 0 || d.x_off[0] < 0 || d.y_off < 0) {
            set_last_error("descriptor " + std::to_string(i) + ": negative offset");
            return HANKEL_EINVAL;
        }
        const int64_t dl = (int64_t)d.m * (d.n[0] - 1) + 1;
        const int64_t L = hankel_fft_length(dl);
        if (L < 0 || L > maxL) {
            set_last_error("descriptor " + std::to_string(i) + ": FFT length beyond the maximum of this entry point");
            return HANKEL_EINVAL;
        }
        if (!tw_at.count((int)L)) {
            tw_at[(int)L] = used;
            used += align256((size_t)L * cs);
        }
        RealJob J;
        std::memset(&J, 0, sizeof(J));
        fft_factor((int)L, &J.P);
        J.single = 1;
        J.mA = d.m;
        J.nA = d.n[0];
        J.dA = (int)dl;
        J.iA = (int)i;
        J.iB = -1;
        J.hA = d.h_off;
        J.xA = d.x_off[0];
        J.yA = d.y_off;
        J.wsA = (int64_t)used;  // byte offset of this tensor's spectrum
        used += align256((size_t)L * cs);
        jobs.push_back(J);
    }
    // each tensor's gradients are written, not summed: descriptors whose h
    // regions or x regions overlap would race
    for (int w = 0; w < 2; ++w) {
        std::vector<std::pair<int64_t, int64_t>> iv;
        for (const auto& J : jobs)
            iv.emplace_back(w == 0 ? J.hA : J.xA, (w == 0 ? J.hA : J.xA) + (w == 0 ? J.dA : J.nA));
        std::sort(iv.begin(), iv.end());
        for (size_t k = 1; k < iv.size(); ++k)
            if (iv[k].first < iv[k - 1].second) {
                set_last_error(std::string("descriptors share ") + (w == 0 ? "h" : "x") +
                               " storage: this entry point writes each tensor's gradients, so overlapping regions "
                               "are not allowed (hankel_txv_backward sums them)");
                return HANKEL_EINVAL;
            }
    }
    if (used > (size_t)HANKEL_STATIC_SCRATCH_BYTES) {
        set_last_error("the batch needs " + std::to_string(used) + " bytes of scratch; the static array holds " +
                       std::to_string((long long)HANKEL_STATIC_SCRATCH_BYTES));
        return HANKEL_EINVAL;
    }
    void* base = nullptr;
    hankel_status s = scratch_base(&base);
    if (s != HANKEL_OK) return s;
    for (auto& J : jobs) J.P.tw_off = (int32_t)tw_at[J.P.L];
    for (auto& kv : tw_at) {
        cudaError_t e = launch_twiddles(sizeof(T) == 8, (char*)base + kv.second, kv.first, st);
        if (e != cudaSuccess) {
            set_last_error(std::string("twiddle kernel: ") + cudaGetErrorString(e));
            return HANKEL_ECUDA;
        }
    }
    std::stable_sort(jobs.begin(), jobs.end(), [](const RealJob& a, const RealJob& b) { return a.P.L > b.P.L; });
    for (size_t i = 0; i < jobs.size(); i += kJobsPerLaunch) {
        StaticJobs pj;
        std::memset(&pj, 0, sizeof(pj));
        const int n = (int)std::min<size_t>(kJobsPerLaunch, jobs.size() - i);
        for (int k = 0; k < n; ++k) pj.job[k] = jobs[i + k];
        const int Lmax = pj.job[0].P.L;
        int nthr = 32;
        while (nthr < 512 && nthr < (Lmax + 15) / 16) nthr <<= 1;
        const size_t smem = RED_BYTES + 2 * smem_elems_host(Lmax) * cs;
        cudaError_t e = grant_smem<T>(smem);
        if (e == cudaSuccess) {
            static_bwd_kernel<T><<<n, nthr, smem, st>>>(pj, (const T*)gy, (const T*)h, (const T*)x, (T*)gh, (T*)gx,
                                                        Lmax);
            e = cudaGetLastError();
        }
        if (e != cudaSuccess) {
            set_last_error(std::string("backward kernel launch: ") + cudaGetErrorString(e));
            return HANKEL_ECUDA;
        }
    }
    return HANKEL_OK;
}

}  // namespace
}  // namespace hk

extern "C" hankel_status hankel_txv_backward_static(const hankel_desc* descs, int64_t count, hankel_dtype dtype,
                                                    const void* grad_y, const void* h, const void* x, void* grad_h,
                                                    void* grad_x, hankel_stream_t stream) {
    if (descs == nullptr || count < 1) {
        hk::set_last_error("need at least one descriptor");
        return HANKEL_EINVAL;
    }
    if (dtype != HANKEL_R32 && dtype != HANKEL_R64) {
        hk::set_last_error("hankel_txv_backward_static takes the real dtypes only");
        return HANKEL_EINVAL;
    }
    if (!grad_y || !h || !x || (!grad_h && !grad_x)) {
        hk::set_last_error("grad_y, h, x and at least one of grad_h / grad_x must be device pointers");
        return HANKEL_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)stream;
    return dtype == HANKEL_R64 ? hk::run_static<double>(descs, count, grad_y, h, x, grad_h, grad_x, st)
                               : hk::run_static<float>(descs, count, grad_y, h, x, grad_h, grad_x, st);
}
