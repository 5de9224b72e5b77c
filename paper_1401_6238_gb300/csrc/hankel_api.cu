// hankel_api.cu -- the C ABI of include/hankel.h: planning (host), validation,
// dispatch of the kernels, status codes.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "general.h"
#include "hankel.h"
#include "jobs.h"
#include "launch.h"

namespace {

thread_local std::string g_err;

hankel_status fail(hankel_status s, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
    return s;
}

hankel_status cuda_fail(cudaError_t e, const char* what) {
    return fail(e == cudaErrorMemoryAllocation ? HANKEL_ENOMEM : HANKEL_ECUDA, "%s: %s", what,
                cudaGetErrorString(e));
}

bool is_double(hankel_dtype d) { return d == HANKEL_R64 || d == HANKEL_C128; }
bool is_complex(hankel_dtype d) { return d == HANKEL_C64 || d == HANKEL_C128; }
size_t real_size(hankel_dtype d) { return is_double(d) ? 8 : 4; }
size_t elem_size(hankel_dtype d) { return real_size(d) * (is_complex(d) ? 2 : 1); }

// ------------------------------------------------------------ FFT lengths
// Radix set of the kernels and a per-point cost model of one Stockham pass
// (shared-memory round trip + butterfly arithmetic, FP32 operations / point).
constexpr int kMaxL = 16384;
// Planner knobs (hankel_set_tuning): the fixed cost of one pass in the
// length/radix cost model, and the points each thread owns (threads per job).
double g_pass_cost = 10.0;
int g_points_per_thread = 16;
std::mutex g_tune_mu;
// Per-length-bin choices (hankel_set_bin_policy), keyed by the persistent
// kernel's FFT lengths; absent bins take the defaults.
struct BinPolicy {
    int path = 0;          // 0: persistent launch, 1: per-length launches
    int fp64_from_m = 99;  // orders m >= this form their spectrum power in FP64
};
std::map<int, BinPolicy> g_bins;
BinPolicy bin_policy(int L) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    const auto it = g_bins.find(L);
    return it == g_bins.end() ? BinPolicy() : it->second;
}
double radix_cost(int r) {
    switch (r) {
        case 2: return 5.0;
        case 3: return 9.3;
        case 4: return 8.5;
        case 5: return 12.8;
        case 7: return 16.5;
        case 8: return 12.75;
        case 16: return 17.4;
    }
    return 1e9;
}

struct LenInfo {
    int L;
    std::vector<int> radix;
    double cost;
};

// Best pass sequence for L = 2^a 3^b 5^c 7^e: the power of two split into
// parts 16/8/4/2 minimising the model, odd primes one pass each.
bool factor(int L, std::vector<int>& out, double& cost) {
    int a = 0, v = L;
    while (v % 2 == 0) { v /= 2; ++a; }
    std::vector<int> odd;
    for (int p : {3, 5, 7})
        while (v % p == 0) { v /= p; odd.push_back(p); }
    if (v != 1) return false;
    // split a into parts of size 4,3,2,1 (log2 of 16,8,4,2)
    double best = 1e18;
    std::vector<int> bestp;
    for (int n4 = 0; n4 * 4 <= a; ++n4)
        for (int n3 = 0; n4 * 4 + n3 * 3 <= a; ++n3)
            for (int n2 = 0; n4 * 4 + n3 * 3 + n2 * 2 <= a; ++n2) {
                int n1 = a - n4 * 4 - n3 * 3 - n2 * 2;
                std::vector<int> p;
                p.insert(p.end(), n4, 16);
                p.insert(p.end(), n3, 8);
                p.insert(p.end(), n2, 4);
                p.insert(p.end(), n1, 2);
                double c = 0;
                for (int r : p) c += g_pass_cost + radix_cost(r);
                if (c < best || (c == best && p.size() < bestp.size())) { best = c; bestp = p; }
            }
    out = bestp;
    out.insert(out.end(), odd.begin(), odd.end());
    std::sort(out.begin(), out.end(), [](int x, int y) { return x > y; });
    cost = 0;
    for (int r : out) cost += g_pass_cost + radix_cost(r);
    cost *= L;
    return !out.empty() && out.size() <= 8;
}

struct LengthTable {
    std::vector<LenInfo> cands;  // sorted by L
    std::vector<int> best_from;  // index of the cheapest candidate at or after i
    LengthTable() {
        for (int L = 2; L <= kMaxL; ++L) {
            LenInfo li;
            li.L = L;
            if (factor(L, li.radix, li.cost)) cands.push_back(li);
        }
        best_from.resize(cands.size());
        int b = (int)cands.size() - 1;
        for (int i = (int)cands.size() - 1; i >= 0; --i) {
            if (cands[i].cost <= cands[b].cost) b = i;
            best_from[i] = b;
        }
    }
    const LenInfo* find(int L) const {
        auto it = std::lower_bound(cands.begin(), cands.end(), L,
                                   [](const LenInfo& li, int v) { return li.L < v; });
        return (it != cands.end() && it->L == L) ? &*it : nullptr;
    }
    const LenInfo* pick(int64_t d) const {
        if (d < 1 || d > kMaxL) return nullptr;
        auto it = std::lower_bound(cands.begin(), cands.end(), (int)d,
                                   [](const LenInfo& li, int v) { return li.L < v; });
        if (it == cands.end()) return nullptr;
        return &cands[best_from[it - cands.begin()]];
    }
};

// The table for the current knobs; rebuilt when hankel_set_tuning changes them.
std::unique_ptr<LengthTable> g_lengths;
const LengthTable& lengths() {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    if (!g_lengths) g_lengths.reset(new LengthTable);
    return *g_lengths;
}

int pow2ceil(int v) {
    int p = 1;
    while (p < v) p <<= 1;
    return p;
}

}  // namespace

namespace hk {
// The planner's pass sequence for FFT length L (tw_off left at 0); false if
// L is not one of the planner's lengths.
bool fft_factor(int L, FftPlan* P) {
    const LenInfo* li = lengths().find(L);
    if (li == nullptr) return false;
    std::memset(P, 0, sizeof(*P));
    P->L = L;
    P->npass = (int)li->radix.size();
    for (int i = 0; i < P->npass && i < 8; ++i) P->radix[i] = (uint8_t)li->radix[i];
    fill_magic(*P);
    return true;
}
// Record the message hankel_last_error() returns for this thread.
void set_last_error(const std::string& msg) { g_err = msg; }
}  // namespace hk

struct hankel_plan_s {
    int device = 0;
    hankel_dtype dtype = HANKEL_R32;
    uint32_t flags = 0;
    std::vector<hankel_desc> descs;
    std::vector<int> Lof;
    bool real_path = false;
    // descriptors whose h or x regions overlap: the fused real path writes
    // gradients per tensor, so their adjoint runs on the general path (which
    // sums over every use)
    bool shared_io = false;
    // fused path for real tensors with a different vector per mode
    bool multi_path = false;
    std::vector<hk::MultiJob> multi_jobs;
    std::vector<hk::RealLaunch> multi_launches;
    hk::MultiJob* d_multi = nullptr;
    // fused real path
    std::vector<hk::RealJob> fwd_jobs, bwd_jobs;
    std::vector<hk::RealLaunch> fwd_launches, bwd_launches;
    hk::RealJob* d_fwd = nullptr;
    hk::RealJob* d_bwd = nullptr;
    // persistent forward kernel (FP32, one vector per tensor): the tensors
    // whose generating length fits its transforms run there, the rest on
    // the per-length launches above
    bool fast = false;
    std::vector<hk::FastJob> fast_jobs;
    std::vector<hk::FastItem> fast_items;
    hk::FastJob* d_fast_jobs = nullptr;
    hk::FastItem* d_fast_items = nullptr;
    int* d_fast_ctr = nullptr;
    void* d_fast_tw = nullptr;  // two-level tables of w_4096, w_3072 and w_5120 (FP32 complex)
    size_t fast_tw3 = 0;        // byte offset of the w_3072 table
    size_t fast_tw5 = 0;        // byte offset of the w_5120 table
    void* d_fast_slab = nullptr;  // per-block slab of the longest length (or null)
    int fast_grid = 0;
    int64_t fast_pairs = 0;  // pair jobs with at least one tensor (the rest pad items)
    bool fast_f64 = false;   // some job of the persistent launch asks for FP64 powers
    bool fast_bwd = false;   // the adjoint of the persistent launch's tensors is persistent too
    int64_t fp64_tensors = 0;  // tensors whose spectrum power is formed in FP64
    // general path (complex data, distinct vectors, BHHB)
    hk::GeneralPlan* gen = nullptr;
    // twiddle tables and workspace
    std::map<int, int> tw_off;
    void* d_tw = nullptr;
    void* d_ws = nullptr;
    size_t ws_bytes = 0;
    int64_t sum_L = 0, max_L = 0;
    int64_t h_elems = 0, x_elems = 0, y_elems = 0;
    // staging buffers of hankel_txv_host
    void *s_h = nullptr, *s_x = nullptr, *s_y = nullptr, *s_a = nullptr;
    // streams the independent launches of one call fork onto, and events
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> events;  // [0] fork, [1 + i] join of streams[i]
    // hankel_txv_host pipeline: sub-plans over contiguous descriptor ranges
    // whose copies in and out overlap the other ranges' kernels
    bool from_descs = true;  // false for plans made from level-k descriptors
    bool chunks_tried = false;
    struct Chunk {
        hankel_plan_s* plan;
        int64_t first;
        int64_t hlo, hhi, xlo, xhi, ylo, yhi;  // element ranges the chunk reads / writes
    };
    std::vector<Chunk> chunks;
    cudaStream_t s_in = nullptr, s_out = nullptr, s_cap = nullptr;
    std::vector<cudaEvent_t> pipe_events;  // [0] start, [1] end, then in / done per chunk
    // the pipeline as a CUDA graph, replayed while the host buffers are the same
    cudaGraphExec_t graph = nullptr;
    const void* gkey[4] = {nullptr, nullptr, nullptr, nullptr};
    cudaEvent_t cap_in = nullptr, cap_out = nullptr;
    // anti-circulant tensors of dimensions the transforms do not cover: the
    // Hankel plan `inner` of the periodic generating vectors, expanded from
    // the caller's c into ws_h before each call (gradients folded back)
    hankel_plan_s* inner = nullptr;
    std::vector<hk::ExpandEntry> expand;
    std::vector<hk::FoldGroup> folds;
    hk::ExpandEntry* d_expand = nullptr;
    hk::FoldGroup* d_folds = nullptr;
    int max_d = 0, max_n = 0;
    void *ws_h = nullptr, *ws_gh = nullptr;
};

namespace {

void free_plan(hankel_plan_s* p);
void free_plan(hankel_plan_s* p) {
    if (!p) return;
    cudaFree(p->d_fwd);
    cudaFree(p->d_bwd);
    cudaFree(p->d_fast_jobs);
    cudaFree(p->d_fast_items);
    cudaFree(p->d_fast_ctr);
    cudaFree(p->d_fast_tw);
    cudaFree(p->d_fast_slab);
    cudaFree(p->d_multi);
    cudaFree(p->d_tw);
    cudaFree(p->d_ws);
    cudaFree(p->s_h);
    cudaFree(p->s_x);
    cudaFree(p->s_y);
    cudaFree(p->s_a);
    for (auto st : p->streams) cudaStreamDestroy(st);
    for (auto ev : p->events) cudaEventDestroy(ev);
    for (auto& c : p->chunks) free_plan(c.plan);
    if (p->s_in) cudaStreamDestroy(p->s_in);
    if (p->s_out) cudaStreamDestroy(p->s_out);
    if (p->s_cap) cudaStreamDestroy(p->s_cap);
    if (p->graph) cudaGraphExecDestroy(p->graph);
    if (p->cap_in) cudaEventDestroy(p->cap_in);
    if (p->cap_out) cudaEventDestroy(p->cap_out);
    for (auto ev : p->pipe_events) cudaEventDestroy(ev);
    if (p->inner) free_plan(p->inner);
    cudaFree(p->d_expand);
    cudaFree(p->d_folds);
    cudaFree(p->ws_h);
    cudaFree(p->ws_gh);
    if (p->gen) hk::general_destroy(p->gen);
    delete p;
}

hankel_status validate(const hankel_desc& d, int64_t i, uint32_t flags, int64_t& gen_len) {
    if (d.m < 2 || d.m > HANKEL_MAX_ORDER)
        return fail(HANKEL_EINVAL, "descriptor %lld: order m=%d outside [2, %d]", (long long)i, d.m,
                    HANKEL_MAX_ORDER);
    int64_t s = 0;
    for (int p = 0; p < d.m; ++p) {
        if (d.n[p] < 1) return fail(HANKEL_EINVAL, "descriptor %lld: n[%d]=%d must be >= 1", (long long)i, p, d.n[p]);
        if ((flags & HANKEL_BLOCK) && d.N[p] < 1)
            return fail(HANKEL_EINVAL, "descriptor %lld: N[%d]=%d must be >= 1", (long long)i, p, d.N[p]);
        s += d.n[p];
    }
    gen_len = s - d.m + 1;
    if (d.h_off < 0 || d.y_off < 0) return fail(HANKEL_EINVAL, "descriptor %lld: negative offset", (long long)i);
    const int nx = (flags & HANKEL_SAME_X) ? 1 : d.m;
    for (int p = 0; p < nx; ++p)
        if (d.x_off[p] < 0) return fail(HANKEL_EINVAL, "descriptor %lld: negative x_off[%d]", (long long)i, p);
    return HANKEL_OK;
}

// A one- or two-level descriptor in the level-k form of the general path.
hankel_mdesc to_levels(const hankel_desc& d, bool block) {
    hankel_mdesc m;
    std::memset(&m, 0, sizeof(m));
    m.m = d.m;
    m.levels = block ? 2 : 1;
    for (int q = 0; q < d.m; ++q) {
        m.n[0][q] = d.n[q];
        m.n[1][q] = block ? d.N[q] : 1;
    }
    m.h_off = d.h_off;
    for (int q = 0; q < HANKEL_MAX_ORDER; ++q) m.x_off[q] = d.x_off[q];
    m.y_off = d.y_off;
    return m;
}

// Per-pass twiddle tables (fft_stage.cuh layout) of every distinct length.
hankel_status upload_twiddles(hankel_plan_s* p, const std::vector<int>& Ls) {
    int64_t total = 0;
    std::vector<hk::FftPlan> plans;
    for (int L : Ls) {
        if (p->tw_off.count(L)) continue;
        hk::FftPlan P;
        hk::fft_factor(L, &P);
        p->tw_off[L] = (int)total;
        P.tw_off = (int)total;
        plans.push_back(P);
        total += std::max(1, hk::stage_twiddle_count(P));
    }
    const size_t cs = 2 * real_size(p->dtype);
    cudaError_t e = cudaMalloc(&p->d_tw, std::max<int64_t>(total, 1) * cs);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(twiddles)");
    for (const auto& P : plans) {
        e = hk::launch_stage_twiddles(is_double(p->dtype), (char*)p->d_tw + (size_t)P.tw_off * cs, P, 0);
        if (e != cudaSuccess) return cuda_fail(e, "twiddle kernel");
    }
    e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(e, "twiddle generation");
    return HANKEL_OK;
}

// Threads per block for a transform of length L: about one radix-16
// butterfly per thread and pass, between one warp and 512 threads.
int nthr_of(int L) {
    const int ppt = g_points_per_thread;
    return std::max(32, std::min(512, pow2ceil((L + ppt - 1) / ppt)));
}

// Largest L whose `buffers` ping-pong arrays fit in one block's shared memory.
constexpr size_t kSmemLimit = 227 * 1024;
int max_len_for(int buffers, size_t csize) {
    int L = 2;
    while (L + 1 <= kMaxL &&
           hk::RED_BYTES + ((size_t)hk::TW_SMEM_HOST + (size_t)buffers * hk::smem_elems_host(L + 1)) * csize <=
               kSmemLimit)
        ++L;
    return L;
}

// Group jobs into launches of one block size and one job kind each (pairs
// need three shared buffers, singles two), largest transforms first.
void make_launches(std::vector<hk::RealJob>& jobs, std::vector<hk::RealLaunch>& launches, bool one_per_launch,
                   int single_buffers, int max_single_L) {
    // kind: 0 pair (three shared buffers), 1 single (two), 2 single with
    // global scratch (shared memory holds only twiddles), 4 / 5 split single
    // on a cluster of four / two blocks (two buffers of L/4 / L/2 each)
    auto kind = [&](const hk::RealJob& j) {
        if (!j.single) return 0;
        if (j.split) return j.split == 2 ? 4 : 5;
        return j.P.L > max_single_L ? 2 : 1;
    };
    std::stable_sort(jobs.begin(), jobs.end(), [&](const hk::RealJob& a, const hk::RealJob& b) {
        if (kind(a) != kind(b)) return kind(a) < kind(b);
        return a.P.L > b.P.L;
    });
    launches.clear();
    for (size_t i = 0; i < jobs.size();) {
        const int L0 = jobs[i].P.L;
        hk::RealLaunch lc{};
        lc.first = (int)i;
        lc.nthr = nthr_of(L0);
        lc.Lmax = L0;
        lc.arrays = kind(jobs[i]) == 0 ? 3 : (kind(jobs[i]) == 1 ? single_buffers : (kind(jobs[i]) >= 3 ? 2 : 0));
        lc.split = jobs[i].split;
        size_t j = i + 1;
        if (!one_per_launch)
            while (j < jobs.size() && nthr_of(jobs[j].P.L) == lc.nthr && kind(jobs[j]) == kind(jobs[i])) ++j;
        lc.count = (int)(j - i);
        launches.push_back(lc);
        i = j;
    }
}

hk::FftPlan fft_plan_of(const hankel_plan_s* p, int L) {
    const LenInfo* li = lengths().find(L);
    hk::FftPlan P;
    P.L = L;
    P.npass = (int)li->radix.size();
    P.tw_off = p->tw_off.at(L);
    for (int i = 0; i < 8; ++i) P.radix[i] = i < P.npass ? (uint8_t)li->radix[i] : 0;
    hk::fill_magic(P);
    return P;
}

// Streams (at most 8) that the independent launches of one call fork onto,
// with the fork/join events.
hankel_status make_streams(hankel_plan_s* p, size_t nlaunch) {
    const size_t nstreams = std::min<size_t>(8, nlaunch);
    if (nstreams < 2) return HANKEL_OK;
    cudaError_t e;
    for (size_t i = 0; i < nstreams; ++i) {
        cudaStream_t st;
        e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
        if (e != cudaSuccess) return cuda_fail(e, "cudaStreamCreate");
        p->streams.push_back(st);
    }
    for (size_t i = 0; i <= nstreams; ++i) {
        cudaEvent_t ev;
        e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        if (e != cudaSuccess) return cuda_fail(e, "cudaEventCreate");
        p->events.push_back(ev);
    }
    return HANKEL_OK;
}

// L / 2 when a single job of length L can run split (L even, L / 2 one of
// the planner's lengths that fits two shared buffers), else 0.
int split_length(const hankel_plan_s* p, int L) {
    const int max_single_L = max_len_for(2, 2 * real_size(p->dtype));
    if (L % 2 != 0 || L / 2 > max_single_L || lengths().find(L / 2) == nullptr) return 0;
    return L / 2;
}

// Four-way split (a cluster of four blocks of length L/4, real_path.cu),
// preferred to the two-way one where L/4 is a transform length: 0 if not.
int split4_length(const hankel_plan_s* p, int L) {
    const int max_single_L = max_len_for(2, 2 * real_size(p->dtype));
    if (L % 4 != 0 || L / 4 > max_single_L || lengths().find(L / 4) == nullptr) return 0;
    return L / 4;
}

// Pair jobs and work items of the persistent forward kernel for the tensors
// marked in `sel`: tensors of one FFT length (and, as far as the counts
// allow, one order) in pairs, each length's jobs padded with empty slots to
// whole items, items longest length first.
hankel_status build_fast(hankel_plan_s* p, const std::vector<char>& sel, const std::vector<char>& want64) {
    const int64_t count = (int64_t)p->descs.size();
    std::vector<std::pair<int, int64_t>> byL;
    for (int64_t i = 0; i < count; ++i)
        if (sel[i]) {
            const hankel_desc& d = p->descs[i];
            byL.emplace_back(hk::fast_length((int64_t)d.n[0] * d.m - d.m + 1), i);
        }
    if (byL.empty()) return HANKEL_OK;
    // longest length first; within a length by order, so that the groups of
    // a warp (short lengths put several in one warp) mostly share m and
    // with it the code of the spectral power
    std::stable_sort(byL.begin(), byL.end(), [&](const std::pair<int, int64_t>& a, const std::pair<int, int64_t>& b) {
        if (a.first != b.first) return a.first > b.first;
        return p->descs[a.second].m < p->descs[b.second].m;
    });
    hk::FastJob empty;
    std::memset(&empty, 0, sizeof(empty));
    empty.mA = empty.mB = 2;
    empty.iA = empty.iB = -1;
    auto put = [&](hk::FastJob& J, int64_t i, bool B) {
        const hankel_desc& d = p->descs[i];
        const int dl = (int)((int64_t)d.n[0] * d.m - d.m + 1);
        if (!B) {
            J.mA = d.m; J.nA = d.n[0]; J.dA = dl; J.iA = (int)i; J.fA = want64[i];
            J.hA = d.h_off; J.xA = d.x_off[0]; J.yA = d.y_off;
        } else {
            J.mB = d.m; J.nB = d.n[0]; J.dB = dl; J.iB = (int)i; J.fB = want64[i];
            J.hB = d.h_off; J.xB = d.x_off[0]; J.yB = d.y_off;
        }
    };
    p->fast_jobs.clear();
    p->fast_items.clear();
    p->fast_pairs = 0;
    p->fast_f64 = false;
    for (const auto& e : byL) p->fast_f64 = p->fast_f64 || want64[e.second];
    for (size_t k = 0; k < byL.size();) {
        const int L = byL[k].first;
        const int G = hk::fast_jobs_per_item(L);
        size_t e = k;
        while (e < byL.size() && byL[e].first == L) ++e;
        std::vector<hk::FastJob> js;
        for (size_t q = k; q < e; q += 2) {
            hk::FastJob J = empty;
            put(J, byL[q].second, false);
            if (q + 1 < e) put(J, byL[q + 1].second, true);
            js.push_back(J);
            ++p->fast_pairs;
        }
        while (js.size() % G) js.push_back(empty);
        for (size_t q = 0; q < js.size(); q += G)
            p->fast_items.push_back(hk::FastItem{L, (int32_t)(p->fast_jobs.size() + q)});
        p->fast_jobs.insert(p->fast_jobs.end(), js.begin(), js.end());
        k = e;
    }
    int sms = 0;
    cudaError_t e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p->device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceGetAttribute");
    p->fast_grid = (int)std::min<int64_t>((int64_t)p->fast_items.size(), (int64_t)sms * hk::fast_blocks_per_sm());
    if ((e = cudaMalloc(&p->d_fast_jobs, p->fast_jobs.size() * sizeof(hk::FastJob))) != cudaSuccess)
        return cuda_fail(e, "cudaMalloc(jobs)");
    if ((e = cudaMalloc(&p->d_fast_items, p->fast_items.size() * sizeof(hk::FastItem))) != cudaSuccess)
        return cuda_fail(e, "cudaMalloc(jobs)");
    // work counters: [0], [1] the forward's, [2], [3] the adjoint's
    if ((e = cudaMalloc(&p->d_fast_ctr, 4 * sizeof(int))) != cudaSuccess) return cuda_fail(e, "cudaMalloc(counter)");
    // items are longest first: the first one's length sizes the slab
    const size_t slab = hk::fast_slab_bytes(p->fast_items.front().L);
    if (slab > 0 && (e = cudaMalloc(&p->d_fast_slab, slab * p->fast_grid)) != cudaSuccess)
        return cuda_fail(e, "cudaMalloc(slab)");
    hk::FftPlan P2, P3, P5;
    std::memset(&P2, 0, sizeof(P2));
    std::memset(&P3, 0, sizeof(P3));
    std::memset(&P5, 0, sizeof(P5));
    P2.L = 4096;
    P3.L = 3072;
    P5.L = 5120;
    const int n2 = hk::stage_twiddle_count(P2), n3 = hk::stage_twiddle_count(P3), n5 = hk::stage_twiddle_count(P5);
    if ((e = cudaMalloc(&p->d_fast_tw, (size_t)(n2 + n3 + n5) * 2 * sizeof(float))) != cudaSuccess)
        return cuda_fail(e, "cudaMalloc(twiddles)");
    p->fast_tw3 = (size_t)n2 * 2 * sizeof(float);
    p->fast_tw5 = (size_t)(n2 + n3) * 2 * sizeof(float);
    e = cudaMemcpy(p->d_fast_jobs, p->fast_jobs.data(), p->fast_jobs.size() * sizeof(hk::FastJob),
                   cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(p->d_fast_items, p->fast_items.data(), p->fast_items.size() * sizeof(hk::FastItem),
                       cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(p->d_fast_ctr, 0, 4 * sizeof(int));
    if (e == cudaSuccess) e = hk::launch_stage_twiddles(false, p->d_fast_tw, P2, 0);
    if (e == cudaSuccess) e = hk::launch_stage_twiddles(false, (char*)p->d_fast_tw + p->fast_tw3, P3, 0);
    if (e == cudaSuccess) e = hk::launch_stage_twiddles(false, (char*)p->d_fast_tw + p->fast_tw5, P5, 0);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(e, "fast path set-up");
    p->fast = true;
    return HANKEL_OK;
}

hankel_status build_real_path(hankel_plan_s* p) {
    const int64_t count = (int64_t)p->descs.size();
    const bool dbl = is_double(p->dtype);
    const size_t cs = 2 * real_size(p->dtype);
    const int max_pair_L = max_len_for(3, cs);
    const int max_single_L = max_len_for(2, cs);
    const bool singles = (p->flags & (HANKEL_STORE_SPECTRA | HANKEL_ONE_PER_LAUNCH)) != 0;
    // workspace: one spectrum (L) per tensor, then 2 L of transform scratch
    // for each tensor longer than shared memory allows
    std::vector<int64_t> ws_off(count), gscratch(count, -1);
    int64_t ws = 0;
    for (int64_t i = 0; i < count; ++i) {
        ws_off[i] = ws;
        ws += p->Lof[i];
    }
    for (int64_t i = 0; i < count; ++i)
        if (p->Lof[i] > max_single_L) {
            gscratch[i] = ws;
            ws += 2 * (int64_t)p->Lof[i];
        }
    auto fill = [&](hk::RealJob& J, int64_t i, bool B) {
        const hankel_desc& d = p->descs[i];
        const int dl = (p->flags & HANKEL_ANTICIRCULANT) ? d.n[0] : (int)(d.n[0] * (int64_t)d.m - d.m + 1);
        if (!B) {
            J.mA = d.m; J.nA = d.n[0]; J.dA = dl; J.iA = (int)i;
            J.hA = d.h_off; J.xA = d.x_off[0]; J.yA = d.y_off; J.wsA = ws_off[i];
            if (gscratch[i] >= 0) J.wsB = gscratch[i];
        } else {
            J.mB = d.m; J.nB = d.n[0]; J.dB = dl; J.iB = (int)i;
            J.hB = d.h_off; J.xB = d.x_off[0]; J.yB = d.y_off; J.wsB = ws_off[i];
        }
    };
    std::vector<int64_t> order(count);
    for (int64_t i = 0; i < count; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int64_t a, int64_t b) { return p->Lof[a] < p->Lof[b]; });
    p->fwd_jobs.clear();
    p->bwd_jobs.clear();
    // FP32 forward products whose generating length fits the persistent
    // kernel's transforms run there, unless their bin's policy says
    // otherwise; FP64 spectrum powers for the whole plan (flag) or for the
    // orders the bin's policy names
    const bool fast_ok = p->dtype == HANKEL_R32 &&
                         !(p->flags & (HANKEL_STORE_SPECTRA | HANKEL_ONE_PER_LAUNCH | HANKEL_ANTICIRCULANT));
    std::vector<char> on_fast(count, 0), want64(count, 0);
    p->fp64_tensors = 0;
    for (int64_t i = 0; i < count; ++i) {
        const hankel_desc& d = p->descs[i];
        const int dl = (p->flags & HANKEL_ANTICIRCULANT) ? d.n[0] : (int)(d.n[0] * (int64_t)d.m - d.m + 1);
        const int Lb = hk::fast_length(dl);
        const BinPolicy bp = Lb > 0 ? bin_policy(Lb) : BinPolicy();
        want64[i] = !dbl && ((p->flags & HANKEL_FP64_POWER) || d.m >= bp.fp64_from_m);
        p->fp64_tensors += want64[i];
        on_fast[i] = fast_ok && Lb > 0 && bp.path == 0;
    }
    std::vector<int64_t> fwd_order;
    for (int64_t a : order)
        if (!on_fast[a]) fwd_order.push_back(a);
    // the adjoint of the persistent launch's tensors runs persistent too,
    // unless some of them share storage (their gradients are sums: the
    // general path) or ask for FP64 spectrum powers
    bool any_fast = false, fast64 = false;
    for (int64_t i = 0; i < count; ++i) {
        any_fast = any_fast || on_fast[i];
        fast64 = fast64 || (on_fast[i] && want64[i]);
    }
    p->fast_bwd = any_fast && !fast64 && !p->shared_io;
    for (size_t k = 0; k < fwd_order.size();) {
        const std::vector<int64_t>& order = fwd_order;
        hk::RealJob J;
        std::memset(&J, 0, sizeof(J));
        const int64_t a = order[k];
        const int L = p->Lof[a];
        J.P = fft_plan_of(p, L);
        fill(J, a, false);
        J.iB = -1;
        if (!singles && L <= max_pair_L && k + 1 < order.size() && p->Lof[order[k + 1]] == L) {
            fill(J, order[k + 1], true);
            J.single = 0;
            k += 2;
        } else if (!singles && L <= max_pair_L) {
            // a leftover tensor runs as a pair with an empty partner, so that
            // it shares the pair launches instead of needing its own
            J.single = 0;
            k += 1;
        } else {
            J.single = 1;
            k += 1;
        }
        p->fwd_jobs.push_back(J);
    }
    // adjoint: tensors of one length in pairs that share the transform of
    // their upstream gradients (three shared buffers), longer ones alone
    const bool pair_bwd = (p->flags & HANKEL_ONE_PER_LAUNCH) == 0;
    if (p->fast_bwd) {
        std::vector<int64_t> rest;
        for (int64_t a : order)
            if (!on_fast[a]) rest.push_back(a);
        order.swap(rest);
    }
    for (size_t k = 0; k < order.size();) {
        hk::RealJob J;
        std::memset(&J, 0, sizeof(J));
        const int64_t a = order[k];
        const int L = p->Lof[a];
        J.P = fft_plan_of(p, L);
        fill(J, a, false);
        J.iB = -1;
        J.single = 1;
        k += 1;
        if (pair_bwd && L <= max_pair_L) {
            J.single = 0;
            if (k < order.size() && p->Lof[order[k]] == L) {
                fill(J, order[k], true);
                k += 1;
            }
        }
        p->bwd_jobs.push_back(J);
    }
    // single jobs too long for one block's shared memory run as split jobs
    // on thread-block clusters: two blocks of length L/2 (split 3), else
    // four of L/4 (split 2), where that is a transform length of the plan
    for (auto* v : {&p->fwd_jobs, &p->bwd_jobs})
        for (auto& J : *v) {
            const int L = J.P.L;
            if (!J.single || L <= max_single_L) continue;
            if (split_length(p, L) > 0) {
                J.split = 3;
                J.twL = p->tw_off.at(L);
                J.P = fft_plan_of(p, L / 2);
            } else if (split4_length(p, L) > 0) {
                J.split = 2;
                J.twL = p->tw_off.at(L);
                J.P = fft_plan_of(p, L / 4);
            }
        }
    const bool opl = (p->flags & HANKEL_ONE_PER_LAUNCH) != 0;
    make_launches(p->fwd_jobs, p->fwd_launches, opl, 2, max_single_L);
    make_launches(p->bwd_jobs, p->bwd_launches, opl, 2, max_single_L);
    // a launch forms FP64 powers when one of its tensors asks for them
    auto mark64 = [&](const std::vector<hk::RealJob>& jobs, std::vector<hk::RealLaunch>& launches) {
        for (auto& lc : launches) {
            lc.fp64 = 0;
            for (int j = lc.first; j < lc.first + lc.count; ++j)
                lc.fp64 |= (jobs[j].iA >= 0 && want64[jobs[j].iA]) || (jobs[j].iB >= 0 && want64[jobs[j].iB]);
        }
    };
    mark64(p->fwd_jobs, p->fwd_launches);
    mark64(p->bwd_jobs, p->bwd_launches);
    for (auto* v : {&p->fwd_launches, &p->bwd_launches})
        for (auto& lc : *v)
            if (hk::real_launch_smem(dbl, lc) > kSmemLimit)
                return fail(HANKEL_EUNSUPPORTED, "FFT length %d needs more shared memory than a block has", lc.Lmax);
    cudaError_t e;
    const size_t jb = sizeof(hk::RealJob);
    e = cudaMalloc(&p->d_fwd, std::max<size_t>(p->fwd_jobs.size(), 1) * jb);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(jobs)");
    e = cudaMalloc(&p->d_bwd, std::max<size_t>(p->bwd_jobs.size(), 1) * jb);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(jobs)");
    e = cudaMemcpy(p->d_fwd, p->fwd_jobs.data(), p->fwd_jobs.size() * jb, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy(jobs)");
    e = cudaMemcpy(p->d_bwd, p->bwd_jobs.data(), p->bwd_jobs.size() * jb, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy(jobs)");
    const size_t nfwd = p->fwd_launches.size() + (fast_ok ? 1 : 0);
    const hankel_status ss = make_streams(p, opl ? 0 : std::max(nfwd, p->bwd_launches.size()));
    if (ss != HANKEL_OK) return ss;
    if (fast_ok) {
        const hankel_status fs = build_fast(p, on_fast, want64);
        if (fs != HANKEL_OK) return fs;
    }
    p->ws_bytes = (size_t)std::max<int64_t>(ws, 1) * 2 * real_size(p->dtype);
    e = cudaMalloc(&p->d_ws, p->ws_bytes);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(workspace)");
    return HANKEL_OK;
}

// The per-length launches (queued first) on the plan's streams and `main`
// (the persistent kernel) on the caller's stream, joined back into it.
template <class F, class G>
hankel_status run_forked_with(hankel_plan_s* p, const std::vector<hk::RealLaunch>& launches, cudaStream_t st,
                              F launch, G main) {
    cudaError_t e;
    if (launches.empty() || p->streams.empty()) {
        for (auto& lc : launches)
            if ((e = launch(lc, st)) != cudaSuccess) return cuda_fail(e, "kernel launch");
        if ((e = main(st)) != cudaSuccess) return cuda_fail(e, "kernel launch");
        return HANKEL_OK;
    }
    const size_t n = std::min(p->streams.size(), launches.size());
    if ((e = cudaEventRecord(p->events[0], st)) != cudaSuccess) return cuda_fail(e, "cudaEventRecord");
    for (size_t i = 0; i < n; ++i)
        if ((e = cudaStreamWaitEvent(p->streams[i], p->events[0], 0)) != cudaSuccess)
            return cuda_fail(e, "cudaStreamWaitEvent");
    for (size_t i = 0; i < launches.size(); ++i)
        if ((e = launch(launches[i], p->streams[i % n])) != cudaSuccess) return cuda_fail(e, "kernel launch");
    if ((e = main(st)) != cudaSuccess) return cuda_fail(e, "kernel launch");
    for (size_t i = 0; i < n; ++i) {
        if ((e = cudaEventRecord(p->events[1 + i], p->streams[i])) != cudaSuccess)
            return cuda_fail(e, "cudaEventRecord");
        if ((e = cudaStreamWaitEvent(st, p->events[1 + i], 0)) != cudaSuccess)
            return cuda_fail(e, "cudaStreamWaitEvent");
    }
    return HANKEL_OK;
}

// Queue independent launches: with the plan's streams, fork from `st`, run
// launch i on stream i mod n, and join back into `st` (graph-capturable);
// without them, run them in order on `st`.
template <class F>
hankel_status run_forked(hankel_plan_s* p, const std::vector<hk::RealLaunch>& launches, cudaStream_t st, F launch) {
    cudaError_t e;
    if (p->streams.empty() || launches.size() < 2) {
        for (auto& lc : launches)
            if ((e = launch(lc, st)) != cudaSuccess) return cuda_fail(e, "kernel launch");
        return HANKEL_OK;
    }
    const size_t n = std::min(p->streams.size(), launches.size());
    if ((e = cudaEventRecord(p->events[0], st)) != cudaSuccess) return cuda_fail(e, "cudaEventRecord");
    for (size_t i = 0; i < n; ++i)
        if ((e = cudaStreamWaitEvent(p->streams[i], p->events[0], 0)) != cudaSuccess)
            return cuda_fail(e, "cudaStreamWaitEvent");
    for (size_t i = 0; i < launches.size(); ++i)
        if ((e = launch(launches[i], p->streams[i % n])) != cudaSuccess) return cuda_fail(e, "kernel launch");
    for (size_t i = 0; i < n; ++i) {
        if ((e = cudaEventRecord(p->events[1 + i], p->streams[i])) != cudaSuccess) return cuda_fail(e, "cudaEventRecord");
        if ((e = cudaStreamWaitEvent(st, p->events[1 + i], 0)) != cudaSuccess)
            return cuda_fail(e, "cudaStreamWaitEvent");
    }
    return HANKEL_OK;
}

// Real tensors with distinct mode vectors: pair tensors of equal FFT length
// (MultiJob), group pairs into launches by block size.
hankel_status build_multi_path(hankel_plan_s* p) {
    const int64_t count = (int64_t)p->descs.size();
    std::vector<int64_t> order(count);
    for (int64_t i = 0; i < count; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int64_t a, int64_t b) { return p->Lof[a] > p->Lof[b]; });
    auto fill = [&](hk::MultiJob& J, int64_t i, bool B) {
        const hankel_desc& d = p->descs[i];
        int64_t sn = 0;
        for (int q = 0; q < d.m; ++q) sn += d.n[q];
        const int dl = (p->flags & HANKEL_ANTICIRCULANT) ? d.n[0] : (int)(sn - d.m + 1);
        if (!B) {
            J.mA = d.m; J.iA = (int)i; J.dA = dl; J.hA = d.h_off; J.yA = d.y_off;
            for (int q = 0; q < d.m; ++q) { J.nA[q] = d.n[q]; J.xA[q] = d.x_off[q]; }
        } else {
            J.mB = d.m; J.iB = (int)i; J.dB = dl; J.hB = d.h_off; J.yB = d.y_off;
            for (int q = 0; q < d.m; ++q) { J.nB[q] = d.n[q]; J.xB[q] = d.x_off[q]; }
        }
    };
    p->multi_jobs.clear();
    for (size_t k = 0; k < order.size();) {
        hk::MultiJob J;
        std::memset(&J, 0, sizeof(J));
        J.P = fft_plan_of(p, p->Lof[order[k]]);
        fill(J, order[k], false);
        J.iB = -1;
        if (k + 1 < order.size() && p->Lof[order[k + 1]] == p->Lof[order[k]]) {
            fill(J, order[k + 1], true);
            k += 2;
        } else {
            k += 1;
        }
        p->multi_jobs.push_back(J);
    }
    // launches: consecutive jobs (lengths descending) with one block size
    const bool opl = (p->flags & HANKEL_ONE_PER_LAUNCH) != 0;
    p->multi_launches.clear();
    for (size_t i = 0; i < p->multi_jobs.size();) {
        hk::RealLaunch lc{};
        lc.first = (int)i;
        lc.nthr = nthr_of(p->multi_jobs[i].P.L);
        lc.split = 0;
        lc.Lmax = p->multi_jobs[i].P.L;
        lc.arrays = 3;
        size_t j = i + 1;
        if (!opl)
            while (j < p->multi_jobs.size() && nthr_of(p->multi_jobs[j].P.L) == lc.nthr) ++j;
        lc.count = (int)(j - i);
        p->multi_launches.push_back(lc);
        i = j;
    }
    for (const auto& lc : p->multi_launches)
        if (hk::real_launch_smem(is_double(p->dtype), lc) > kSmemLimit)
            return fail(HANKEL_EUNSUPPORTED, "FFT length %d needs more shared memory than a block has", lc.Lmax);
    const size_t jb = sizeof(hk::MultiJob);
    cudaError_t e = cudaMalloc(&p->d_multi, std::max<size_t>(p->multi_jobs.size(), 1) * jb);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(jobs)");
    e = cudaMemcpy(p->d_multi, p->multi_jobs.data(), p->multi_jobs.size() * jb, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy(jobs)");
    return make_streams(p, opl ? 0 : p->multi_launches.size());
}

// Device address of page-locked host memory that is mapped into the device
// address space, or nullptr for any other pointer.
const void* mapped_host(const void* ptr) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return (a.type == cudaMemoryTypeHost) ? a.devicePointer : nullptr;
}

// Element ranges of h, x and y that one descriptor reads or writes.
void desc_ranges(const hankel_desc& d, uint32_t flags, int64_t r[6]) {
    const bool block = flags & HANKEL_BLOCK, anti = flags & HANKEL_ANTICIRCULANT;
    int64_t sn = 0, sN = 0;
    for (int q = 0; q < d.m; ++q) {
        sn += d.n[q];
        sN += block ? d.N[q] : 1;
    }
    const int64_t N0 = block ? d.N[0] : 1;
    const int64_t hl = anti ? (int64_t)d.n[0] * N0 : (sn - d.m + 1) * (block ? sN - d.m + 1 : 1);
    r[0] = d.h_off;
    r[1] = d.h_off + hl;
    const int nx = (flags & HANKEL_SAME_X) ? 1 : d.m;
    r[2] = INT64_MAX;
    r[3] = 0;
    for (int q = 0; q < nx; ++q) {
        r[2] = std::min<int64_t>(r[2], d.x_off[q]);
        r[3] = std::max<int64_t>(r[3], d.x_off[q] + (int64_t)d.n[q] * (block ? d.N[q] : 1));
    }
    r[4] = d.y_off;
    r[5] = d.y_off + (int64_t)d.n[0] * N0;
}

// Split a plan's descriptors into contiguous ranges with one sub-plan each
// (made once, on the first pipelined hankel_txv_host).
hankel_status build_chunks(hankel_plan_s* p) {
    const int64_t count = (int64_t)p->descs.size();
    // Range sizes by input bytes: small at both ends, so that the first copy
    // in (which nothing overlaps) and the last range's kernels and copy out
    // (which overlap nothing) are short; each middle range's kernels finish
    // while the next range is still being copied in.
    static const double kShare[] = {0.04, 0.12, 0.20, 0.24, 0.20, 0.12, 0.08};
    constexpr int nchunks = (int)(sizeof(kShare) / sizeof(kShare[0]));
    std::vector<double> cum(count + 1, 0.0);
    for (int64_t i = 0; i < count; ++i) {
        int64_t r[6];
        desc_ranges(p->descs[i], p->flags, r);
        cum[i + 1] = cum[i] + (double)(r[1] - r[0]) + (double)(r[3] - r[2]);
    }
    std::vector<int64_t> cut(nchunks + 1, count);
    cut[0] = 0;
    double acc = 0.0;
    for (int c = 1; c < nchunks; ++c) {
        acc += kShare[c - 1];
        cut[c] = std::lower_bound(cum.begin(), cum.end(), acc * cum[count]) - cum.begin();
        cut[c] = std::max(cut[c], cut[c - 1]);
    }
    for (int c = 0; c < nchunks; ++c) {
        const int64_t c0 = cut[c], c1 = std::min<int64_t>(cut[c + 1], count);
        if (c1 <= c0) continue;
        hankel_plan_s::Chunk ch{nullptr, c0, INT64_MAX, 0, INT64_MAX, 0, INT64_MAX, 0};
        for (int64_t i = c0; i < c1; ++i) {
            int64_t r[6];
            desc_ranges(p->descs[i], p->flags, r);
            ch.hlo = std::min(ch.hlo, r[0]);
            ch.hhi = std::max(ch.hhi, r[1]);
            ch.xlo = std::min(ch.xlo, r[2]);
            ch.xhi = std::max(ch.xhi, r[3]);
            ch.ylo = std::min(ch.ylo, r[4]);
            ch.yhi = std::max(ch.yhi, r[5]);
        }
        const hankel_status s = hankel_plan(&ch.plan, p->descs.data() + c0, c1 - c0, p->dtype, p->flags);
        if (s != HANKEL_OK) return s;
        p->chunks.push_back(ch);
    }
    cudaError_t e;
    if ((e = cudaStreamCreateWithFlags(&p->s_in, cudaStreamNonBlocking)) != cudaSuccess)
        return cuda_fail(e, "cudaStreamCreate");
    if ((e = cudaStreamCreateWithFlags(&p->s_out, cudaStreamNonBlocking)) != cudaSuccess)
        return cuda_fail(e, "cudaStreamCreate");
    if ((e = cudaStreamCreateWithFlags(&p->s_cap, cudaStreamNonBlocking)) != cudaSuccess)
        return cuda_fail(e, "cudaStreamCreate");
    if ((e = cudaEventCreateWithFlags(&p->cap_in, cudaEventDisableTiming)) != cudaSuccess)
        return cuda_fail(e, "cudaEventCreate");
    if ((e = cudaEventCreateWithFlags(&p->cap_out, cudaEventDisableTiming)) != cudaSuccess)
        return cuda_fail(e, "cudaEventCreate");
    for (size_t i = 0; i < 2 + 2 * p->chunks.size(); ++i) {
        cudaEvent_t ev;
        if ((e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess)
            return cuda_fail(e, "cudaEventCreate");
        p->pipe_events.push_back(ev);
    }
    return HANKEL_OK;
}

// Enqueue the whole pipeline on stream s: copies in on s_in, each range's
// kernels on s, copies out on s_out, all joined back into s.
hankel_status enqueue_pipeline(hankel_plan_s* p, const void* h, const void* x, void* y, void* alpha, cudaStream_t s) {
    const size_t es = elem_size(p->dtype);
    cudaError_t e;
    cudaEvent_t ev_start = p->pipe_events[0], ev_end = p->pipe_events[1];
    if ((e = cudaEventRecord(ev_start, s)) != cudaSuccess) return cuda_fail(e, "cudaEventRecord");
    if ((e = cudaStreamWaitEvent(p->s_in, ev_start, 0)) != cudaSuccess) return cuda_fail(e, "cudaStreamWaitEvent");
    if ((e = cudaStreamWaitEvent(p->s_out, ev_start, 0)) != cudaSuccess) return cuda_fail(e, "cudaStreamWaitEvent");
    for (size_t c = 0; c < p->chunks.size(); ++c) {
        const auto& ch = p->chunks[c];
        cudaEvent_t ev_in = p->pipe_events[2 + 2 * c], ev_done = p->pipe_events[3 + 2 * c];
        if ((e = cudaMemcpyAsync((char*)p->s_h + ch.hlo * es, (const char*)h + ch.hlo * es, (ch.hhi - ch.hlo) * es,
                                 cudaMemcpyHostToDevice, p->s_in)) != cudaSuccess)
            return cuda_fail(e, "H2D");
        if ((e = cudaMemcpyAsync((char*)p->s_x + ch.xlo * es, (const char*)x + ch.xlo * es, (ch.xhi - ch.xlo) * es,
                                 cudaMemcpyHostToDevice, p->s_in)) != cudaSuccess)
            return cuda_fail(e, "H2D");
        if ((e = cudaEventRecord(ev_in, p->s_in)) != cudaSuccess) return cuda_fail(e, "cudaEventRecord");
        if ((e = cudaStreamWaitEvent(s, ev_in, 0)) != cudaSuccess) return cuda_fail(e, "cudaStreamWaitEvent");
        void* ya = y ? p->s_y : nullptr;
        void* aa = alpha ? (void*)((char*)p->s_a + ch.first * es) : nullptr;
        const hankel_stream_t hs = (hankel_stream_t)s;
        const hankel_status st = (p->flags & HANKEL_BLOCK) ? hankel_txv_block(ch.plan, p->s_h, p->s_x, ya, aa, hs)
                                                           : hankel_txv(ch.plan, p->s_h, p->s_x, ya, aa, hs);
        if (st != HANKEL_OK) return st;
        if ((e = cudaEventRecord(ev_done, s)) != cudaSuccess) return cuda_fail(e, "cudaEventRecord");
        if (y) {
            // ranges copied out later repeat any value copied earlier, so the
            // last copy of every output is the computed one
            if ((e = cudaStreamWaitEvent(p->s_out, ev_done, 0)) != cudaSuccess)
                return cuda_fail(e, "cudaStreamWaitEvent");
            if ((e = cudaMemcpyAsync((char*)y + ch.ylo * es, (const char*)p->s_y + ch.ylo * es, (ch.yhi - ch.ylo) * es,
                                     cudaMemcpyDeviceToHost, p->s_out)) != cudaSuccess)
                return cuda_fail(e, "D2H");
        }
    }
    if (alpha && (e = cudaMemcpyAsync(alpha, p->s_a, p->descs.size() * es, cudaMemcpyDeviceToHost, s)) != cudaSuccess)
        return cuda_fail(e, "D2H");
    if ((e = cudaEventRecord(ev_end, p->s_out)) != cudaSuccess) return cuda_fail(e, "cudaEventRecord");
    if ((e = cudaStreamWaitEvent(s, ev_end, 0)) != cudaSuccess) return cuda_fail(e, "cudaStreamWaitEvent");
    return HANKEL_OK;
}

// Record the pipeline for these host buffers as a CUDA graph (after an eager
// run has finished, so every kernel attribute is already set).  On any
// failure the plan keeps running the pipeline eagerly.
void capture_pipeline(hankel_plan_s* p, const void* h, const void* x, void* y, void* alpha) {
    if (p->graph) {
        cudaGraphExecDestroy(p->graph);
        p->graph = nullptr;
    }
    cudaGraph_t graph = nullptr;
    if (cudaStreamBeginCapture(p->s_cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        return;
    }
    const hankel_status s = enqueue_pipeline(p, h, x, y, alpha, p->s_cap);
    const cudaError_t e = cudaStreamEndCapture(p->s_cap, &graph);
    if (s == HANKEL_OK && e == cudaSuccess && graph != nullptr &&
        cudaGraphInstantiate(&p->graph, graph, 0) == cudaSuccess) {
        p->gkey[0] = h;
        p->gkey[1] = x;
        p->gkey[2] = y;
        p->gkey[3] = alpha;
    } else {
        p->graph = nullptr;
        cudaGetLastError();
    }
    if (graph) cudaGraphDestroy(graph);
}

// Whether an anti-circulant plan needs the periodic expansion: some
// dimension n is not one of the transform lengths.
bool needs_expansion(const hankel_desc* descs, int64_t count) {
    for (int64_t i = 0; i < count; ++i)
        if (descs[i].n[0] >= 2 && (lengths().find(descs[i].n[0]) == nullptr || descs[i].n[0] > kMaxL)) return true;
    return false;
}

hankel_status plan_expanded(hankel_plan_t* out, const hankel_desc* descs, int64_t count, hankel_dtype dtype,
                            uint32_t flags) {
    std::vector<hankel_desc> in(descs, descs + count);
    auto* p = new (std::nothrow) hankel_plan_s;
    if (!p) return fail(HANKEL_ENOMEM, "host allocation failed");
    p->dtype = dtype;
    p->flags = flags;
    cudaGetDevice(&p->device);
    p->descs.assign(descs, descs + count);
    std::map<std::pair<int64_t, int>, std::vector<int>> groups;
    int64_t ws = 0;
    for (int64_t i = 0; i < count; ++i) {
        const hankel_desc& D = descs[i];
        for (int q = 1; q < D.m; ++q)
            if (D.n[q] != D.n[0]) {
                free_plan(p);
                return fail(HANKEL_EINVAL, "descriptor %lld: anti-circulant tensors are square", (long long)i);
            }
        if (D.n[0] < 2) {
            free_plan(p);
            return fail(HANKEL_EINVAL, "descriptor %lld: anti-circulant dimension n=%d must be >= 2", (long long)i,
                        D.n[0]);
        }
        const int64_t d = (int64_t)D.m * (D.n[0] - 1) + 1;
        const LenInfo* li = lengths().pick(d);
        if (!li || li->L > kMaxL) {
            free_plan(p);
            return fail(HANKEL_EUNSUPPORTED, "descriptor %lld: anti-circulant dimension n=%d is not an FFT length "
                        "and its periodic embedding d=%lld exceeds the maximum FFT length %lld",
                        (long long)i, D.n[0], (long long)d, (long long)kMaxL);
        }
        p->expand.push_back({D.h_off, ws, D.n[0], (int32_t)d});
        groups[std::make_pair(D.h_off, D.n[0])].push_back((int)i);
        in[i].h_off = ws;
        ws += (d + 3) / 4 * 4;
        p->max_d = std::max<int>(p->max_d, (int)d);
        p->max_n = std::max<int>(p->max_n, D.n[0]);
        p->h_elems = std::max<int64_t>(p->h_elems, D.h_off + D.n[0]);
    }
    // fold groups: entries sharing c, listed contiguously
    std::vector<hk::ExpandEntry> ordered;
    for (auto& kv : groups) {
        hk::FoldGroup G{kv.first.first, kv.first.second, (int32_t)ordered.size(), (int32_t)kv.second.size()};
        for (int i : kv.second) ordered.push_back(p->expand[i]);
        p->folds.push_back(G);
    }
    hankel_status s = hankel_plan(&p->inner, in.data(), count, dtype, flags & ~(uint32_t)HANKEL_ANTICIRCULANT);
    if (s != HANKEL_OK) { free_plan(p); return s; }
    const size_t es = elem_size(dtype);
    cudaError_t e;
    if ((e = cudaMalloc(&p->ws_h, std::max<int64_t>(ws, 1) * es)) != cudaSuccess) { free_plan(p); return cuda_fail(e, "cudaMalloc(expansion)"); }
    if ((e = cudaMalloc(&p->ws_gh, std::max<int64_t>(ws, 1) * es)) != cudaSuccess) { free_plan(p); return cuda_fail(e, "cudaMalloc(expansion)"); }
    if ((e = cudaMalloc(&p->d_expand, p->expand.size() * sizeof(hk::ExpandEntry))) != cudaSuccess) { free_plan(p); return cuda_fail(e, "cudaMalloc(expansion)"); }
    if ((e = cudaMalloc(&p->d_folds, p->folds.size() * sizeof(hk::FoldGroup) + ordered.size() * sizeof(hk::ExpandEntry))) != cudaSuccess) { free_plan(p); return cuda_fail(e, "cudaMalloc(expansion)"); }
    e = cudaMemcpy(p->d_expand, p->expand.data(), p->expand.size() * sizeof(hk::ExpandEntry), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(p->d_folds, p->folds.data(), p->folds.size() * sizeof(hk::FoldGroup), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(reinterpret_cast<char*>(p->d_folds) + p->folds.size() * sizeof(hk::FoldGroup), ordered.data(),
                       ordered.size() * sizeof(hk::ExpandEntry), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) { free_plan(p); return cuda_fail(e, "cudaMemcpy(expansion)"); }
    p->x_elems = p->inner->x_elems;
    p->y_elems = p->inner->y_elems;
    p->sum_L = p->inner->sum_L;
    p->max_L = p->inner->max_L;
    *out = p;
    return HANKEL_OK;
}

// The fold groups' entries (ordered by group) follow the groups in d_folds.
const hk::ExpandEntry* fold_entries(const hankel_plan_s* p) {
    return reinterpret_cast<const hk::ExpandEntry*>(reinterpret_cast<const char*>(p->d_folds) +
                                                    p->folds.size() * sizeof(hk::FoldGroup));
}

// The general-path program of a plan (made on first use for plans whose
// forward products run on a fused path but whose adjoint runs here).
hankel_status ensure_general(hankel_plan_s* p) {
    if (p->gen) return HANKEL_OK;
    const bool block = (p->flags & HANKEL_BLOCK) != 0;
    std::vector<hankel_mdesc> md(p->descs.size());
    for (size_t i = 0; i < p->descs.size(); ++i) md[i] = to_levels(p->descs[i], block);
    int64_t he, xe, ye, sl, ml;
    // its forward never runs, so it keeps no spectra for the adjoint
    return hk::general_create(&p->gen, md, p->dtype, p->flags & ~(uint32_t)HANKEL_STORE_SPECTRA, &he, &xe, &ye, &sl,
                              &ml, g_err);
}

// Whether any two descriptors' h regions, or any two x regions, overlap.
bool regions_overlap(const std::vector<hankel_desc>& descs, uint32_t flags) {
    std::vector<std::pair<int64_t, int64_t>> hs, xs;
    for (const auto& d : descs) {
        int64_t r[6];
        desc_ranges(d, flags, r);
        hs.emplace_back(r[0], r[1]);
        const int nx = (flags & HANKEL_SAME_X) ? 1 : d.m;
        for (int q = 0; q < nx; ++q) xs.emplace_back(d.x_off[q], d.x_off[q] + d.n[q]);
    }
    for (auto* v : {&hs, &xs}) {
        std::sort(v->begin(), v->end());
        for (size_t i = 1; i < v->size(); ++i)
            if ((*v)[i].first < (*v)[i - 1].second) return true;
    }
    return false;
}

}  // namespace

extern "C" {

hankel_status hankel_plan(hankel_plan_t* out, const hankel_desc* descs, int64_t count, hankel_dtype dtype,
                          uint32_t flags) {
    if (out == nullptr) return fail(HANKEL_EINVAL, "out is NULL");
    *out = nullptr;
    if (descs == nullptr || count < 1) return fail(HANKEL_EINVAL, "need at least one descriptor");
    if (dtype < HANKEL_R32 || dtype > HANKEL_C128) return fail(HANKEL_EINVAL, "unknown dtype %d", (int)dtype);
    if (flags & ~(uint32_t)0x3F) return fail(HANKEL_EINVAL, "unknown flag bits 0x%x", flags);
    if ((flags & HANKEL_ANTICIRCULANT) && !(flags & HANKEL_BLOCK) && needs_expansion(descs, count)) {
        for (int64_t i = 0; i < count; ++i) {
            int64_t d;
            const hankel_status s = validate(descs[i], i, flags, d);
            if (s != HANKEL_OK) return s;
        }
        return plan_expanded(out, descs, count, dtype, flags);
    }
    auto* p = new (std::nothrow) hankel_plan_s;
    if (!p) return fail(HANKEL_ENOMEM, "host allocation failed");
    p->dtype = dtype;
    p->flags = flags;
    cudaGetDevice(&p->device);
    p->descs.assign(descs, descs + count);
    const bool block = (flags & HANKEL_BLOCK) != 0;
    const int64_t maxL = kMaxL;
    std::vector<int> Ls;
    for (int64_t i = 0; i < count; ++i) {
        int64_t d;
        hankel_status s = validate(descs[i], i, flags, d);
        if (s != HANKEL_OK) { free_plan(p); return s; }
        const hankel_desc& D = descs[i];
        const int nx = (flags & HANKEL_SAME_X) ? 1 : D.m;
        if (flags & HANKEL_ANTICIRCULANT) {
            for (int q = 1; q < D.m; ++q)
                if (D.n[q] != D.n[0] || (block && D.N[q] != D.N[0])) {
                    free_plan(p);
                    return fail(HANKEL_EINVAL, "descriptor %lld: anti-circulant tensors are square", (long long)i);
                }
            if (D.n[0] < 2) {
                free_plan(p);
                return fail(HANKEL_EINVAL, "descriptor %lld: anti-circulant dimension n=%d must be >= 2",
                            (long long)i, D.n[0]);
            }
            d = D.n[0];  // the compressed generating vector has n entries
            if (!block && (lengths().find((int)d) == nullptr || d > maxL)) {
                free_plan(p);
                return fail(HANKEL_EUNSUPPORTED, "descriptor %lld: anti-circulant dimension n=%lld is not an FFT "
                            "length of this build (2,3,5,7-smooth, at most %lld)", (long long)i, (long long)d,
                            (long long)maxL);
            }
        }
        if (!block) {
            const LenInfo* li = (flags & HANKEL_ANTICIRCULANT) ? lengths().find((int)d) : lengths().pick(d);
            if (!li || li->L > maxL) {
                free_plan(p);
                return fail(HANKEL_EUNSUPPORTED, "descriptor %lld: generating length d=%lld exceeds the maximum "
                            "FFT length %lld of this build", (long long)i, (long long)d, (long long)maxL);
            }
            p->Lof.push_back(li->L);
            Ls.push_back(li->L);
            p->sum_L += li->L;
            p->max_L = std::max<int64_t>(p->max_L, li->L);
            p->h_elems = std::max<int64_t>(p->h_elems, D.h_off + d);
            for (int q = 0; q < nx; ++q) p->x_elems = std::max<int64_t>(p->x_elems, D.x_off[q] + D.n[q]);
            p->y_elems = std::max<int64_t>(p->y_elems, D.y_off + D.n[0]);
        }
    }
    bool square = true;
    if (!block)
        for (auto& D : p->descs)
            for (int q = 1; q < D.m; ++q) square = square && D.n[q] == D.n[0];
    p->real_path = !block && !is_complex(dtype) && (flags & HANKEL_SAME_X) && square;
    if (p->real_path) p->shared_io = regions_overlap(p->descs, flags);
    // real tensors with a vector per mode: the fused m + 1 transform kernel
    // when every length fits its three shared buffers
    p->multi_path = !block && !is_complex(dtype) && !(flags & (HANKEL_SAME_X | HANKEL_STORE_SPECTRA)) &&
                    p->max_L <= max_len_for(3, 2 * real_size(dtype));
    hankel_status s = HANKEL_OK;
    if (p->multi_path) {
        s = upload_twiddles(p, Ls);
        if (s == HANKEL_OK) s = build_multi_path(p);
    } else if (p->real_path) {
        // split jobs also need the tables of half their length
        const int max_single_L = max_len_for(2, 2 * real_size(dtype));
        const size_t nL = Ls.size();
        for (size_t i = 0; i < nL; ++i)
            if (Ls[i] > max_single_L) {
                if (split_length(p, Ls[i]) > 0)
                    Ls.push_back(Ls[i] / 2);
                else if (split4_length(p, Ls[i]) > 0)
                    Ls.push_back(Ls[i] / 4);
            }
        s = upload_twiddles(p, Ls);
        if (s == HANKEL_OK) s = build_real_path(p);
    } else {
        // the general path takes level-k descriptors: level 1 (Hankel) or,
        // with HANKEL_BLOCK, level 2 (BHHB: block sizes n, block counts N)
        std::vector<hankel_mdesc> md(p->descs.size());
        for (size_t i = 0; i < p->descs.size(); ++i) md[i] = to_levels(p->descs[i], block);
        s = hk::general_create(&p->gen, md, dtype, flags, &p->h_elems, &p->x_elems, &p->y_elems, &p->sum_L,
                               &p->max_L, g_err);
    }
    if (s != HANKEL_OK) { free_plan(p); return s; }
    *out = p;
    return HANKEL_OK;
}

hankel_status hankel_plan_multilevel(hankel_plan_t* out, const hankel_mdesc* descs, int64_t count, hankel_dtype dtype,
                                     uint32_t flags) {
    if (out == nullptr) return fail(HANKEL_EINVAL, "out is NULL");
    *out = nullptr;
    if (descs == nullptr || count < 1) return fail(HANKEL_EINVAL, "need at least one descriptor");
    if (dtype < HANKEL_R32 || dtype > HANKEL_C128) return fail(HANKEL_EINVAL, "unknown dtype %d", (int)dtype);
    if (flags & ~(uint32_t)(HANKEL_SAME_X | HANKEL_STORE_SPECTRA | HANKEL_ANTICIRCULANT))
        return fail(HANKEL_EINVAL, "flags 0x%x: only HANKEL_SAME_X, HANKEL_STORE_SPECTRA and HANKEL_ANTICIRCULANT apply",
                    flags);
    for (int64_t i = 0; i < count; ++i) {
        const hankel_mdesc& d = descs[i];
        if (d.m < 2 || d.m > HANKEL_MAX_ORDER)
            return fail(HANKEL_EINVAL, "descriptor %lld: order m=%d outside [2, %d]", (long long)i, d.m,
                        HANKEL_MAX_ORDER);
        if (d.levels < 1 || d.levels > HANKEL_MAX_LEVELS)
            return fail(HANKEL_EINVAL, "descriptor %lld: levels=%d outside [1, %d]", (long long)i, d.levels,
                        HANKEL_MAX_LEVELS);
        for (int l = 0; l < d.levels; ++l)
            for (int q = 0; q < d.m; ++q)
                if (d.n[l][q] < 1)
                    return fail(HANKEL_EINVAL, "descriptor %lld: n[%d][%d]=%d must be >= 1", (long long)i, l, q,
                                d.n[l][q]);
        if (d.h_off < 0 || d.y_off < 0) return fail(HANKEL_EINVAL, "descriptor %lld: negative offset", (long long)i);
        const int nx = (flags & HANKEL_SAME_X) ? 1 : d.m;
        for (int q = 0; q < nx; ++q)
            if (d.x_off[q] < 0) return fail(HANKEL_EINVAL, "descriptor %lld: negative x_off[%d]", (long long)i, q);
    }
    auto* p = new (std::nothrow) hankel_plan_s;
    if (!p) return fail(HANKEL_ENOMEM, "host allocation failed");
    p->dtype = dtype;
    p->flags = flags | HANKEL_BLOCK;  // computes through hankel_txv_block
    p->from_descs = false;
    cudaGetDevice(&p->device);
    std::vector<hankel_mdesc> md(descs, descs + count);
    p->descs.resize(count);  // only the count is read back (hankel_plan_query, staging sizes)
    hankel_status s = hk::general_create(&p->gen, md, dtype, flags, &p->h_elems, &p->x_elems, &p->y_elems,
                                         &p->sum_L, &p->max_L, g_err);
    if (s != HANKEL_OK) { free_plan(p); return s; }
    *out = p;
    return HANKEL_OK;
}

hankel_status hankel_txv(hankel_plan_t p, const void* h, const void* x, void* y, void* alpha, hankel_stream_t stream) {
    if (!p) return fail(HANKEL_EINVAL, "plan is NULL");
    if (p->flags & HANKEL_BLOCK) return fail(HANKEL_EINVAL, "plan was made for BHHB tensors: use hankel_txv_block");
    if (!h || !x) return fail(HANKEL_EINVAL, "h and x must be device pointers");
    if (!y && !alpha) return fail(HANKEL_EINVAL, "nothing to compute: y and alpha are both NULL");
    cudaStream_t st = (cudaStream_t)stream;
    const bool dbl = is_double(p->dtype);
    if (p->inner) {
        const cudaError_t e = hk::launch_expand((int)elem_size(p->dtype), p->d_expand, (int)p->expand.size(), p->max_d,
                                                h, p->ws_h, st);
        if (e != cudaSuccess) return cuda_fail(e, "expansion kernel");
        return hankel_txv(p->inner, p->ws_h, x, y, alpha, stream);
    }
    if (p->multi_path)
        return run_forked(p, p->multi_launches, st, [&](const hk::RealLaunch& lc, cudaStream_t s) {
            return hk::launch_real_multi(dbl, lc, p->d_multi, h, x, y, alpha, p->d_tw, s);
        });
    if (!p->real_path) return hk::general_forward(p->gen, h, x, y, alpha, st, g_err);
    auto fwd = [&](const hk::RealLaunch& lc, cudaStream_t s) {
        return hk::launch_real_forward(dbl, lc, p->d_fwd, h, x, y, alpha, p->d_tw, p->d_ws,
                                       (int)(p->flags | (lc.fp64 ? HANKEL_FP64_POWER : 0u)), s);
    };
    if (!p->fast) return run_forked(p, p->fwd_launches, st, fwd);
    auto fast = [&](cudaStream_t s) {
        const char* t2 = (const char*)p->d_fast_tw;
        return hk::launch_fast_forward(p->d_fast_items, (int)p->fast_items.size(), p->fast_grid, p->d_fast_jobs, h, x,
                                       y, alpha, t2, t2 + p->fast_tw3, t2 + p->fast_tw5, p->d_fast_slab,
                                       p->d_fast_ctr, p->fast_f64 ? (int)HANKEL_FP64_POWER : 0, s);
    };
    return run_forked_with(p, p->fwd_launches, st, fwd, fast);
}

hankel_status hankel_txv_host(hankel_plan_t p, const void* h, const void* x, void* y, void* alpha,
                              hankel_stream_t stream) {
    if (!p) return fail(HANKEL_EINVAL, "plan is NULL");
    if (!h || !x) return fail(HANKEL_EINVAL, "h and x must be host pointers");
    if (!y && !alpha) return fail(HANKEL_EINVAL, "nothing to compute: y and alpha are both NULL");
    {
        // page-locked host memory mapped into the device address space: the
        // kernels read the inputs and write the outputs across the host link
        // directly, with no staging copies
        const void* dh = mapped_host(h);
        const void* dx = mapped_host(x);
        void* dy = y ? const_cast<void*>(mapped_host(y)) : nullptr;
        void* da = alpha ? const_cast<void*>(mapped_host(alpha)) : nullptr;
        if (dh && dx && (!y || dy) && (!alpha || da)) {
            const hankel_status s = (p->flags & HANKEL_BLOCK) ? hankel_txv_block(p, dh, dx, dy, da, stream)
                                                              : hankel_txv(p, dh, dx, dy, da, stream);
            if (s != HANKEL_OK) return s;
            const cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
            return e == cudaSuccess ? HANKEL_OK : cuda_fail(e, "stream synchronize");
        }
    }
    const size_t es = elem_size(p->dtype);
    const size_t hb = (size_t)std::max<int64_t>(p->h_elems, 1) * es;
    const size_t xb = (size_t)std::max<int64_t>(p->x_elems, 1) * es;
    const size_t yb = (size_t)std::max<int64_t>(p->y_elems, 1) * es;
    const size_t ab = (size_t)p->descs.size() * es;
    cudaError_t e;
    if (!p->s_h) {
        // all four staging buffers or none (a failed call leaves the plan as it was)
        void* sb[4] = {nullptr, nullptr, nullptr, nullptr};
        const size_t bytes[4] = {hb, xb, yb, ab};
        for (int i = 0; i < 4; ++i) {
            if ((e = cudaMalloc(&sb[i], bytes[i])) != cudaSuccess) {
                for (int j = 0; j < i; ++j) cudaFree(sb[j]);
                return cuda_fail(e, "cudaMalloc(staging)");
            }
        }
        p->s_h = sb[0];
        p->s_x = sb[1];
        p->s_y = sb[2];
        p->s_a = sb[3];
    }
    cudaStream_t st = (cudaStream_t)stream;
    // Large batches run as a pipeline of contiguous descriptor ranges: the
    // copies in of range c + 1 and the copy out of range c - 1 overlap the
    // kernels of range c.
    const bool pipe = p->from_descs && (int64_t)p->descs.size() >= 256 && hb + xb >= (8u << 20);
    if (pipe && !p->chunks_tried) {
        p->chunks_tried = true;
        if (build_chunks(p) != HANKEL_OK) {
            for (auto& c : p->chunks) free_plan(c.plan);
            p->chunks.clear();
        }
    }
    if (pipe && !p->chunks.empty()) {
        // the pipeline runs on the plan's own stream s_cap, ordered after the
        // caller's stream and joined back into it; with the same host buffers
        // as the previous call it is one CUDA graph launch (the host cost of
        // the ~200 calls that enqueue it would otherwise pace the copies)
        const void* key[4] = {h, x, y, alpha};
        const bool replay = p->graph && std::equal(key, key + 4, p->gkey);
        if ((e = cudaEventRecord(p->cap_in, st)) != cudaSuccess) return cuda_fail(e, "cudaEventRecord");
        if ((e = cudaStreamWaitEvent(p->s_cap, p->cap_in, 0)) != cudaSuccess) return cuda_fail(e, "cudaStreamWaitEvent");
        if (replay) {
            if ((e = cudaGraphLaunch(p->graph, p->s_cap)) != cudaSuccess) return cuda_fail(e, "cudaGraphLaunch");
        } else {
            const hankel_status s = enqueue_pipeline(p, h, x, y, alpha, p->s_cap);
            if (s != HANKEL_OK) return s;
        }
        if ((e = cudaEventRecord(p->cap_out, p->s_cap)) != cudaSuccess) return cuda_fail(e, "cudaEventRecord");
        if ((e = cudaStreamWaitEvent(st, p->cap_out, 0)) != cudaSuccess) return cuda_fail(e, "cudaStreamWaitEvent");
        if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_fail(e, "stream synchronize");
        if (!replay) capture_pipeline(p, h, x, y, alpha);
        return HANKEL_OK;
    }
    if ((e = cudaMemcpyAsync(p->s_h, h, hb, cudaMemcpyHostToDevice, st)) != cudaSuccess) return cuda_fail(e, "H2D");
    if ((e = cudaMemcpyAsync(p->s_x, x, xb, cudaMemcpyHostToDevice, st)) != cudaSuccess) return cuda_fail(e, "H2D");
    hankel_status s = (p->flags & HANKEL_BLOCK)
                          ? hankel_txv_block(p, p->s_h, p->s_x, y ? p->s_y : nullptr, alpha ? p->s_a : nullptr, stream)
                          : hankel_txv(p, p->s_h, p->s_x, y ? p->s_y : nullptr, alpha ? p->s_a : nullptr, stream);
    if (s != HANKEL_OK) return s;
    if (y && (e = cudaMemcpyAsync(y, p->s_y, yb, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
        return cuda_fail(e, "D2H");
    if (alpha && (e = cudaMemcpyAsync(alpha, p->s_a, ab, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
        return cuda_fail(e, "D2H");
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_fail(e, "stream synchronize");
    return HANKEL_OK;
}

hankel_status hankel_txv_block(hankel_plan_t p, const void* H, const void* X, void* Y, void* alpha,
                               hankel_stream_t stream) {
    if (!p) return fail(HANKEL_EINVAL, "plan is NULL");
    if (!(p->flags & HANKEL_BLOCK)) return fail(HANKEL_EINVAL, "plan was not made with HANKEL_BLOCK");
    if (!H || !X) return fail(HANKEL_EINVAL, "H and X must be device pointers");
    if (!Y && !alpha) return fail(HANKEL_EINVAL, "nothing to compute: Y and alpha are both NULL");
    return hk::general_forward(p->gen, H, X, Y, alpha, (cudaStream_t)stream, g_err);
}

hankel_status hankel_txv_backward(hankel_plan_t p, const void* grad_y, const void* h, const void* x, void* grad_h,
                                  void* grad_x, hankel_stream_t stream) {
    if (!p) return fail(HANKEL_EINVAL, "plan is NULL");
    if (!grad_y || !h || !x) return fail(HANKEL_EINVAL, "grad_y, h and x must be device pointers");
    if (!grad_h && !grad_x) return fail(HANKEL_EINVAL, "nothing to compute: grad_h and grad_x are both NULL");
    cudaStream_t st = (cudaStream_t)stream;
    if (p->inner) {
        cudaError_t e = hk::launch_expand((int)elem_size(p->dtype), p->d_expand, (int)p->expand.size(), p->max_d, h,
                                          p->ws_h, st);
        if (e != cudaSuccess) return cuda_fail(e, "expansion kernel");
        const hankel_status s =
            hankel_txv_backward(p->inner, grad_y, p->ws_h, x, grad_h ? p->ws_gh : nullptr, grad_x, stream);
        if (s != HANKEL_OK || !grad_h) return s;
        e = hk::launch_fold(is_double(p->dtype), is_complex(p->dtype), fold_entries(p), p->d_folds,
                            (int)p->folds.size(), p->max_n, p->ws_gh, grad_h, st);
        return e == cudaSuccess ? HANKEL_OK : cuda_fail(e, "fold kernel");
    }
    if (p->multi_path || (p->real_path && p->shared_io)) {
        // the adjoint of the distinct-vector products, and of fused plans
        // whose tensors share h or x storage, runs on the general path
        const hankel_status s = ensure_general(p);
        if (s != HANKEL_OK) return s;
        return hk::general_backward(p->gen, grad_y, h, x, grad_h, grad_x, st, g_err);
    }
    if (!p->real_path) return hk::general_backward(p->gen, grad_y, h, x, grad_h, grad_x, st, g_err);
    const bool dbl = is_double(p->dtype);
    const int stored = (p->flags & HANKEL_STORE_SPECTRA) ? 1 : 0;
    auto bwd = [&](const hk::RealLaunch& lc, cudaStream_t s) {
        return hk::launch_real_backward(dbl, lc, p->d_bwd, grad_y, h, x, grad_h, grad_x, p->d_tw, p->d_ws,
                                        (int)(p->flags | (lc.fp64 ? HANKEL_FP64_POWER : 0u)), stored, s);
    };
    if (!p->fast_bwd) return run_forked(p, p->bwd_launches, st, bwd);
    auto fast = [&](cudaStream_t s) {
        const char* t2 = (const char*)p->d_fast_tw;
        return hk::launch_fast_backward(p->d_fast_items, (int)p->fast_items.size(), p->fast_grid, p->d_fast_jobs,
                                        grad_y, h, x, grad_h, grad_x, t2, t2 + p->fast_tw3, t2 + p->fast_tw5,
                                        p->d_fast_slab, p->d_fast_ctr, s);
    };
    return run_forked_with(p, p->bwd_launches, st, bwd, fast);
}

hankel_status hankel_plan_query(hankel_plan_t p, hankel_plan_info* info) {
    if (!p || !info) return fail(HANKEL_EINVAL, "NULL argument");
    std::memset(info, 0, sizeof(*info));
    info->count = (int64_t)p->descs.size();
    info->sum_length = p->sum_L;
    info->max_length = p->max_L;
    info->h_elems = p->h_elems;
    info->x_elems = p->x_elems;
    info->y_elems = p->y_elems;
    if (p->inner) {
        hankel_plan_info in;
        hankel_plan_query(p->inner, &in);
        info->jobs = in.jobs;
        info->launches = in.launches + 1;
        info->distinct_lengths = in.distinct_lengths;
        info->workspace_bytes = in.workspace_bytes;
        info->fp64_power_tensors = in.fp64_power_tensors;
    } else if (p->multi_path) {
        info->jobs = (int64_t)p->multi_jobs.size();
        info->launches = (int64_t)p->multi_launches.size();
        info->distinct_lengths = (int64_t)p->tw_off.size();
        info->workspace_bytes = 0;
    } else if (p->real_path) {
        info->jobs = (int64_t)p->fwd_jobs.size() + p->fast_pairs;
        info->launches = (int64_t)p->fwd_launches.size() + (p->fast ? 1 : 0);
        info->distinct_lengths = (int64_t)p->tw_off.size();
        info->workspace_bytes = (int64_t)p->ws_bytes;
        info->fp64_power_tensors = p->fp64_tensors;
        info->backward_launches = (int64_t)p->bwd_launches.size() + (p->fast_bwd ? 1 : 0);
    } else {
        hk::general_info(p->gen, &info->jobs, &info->launches, &info->distinct_lengths, &info->workspace_bytes);
    }
    if (!p->real_path && !p->inner && (p->flags & HANKEL_FP64_POWER) && !is_double(p->dtype))
        info->fp64_power_tensors = info->count;
    return HANKEL_OK;
}

hankel_status hankel_set_tuning(double pass_cost, int points_per_thread) {
    if (!(pass_cost >= 0.0 && pass_cost <= 1000.0))
        return fail(HANKEL_EINVAL, "pass_cost %g outside [0, 1000]", pass_cost);
    if (points_per_thread != 8 && points_per_thread != 16 && points_per_thread != 32 && points_per_thread != 64)
        return fail(HANKEL_EINVAL, "points_per_thread %d is not 8, 16, 32 or 64", points_per_thread);
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_pass_cost = pass_cost;
    g_points_per_thread = points_per_thread;
    g_lengths.reset();  // rebuilt with the new cost model on next use
    return HANKEL_OK;
}

hankel_status hankel_get_tuning(double* pass_cost, int* points_per_thread) {
    if (!pass_cost || !points_per_thread) return fail(HANKEL_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lk(g_tune_mu);
    *pass_cost = g_pass_cost;
    *points_per_thread = g_points_per_thread;
    return HANKEL_OK;
}

hankel_status hankel_set_bin_policy(int32_t nbins, const int32_t* L, const int32_t* path, const int32_t* fp64_from_m) {
    if (nbins < 0) return fail(HANKEL_EINVAL, "nbins %d is negative", nbins);
    if (nbins > 0 && (!L || !path || !fp64_from_m)) return fail(HANKEL_EINVAL, "NULL argument");
    for (int32_t i = 0; i < nbins; ++i) {
        if (!hk::fast_length_ok(L[i])) return fail(HANKEL_EINVAL, "%d is not a length bin", L[i]);
        if (path[i] != 0 && path[i] != 1) return fail(HANKEL_EINVAL, "path %d of bin %d is not 0 or 1", path[i], L[i]);
        if (fp64_from_m[i] < 2 || fp64_from_m[i] > 99)
            return fail(HANKEL_EINVAL, "fp64_from_m %d of bin %d outside [2, 99]", fp64_from_m[i], L[i]);
    }
    std::lock_guard<std::mutex> lk(g_tune_mu);
    if (nbins == 0) g_bins.clear();
    for (int32_t i = 0; i < nbins; ++i) {
        BinPolicy bp;
        bp.path = path[i];
        bp.fp64_from_m = fp64_from_m[i];
        g_bins[L[i]] = bp;
    }
    return HANKEL_OK;
}

hankel_status hankel_get_bin_policy(int32_t L, int32_t* path, int32_t* fp64_from_m) {
    if (!path || !fp64_from_m) return fail(HANKEL_EINVAL, "NULL argument");
    if (!hk::fast_length_ok(L)) return fail(HANKEL_EINVAL, "%d is not a length bin", L);
    const BinPolicy bp = bin_policy(L);
    *path = bp.path;
    *fp64_from_m = bp.fp64_from_m;
    return HANKEL_OK;
}

int64_t hankel_fft_length(int64_t d) {
    const LenInfo* li = lengths().pick(d);
    return li ? li->L : -1;
}

void hankel_plan_destroy(hankel_plan_t p) {
    if (!p) return;
    cudaDeviceSynchronize();
    free_plan(p);
}

const char* hankel_last_error(void) { return g_err.c_str(); }

const char* hankel_version(void) { return "hankel-gb300 0.1 (sm_103a)"; }

}  // extern "C"
