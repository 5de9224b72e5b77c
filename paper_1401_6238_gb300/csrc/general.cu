// general.cu -- the general path: complex or real data, a different vector
// in every mode, alpha with its own x_1, shared operands, and block tensors
// of any level (Section 2.2: level 1 Hankel, level 2 BHHB, level k a block
// Hankel tensor whose blocks are level-(k-1) tensors).
//
// Everything is expressed on k-dimensional spectral arrays of size
// L_0 x ... x L_{k-1} (column-major: level 0 fastest, stride st_l =
// L_0 ... L_{l-1}).  L_l >= D_l = sum_p n[l][p] - m + 1; a level whose D_l
// is 1 keeps L_l = 1 and is never transformed.
//
// Forward (Section 3; the k-dimensional form its closing remark states):
//   1. every distinct operand gets its spectrum array once:
//        X^_p = fftn(X~_p),   H^ = ifftn(G~) = conj(fftn(conj G~)) / prod L
//      as line transforms along level 0 (over the operand's nonzero lines
//      only), then level 1 (lines whose higher coordinates are inside the
//      operand), and so on;
//   2. per descriptor: Y~ = fftn(H^ .* X^_2 .* ... .* X^_m), transformed along
//      the highest level first keeping only coordinates < n[l][0], down to
//      level 0, whose lines store the crop Y into y;
//   3. alpha = sum over the array of H^ .* X^_1 .* ... .* X^_m.
// Backward (adjoint, not in the paper; G = fftn(grad_y~); (-c) is the
// coordinate-wise negation mod L):
//   grad_G  = ifftn( sum_t G_t .* prod_p conj(X^_{t,p}(-c)) ) cropped to D
//   grad_X  = conj(fftn( sum_{(t,p)} H^_t .* conj(G_t(-c)) .* prod_{q!=p} X^_{t,q} )) cropped
// where the sums run over every descriptor (and mode) that uses the operand,
// so shared operands receive the summed gradient.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cstring>
#include <functional>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "fft_stage.cuh"
#include "general.h"
#include "launch.h"

namespace hk {

namespace {

constexpr int MAXOPS = HANKEL_MAX_ORDER + 1;
constexpr int MAXLV = HANKEL_MAX_LEVELS;

enum { SRC_OPERAND = 0, SRC_PRODUCT = 1 };
enum { BUF_WS = 0, BUF_OUT = 1 };
enum { ROLE_SPECTRUM = 0, ROLE_PRODUCT = 1 };

// One line transform: a block loads a line (of an input operand, or of a
// product of spectral arrays), transforms it and stores a prefix of it.
struct LineTask {
    FftPlan P;
    int32_t src_mode;
    int32_t src_len, src_stride;
    int32_t src_conj;
    int64_t src;  // SRC_OPERAND: element offset in the input buffer
    // SRC_PRODUCT: element i is prod_q ws[ops[q] + loff + i * lstride]
    int32_t nops;
    int64_t loff, lstride;
    int64_t ops[MAXOPS];
    // sink
    int32_t dst_buf, dst_len, dst_stride, dst_conj, dst_real;
    int64_t dst;
    double scale;
    int32_t out_sel;  // BUF_OUT sinks: 0 y, 1 grad_h, 2 grad_x
};

// An operand line reads the h buffer when it is read conjugated (the
// ifft of the generating array), the x buffer otherwise; one launch may hold
// lines of both.
__host__ __device__ inline bool reads_h(const LineTask& t) { return t.src_conj != 0; }

struct AlphaTask {
    int32_t nops, idx;
    int64_t count;
    int64_t ops[MAXOPS];
};

// Elementwise spectral sum of products into one array (backward).
struct Term {
    int32_t nops;
    uint32_t rev_mask;  // operand q read at (-c) and conjugated
    int64_t ops[MAXOPS];
};
struct AccTask {
    int32_t k, t0, t1;
    int32_t L[MAXLV];
    int64_t count, dst;
    int32_t bfirst, nblk;  // blocks of the accumulate launch given to this task (by its work)
};

struct Launch {
    int kind;  // 0 line, 1 alpha, 2 accumulate
    int first, count, L;
    int role;  // ROLE_SPECTRUM: spectra, always run; ROLE_PRODUCT: only when y is wanted
    int what;  // buffers of a run: 0 workspace source, 1 operands (h and x), 3 gradient sinks
};

template <typename T>
struct OperandLoad {
    const void* base;
    int len, stride, conj, real;
    __device__ __forceinline__ cx<T> operator()(int i) const {
        if (i >= len) return mk<T>(T(0), T(0));
        cx<T> v;
        if (real) {
            v = mk<T>(reinterpret_cast<const T*>(base)[(int64_t)i * stride], T(0));
        } else {
            v = reinterpret_cast<const cx<T>*>(base)[(int64_t)i * stride];
        }
        return conj ? conjg(v) : v;
    }
};

template <typename T>
struct ProductLoad {
    const cx<T>* ws;
    const int64_t* ops;  // shared-memory copy of the task's array offsets
    int nops, len, conj;
    int64_t loff, lstride;
    __device__ __forceinline__ cx<T> operator()(int i) const {
        if (i >= len) return mk<T>(T(0), T(0));
        const int64_t e = loff + (int64_t)i * lstride;
        cx<T> v = ws[ops[0] + e];
        for (int q = 1; q < nops; ++q) v = cmul(v, ws[ops[q] + e]);
        return conj ? conjg(v) : v;
    }
};

template <typename T>
struct LineSink {
    void* base;
    int len, stride, conj, real;
    T scale;
    __device__ __forceinline__ void operator()(int i, cx<T> v) const {
        if (i >= len) return;
        if (conj) v = conjg(v);
        v = scal(v, scale);
        if (real)
            reinterpret_cast<T*>(base)[(int64_t)i * stride] = v.x;
        else
            reinterpret_cast<cx<T>*>(base)[(int64_t)i * stride] = v;
    }
};

// shared-memory slots of the twiddle table (lengths up to 16384)
constexpr int TWG_SMEM = tw_table_elems(16384);

// The caller's buffers a launch of lines may touch: operand lines read h or
// x (reads_h), output sinks write y, grad_h or grad_x (out_sel 0, 1, 2); a
// null sink is a result the caller did not ask for, whose lines store nothing.
struct LineBufs {
    const void* in_h;
    const void* in_x;
    void* y;
    void* grad_h;
    void* grad_x;
};

// Loader of an operand line (bit 1 of dst_real flags a real input operand).
template <typename T>
__device__ __forceinline__ OperandLoad<T> operand_load(const LineTask& t, const LineBufs& b) {
    const bool real = t.dst_real & 2;
    const void* in = reads_h(t) ? b.in_h : b.in_x;
    return OperandLoad<T>{(const char*)in + t.src * (real ? sizeof(T) : sizeof(cx<T>)), t.src_len, t.src_stride,
                          t.src_conj, real ? 1 : 0};
}

// Sink of a line: plan workspace, or the caller's buffer that out_sel names
// (bit 0 of dst_real: real output); a null buffer stores nothing.
template <typename T>
__device__ __forceinline__ LineSink<T> line_sink(const LineTask& t, const LineBufs& b, cx<T>* ws) {
    const int real = t.dst_real & 1;
    if (t.dst_buf == BUF_WS) return LineSink<T>{ws + t.dst, t.dst_len, t.dst_stride, t.dst_conj, real, (T)t.scale};
    void* out = (t.out_sel == 0) ? b.y : (t.out_sel == 1) ? b.grad_h : b.grad_x;
    if (out == nullptr) return LineSink<T>{nullptr, 0, t.dst_stride, t.dst_conj, real, (T)t.scale};
    return LineSink<T>{(char*)out + t.dst * (real ? sizeof(T) : sizeof(cx<T>)), t.dst_len, t.dst_stride, t.dst_conj,
                       real, (T)t.scale};
}

// One line per block: the line's input (an operand line, or a product of
// spectral arrays) is staged in shared memory, transformed by the stage
// transform (fft_stage.cuh) and its prefix stored through the sink.  All
// reads of the line finish before the first store, so a sink may overwrite
// the line the source read.
template <typename T>
__global__ void __launch_bounds__(512) line_kernel(const LineTask* __restrict__ tasks, int first, LineBufs io,
                                                   cx<T>* ws, const cx<T>* __restrict__ tw_all, int Lmax) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int64_t ops_s[MAXOPS];
    cx<T>* tws = reinterpret_cast<cx<T>*>(smem_raw + RED_BYTES);
    cx<T>* b0 = tws + TWG_SMEM;
    cx<T>* b1 = b0 + smem_elems(Lmax);
    const LineTask& t = tasks[first + blockIdx.x];
    const Group g{(int)threadIdx.x, (int)blockDim.x, 0};
    const FftPlan P = t.P;
    const TwTab<T> tw = load_twiddles(tws, tw_all + P.tw_off, P.L, g);
    if (g.tid < MAXOPS) ops_s[g.tid] = t.ops[g.tid];
    g.sync();
    if (t.src_mode == SRC_OPERAND) {
        const OperandLoad<T> ld = operand_load<T>(t, io);
        for (int i = g.tid; i < P.L; i += g.nthr) b0[sp(i)] = ld(i);
    } else {
        const ProductLoad<T> ld{ws, ops_s, t.nops, t.src_len, t.src_conj, t.loff, t.lstride};
        for (int i = g.tid; i < P.L; i += g.nthr) b0[sp(i)] = ld(i);
    }
    g.sync();
    fft_stage<T>(P, GLd<T>{nullptr, 0, nullptr, 0}, b0, b1, b0, line_sink<T>(t, io, ws), false, tw, g);
}

// Short lines, several per warp (lines of one launch share their length L):
// a group of `gth` < 32 lanes transforms one line, synchronising with the
// other groups of its warp (__syncwarp over the lanes that hold a line: the
// groups of a warp run the same pass sequence), so a warp keeps 32 / gth
// lines in flight instead of one line with mostly idle lanes.  The block
// loads the twiddle table once.  Built for three resident blocks per SM.
template <typename T>
__global__ void __launch_bounds__(256, 3) line_group_kernel(const LineTask* __restrict__ tasks, int first, int count,
                                                         int lpb, int gth, LineBufs io, cx<T>* ws,
                                                         const cx<T>* __restrict__ tw_all, int L) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cx<T>* tws = reinterpret_cast<cx<T>*>(smem_raw + RED_BYTES);
    cx<T>* bufs = tws + TWG_SMEM;
    const int E = smem_elems(L);
    int64_t* ops_all = reinterpret_cast<int64_t*>(bufs + (size_t)2 * lpb * E);
    const int tid = threadIdx.x;
    const int base = first + blockIdx.x * lpb;
    const int nl = min(lpb, first + count - base);
    const TwTab<T> tw = load_twiddles(tws, tw_all + tasks[base].P.tw_off, L, Group{tid, (int)blockDim.x, 0});
    for (int w = tid; w < nl * MAXOPS; w += blockDim.x) ops_all[w] = tasks[base + w / MAXOPS].ops[w % MAXOPS];
    __syncthreads();
    const int j = tid / gth;
    if (j >= nl) return;
    // lanes of this warp that hold a line
    const int lane = tid & 31, warp_first_line = (tid - lane) / gth;
    const int lines_here = min(32 / gth, nl - warp_first_line);
    const unsigned mask = (lines_here * gth >= 32) ? 0xffffffffu : ((1u << (lines_here * gth)) - 1u);
    Group g{tid - j * gth, gth, -1};
    g.mask = mask;
    const LineTask& t = tasks[base + j];
    cx<T>* b0 = bufs + (2 * j) * E;
    cx<T>* b1 = b0 + E;
    if (t.src_mode == SRC_OPERAND) {
        const OperandLoad<T> ld = operand_load<T>(t, io);
        for (int i = g.tid; i < L; i += g.nthr) b0[sp(i)] = ld(i);
    } else {
        const ProductLoad<T> ld{ws, ops_all + j * MAXOPS, t.nops, t.src_len, t.src_conj, t.loff, t.lstride};
        for (int i = g.tid; i < L; i += g.nthr) b0[sp(i)] = ld(i);
    }
    g.sync();
    fft_stage<T>(t.P, GLd<T>{nullptr, 0, nullptr, 0}, b0, b1, b0, line_sink<T>(t, io, ws), false, tw, g);
}

template <typename T>
__global__ void __launch_bounds__(256) alpha_kernel(const AlphaTask* __restrict__ tasks, int first,
                                                    const cx<T>* __restrict__ ws, void* alpha, int real) {
    __shared__ double red[64];
    const AlphaTask& t = tasks[first + blockIdx.x];
    const Group g{(int)threadIdx.x, (int)blockDim.x, 0};
    // products in T precision, their sum in FP64 (FP64 arithmetic is slow on
    // this part: one conversion and one FP64 add per element and component)
    double sr = 0.0, si = 0.0;
    for (int64_t e = g.tid; e < t.count; e += g.nthr) {
        cx<T> v = ws[t.ops[0] + e];
        for (int q = 1; q < t.nops; ++q) v = cmul(v, ws[t.ops[q] + e]);
        sr += (double)v.x;
        si += (double)v.y;
    }
    sr = group_sum(sr, red, g);
    si = group_sum(si, red, g);
    if (g.tid == 0) {
        if (real)
            reinterpret_cast<T*>(alpha)[t.idx] = (T)sr;
        else
            reinterpret_cast<cx<T>*>(alpha)[t.idx] = mk<T>((T)sr, (T)si);
    }
}

template <typename T>
__global__ void __launch_bounds__(256) accumulate_kernel(const AccTask* __restrict__ tasks, int first, int ntasks,
                                                         const Term* __restrict__ terms, cx<T>* ws) {
    // the task owning this block: the last one whose first block is <= blockIdx.x
    int lo = first, hi = first + ntasks - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (tasks[mid].bfirst <= (int)blockIdx.x)
            lo = mid;
        else
            hi = mid - 1;
    }
    const AccTask& t = tasks[lo];
    const int n = (int)t.count;  // arrays hold fewer than 2^31 elements (checked at plan time)
    const int b = (int)blockIdx.x - t.bfirst;
    for (int e = b * blockDim.x + threadIdx.x; e < n; e += t.nblk * blockDim.x) {
        // offset of the coordinate-wise negation (-c) mod L
        int re = 0, rest = e, st = 1;
        for (int l = 0; l < t.k; ++l) {
            const int L = t.L[l];
            const int q = rest / L, c = rest - q * L;
            rest = q;
            re += (c == 0 ? 0 : L - c) * st;
            st *= L;
        }
        cx<T> acc = mk<T>(T(0), T(0));
        for (int j = t.t0; j < t.t1; ++j) {
            const Term& tm = terms[j];
            cx<T> v = mk<T>(T(1), T(0));
            for (int q = 0; q < tm.nops; ++q) {
                const cx<T> w = (tm.rev_mask & (1u << q)) ? conjg(ws[tm.ops[q] + re]) : ws[tm.ops[q] + e];
                v = (q == 0) ? w : cmul(v, w);
            }
            acc = acc + v;
        }
        ws[t.dst + e] = acc;
    }
}

// Geometry of one spectral array: per-level lengths and strides.
struct Geo {
    int k = 1;
    int L[MAXLV] = {1, 1, 1, 1};
    int64_t st[MAXLV] = {1, 1, 1, 1};
    int64_t total = 1;
    void finish() {
        total = 1;
        for (int l = 0; l < k; ++l) {
            st[l] = total;
            total *= L[l];
        }
    }
    int top() const {  // highest transformed level (level 0 always is)
        int t = 0;
        for (int l = 0; l < k; ++l)
            if (L[l] > 1) t = l;
        return t;
    }
};

// Column-major strides of an array with extents ext[0..k).
void cm_strides(int k, const int* ext, int64_t* st) {
    int64_t s = 1;
    for (int l = 0; l < k; ++l) {
        st[l] = s;
        s *= ext[l];
    }
}

// Visit every line along level `l` of a k-dimensional array whose other
// coordinates run over [0, ext[j]); the callback gets the coordinates.
void for_lines(int k, int l, const int* ext, const std::function<void(const int*)>& fn) {
    int c[MAXLV] = {0, 0, 0, 0};
    for (int j = 0; j < k; ++j)
        if (j != l && ext[j] <= 0) return;
    while (true) {
        fn(c);
        int j = 0;
        for (; j < k; ++j) {
            if (j == l) continue;
            if (++c[j] < ext[j]) break;
            c[j] = 0;
        }
        if (j == k) return;
    }
}

int64_t dot(int k, const int* c, const int64_t* st, int skip) {
    int64_t o = 0;
    for (int j = 0; j < k; ++j)
        if (j != skip) o += (int64_t)c[j] * st[j];
    return o;
}

}  // namespace

// ------------------------------------------------------------------- plan

struct GeneralPlan {
    hankel_dtype dtype;
    uint32_t flags;
    bool dbl, cplx;
    std::vector<hankel_mdesc> descs;
    struct Op {
        bool is_h;
        int64_t off;
        int rows[MAXLV];  // extents of the operand along each level
        Geo geo;
        int64_t plane;
    };
    std::vector<Op> ops;
    struct D {
        int m;
        Geo geo;
        int n1[MAXLV];  // output extents
        int hop, xop[HANKEL_MAX_ORDER];  // operand index of h and x_1..x_m
        int64_t temp, gplane;
    };
    std::vector<D> ds;
    std::map<int, int> tw_off;
    int64_t tw_elems = 0, ws_elems = 0;
    void* d_tw = nullptr;
    void* d_ws = nullptr;
    size_t ws_bytes = 0;
    std::vector<LineTask> fwd_lines, bwd_lines;
    std::vector<AlphaTask> alphas;
    std::vector<Term> terms;
    std::vector<AccTask> accs;
    int acc_blocks = 0;
    std::vector<Launch> fwd_prog, bwd_prog_spec, bwd_prog_rest;
    LineTask *d_fwd = nullptr, *d_bwd = nullptr;
    AlphaTask* d_alpha = nullptr;
    Term* d_terms = nullptr;
    AccTask* d_accs = nullptr;
};

namespace {

size_t csize(const GeneralPlan* g) { return (g->dbl ? 8 : 4) * 2; }

FftPlan plan_for(GeneralPlan* g, int L) {
    FftPlan P;
    std::memset(&P, 0, sizeof(P));
    fft_factor(L, &P);  // the planner's pass sequence for this length
    P.tw_off = g->tw_off.at(L);
    return P;
}

LineTask blank_task() {
    LineTask t;
    std::memset(&t, 0, sizeof(t));
    t.scale = 1.0;
    t.src_stride = 1;
    t.dst_stride = 1;
    return t;
}

// Per-level launches of a multi-phase emission: phases[l] holds the launches
// of phase l (one per transform length).
using Phases = std::vector<std::vector<Launch>>;

void add_launch(Phases& ph, int phase, int first, int count, int L, int role) {
    if (count == 0) return;
    if ((int)ph.size() <= phase) ph.resize(phase + 1);
    ph[phase].push_back({0, first, count, L, role, 0});
}

// Spectrum array of an operand whose data (extents rows[], column-major) is
// at `src` in the input buffer: level-0 lines read the input (zero-padded),
// every higher transformed level works in place on the array.  For the
// generating tensor (is_h) the result is ifftn = conj(fftn(conj .)) / total.
void emit_spectrum(GeneralPlan* g, bool is_h, int64_t src, const int* rows, const Geo& geo, int64_t plane,
                   std::vector<LineTask>& lines, Phases& ph) {
    const int top = geo.top();
    const double sc = is_h ? 1.0 / (double)geo.total : 1.0;
    int64_t rs[MAXLV];
    cm_strides(geo.k, rows, rs);
    for (int l = 0; l < geo.k; ++l) {
        if (geo.L[l] == 1) continue;
        int ext[MAXLV];
        for (int j = 0; j < geo.k; ++j) ext[j] = j < l ? geo.L[j] : rows[j];
        const int first = (int)lines.size();
        for_lines(geo.k, l, ext, [&](const int* c) {
            LineTask t = blank_task();
            t.P = plan_for(g, geo.L[l]);
            if (l == 0) {
                t.src_mode = SRC_OPERAND;
                t.src = src + dot(geo.k, c, rs, 0);
                t.src_conj = is_h;
                t.dst_real = g->cplx ? 0 : 2;  // input real flag in bit 1
            } else {
                t.src_mode = SRC_PRODUCT;
                t.nops = 1;
                t.ops[0] = plane;
                t.loff = dot(geo.k, c, geo.st, l);
                t.lstride = geo.st[l];
            }
            t.src_len = rows[l];
            t.dst_buf = BUF_WS;
            t.dst = plane + dot(geo.k, c, geo.st, l);
            t.dst_stride = (int)geo.st[l];
            t.dst_len = geo.L[l];
            if (l == top) {
                t.dst_conj = is_h;
                t.scale = sc;
            }
            lines.push_back(t);
        });
        add_launch(ph, l, first, (int)lines.size() - first, geo.L[l], ROLE_SPECTRUM);
    }
}

// Inverse-direction transform of a spectral array (the product of `planes`,
// or an array already in `temp`), highest transformed level first, cropped
// to extents out[] and finally stored along level 0 to the destination
// (column-major with extents out[]).  Intermediate levels write into `temp`
// (a full-size array; it may be the source array itself).
void emit_crop_transform(GeneralPlan* g, const Geo& geo, const std::vector<int64_t>& planes, bool conj_in,
                         const int* out, int64_t temp, int dst_buf, int64_t dst, bool conj_out, double scale,
                         bool real_out, int out_sel, std::vector<LineTask>& lines, Phases& ph, int role) {
    int64_t os[MAXLV];
    cm_strides(geo.k, out, os);
    std::vector<int> act;
    for (int l = geo.k - 1; l >= 0; --l)
        if (geo.L[l] > 1 || l == 0) act.push_back(l);
    for (size_t s = 0; s < act.size(); ++s) {
        const int l = act[s];
        const bool first_stage = (s == 0);
        int ext[MAXLV];
        for (int j = 0; j < geo.k; ++j) ext[j] = j < l ? geo.L[j] : out[j];
        const int first = (int)lines.size();
        for_lines(geo.k, l, ext, [&](const int* c) {
            LineTask t = blank_task();
            t.P = plan_for(g, geo.L[l]);
            t.src_mode = SRC_PRODUCT;
            if (first_stage) {
                t.nops = (int)planes.size();
                for (int q = 0; q < t.nops; ++q) t.ops[q] = planes[q];
                t.src_conj = conj_in;
            } else {
                t.nops = 1;
                t.ops[0] = temp;
            }
            t.loff = dot(geo.k, c, geo.st, l);
            t.lstride = geo.st[l];
            t.src_len = geo.L[l];
            if (l == 0) {
                t.dst_buf = dst_buf;
                t.dst = dst + dot(geo.k, c, os, 0);
                t.dst_len = out[0];
                t.dst_conj = conj_out;
                t.scale = scale;
                t.dst_real = real_out ? 1 : 0;
                t.out_sel = out_sel;
            } else {
                t.dst_buf = BUF_WS;
                t.dst = temp + t.loff;
                t.dst_stride = (int)geo.st[l];
                t.dst_len = out[l];
            }
            lines.push_back(t);
        });
        add_launch(ph, (int)s, first, (int)lines.size() - first, geo.L[l], role);
    }
}

// Threads per block of a one-line launch of length L.
int nthr_for(int L) {
    int p = 1;
    while (p < (L + 15) / 16) p <<= 1;
    return std::max(32, std::min(512, p));
}

// Buffers a line task reads and writes: 0 workspace source, 1 an operand
// buffer (h or x), 3 a gradient sink (grad_h or grad_x).  The kernels take
// every buffer and each line picks its own (LineBufs), so these classes only
// order the launches of a phase.
int task_class(const LineTask& t) {
    if (t.dst_buf == BUF_OUT && t.out_sel != 0) return 3;
    if (t.src_mode == SRC_OPERAND) return 1;
    return 0;
}

// Lines that may share a launch: one length each up to 256 (several lines
// per warp need one pass sequence), above that every length with the same
// block size (one line per block, shared memory sized for the longest).
int len_bucket(int L) { return L <= 256 ? L : (1 << 20) + nthr_for(L); }

// Flatten phases into one program; `cuts` receives the phase boundaries.
// Inside a phase (independent tasks) launches are ordered by the buffers
// they use and by length bucket, so that merge() can join them.
void flatten(const Phases& ph, std::vector<Launch>& prog, std::vector<int>& cuts, const std::vector<LineTask>& lines) {
    for (auto p : ph) {
        std::stable_sort(p.begin(), p.end(), [&](const Launch& a, const Launch& b) {
            const int ca = a.kind == 0 ? task_class(lines[a.first]) : -1;
            const int cb = b.kind == 0 ? task_class(lines[b.first]) : -1;
            if (ca != cb) return ca < cb;
            if (len_bucket(a.L) != len_bucket(b.L)) return len_bucket(a.L) < len_bucket(b.L);
            return a.L > b.L;
        });
        prog.insert(prog.end(), p.begin(), p.end());
        cuts.push_back((int)prog.size());
    }
}

// Group consecutive launches of the same kind, length bucket and role
// (independent tasks of one phase) to cut launch counts; a merged launch
// carries the longest length.
std::vector<Launch> merge(const std::vector<Launch>& in, const std::vector<int>& barriers) {
    std::vector<Launch> out;
    size_t bi = 0;
    for (size_t i = 0; i < in.size(); ++i) {
        bool cut = false;
        while (bi < barriers.size() && barriers[bi] <= (int)i) {
            if (barriers[bi] == (int)i) cut = true;
            ++bi;
        }
        if (!out.empty() && !cut && out.back().kind == in[i].kind && len_bucket(out.back().L) == len_bucket(in[i].L) &&
            out.back().role == in[i].role && out.back().first + out.back().count == in[i].first) {
            out.back().count += in[i].count;
            out.back().L = std::max(out.back().L, in[i].L);
        } else {
            out.push_back(in[i]);
        }
    }
    return out;
}

// Reorder the task table so that the tasks of consecutive launches of every
// program are contiguous (launches of one phase can then be merged).
void compact(std::vector<LineTask>& lines, std::vector<std::vector<Launch>*> progs) {
    std::vector<LineTask> out;
    out.reserve(lines.size());
    for (auto* prog : progs)
        for (auto& l : *prog) {
            if (l.kind != 0) continue;
            const int nf = (int)out.size();
            out.insert(out.end(), lines.begin() + l.first, lines.begin() + l.first + l.count);
            l.first = nf;
        }
    lines.swap(out);
}

// Split every line launch into runs of tasks that read the same input
// buffer and write the same output buffer (done once, at plan time).
std::vector<Launch> split_runs(const std::vector<Launch>& prog, const std::vector<LineTask>& lines) {
    const auto cls = task_class;
    std::vector<Launch> out;
    for (const Launch& l : prog) {
        if (l.kind != 0) {
            out.push_back(l);
            out.back().what = 0;
            continue;
        }
        int i = l.first;
        while (i < l.first + l.count) {
            const int what = cls(lines[i]);
            int j = i + 1;
            while (j < l.first + l.count && cls(lines[j]) == what) ++j;
            out.push_back({0, i, j - i, l.L, l.role, what});
            i = j;
        }
    }
    return out;
}

hankel_status cuerr(cudaError_t e, const char* what, std::string& err) {
    err = std::string(what) + ": " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? HANKEL_ENOMEM : HANKEL_ECUDA;
}

template <typename V>
hankel_status upload(const std::vector<V>& v, V** d, std::string& err) {
    cudaError_t e = cudaMalloc((void**)d, std::max<size_t>(v.size(), 1) * sizeof(V));
    if (e != cudaSuccess) return cuerr(e, "cudaMalloc(tasks)", err);
    if (!v.empty()) {
        e = cudaMemcpy(*d, v.data(), v.size() * sizeof(V), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return cuerr(e, "cudaMemcpy(tasks)", err);
    }
    return HANKEL_OK;
}

size_t line_smem(const GeneralPlan* g, int L) {
    return RED_BYTES + ((size_t)TWG_SMEM + 2 * smem_elems_host(L)) * csize(g);
}

// Lanes per line of the grouped kernel for length L: about one radix-16
// butterfly per lane, at least 4; 32 or more means one line per block.
int group_lanes(int L) {
    int p = 4;
    while (p < 32 && p * 16 < L) p <<= 1;
    return p;
}

size_t group_smem(const GeneralPlan* g, int L, int lpb) {
    return RED_BYTES + ((size_t)TWG_SMEM + (size_t)lpb * 2 * smem_elems_host(L)) * csize(g) +
           (size_t)lpb * MAXOPS * sizeof(int64_t);
}

// Raise a kernel's dynamic shared-memory limit only when a launch needs more
// than was granted (no attribute calls in steady state, so the launches can
// be captured into CUDA graphs); grants are kept per device and kernel,
// under a lock (plans may run on several host threads).
cudaError_t grant_smem(const void* fn, size_t bytes) {
    static std::mutex mu;
    static std::map<std::pair<int, const void*>, size_t> granted;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lk(mu);
    size_t& have = granted[std::make_pair(dev, fn)];
    if (bytes <= have) return cudaSuccess;
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess) have = bytes;
    return e;
}

template <typename T>
cudaError_t run_lines(GeneralPlan* g, const Launch& l, const LineTask* d_tasks, const LineBufs& io,
                      cudaStream_t st) {
    const int gth = group_lanes(l.L);
    if (gth < 32) {
        // whole warps of lines, as many as let three blocks share an SM's
        // shared memory (the kernel is built for three resident blocks)
        const int per_warp = 32 / gth;
        int lpb = 256 / gth;
        while (lpb > per_warp && 3 * group_smem(g, l.L, lpb) > 227 * 1024) lpb -= per_warp;
        const size_t smem = group_smem(g, l.L, lpb);
        cudaError_t e = grant_smem(reinterpret_cast<const void*>(line_group_kernel<T>), smem);
        if (e != cudaSuccess) return e;
        const int blocks = (l.count + lpb - 1) / lpb;
        line_group_kernel<T><<<blocks, lpb * gth, smem, st>>>(d_tasks, l.first, l.count, lpb, gth, io,
                                                              (cx<T>*)g->d_ws, (const cx<T>*)g->d_tw, l.L);
        return cudaGetLastError();
    }
    const size_t smem = line_smem(g, l.L);
    cudaError_t e = grant_smem(reinterpret_cast<const void*>(line_kernel<T>), smem);
    if (e != cudaSuccess) return e;
    line_kernel<T><<<l.count, nthr_for(l.L), smem, st>>>(d_tasks, l.first, io, (cx<T>*)g->d_ws,
                                                       (const cx<T>*)g->d_tw, l.L);
    return cudaGetLastError();
}

}  // namespace

namespace {

// Host half of plan creation: operands, array offsets, twiddle offsets and
// the launch programs.  Touches no device (the task tables can be built and
// inspected without a GPU).
hankel_status build_programs(GeneralPlan* g, const std::vector<hankel_mdesc>& descs, int64_t* h_elems,
                             int64_t* x_elems, int64_t* y_elems, int64_t* sum_L, int64_t* max_L, std::string& err) {
    const bool same_x = (g->flags & HANKEL_SAME_X) != 0;
    const size_t cs = csize(g);
    int maxL = 2;
    while (maxL < 16384 && RED_BYTES + ((size_t)TWG_SMEM + 2 * smem_elems_host(maxL + 1)) * cs <= 227 * 1024) ++maxL;
    std::map<std::vector<int64_t>, int> opidx;
    int64_t cursor = 0;
    auto add_op = [&](bool is_h, int64_t off, const int* rows, const Geo& geo) {
        std::vector<int64_t> key{(int64_t)is_h, off, geo.k};
        for (int l = 0; l < geo.k; ++l) {
            key.push_back(rows[l]);
            key.push_back(geo.L[l]);
        }
        auto it = opidx.find(key);
        if (it != opidx.end()) return it->second;
        GeneralPlan::Op op;
        op.is_h = is_h;
        op.off = off;
        for (int l = 0; l < MAXLV; ++l) op.rows[l] = l < geo.k ? rows[l] : 1;
        op.geo = geo;
        op.plane = cursor;
        cursor += geo.total;
        g->ops.push_back(op);
        opidx[key] = (int)g->ops.size() - 1;
        return (int)g->ops.size() - 1;
    };
    *h_elems = *x_elems = *y_elems = 0;
    *sum_L = *max_L = 0;
    for (size_t i = 0; i < descs.size(); ++i) {
        const hankel_mdesc& d = descs[i];
        GeneralPlan::D D{};
        D.m = d.m;
        D.geo.k = d.levels;
        int gs[MAXLV];
        const bool anti = (g->flags & HANKEL_ANTICIRCULANT) != 0;
        for (int l = 0; l < d.levels; ++l) {
            int64_t s = 0;
            for (int p = 0; p < d.m; ++p) s += d.n[l][p];
            if (anti) {
                // compressed generating data: n entries per level, transformed at length exactly n
                for (int p = 1; p < d.m; ++p)
                    if (d.n[l][p] != d.n[l][0]) {
                        err = "descriptor " + std::to_string(i) + ": anti-circulant tensors are square";
                        return HANKEL_EINVAL;
                    }
                if (l == 0 && d.n[0][0] < 2) {
                    err = "descriptor " + std::to_string(i) + ": anti-circulant dimension must be >= 2";
                    return HANKEL_EINVAL;
                }
                gs[l] = d.n[l][0];
            } else {
                gs[l] = (int)(s - d.m + 1);
            }
            // level 0 is always transformed (length >= 2); a level with D_l = 1 is not
            const int64_t L = (l > 0 && gs[l] == 1) ? 1 : (anti ? (int64_t)gs[l] : hankel_fft_length(gs[l]));
            FftPlan probe;
            if (L < 0 || L > maxL || (L > 1 && !fft_factor((int)L, &probe))) {
                err = "descriptor " + std::to_string(i) +
                      (anti ? ": anti-circulant dimension " + std::to_string(gs[l]) +
                                  " is not an FFT length of this build (2,3,5,7-smooth, within the maximum)"
                            : std::string(": FFT length beyond the supported maximum of this build"));
                return HANKEL_EUNSUPPORTED;
            }
            D.geo.L[l] = (int)L;
            D.n1[l] = d.n[l][0];
            if (L > 1) g->tw_off[(int)L] = 0;
            *max_L = std::max<int64_t>(*max_L, L);
        }
        D.geo.finish();
        if (D.geo.total > INT32_MAX) {
            err = "descriptor " + std::to_string(i) + ": padded array of " + std::to_string(D.geo.total) +
                  " elements exceeds this build's 2^31 limit";
            return HANKEL_EUNSUPPORTED;
        }
        D.hop = add_op(true, d.h_off, gs, D.geo);
        int64_t hsz = 1, ysz = 1;
        for (int l = 0; l < d.levels; ++l) {
            hsz *= gs[l];
            ysz *= D.n1[l];
        }
        for (int p = 0; p < d.m; ++p) {
            const int q = same_x ? 0 : p;
            const int64_t xo = d.x_off[q];
            int rows[MAXLV];
            int64_t xsz = 1;
            for (int l = 0; l < d.levels; ++l) {
                rows[l] = d.n[l][q];
                xsz *= rows[l];
            }
            D.xop[p] = add_op(false, xo, rows, D.geo);
            *x_elems = std::max<int64_t>(*x_elems, xo + xsz);
        }
        *h_elems = std::max<int64_t>(*h_elems, d.h_off + hsz);
        *y_elems = std::max<int64_t>(*y_elems, d.y_off + ysz);
        *sum_L += D.geo.total;
        g->ds.push_back(D);
    }
    // temp arrays (forward, more than one transformed level), G arrays and
    // S arrays (backward)
    for (auto& D : g->ds) {
        D.temp = cursor;
        if (D.geo.top() > 0) cursor += D.geo.total;
        D.gplane = cursor;
        cursor += D.geo.total;
    }
    std::vector<int64_t> splane(g->ops.size());
    for (size_t o = 0; o < g->ops.size(); ++o) {
        splane[o] = cursor;
        cursor += g->ops[o].geo.total;
    }
    // twiddle table offsets (the tables are generated on the device later)
    int64_t tw_total = 0;
    for (auto& kv : g->tw_off) {
        kv.second = (int)tw_total;
        tw_total += tw_table_elems(kv.first);
    }
    g->tw_elems = tw_total;
    g->ws_elems = cursor;

    // ---- forward program: operand spectra by level, then product stages
    {
        Phases spec, prod;
        for (const auto& op : g->ops) emit_spectrum(g, op.is_h, op.off, op.rows, op.geo, op.plane, g->fwd_lines, spec);
        for (size_t i = 0; i < g->ds.size(); ++i) {
            const auto& D = g->ds[i];
            std::vector<int64_t> planes{g->ops[D.hop].plane};
            for (int p = 1; p < D.m; ++p) planes.push_back(g->ops[D.xop[p]].plane);
            emit_crop_transform(g, D.geo, planes, false, D.n1, D.temp, BUF_OUT, descs[i].y_off, false, 1.0, !g->cplx, 0,
                                g->fwd_lines, prod, ROLE_PRODUCT);
        }
        std::vector<Launch> prog;
        std::vector<int> cuts;
        flatten(spec, prog, cuts, g->fwd_lines);
        flatten(prod, prog, cuts, g->fwd_lines);
        compact(g->fwd_lines, {&prog});
        g->fwd_prog = split_runs(merge(prog, cuts), g->fwd_lines);
    }
    for (size_t i = 0; i < g->ds.size(); ++i) {
        const auto& D = g->ds[i];
        AlphaTask a;
        std::memset(&a, 0, sizeof(a));
        a.nops = D.m + 1;
        a.ops[0] = g->ops[D.hop].plane;
        for (int p = 0; p < D.m; ++p) a.ops[1 + p] = g->ops[D.xop[p]].plane;
        a.count = D.geo.total;
        a.idx = (int)i;
        g->alphas.push_back(a);
    }

    // ---- backward program: spectra, G arrays, spectral sums, gradients
    {
        Phases bspec, gspec, tails;
        for (const auto& op : g->ops)
            emit_spectrum(g, op.is_h, op.off, op.rows, op.geo, op.plane, g->bwd_lines, bspec);
        for (size_t i = 0; i < g->ds.size(); ++i) {
            const auto& D = g->ds[i];
            emit_spectrum(g, false, descs[i].y_off, D.n1, D.geo, D.gplane, g->bwd_lines, gspec);
        }
        std::vector<std::vector<Term>> hterms(g->ops.size()), xterms(g->ops.size());
        for (const auto& D : g->ds) {
            Term th;
            std::memset(&th, 0, sizeof(th));
            th.ops[th.nops++] = D.gplane;
            for (int p = 1; p < D.m; ++p) {
                th.rev_mask |= 1u << th.nops;
                th.ops[th.nops++] = g->ops[D.xop[p]].plane;
            }
            hterms[D.hop].push_back(th);
            for (int p = 1; p < D.m; ++p) {
                Term tx;
                std::memset(&tx, 0, sizeof(tx));
                tx.ops[tx.nops++] = g->ops[D.hop].plane;
                tx.rev_mask |= 1u << tx.nops;
                tx.ops[tx.nops++] = D.gplane;
                for (int q = 1; q < D.m; ++q)
                    if (q != p) tx.ops[tx.nops++] = g->ops[D.xop[q]].plane;
                xterms[D.xop[p]].push_back(tx);
            }
        }
        for (size_t o = 0; o < g->ops.size(); ++o) {
            const auto& op = g->ops[o];
            const auto& tl = op.is_h ? hterms[o] : xterms[o];
            if (tl.empty()) continue;
            AccTask a;
            std::memset(&a, 0, sizeof(a));
            a.k = op.geo.k;
            for (int l = 0; l < MAXLV; ++l) a.L[l] = l < op.geo.k ? op.geo.L[l] : 1;
            a.count = op.geo.total;
            a.t0 = (int)g->terms.size();
            g->terms.insert(g->terms.end(), tl.begin(), tl.end());
            a.t1 = (int)g->terms.size();
            a.dst = splane[o];
            // blocks in proportion to the work (elements x terms), about 8
            // element-terms per thread
            const int64_t work = a.count * (a.t1 - a.t0);
            a.nblk = (int)std::max<int64_t>(1, std::min<int64_t>(8192, (work + 2047) / 2048));
            a.bfirst = g->acc_blocks;
            g->acc_blocks += a.nblk;
            g->accs.push_back(a);
            // grad_G = ifftn(S) = conj(fftn(conj S)) / total; grad_X = conj(fftn(S)); both cropped
            const bool h = op.is_h;
            emit_crop_transform(g, op.geo, {splane[o]}, h, op.rows, splane[o], BUF_OUT, op.off, true,
                                h ? 1.0 / (double)op.geo.total : 1.0, !g->cplx, h ? 1 : 2, g->bwd_lines, tails,
                                ROLE_PRODUCT);
        }
        std::vector<Launch> spec_list, rest;
        std::vector<int> spec_cuts, rest_cuts;
        flatten(bspec, spec_list, spec_cuts, g->bwd_lines);
        flatten(gspec, rest, rest_cuts, g->bwd_lines);
        if (!g->accs.empty()) rest.push_back({2, 0, (int)g->accs.size(), 0, ROLE_PRODUCT, 0});
        rest_cuts.push_back((int)rest.size());
        flatten(tails, rest, rest_cuts, g->bwd_lines);
        compact(g->bwd_lines, {&spec_list, &rest});
        g->bwd_prog_spec = split_runs(merge(spec_list, spec_cuts), g->bwd_lines);
        g->bwd_prog_rest = split_runs(merge(rest, rest_cuts), g->bwd_lines);
    }
    return HANKEL_OK;
}

}  // namespace

hankel_status general_create(GeneralPlan** out, const std::vector<hankel_mdesc>& descs, hankel_dtype dtype,
                             uint32_t flags, int64_t* h_elems, int64_t* x_elems, int64_t* y_elems, int64_t* sum_L,
                             int64_t* max_L, std::string& err) {
    *out = nullptr;
    auto* g = new GeneralPlan;
    g->dtype = dtype;
    g->flags = flags;
    g->dbl = (dtype == HANKEL_R64 || dtype == HANKEL_C128);
    g->cplx = (dtype == HANKEL_C64 || dtype == HANKEL_C128);
    g->descs = descs;
    hankel_status s = build_programs(g, descs, h_elems, x_elems, y_elems, sum_L, max_L, err);
    if (s != HANKEL_OK) {
        delete g;
        return s;
    }
    const size_t cs = csize(g);
    cudaError_t e = cudaMalloc(&g->d_tw, std::max<int64_t>(g->tw_elems, 1) * cs);
    if (e != cudaSuccess) { delete g; return cuerr(e, "cudaMalloc(twiddles)", err); }
    for (auto& kv : g->tw_off) {
        FftPlan TP;
        std::memset(&TP, 0, sizeof(TP));
        TP.L = kv.first;
        e = launch_stage_twiddles(g->dbl, (char*)g->d_tw + (size_t)kv.second * cs, TP, 0);
        if (e != cudaSuccess) { general_destroy(g); return cuerr(e, "twiddle kernel", err); }
    }
    g->ws_bytes = (size_t)std::max<int64_t>(g->ws_elems, 1) * cs;
    e = cudaMalloc(&g->d_ws, g->ws_bytes);
    if (e != cudaSuccess) { general_destroy(g); return cuerr(e, "cudaMalloc(workspace)", err); }
    if ((s = upload(g->fwd_lines, &g->d_fwd, err)) != HANKEL_OK) { general_destroy(g); return s; }
    if ((s = upload(g->bwd_lines, &g->d_bwd, err)) != HANKEL_OK) { general_destroy(g); return s; }
    if ((s = upload(g->alphas, &g->d_alpha, err)) != HANKEL_OK) { general_destroy(g); return s; }
    if ((s = upload(g->terms, &g->d_terms, err)) != HANKEL_OK) { general_destroy(g); return s; }
    if ((s = upload(g->accs, &g->d_accs, err)) != HANKEL_OK) { general_destroy(g); return s; }
    e = cudaDeviceSynchronize();
    if (e != cudaSuccess) { general_destroy(g); return cuerr(e, "plan set-up", err); }
    *out = g;
    return HANKEL_OK;
}

namespace {

// Run a program whose launches were split at plan time (split_runs) into
// runs reading one input buffer and writing one output buffer.
template <typename Skip, typename Run>
cudaError_t run_program(const std::vector<Launch>& runs, Skip skip, Run run) {
    for (const Launch& l : runs) {
        if (skip(l)) continue;
        cudaError_t e = run(l, l.what);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace

hankel_status general_forward(GeneralPlan* g, const void* h, const void* x, void* y, void* alpha, cudaStream_t st,
                              std::string& err) {
    if (!g) {
        err = "plan has no general program";
        return HANKEL_EINVAL;
    }
    cudaError_t e = run_program(
        g->fwd_prog, [&](const Launch& l) { return l.role == ROLE_PRODUCT && y == nullptr; },
        [&](const Launch& l, int) {
            const LineBufs io{h, x, y, nullptr, nullptr};
            return g->dbl ? run_lines<double>(g, l, g->d_fwd, io, st) : run_lines<float>(g, l, g->d_fwd, io, st);
        });
    if (e != cudaSuccess) return cuerr(e, "general forward launch", err);
    if (alpha != nullptr) {
        if (g->dbl)
            alpha_kernel<double><<<(int)g->alphas.size(), 256, 0, st>>>(g->d_alpha, 0, (const cx<double>*)g->d_ws,
                                                                         alpha, !g->cplx);
        else
            alpha_kernel<float><<<(int)g->alphas.size(), 256, 0, st>>>(g->d_alpha, 0, (const cx<float>*)g->d_ws,
                                                                        alpha, !g->cplx);
        e = cudaGetLastError();
        if (e != cudaSuccess) return cuerr(e, "alpha launch", err);
    }
    return HANKEL_OK;
}

hankel_status general_backward(GeneralPlan* g, const void* gy, const void* h, const void* x, void* gh, void* gx,
                               cudaStream_t st, std::string& err) {
    if (!g) {
        err = "plan has no general program";
        return HANKEL_EINVAL;
    }
    auto lines = [&](const Launch& l, const LineBufs& io) {
        return g->dbl ? run_lines<double>(g, l, g->d_bwd, io, st) : run_lines<float>(g, l, g->d_bwd, io, st);
    };
    cudaError_t e = cudaSuccess;
    if (!(g->flags & HANKEL_STORE_SPECTRA)) {
        e = run_program(
            g->bwd_prog_spec, [](const Launch&) { return false; },
            [&](const Launch& l, int) { return lines(l, LineBufs{h, x, nullptr, nullptr, nullptr}); });
        if (e != cudaSuccess) return cuerr(e, "backward spectra launch", err);
    }
    e = run_program(
        g->bwd_prog_rest, [](const Launch&) { return false; },
        [&](const Launch& l, int what) -> cudaError_t {
            if (l.kind == 2) {  // one launch over every accumulate task
                if (g->dbl)
                    accumulate_kernel<double><<<g->acc_blocks, 256, 0, st>>>(g->d_accs, l.first, l.count, g->d_terms,
                                                                             (cx<double>*)g->d_ws);
                else
                    accumulate_kernel<float><<<g->acc_blocks, 256, 0, st>>>(g->d_accs, l.first, l.count, g->d_terms,
                                                                            (cx<float>*)g->d_ws);
                return cudaGetLastError();
            }
            if (what == 3 && gh == nullptr && gx == nullptr) return cudaSuccess;  // no gradient wanted
            // G arrays read grad_y, the rest read workspace; gradient lines store
            // into grad_h (sel 1) or grad_x (sel 2) when the caller passed it
            return lines(l, LineBufs{gy, gy, nullptr, gh, gx});
        });
    if (e != cudaSuccess) return cuerr(e, "backward launch", err);
    return HANKEL_OK;
}

void general_info(GeneralPlan* g, int64_t* jobs, int64_t* launches, int64_t* lengths, int64_t* ws) {
    *jobs = g ? (int64_t)g->ds.size() : 0;
    *launches = g ? (int64_t)g->fwd_prog.size() : 0;
    *lengths = g ? (int64_t)g->tw_off.size() : 0;
    *ws = g ? (int64_t)g->ws_bytes : 0;
}

void general_destroy(GeneralPlan* g) {
    if (!g) return;
    cudaFree(g->d_tw);
    cudaFree(g->d_ws);
    cudaFree(g->d_fwd);
    cudaFree(g->d_bwd);
    cudaFree(g->d_alpha);
    cudaFree(g->d_terms);
    cudaFree(g->d_accs);
    delete g;
}

}  // namespace hk
