// general.cu -- the general path: complex or real data, a different vector
// in every mode, alpha with its own x_1, shared operands, and BHHB tensors.
//
// Everything is expressed on P x Q spectral planes (column-major, element
// (r, c) at r + P c).  A one-level tensor is the case Q = 1 (P = L >= d), a
// BHHB tensor has P >= sum n - m + 1 and Q >= sum N - m + 1 (Section 3, the
// block procedures: embed every Hankel block, then the block level).
//
// Forward (Section 3):
//   1. every distinct operand gets its spectrum plane once:
//        X^_p = fft2(X~_p),   H^ = ifft2(H~) = conj(fft2(conj H~)) / (P Q)
//      as line transforms along dim 0 (only the operand's nonzero columns)
//      then along dim 1 (Q > 1 only);
//   2. per descriptor: Y~ = fft2(H^ .* X^_2 .* ... .* X^_m), transformed along
//      dim 1 first keeping only the columns c < N_1, then along dim 0 keeping
//      rows r < n_1 (Y = Y~[0:n_1, 0:N_1]);
//   3. alpha = sum_{r,c} H^ .* X^_1 .* ... .* X^_m.
// Backward (adjoint, not in the paper; G = fft2(grad_y~)):
//   grad_H  = ifft2( sum_t G_t .* prod_p conj(X^_{t,p}(-r,-c)) )[0:d1, 0:d2]
//   grad_X  = conj(fft2( sum_{(t,p)} H^_t .* conj(G_t(-r,-c)) .* prod_{q!=p} X^_{t,q} ))[0:n_p, 0:N_p]
// where the sums run over every descriptor (and mode) that uses the operand,
// so shared operands receive the summed gradient.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <map>
#include <string>
#include <tuple>
#include <vector>

#include "fft_stage.cuh"
#include "general.h"
#include "launch.h"

namespace hk {

namespace {

constexpr int MAXOPS = HANKEL_MAX_ORDER + 1;

enum { SRC_OPERAND = 0, SRC_PRODUCT = 1 };
enum { BUF_WS = 0, BUF_OUT = 1 };

// One line transform: a block loads a line (of an input operand, or of a
// product of spectral planes), transforms it and stores a prefix of it.
struct LineTask {
    FftPlan P;
    int32_t src_mode;
    int32_t src_len, src_stride;
    int32_t src_conj;
    int64_t src;  // SRC_OPERAND: element offset in the input buffer
    // SRC_PRODUCT: product of nops planes at coordinates along the line
    int32_t nops, along, fixed, Pp, Qp;
    uint32_t rev_mask;  // operand q read at (-r, -c) and conjugated
    int64_t ops[MAXOPS];
    // sink
    int32_t dst_buf, dst_len, dst_stride, dst_conj, dst_real;
    int64_t dst;
    double scale;
    int32_t inplace;  // the sink overwrites the line the source reads
    int32_t out_sel;  // BUF_OUT sinks: 0 y, 1 grad_h, 2 grad_x
};

struct AlphaTask {
    int32_t nops, Pp, Qp, idx;
    int64_t ops[MAXOPS];
};

// Elementwise spectral sum of products into one plane (backward).
struct Term {
    int32_t nops;
    uint32_t rev_mask;
    int64_t ops[MAXOPS];
};
struct AccTask {
    int32_t Pp, Qp, t0, t1;
    int64_t dst;
};

struct Launch {
    int kind;  // 0 line, 1 alpha, 2 accumulate
    int first, count, L;
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
__device__ __forceinline__ cx<T> plane_at(const cx<T>* ws, const int64_t* ops, int nops, uint32_t rev, int r, int c,
                                          int P, int Q) {
    cx<T> v = mk<T>(T(1), T(0));
    for (int q = 0; q < nops; ++q) {
        cx<T> w;
        if (rev & (1u << q)) {
            const int rr = (r == 0) ? 0 : P - r, cc = (c == 0) ? 0 : Q - c;
            w = conjg(ws[ops[q] + rr + (int64_t)P * cc]);
        } else {
            w = ws[ops[q] + r + (int64_t)P * c];
        }
        v = (q == 0) ? w : cmul(v, w);
    }
    return v;
}

template <typename T>
struct ProductLoad {
    const cx<T>* ws;
    const int64_t* ops;  // shared-memory copy of the task's plane offsets
    int nops, along, fixed, P, Q, len, conj;
    uint32_t rev;
    __device__ __forceinline__ cx<T> operator()(int i) const {
        if (i >= len) return mk<T>(T(0), T(0));
        const int r = along == 0 ? i : fixed;
        const int c = along == 0 ? fixed : i;
        const cx<T> v = plane_at(ws, ops, nops, rev, r, c, P, Q);
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

// One line per block: the line's input (an operand column/row, or a product
// of spectral planes) is staged in shared memory, transformed by the stage
// transform (fft_stage.cuh) and its prefix stored through the sink.  All
// reads of the line finish before the first store, so a sink may overwrite
// the line the source read.
template <typename T>
__global__ void __launch_bounds__(512) line_kernel(const LineTask* __restrict__ tasks, int first,
                                                   const void* __restrict__ in, void* out, cx<T>* ws,
                                                   const cx<T>* __restrict__ tw_all, int Lmax) {
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
        const bool real = t.dst_real & 2;  // bit 1 of dst_real flags a real input operand
        const void* sbase = (const char*)in + t.src * (real ? sizeof(T) : sizeof(cx<T>));
        const OperandLoad<T> ld{sbase, t.src_len, t.src_stride, t.src_conj, real ? 1 : 0};
        for (int i = g.tid; i < P.L; i += g.nthr) b0[sp(i)] = ld(i);
    } else {
        const ProductLoad<T> ld{ws, ops_s, t.nops, t.along, t.fixed, t.Pp, t.Qp, t.src_len, t.src_conj, t.rev_mask};
        for (int i = g.tid; i < P.L; i += g.nthr) b0[sp(i)] = ld(i);
    }
    g.sync();
    void* dbase = (t.dst_buf == BUF_WS) ? (void*)(ws + t.dst)
                                        : (void*)((char*)out + t.dst * ((t.dst_real & 1) ? sizeof(T) : sizeof(cx<T>)));
    fft_stage<T>(P, GLd<T>{nullptr, 0, nullptr, 0}, b0, b1, b0,
                 LineSink<T>{dbase, t.dst_len, t.dst_stride, t.dst_conj, t.dst_real & 1, (T)t.scale}, false, tw, g);
}

template <typename T>
__global__ void __launch_bounds__(256) alpha_kernel(const AlphaTask* __restrict__ tasks, int first,
                                                    const cx<T>* __restrict__ ws, void* alpha, int real) {
    __shared__ double red[64];
    const AlphaTask& t = tasks[first + blockIdx.x];
    const Group g{(int)threadIdx.x, (int)blockDim.x, 0};
    double sr = 0.0, si = 0.0;
    const int64_t n = (int64_t)t.Pp * t.Qp;
    for (int64_t e = g.tid; e < n; e += g.nthr) {
        cx<double> v = mk<double>(1.0, 0.0);
        for (int q = 0; q < t.nops; ++q) {
            const cx<T> w = ws[t.ops[q] + e];
            v = cmul(v, mk<double>((double)w.x, (double)w.y));
        }
        sr += v.x;
        si += v.y;
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
__global__ void __launch_bounds__(256) accumulate_kernel(const AccTask* __restrict__ tasks, int first,
                                                         const Term* __restrict__ terms, cx<T>* ws) {
    const AccTask& t = tasks[first + blockIdx.y];
    const int64_t n = (int64_t)t.Pp * t.Qp;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(e % t.Pp), c = (int)(e / t.Pp);
        cx<T> acc = mk<T>(T(0), T(0));
        for (int k = t.t0; k < t.t1; ++k) {
            const Term& tm = terms[k];
            acc = acc + plane_at(ws, tm.ops, tm.nops, tm.rev_mask, r, c, t.Pp, t.Qp);
        }
        ws[t.dst + e] = acc;
    }
}

}  // namespace

// ------------------------------------------------------------------- plan

struct GeneralPlan {
    hankel_dtype dtype;
    uint32_t flags;
    bool dbl, cplx, block;
    std::vector<hankel_desc> descs;
    struct Op {
        bool is_h;
        int64_t off;
        int rows, cols, P, Q;
        int64_t plane;
    };
    std::vector<Op> ops;
    struct D {
        int m, P, Q, n1, N1, d1, d2;
        int hop, xop[HANKEL_MAX_ORDER];  // operand index of h and x_1..x_m
        int64_t temp, gplane;
    };
    std::vector<D> ds;
    std::map<int, int> tw_off;
    void* d_tw = nullptr;
    cx<float>* ws32 = nullptr;
    void* d_ws = nullptr;
    size_t ws_bytes = 0;
    // forward / backward programs
    std::vector<LineTask> fwd_lines, bwd_lines;
    std::vector<AlphaTask> alphas;
    std::vector<Term> terms;
    std::vector<AccTask> accs;
    std::vector<Launch> fwd_prog, bwd_prog_spec, bwd_prog_rest;
    std::vector<Launch> alpha_prog;
    LineTask *d_fwd = nullptr, *d_bwd = nullptr;
    AlphaTask* d_alpha = nullptr;
    Term* d_terms = nullptr;
    AccTask* d_accs = nullptr;
    bool want_grad_h = true, want_grad_x = true;
    // backward gradient targets
    std::vector<int64_t> h_targets, x_targets;  // operand indices
};

namespace {

size_t csize(const GeneralPlan* g) { return (g->dbl ? 8 : 4) * 2; }

int64_t fft_len(int64_t d) { return hankel_fft_length(d); }

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

// Spectrum plane of operand o: dim-0 lines over its nonzero columns, then
// dim-1 lines (Q > 1).  h operands become ifft2 (conj in, conj + 1/(PQ) out).
void emit_operand_spectrum(GeneralPlan* g, int o, std::vector<LineTask>& lines, std::vector<Launch>& prog) {
    const auto& op = g->ops[o];
    const bool last_is_dim0 = (op.Q == 1);
    const double sc = op.is_h ? 1.0 / ((double)op.P * op.Q) : 1.0;
    int first = (int)lines.size();
    for (int j = 0; j < op.cols; ++j) {
        LineTask t = blank_task();
        t.P = plan_for(g, op.P);
        t.src_mode = SRC_OPERAND;
        t.src = op.off + (int64_t)j * op.rows;
        t.src_len = op.rows;
        t.src_conj = op.is_h;
        t.dst_buf = BUF_WS;
        t.dst = op.plane + (int64_t)j * op.P;
        t.dst_len = op.P;
        t.dst_real = g->cplx ? 0 : 2;  // input real flag in bit 1
        if (last_is_dim0) {
            t.dst_conj = op.is_h;
            t.scale = sc;
        }
        lines.push_back(t);
    }
    prog.push_back({0, first, (int)lines.size() - first, op.P});
    if (op.Q > 1) {
        first = (int)lines.size();
        for (int r = 0; r < op.P; ++r) {
            LineTask t = blank_task();
            t.P = plan_for(g, op.Q);
            t.src_mode = SRC_PRODUCT;
            t.nops = 1;
            t.ops[0] = op.plane;
            t.along = 1;
            t.fixed = r;
            t.Pp = op.P;
            t.Qp = op.Q;
            t.src_len = op.cols;
            t.dst_buf = BUF_WS;
            t.dst = op.plane + r;
            t.dst_stride = op.P;
            t.dst_len = op.Q;
            t.dst_conj = op.is_h;
            t.scale = sc;
            t.inplace = 1;
            lines.push_back(t);
        }
        prog.push_back({0, first, (int)lines.size() - first, op.Q});
    }
}

// Two-pass transform of a product of planes, cropped to rows x cols and stored
// to a destination matrix (column-major, leading dimension ld):
// dim 1 first over all P rows into `temp` (keeping cols columns), then dim 0.
void emit_product_transform(GeneralPlan* g, int P, int Q, const std::vector<int64_t>& planes, uint32_t rev,
                            bool conj_in, int rows, int cols, int64_t temp, int dst_buf, int64_t dst, int64_t ld,
                            bool conj_out, double scale, bool real_out, std::vector<LineTask>& lines,
                            std::vector<Launch>& prog) {
    if (Q > 1) {
        int first = (int)lines.size();
        for (int r = 0; r < P; ++r) {
            LineTask t = blank_task();
            t.P = plan_for(g, Q);
            t.src_mode = SRC_PRODUCT;
            t.nops = (int)planes.size();
            for (int q = 0; q < t.nops; ++q) t.ops[q] = planes[q];
            t.rev_mask = rev;
            t.src_conj = conj_in;
            t.along = 1;
            t.fixed = r;
            t.Pp = P;
            t.Qp = Q;
            t.src_len = Q;
            t.dst_buf = BUF_WS;
            t.dst = temp + r;
            t.dst_stride = P;
            t.dst_len = cols;
            lines.push_back(t);
        }
        prog.push_back({0, first, (int)lines.size() - first, Q});
    }
    int first = (int)lines.size();
    for (int c = 0; c < cols; ++c) {
        LineTask t = blank_task();
        t.P = plan_for(g, P);
        t.src_mode = SRC_PRODUCT;
        if (Q > 1) {
            t.nops = 1;
            t.ops[0] = temp;
            t.Qp = cols;
        } else {
            t.nops = (int)planes.size();
            for (int q = 0; q < t.nops; ++q) t.ops[q] = planes[q];
            t.rev_mask = rev;
            t.src_conj = conj_in;
            t.Qp = Q;
        }
        t.along = 0;
        t.fixed = c;
        t.Pp = P;
        t.src_len = P;
        t.dst_buf = dst_buf;
        t.dst = dst + (int64_t)c * ld;
        t.dst_len = rows;
        t.dst_conj = conj_out;
        t.scale = scale;
        t.dst_real = real_out ? 1 : 0;
        lines.push_back(t);
    }
    prog.push_back({0, first, (int)lines.size() - first, P});
}

// Group consecutive launches of the same kind and length (independent tasks
// of one phase) to cut launch counts.
std::vector<Launch> merge(const std::vector<Launch>& in, const std::vector<int>& barriers) {
    std::vector<Launch> out;
    size_t bi = 0;
    for (size_t i = 0; i < in.size(); ++i) {
        bool cut = false;
        while (bi < barriers.size() && barriers[bi] <= (int)i) {
            if (barriers[bi] == (int)i) cut = true;
            ++bi;
        }
        if (!out.empty() && !cut && out.back().kind == in[i].kind && out.back().L == in[i].L &&
            out.back().first + out.back().count == in[i].first)
            out.back().count += in[i].count;
        else
            out.push_back(in[i]);
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

int nthr_for(int L) {
    int p = 1;
    while (p < (L + 15) / 16) p <<= 1;
    return std::max(32, std::min(512, p));
}

template <typename T>
cudaError_t run_lines(GeneralPlan* g, const std::vector<Launch>& prog, const LineTask* d_tasks, const void* in,
                      void* out, cudaStream_t st) {
    for (const Launch& l : prog) {
        const size_t smem = line_smem(g, l.L);
        // raise the limit only when needed (no attribute calls in steady state,
        // so the launches can be captured into CUDA graphs); per device
        static size_t granted[64] = {0};
        int dev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e != cudaSuccess) return e;
        if (smem > granted[dev & 63]) {
            e = cudaFuncSetAttribute(line_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
            granted[dev & 63] = smem;
        }
        line_kernel<T><<<l.count, nthr_for(l.L), smem, st>>>(d_tasks, l.first, in, out, (cx<T>*)g->d_ws,
                                                           (const cx<T>*)g->d_tw, l.L);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace

hankel_status general_create(GeneralPlan** out, const std::vector<hankel_desc>& descs, hankel_dtype dtype,
                             uint32_t flags, int64_t* h_elems, int64_t* x_elems, int64_t* y_elems, int64_t* sum_L,
                             int64_t* max_L, std::string& err) {
    *out = nullptr;
    auto* g = new GeneralPlan;
    g->dtype = dtype;
    g->flags = flags;
    g->dbl = (dtype == HANKEL_R64 || dtype == HANKEL_C128);
    g->cplx = (dtype == HANKEL_C64 || dtype == HANKEL_C128);
    g->block = (flags & HANKEL_BLOCK) != 0;
    g->descs = descs;
    const bool same_x = (flags & HANKEL_SAME_X) != 0;
    const size_t cs = csize(g);
    const int maxL = (int)std::min<int64_t>(16384, [&] {
        int L = 2;
        while (L < 16384 && RED_BYTES + ((size_t)TWG_SMEM + 2 * smem_elems_host(L + 1)) * cs <= 227 * 1024) ++L;
        return (int64_t)L;
    }());
    std::map<std::tuple<int, int64_t, int, int, int, int>, int> opidx;
    int64_t plane_cursor = 0;
    auto add_op = [&](bool is_h, int64_t off, int rows, int cols, int P, int Q) {
        auto key = std::make_tuple((int)is_h, off, rows, cols, P, Q);
        auto it = opidx.find(key);
        if (it != opidx.end()) return it->second;
        GeneralPlan::Op op{is_h, off, rows, cols, P, Q, plane_cursor};
        plane_cursor += (int64_t)P * Q;
        g->ops.push_back(op);
        opidx[key] = (int)g->ops.size() - 1;
        return (int)g->ops.size() - 1;
    };
    *h_elems = *x_elems = *y_elems = 0;
    *sum_L = *max_L = 0;
    for (size_t i = 0; i < descs.size(); ++i) {
        const hankel_desc& d = descs[i];
        GeneralPlan::D D;
        std::memset(&D, 0, sizeof(D));
        D.m = d.m;
        int64_t sn = 0, sN = 0;
        for (int p = 0; p < d.m; ++p) {
            sn += d.n[p];
            sN += g->block ? d.N[p] : 1;
        }
        D.d1 = (int)(sn - d.m + 1);
        D.d2 = (int)(sN - d.m + 1);
        const int64_t P = fft_len(D.d1), Q = g->block ? fft_len(D.d2) : 1;
        if (P < 0 || Q < 0 || P > maxL || Q > maxL) {
            err = "descriptor " + std::to_string(i) + ": FFT length beyond the supported maximum of this build";
            delete g;
            return HANKEL_EUNSUPPORTED;
        }
        D.P = (int)P;
        D.Q = (int)Q;
        D.n1 = d.n[0];
        D.N1 = g->block ? d.N[0] : 1;
        D.hop = add_op(true, d.h_off, D.d1, D.d2, D.P, D.Q);
        for (int p = 0; p < d.m; ++p) {
            const int64_t xo = same_x ? d.x_off[0] : d.x_off[p];
            const int Np = g->block ? d.N[p] : 1;
            const int np_ = same_x ? d.n[0] : d.n[p];
            D.xop[p] = add_op(false, xo, np_, same_x ? (g->block ? d.N[0] : 1) : Np, D.P, D.Q);
            *x_elems = std::max<int64_t>(*x_elems, xo + (int64_t)np_ * Np);
        }
        *h_elems = std::max<int64_t>(*h_elems, d.h_off + (int64_t)D.d1 * D.d2);
        *y_elems = std::max<int64_t>(*y_elems, d.y_off + (int64_t)D.n1 * D.N1);
        *sum_L += P * Q;
        *max_L = std::max<int64_t>(*max_L, std::max(P, Q));
        g->tw_off[(int)P] = 0;
        g->tw_off[(int)Q] = 0;
        g->ds.push_back(D);
    }
    // temp planes (forward, BHHB only), G planes and S planes (backward)
    for (auto& D : g->ds) {
        D.temp = plane_cursor;
        if (D.Q > 1) plane_cursor += (int64_t)D.P * D.N1;
        D.gplane = plane_cursor;
        plane_cursor += (int64_t)D.P * D.Q;
    }
    std::vector<int64_t> splane(g->ops.size());
    for (size_t o = 0; o < g->ops.size(); ++o) {
        splane[o] = plane_cursor;
        plane_cursor += (int64_t)g->ops[o].P * g->ops[o].Q;
    }
    // twiddles
    int64_t tw_total = 0;
    for (auto& kv : g->tw_off) {
        kv.second = (int)tw_total;
        tw_total += tw_table_elems(kv.first);
    }
    cudaError_t e = cudaMalloc(&g->d_tw, std::max<int64_t>(tw_total, 1) * cs);
    if (e != cudaSuccess) { delete g; return cuerr(e, "cudaMalloc(twiddles)", err); }
    for (auto& kv : g->tw_off) {
        if (kv.first < 2) continue;  // Q = 1: no transform along that axis
        FftPlan TP;
        std::memset(&TP, 0, sizeof(TP));
        TP.L = kv.first;
        e = launch_stage_twiddles(g->dbl, (char*)g->d_tw + (size_t)kv.second * cs, TP, 0);
        if (e != cudaSuccess) { general_destroy(g); return cuerr(e, "twiddle kernel", err); }
    }
    g->ws_bytes = (size_t)std::max<int64_t>(plane_cursor, 1) * cs;
    e = cudaMalloc(&g->d_ws, g->ws_bytes);
    if (e != cudaSuccess) { general_destroy(g); return cuerr(e, "cudaMalloc(workspace)", err); }

    // ---- forward program
    std::vector<Launch> prog;
    std::vector<int> cuts;
    for (size_t o = 0; o < g->ops.size(); ++o) emit_operand_spectrum(g, (int)o, g->fwd_lines, prog);
    // keep spectra dim-0 / dim-1 phases ordered: cut between phases by
    // reordering: all dim-0 launches first, then all dim-1 launches
    {
        std::vector<Launch> d0, d1;
        for (auto& l : prog) {
            const LineTask& t = g->fwd_lines[l.first];
            ((t.src_mode == SRC_OPERAND) ? d0 : d1).push_back(l);
        }
        prog = d0;
        cuts.push_back((int)prog.size());
        prog.insert(prog.end(), d1.begin(), d1.end());
        cuts.push_back((int)prog.size());
    }
    const size_t spec_end = prog.size();
    std::vector<Launch> pd1, pd0;
    for (size_t i = 0; i < g->ds.size(); ++i) {
        const auto& D = g->ds[i];
        std::vector<int64_t> planes{g->ops[D.hop].plane};
        for (int p = 1; p < D.m; ++p) planes.push_back(g->ops[D.xop[p]].plane);
        std::vector<Launch> tmp;
        emit_product_transform(g, D.P, D.Q, planes, 0u, false, D.n1, D.N1, D.temp, BUF_OUT, descs[i].y_off, D.n1,
                               false, 1.0, !g->cplx, g->fwd_lines, tmp);
        if (tmp.size() == 2) {
            pd1.push_back(tmp[0]);
            pd0.push_back(tmp[1]);
        } else {
            pd0.push_back(tmp[0]);
        }
    }
    prog.insert(prog.end(), pd1.begin(), pd1.end());
    cuts.push_back((int)prog.size());
    prog.insert(prog.end(), pd0.begin(), pd0.end());
    compact(g->fwd_lines, {&prog});
    g->fwd_prog = merge(prog, cuts);
    (void)spec_end;
    for (size_t i = 0; i < g->ds.size(); ++i) {
        const auto& D = g->ds[i];
        AlphaTask a;
        std::memset(&a, 0, sizeof(a));
        a.nops = D.m + 1;
        a.ops[0] = g->ops[D.hop].plane;
        for (int p = 0; p < D.m; ++p) a.ops[1 + p] = g->ops[D.xop[p]].plane;
        a.Pp = D.P;
        a.Qp = D.Q;
        a.idx = (int)i;
        g->alphas.push_back(a);
    }

    // ---- backward program: G planes, spectral sums, transforms to gradients
    std::vector<Launch> bspec, bg0, bg1, spec_list;
    std::vector<int> spec_cuts;
    for (size_t o = 0; o < g->ops.size(); ++o) emit_operand_spectrum(g, (int)o, g->bwd_lines, bspec);
    {
        std::vector<Launch> d0, d1;
        for (auto& l : bspec) ((g->bwd_lines[l.first].src_mode == SRC_OPERAND) ? d0 : d1).push_back(l);
        std::vector<int> c2{(int)d0.size()};
        d0.insert(d0.end(), d1.begin(), d1.end());
        c2.push_back((int)d0.size());
        spec_list = d0;
        spec_cuts = c2;
    }
    // G_t = fft2(grad_y~): dim-0 over the N1 nonzero columns, then dim 1
    for (size_t i = 0; i < g->ds.size(); ++i) {
        const auto& D = g->ds[i];
        int first = (int)g->bwd_lines.size();
        for (int c = 0; c < D.N1; ++c) {
            LineTask t = blank_task();
            t.P = plan_for(g, D.P);
            t.src_mode = SRC_OPERAND;
            t.src = descs[i].y_off + (int64_t)c * D.n1;
            t.src_len = D.n1;
            t.dst_buf = BUF_WS;
            t.dst = D.gplane + (int64_t)c * D.P;
            t.dst_len = D.P;
            t.dst_real = g->cplx ? 0 : 2;
            g->bwd_lines.push_back(t);
        }
        bg0.push_back({0, first, (int)g->bwd_lines.size() - first, D.P});
        if (D.Q > 1) {
            first = (int)g->bwd_lines.size();
            for (int r = 0; r < D.P; ++r) {
                LineTask t = blank_task();
                t.P = plan_for(g, D.Q);
                t.src_mode = SRC_PRODUCT;
                t.nops = 1;
                t.ops[0] = D.gplane;
                t.along = 1;
                t.fixed = r;
                t.Pp = D.P;
                t.Qp = D.Q;
                t.src_len = D.N1;
                t.dst_buf = BUF_WS;
                t.dst = D.gplane + r;
                t.dst_stride = D.P;
                t.dst_len = D.Q;
                t.inplace = 1;
                g->bwd_lines.push_back(t);
            }
            bg1.push_back({0, first, (int)g->bwd_lines.size() - first, D.Q});
        }
    }
    // spectral sums per gradient target
    std::vector<std::vector<Term>> hterms(g->ops.size()), xterms(g->ops.size());
    for (size_t i = 0; i < g->ds.size(); ++i) {
        const auto& D = g->ds[i];
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
    std::vector<Launch> bacc;
    std::vector<LineTask> tail_lines;
    std::vector<Launch> bt1, bt0;
    for (size_t o = 0; o < g->ops.size(); ++o) {
        const auto& op = g->ops[o];
        const auto& tl = op.is_h ? hterms[o] : xterms[o];
        if (tl.empty()) continue;
        AccTask a;
        a.Pp = op.P;
        a.Qp = op.Q;
        a.t0 = (int)g->terms.size();
        g->terms.insert(g->terms.end(), tl.begin(), tl.end());
        a.t1 = (int)g->terms.size();
        a.dst = splane[o];
        g->accs.push_back(a);
        (op.is_h ? g->h_targets : g->x_targets).push_back((int64_t)o);
        // grad_h = ifft2(S) = conj(fft2(conj S))/(PQ); grad_x = conj(fft2(S)); both cropped
        std::vector<Launch> tmp;
        const bool h = op.is_h;
        const int64_t temp = splane[o];  // dim-1 pass writes back into S (its first `cols` columns)
        if (op.Q > 1) {
            // dim 1 in place on S (conj in for h), keep the first `cols` columns
            int first = (int)g->bwd_lines.size();
            for (int r = 0; r < op.P; ++r) {
                LineTask t = blank_task();
                t.P = plan_for(g, op.Q);
                t.src_mode = SRC_PRODUCT;
                t.nops = 1;
                t.ops[0] = splane[o];
                t.src_conj = h;
                t.along = 1;
                t.fixed = r;
                t.Pp = op.P;
                t.Qp = op.Q;
                t.src_len = op.Q;
                t.dst_buf = BUF_WS;
                t.dst = splane[o] + r;
                t.dst_stride = op.P;
                t.dst_len = op.cols;
                t.inplace = 1;
                g->bwd_lines.push_back(t);
            }
            bt1.push_back({0, first, (int)g->bwd_lines.size() - first, op.Q});
        }
        int first = (int)g->bwd_lines.size();
        for (int c = 0; c < op.cols; ++c) {
            LineTask t = blank_task();
            t.P = plan_for(g, op.P);
            t.src_mode = SRC_PRODUCT;
            t.nops = 1;
            t.ops[0] = temp;
            t.src_conj = (op.Q > 1) ? 0 : h;
            t.along = 0;
            t.fixed = c;
            t.Pp = op.P;
            t.Qp = op.Q;
            t.src_len = op.P;
            t.dst_buf = BUF_OUT;
            t.dst = (h ? 0 : 0) + op.off + (int64_t)c * op.rows;
            t.dst_len = op.rows;
            t.dst_conj = 1;
            t.scale = h ? 1.0 / ((double)op.P * op.Q) : 1.0;
            t.dst_real = g->cplx ? 0 : 1;
            t.out_sel = h ? 1 : 2;
            g->bwd_lines.push_back(t);
            (void)tmp;
        }
        bt0.push_back({0, first, (int)g->bwd_lines.size() - first, op.P});
        bacc.push_back({2, (int)g->accs.size() - 1, 1, 0});
    }
    {
        std::vector<Launch> rest;
        std::vector<int> c3;
        rest.insert(rest.end(), bg0.begin(), bg0.end());
        c3.push_back((int)rest.size());
        rest.insert(rest.end(), bg1.begin(), bg1.end());
        c3.push_back((int)rest.size());
        // accumulate launches are emitted as one launch over all targets
        if (!g->accs.empty()) rest.push_back({2, 0, (int)g->accs.size(), 0});
        c3.push_back((int)rest.size());
        rest.insert(rest.end(), bt1.begin(), bt1.end());
        c3.push_back((int)rest.size());
        rest.insert(rest.end(), bt0.begin(), bt0.end());
        compact(g->bwd_lines, {&spec_list, &rest});
        g->bwd_prog_spec = merge(spec_list, spec_cuts);
        g->bwd_prog_rest = merge(rest, c3);
    }
    hankel_status s;
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

hankel_status general_forward(GeneralPlan* g, const void* h, const void* x, void* y, void* alpha, cudaStream_t st,
                              std::string& err) {
    if (!g) {
        err = "plan has no general program";
        return HANKEL_EINVAL;
    }
    // phase 1: operand spectra (h operands read `h`, x operands read `x`)
    cudaError_t e = cudaSuccess;
    for (const Launch& l : g->fwd_prog) {
        const LineTask& t0 = g->fwd_lines[l.first];
        const bool spectra = (t0.dst_buf == BUF_WS && (t0.src_mode == SRC_OPERAND || t0.inplace));
        if (!spectra && y == nullptr) continue;  // product transforms only when y is wanted
        // launches mix h and x operands; split by operand kind within the launch
        int i = l.first;
        while (i < l.first + l.count) {
            int j = i;
            bool ish = false;
            if (g->fwd_lines[i].src_mode == SRC_OPERAND) {
                // find operand kind from its conj flag (h operands are conjugated on load)
                ish = g->fwd_lines[i].src_conj != 0;
                while (j < l.first + l.count && g->fwd_lines[j].src_mode == SRC_OPERAND &&
                       (g->fwd_lines[j].src_conj != 0) == ish)
                    ++j;
            } else {
                j = l.first + l.count;
            }
            Launch sub{0, i, j - i, l.L};
            std::vector<Launch> one{sub};
            e = g->dbl ? run_lines<double>(g, one, g->d_fwd, ish ? h : x, y, st)
                       : run_lines<float>(g, one, g->d_fwd, ish ? h : x, y, st);
            if (e != cudaSuccess) return cuerr(e, "general forward launch", err);
            i = j;
        }
    }
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
    cudaError_t e;
    auto run_sub = [&](const Launch& l, const void* in, void* out) {
        std::vector<Launch> one{l};
        return g->dbl ? run_lines<double>(g, one, g->d_bwd, in, out, st)
                      : run_lines<float>(g, one, g->d_bwd, in, out, st);
    };
    if (!(g->flags & HANKEL_STORE_SPECTRA)) {
        for (const Launch& l : g->bwd_prog_spec) {
            int i = l.first;
            while (i < l.first + l.count) {
                int j = i;
                bool ish = false;
                if (g->bwd_lines[i].src_mode == SRC_OPERAND) {
                    ish = g->bwd_lines[i].src_conj != 0;
                    while (j < l.first + l.count && g->bwd_lines[j].src_mode == SRC_OPERAND &&
                           (g->bwd_lines[j].src_conj != 0) == ish)
                        ++j;
                } else {
                    j = l.first + l.count;
                }
                e = run_sub({0, i, j - i, l.L}, ish ? h : x, nullptr);
                if (e != cudaSuccess) return cuerr(e, "backward spectra launch", err);
                i = j;
            }
        }
    }
    for (const Launch& l : g->bwd_prog_rest) {
        if (l.kind == 2) {
            dim3 grid(64, l.count);
            if (g->dbl)
                accumulate_kernel<double><<<grid, 256, 0, st>>>(g->d_accs, l.first, g->d_terms, (cx<double>*)g->d_ws);
            else
                accumulate_kernel<float><<<grid, 256, 0, st>>>(g->d_accs, l.first, g->d_terms, (cx<float>*)g->d_ws);
            e = cudaGetLastError();
            if (e != cudaSuccess) return cuerr(e, "accumulate launch", err);
            continue;
        }
        const LineTask& t0 = g->bwd_lines[l.first];
        if (t0.dst_buf == BUF_OUT) {
            // gradient stores: split the launch into grad_h and grad_x runs
            int i = l.first;
            while (i < l.first + l.count) {
                const int sel = g->bwd_lines[i].out_sel;
                int j = i + 1;
                while (j < l.first + l.count && g->bwd_lines[j].out_sel == sel) ++j;
                void* dst = (sel == 1) ? gh : gx;
                if (dst != nullptr) {
                    e = run_sub({0, i, j - i, l.L}, nullptr, dst);
                    if (e != cudaSuccess) return cuerr(e, "backward launch", err);
                }
                i = j;
            }
        } else {
            e = run_sub(l, gy, nullptr);
            if (e != cudaSuccess) return cuerr(e, "backward launch", err);
        }
    }
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
