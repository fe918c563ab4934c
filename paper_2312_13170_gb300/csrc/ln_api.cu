// The C ABI of libloopnest: argument validation, aliasing checks, workspace
// planning and dispatch to the plain, FP32-tiled and tcgen05 engines.
#include <algorithm>
#include <atomic>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "ln_gs.h"
#include "ln_internal.h"
#include "ln_stats.h"

namespace ln {

namespace {
thread_local char g_msg[512] = "";
}

ln_status fail(ln_status s, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_msg, sizeof(g_msg), fmt, ap);
    va_end(ap);
    return s;
}

void clear_error() { g_msg[0] = '\0'; }

ln_status check_launch(const char *what) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(LN_ERR_CUDA, "%s launch failed: %s", what, cudaGetErrorString(e));
    return LN_SUCCESS;
}

// ------------------------------------------------------------------ launch accounting
void record_event(cudaEvent_t e, cudaStream_t st);

// Alive around launches that the library issues back to back on one stream
// (see the definition below).
struct SpanHold {
    SpanHold();
    ~SpanHold();
    SpanHold(const SpanHold &) = delete;
    SpanHold &operator=(const SpanHold &) = delete;
};

namespace {
// One timed run: a start and a stop event around `launches` kernel launches.
struct TimedRun {
    cudaEvent_t start = nullptr, stop = nullptr;
    int launches = 0;
};
struct TimingState {
    int mode = 0;  // 0 off, 1 every launch, 2 spans (see ln_timing_enable)
    std::vector<TimedRun> pending[FAM_COUNT];
    std::vector<TimedRun> pool;
    int hold = 0;  // SpanHold scopes alive
    // a span whose stop event is not recorded yet: the last launch of family
    // `open_f` on stream `open_st`, inside a SpanHold
    bool open = false;
    Family open_f = FAM_UMMA;
    cudaStream_t open_st = nullptr;
    int open_slot = -1;
};
TimingState g_timing;
std::atomic<long long> g_launches{0};
const char *const kFamilies[FAM_COUNT] = {"umma", "pack", "simt", "plain", "stats"};

void close_span() {
    if (!g_timing.open) return;
    g_timing.open = false;
    record_event(g_timing.pending[g_timing.open_f][g_timing.open_slot].stop, g_timing.open_st);
}
}  // namespace

// Inside stream capture a plain event record is only a dependency marker; an
// external record becomes a graph node that timestamps every replay.
void record_event(cudaEvent_t e, cudaStream_t st) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusActive)
        cudaEventRecordWithFlags(e, st, cudaEventRecordExternal);
    else
        cudaEventRecord(e, st);
}

LaunchScope::LaunchScope(Family fam, cudaStream_t s) : slot(-1), st(s), f(fam) {
    g_launches.fetch_add(1, std::memory_order_relaxed);
    if (!g_timing.mode) return;
    if (g_timing.open) {
        if (g_timing.open_f == f && g_timing.open_st == st) {
            // the previous launch on this stream was of the same family, inside
            // a SpanHold: this one joins its span, with no event between them
            g_timing.open = false;
            slot = g_timing.open_slot;
            ++g_timing.pending[f][slot].launches;
            return;
        }
        close_span();
    }
    TimedRun r;
    if (!g_timing.pool.empty()) {
        r = g_timing.pool.back();
        g_timing.pool.pop_back();
    } else if (cudaEventCreate(&r.start) != cudaSuccess || cudaEventCreate(&r.stop) != cudaSuccess) {
        return;
    }
    r.launches = 1;
    record_event(r.start, st);
    g_timing.pending[f].push_back(r);
    slot = (int)g_timing.pending[f].size() - 1;
}

LaunchScope::~LaunchScope() {
    if (slot < 0) return;
    if (g_timing.mode == 2 && g_timing.hold > 0) {  // the next launch may join
        g_timing.open = true;
        g_timing.open_f = f;
        g_timing.open_st = st;
        g_timing.open_slot = slot;
        return;
    }
    record_event(g_timing.pending[f][slot].stop, st);
}

// Marks launches that the library issues back to back on one stream with
// programmatic launch overlap (the chain's two contractions): in span mode
// they share one event pair, since an event recorded between them would
// serialise the second launch behind the first's last CTA. Only for launches
// on a single stream: a span left open on a forked stream would be closed
// after that stream's join.
SpanHold::SpanHold() { ++g_timing.hold; }
SpanHold::~SpanHold() {
    if (--g_timing.hold == 0) close_span();
}

// ------------------------------------------------------------------ tuning knobs
namespace {
std::atomic<int> g_chunk_kt{2};
std::atomic<int> g_tile_n{0};
std::atomic<int> g_pack_threads{512};
std::atomic<int> g_split_k{0};
std::atomic<int> g_gs_rows{4};
std::atomic<int> g_stream_k{2};
std::atomic<int> g_pair{1};
std::atomic<int> g_stage_beta{1};
std::atomic<int> g_stage_out{1};
std::atomic<int> g_simt_tile{0};
std::atomic<int> g_sym_wide{0};
std::atomic<int> g_simt_exact{1};
}  // namespace

int tune_chunk_kt() { return g_chunk_kt.load(std::memory_order_relaxed); }
int tune_tile_n() { return g_tile_n.load(std::memory_order_relaxed); }
int tune_pack_threads() { return g_pack_threads.load(std::memory_order_relaxed); }
int tune_split_k() { return g_split_k.load(std::memory_order_relaxed); }
int tune_gs_rows() { return g_gs_rows.load(std::memory_order_relaxed); }
int tune_stream_k() { return g_stream_k.load(std::memory_order_relaxed); }
int tune_pair() { return g_pair.load(std::memory_order_relaxed); }
int tune_stage_beta() { return g_stage_beta.load(std::memory_order_relaxed); }
int tune_stage_out() { return g_stage_out.load(std::memory_order_relaxed); }
int tune_simt_tile() { return g_simt_tile.load(std::memory_order_relaxed); }
int tune_sym_wide() { return g_sym_wide.load(std::memory_order_relaxed); }
int tune_simt_exact() { return g_simt_exact.load(std::memory_order_relaxed); }

bool inject_timeout_requested() {
    const char *v = getenv("LN_FAULT_INJECT");
    return v && strcmp(v, "timeout") == 0;
}

ln_status check_dims(std::initializer_list<long long> dims) {
    for (long long d : dims)
        if (d < 0 || d > MAX_DIM) return fail(LN_ERR_INVALID_VALUE, "size %lld out of range [0, %lld]", d, MAX_DIM);
    return LN_SUCCESS;
}

int sm_count() {
    static int cache[64] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 1;
    if (cache[dev] == 0) {
        int n = 0;
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        cache[dev] = n > 0 ? n : 1;
    }
    return cache[dev];
}

namespace {

// ------------------------------------------------------------------ workspace planning
// A bump allocator over the caller's workspace. With base == nullptr it only
// counts, so the size query and the call run the very same plan.
struct Ws {
    char *base;
    size_t off = 0;
    explicit Ws(void *b) : base(static_cast<char *>(b)) {}
    template <class T>
    T *take(size_t bytes) {
        off = align_up(off, 256);
        T *p = base ? reinterpret_cast<T *>(base + off) : nullptr;
        off += align_up(bytes, 256);
        return p;
    }
};

// Split-K workspace shared by contractions that run one after another in
// stream order (sized for the largest of them).
struct SplitArea {
    float *part = nullptr;
    int *cnt = nullptr;
};

// Split-K (umma_ksplit) or stream-K (umma_streamk) of one tcgen05
// contraction, and their workspace.
struct SplitPlan {
    int ksplit = 1;
    float *part = nullptr;
    int *cnt = nullptr;
    int streamk = 0;
    float *skpart = nullptr;
    int *skflag = nullptr;
};

void plan_split(Ws &w, long long tiles, int ktot, int bn, SplitPlan &sp) {
    sp.ksplit = umma_ksplit(tiles, ktot);
    if (sp.ksplit > 1) {
        sp.part = w.take<float>(umma_split_part_bytes(tiles, sp.ksplit, bn));
        sp.cnt = w.take<int>(umma_split_cnt_bytes(tiles, bn));
        return;
    }
    sp.streamk = umma_streamk(tiles, ktot);
    if (sp.streamk) {
        sp.skpart = w.take<float>(umma_streamk_part_bytes(bn));
        sp.skflag = w.take<int>(umma_streamk_flag_bytes());
    }
}

// Stream-K flags start at zero: cleared before the first kernel of the call,
// so that the call's kernels still follow each other with programmatic
// dependent launch.
ln_status zero_streamk_flags(const SplitPlan &sp, cudaStream_t st) {
    if (sp.streamk) LN_CUDA_TRY(cudaMemsetAsync(sp.skflag, 0, umma_streamk_flag_bytes(), st));
    return LN_SUCCESS;
}

// dims: (M, N, K) of general contractions
void plan_split_area(Ws &w, const int (*dims)[3], int nd, int P, SplitArea &a) {
    size_t pbytes = 0, cbytes = 0;
    for (int i = 0; i < nd; ++i) {
        const int bn = umma_tile_n(P, 0, dims[i][0], dims[i][1]);
        const long long tiles = ceil_div(dims[i][0], PK_ROWS) * ceil_div(dims[i][1], bn);
        const int ks = umma_ksplit(tiles, (int)ceil_div(dims[i][2], PK_K));
        if (ks > 1) {
            pbytes = std::max(pbytes, umma_split_part_bytes(tiles, ks, bn));
            cbytes = std::max(cbytes, umma_split_cnt_bytes(tiles, bn));
        }
    }
    if (pbytes) {
        a.part = w.take<float>(pbytes);
        a.cnt = w.take<int>(cbytes);
    }
}

void apply_split(UmmaProblem &pb, const SplitPlan &sp) {
    pb.ksplit = sp.ksplit;
    pb.kpart = sp.part;
    pb.kcnt = sp.cnt;
    pb.streamk = sp.streamk;
    pb.skpart = sp.skpart;
    pb.skflag = sp.skflag;
}

// ------------------------------------------------------------------ host-resident operands
// The address kernels use for `p`: device and managed memory as is; pinned
// (page-locked or registered) host memory through its device mapping (read
// and written by the kernels over the host link, no staging copy); pageable
// host memory only where the GPU reports coherent pageable access (e.g.
// NVLink-C2C systems), else LN_ERR_INVALID_VALUE before anything is launched.
template <class T>
ln_status device_view(T *p, T **out, const char *name) {
    *out = p;
    if (!p) return LN_SUCCESS;
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return fail(LN_ERR_INVALID_VALUE, "%s: not a pointer this process can use", name);
    }
    switch (a.type) {
        case cudaMemoryTypeDevice:
        case cudaMemoryTypeManaged: return LN_SUCCESS;
        case cudaMemoryTypeHost:
            if (!a.devicePointer) return fail(LN_ERR_INVALID_VALUE, "%s: pinned host buffer without a device mapping", name);
            *out = static_cast<T *>(a.devicePointer);
            return LN_SUCCESS;
        default: {
            int dev = 0, pageable = 0;
            LN_CUDA_TRY(cudaGetDevice(&dev));
            LN_CUDA_TRY(cudaDeviceGetAttribute(&pageable, cudaDevAttrPageableMemoryAccess, dev));
            if (!pageable)
                return fail(LN_ERR_INVALID_VALUE, "%s: pageable host memory is not accessible from this GPU (pin it)",
                            name);
            return LN_SUCCESS;
        }
    }
}

// ------------------------------------------------------------------ a second stream
// For independent contractions that fit on the GPU together: one extra stream
// and two events per host thread and device, created on first use outside
// graph capture (a call that finds none while its stream is capturing runs
// everything in its own stream).
struct SideStream {
    cudaStream_t s = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr, mid_a = nullptr, mid_b = nullptr;
};
thread_local SideStream t_side[64];

SideStream *side_stream(cudaStream_t st) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        cudaGetLastError();
        return nullptr;
    }
    SideStream &g = t_side[dev];
    if (!g.s) {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
            cudaGetLastError();
            return nullptr;
        }
        if (cudaStreamCreateWithFlags(&g.s, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&g.fork, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&g.join, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&g.mid_a, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&g.mid_b, cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            g = SideStream{};
            return nullptr;
        }
    }
    return &g;
}

// ------------------------------------------------------------------ validation helpers
struct Span {
    const void *p;
    size_t bytes;
};

Span mspan(const void *p, long long rows, long long cols, long long ld, size_t elem = 4) {
    if (!p || rows <= 0 || cols <= 0) return {p, 0};
    return {p, (size_t)(((rows - 1) * ld + cols) * (long long)elem)};
}

bool overlap(Span a, Span b) {
    if (!a.p || !b.p || a.bytes == 0 || b.bytes == 0) return false;
    auto x = reinterpret_cast<uintptr_t>(a.p), y = reinterpret_cast<uintptr_t>(b.p);
    return x < y + b.bytes && y < x + a.bytes;
}


ln_status check_form(ln_form form, ln_precision prec) {
    if (form != LN_FORM_PLAIN && form != LN_FORM_INTERNALIZED)
        return fail(LN_ERR_INVALID_VALUE, "unknown form %d", (int)form);
    if (prec < LN_PREC_FP32 || prec > LN_PREC_3XTF32) return fail(LN_ERR_INVALID_VALUE, "unknown precision %d", (int)prec);
    if (form == LN_FORM_PLAIN && prec != LN_PREC_FP32)
        return fail(LN_ERR_UNSUPPORTED, "the plain form computes in FP32 only (precision %d requested)", (int)prec);
    return LN_SUCCESS;
}

ln_status check_ws(void *ws, size_t have, size_t need) {
    if (need == 0) return LN_SUCCESS;
    if (!ws) return fail(LN_ERR_WORKSPACE, "workspace of %zu bytes required, got NULL", need);
    if (have < need) return fail(LN_ERR_WORKSPACE, "workspace of %zu bytes required, got %zu", need, have);
    if (reinterpret_cast<uintptr_t>(ws) & 255) return fail(LN_ERR_MISALIGNED, "workspace must be 256-byte aligned");
    return LN_SUCCESS;
}

#define LN_TRY(expr)                           \
    do {                                       \
        ln_status s_ = (expr);                 \
        if (s_ != LN_SUCCESS) return s_;       \
    } while (0)

inline bool tensor_prec(ln_precision p) { return prec_terms(p) > 0; }
inline cudaStream_t S(void *s) { return static_cast<cudaStream_t>(s); }

// ------------------------------------------------------------------ generic contraction
// out(i,j) <- epi( sum_k opA(i,k) * opB(k,j) ), M x N x K, with
//   opA(i,k) = A[i*lda+k] (a_t == 0) or A[k*lda+i] (a_t == 1)
//   opB(k,j) = B[k*ldb+j] (b_t == 0) or B[j*ldb+k] (b_t == 1)
struct Operand {
    const float *p;
    long long ld;
    int t;
};

// Tile geometry of a general (non-symmetric) tcgen05 contraction: mt row
// tiles of 128, nt column tiles of the engine's width, kt k tiles of 64; the
// packed N-side operand holds yrt = nt * width/128 row tiles (zero padded).
struct ContractPlan {
    char *px = nullptr, *py = nullptr;
    int mt = 0, nt = 0, kt = 0, yrt = 0, bn = 256;
    SplitPlan split;
};

void contract_geometry(int M, int N, int K, int P, ContractPlan &cp) {
    const int bn = umma_tile_n(P, 0, M, N);
    cp.bn = bn;
    cp.mt = (int)ceil_div(M, PK_ROWS);
    cp.nt = (int)ceil_div(N, bn);
    cp.kt = (int)ceil_div(K, PK_K);
    cp.yrt = cp.nt * (bn / PK_ROWS);
}

size_t contract_pack_bytes(const ContractPlan &cp, int P) {
    return align_up(packed_bytes(cp.mt, cp.kt, P), 256) + packed_bytes(cp.yrt, cp.kt, P);
}

void plan_contract(Ws &w, int M, int N, int K, ln_form form, ln_precision prec, ContractPlan &cp) {
    if (form != LN_FORM_INTERNALIZED || !tensor_prec(prec)) return;
    const int P = prec_terms(prec);
    contract_geometry(M, N, K, P, cp);
    cp.px = w.take<char>(packed_bytes(cp.mt, cp.kt, P));
    cp.py = w.take<char>(packed_bytes(cp.yrt, cp.kt, P));
    plan_split(w, (long long)cp.mt * cp.nt, cp.kt, cp.bn, cp.split);
}

ln_status run_contract(int M, int N, int K, Operand a, Operand b, const EpiParams &epi, ln_form form,
                       ln_precision prec, const ContractPlan &cp, cudaStream_t st) {
    if (M == 0 || N == 0) return LN_SUCCESS;
    if (form == LN_FORM_PLAIN || K == 0) {
        long long sai = a.t ? 1 : a.ld, sak = a.t ? a.ld : 1;
        long long sbk = b.t ? 1 : b.ld, sbj = b.t ? b.ld : 1;
        return plain_gemm(M, N, K, a.p, sai, sak, b.p, sbk, sbj, epi, st);
    }
    if (!tensor_prec(prec)) {
        SimtOperands op{};
        op.A[0] = op.A[1] = a.p;
        op.B[0] = op.B[1] = b.p;
        op.lda[0] = op.lda[1] = a.ld;
        op.ldb[0] = op.ldb[1] = b.ld;
        op.a_t = a.t;
        op.b_t = b.t;
        op.nseg = 1;
        return simt_contract(M, N, K, op, epi, st);
    }
    const int P = prec_terms(prec);
    PackSrc ps[2] = {{a.p, a.ld, a.t ? 1 : 0, M, K, nullptr, nullptr, cp.px, cp.mt, cp.kt},
                     {b.p, b.ld, b.t ? 0 : 1, N, K, nullptr, nullptr, cp.py, cp.yrt, cp.kt}};
    for (PackSrc &q : ps) q.tf32 = is_tf32(prec);
    LN_TRY(zero_streamk_flags(cp.split, st));
    LN_TRY(pack_operands(ps, 2, P, st));
    UmmaProblem pb{};
    pb.seg[0] = {cp.px, cp.py};
    pb.nseg = 1;
    pb.kt = cp.kt;
    pb.x_kt = cp.kt;
    pb.y_kt = cp.kt;
    pb.mt = cp.mt;
    pb.nt = cp.nt;
    pb.sym = 0;
    pb.chunk_kt = tune_chunk_kt();
    pb.tf32 = is_tf32(prec);
    pb.inject_timeout = inject_timeout_requested();
    apply_split(pb, cp.split);
    pb.bn = cp.bn;
    pb.epi = epi;
    return umma_contract(pb, P, st);
}

EpiParams epi_gemm(int M, int N, float alpha, float beta, float *C, long long ldc) {
    EpiParams e{};
    e.mode = EPI_GEMM;
    e.M = M;
    e.N = N;
    e.alpha = alpha;
    e.beta = beta;
    e.C = C;
    e.ldc = ldc;
    return e;
}

EpiParams epi_store(int M, int N, float alpha, float *C, long long ldc) {
    EpiParams e = epi_gemm(M, N, alpha, 0.0f, C, ldc);
    e.mode = EPI_STORE;
    return e;
}

// ------------------------------------------------------------------ chain
// FP32 forms keep T = A*B in FP32. The tensor-core form never materialises T
// in FP32: the first contraction's epilogue writes it straight into the packed
// split operand of the second (rows = ni, K = nj, k-tile pitch 2*ceil(nj/128)).
struct ChainPlan {
    float *T = nullptr;
    char *pa = nullptr, *pb = nullptr, *pt = nullptr, *pc = nullptr;
    ContractPlan g1, g2;
    int ktT = 0;
    SplitPlan s1, s2;
};

void plan_chain(Ws &w, int ni, int nj, int nk, int nl, ln_form form, ln_precision prec, ChainPlan &p) {
    if (form != LN_FORM_INTERNALIZED || !tensor_prec(prec)) {
        p.T = w.take<float>(sizeof(float) * (size_t)ni * nj);
        return;
    }
    const int P = prec_terms(prec);
    contract_geometry(ni, nj, nk, P, p.g1);
    contract_geometry(ni, nl, nj, P, p.g2);
    p.ktT = p.g1.yrt * (PK_ROWS / PK_K);  // the first contraction's column tiles, in k tiles of T
    p.pa = w.take<char>(packed_bytes(p.g1.mt, p.g1.kt, P));
    p.pb = w.take<char>(packed_bytes(p.g1.yrt, p.g1.kt, P));
    p.pt = w.take<char>(packed_bytes(p.g1.mt, p.ktT, P));
    p.pc = w.take<char>(packed_bytes(p.g2.yrt, p.g2.kt, P));
    plan_split(w, (long long)p.g1.mt * p.g1.nt, p.g1.kt, p.g1.bn, p.s1);
    plan_split(w, (long long)p.g2.mt * p.g2.nt, p.g2.kt, p.g2.bn, p.s2);
}

// ------------------------------------------------------------------ 3mm
// FP32 forms keep E = A B and F = C D in the workspace. Tensor-core forms: the
// first product's epilogue writes E as the packed row operand of G = E F; the
// second product computes F^T = D^T C^T, whose packing epilogue writes exactly
// the packed column operand of G (rows = G's columns, K = nj).
struct Mm3Plan {
    float *E = nullptr, *F = nullptr;
    char *pa = nullptr, *pb = nullptr, *pc = nullptr, *pd = nullptr, *pe = nullptr, *pf = nullptr;
    ContractPlan gE, gF, gG;  // E = A B; F^T = D^T C^T; G = E F
    int ktE = 0, ktF = 0, rowsF = 0;
    SplitPlan sE, sF, sG;
};

void plan_3mm(Ws &w, int ni, int nj, int nk, int nl, int nm, ln_form form, ln_precision prec, Mm3Plan &p) {
    if (form != LN_FORM_INTERNALIZED || !tensor_prec(prec)) {
        p.E = w.take<float>(sizeof(float) * (size_t)ni * nj);
        p.F = w.take<float>(sizeof(float) * (size_t)nj * nl);
        return;
    }
    const int P = prec_terms(prec);
    contract_geometry(ni, nj, nk, P, p.gE);
    contract_geometry(nl, nj, nm, P, p.gF);
    contract_geometry(ni, nl, nj, P, p.gG);
    p.ktE = p.gE.yrt * (PK_ROWS / PK_K);        // k tiles the first product writes (K of G = nj)
    p.ktF = p.gF.yrt * (PK_ROWS / PK_K);        // k tiles the second product writes
    p.rowsF = std::max(p.gF.mt, p.gG.yrt);      // G reads gG.yrt row tiles of F^T
    p.pa = w.take<char>(packed_bytes(p.gE.mt, p.gE.kt, P));
    p.pb = w.take<char>(packed_bytes(p.gE.yrt, p.gE.kt, P));
    p.pd = w.take<char>(packed_bytes(p.gF.mt, p.gF.kt, P));
    p.pc = w.take<char>(packed_bytes(p.gF.yrt, p.gF.kt, P));
    p.pe = w.take<char>(packed_bytes(p.gE.mt, p.ktE, P));
    p.pf = w.take<char>(packed_bytes(p.rowsF, p.ktF, P));
    plan_split(w, (long long)p.gE.mt * p.gE.nt, p.gE.kt, p.gE.bn, p.sE);
    plan_split(w, (long long)p.gF.mt * p.gF.nt, p.gF.kt, p.gF.bn, p.sF);
    plan_split(w, (long long)p.gG.mt * p.gG.nt, p.gG.kt, p.gG.bn, p.sG);
}

// ------------------------------------------------------------------ covariance / correlation
struct CovPlan {
    double *mean = nullptr, *ss = nullptr, *partials = nullptr;
    float *hi = nullptr, *lo = nullptr, *rs = nullptr;
    char *pack = nullptr;
    int mt = 0, kt = 0;
    int bn = 128, prt = 0;  // symmetric tile width, packed 128-row tiles
    SplitPlan split;
};

void plan_cov(Ws &w, int n, int m, ln_form form, ln_precision prec, CovPlan &p) {
    p.mean = w.take<double>(sizeof(double) * m);
    p.ss = w.take<double>(sizeof(double) * m);
    p.hi = w.take<float>(sizeof(float) * m);
    p.lo = w.take<float>(sizeof(float) * m);
    p.rs = w.take<float>(sizeof(float) * m);
    if (form == LN_FORM_INTERNALIZED) p.partials = w.take<double>(col_stats_partials_bytes(n, m));
    if (form == LN_FORM_INTERNALIZED && tensor_prec(prec)) {
        p.mt = (int)ceil_div(m, PK_ROWS);
        p.kt = (int)ceil_div(n, PK_K);
        p.bn = umma_sym_tile_n(prec_terms(prec), p.mt, p.kt);
        p.prt = sym_packed_rt(p.mt, p.bn);
        p.pack = w.take<char>(packed_bytes(p.prt, p.kt, prec_terms(prec)));
        plan_split(w, sym_tiles(p.mt, p.bn), p.kt, p.bn, p.split);
    }
}

// stats (nullable): 2*m doubles, mean then ss, written for the adjoint; the
// statistics passes then write there instead of into the workspace.
ln_status run_cov(bool corr, int n, int m, const float *X, int ldx, float *out, int ldo, double *stats, void *ws,
                  size_t wsb, ln_form form, ln_precision prec, cudaStream_t st) {
    LN_TRY(check_dims({n, m}));
    LN_TRY(check_form(form, prec));
    if (m == 0) return LN_SUCCESS;
    if (n < 2) return fail(LN_ERR_INVALID_VALUE, "covariance/correlation need nsamples >= 2 (got %d)", n);
    if (!X || !out) return fail(LN_ERR_INVALID_VALUE, "NULL X or output");
    if (ldx < m || ldo < m) return fail(LN_ERR_INVALID_VALUE, "leading dimension smaller than nfeat");
    if (overlap(mspan(out, m, m, ldo), mspan(X, n, m, ldx))) return fail(LN_ERR_ALIASING, "output overlaps X");
    if (stats) {
        const Span ss{stats, sizeof(double) * 2 * (size_t)m};
        if (overlap(ss, mspan(out, m, m, ldo)) || overlap(ss, mspan(X, n, m, ldx)))
            return fail(LN_ERR_ALIASING, "statistics overlap X or the output");
        if (reinterpret_cast<uintptr_t>(stats) & 7) return fail(LN_ERR_INVALID_VALUE, "statistics not 8-byte aligned");
    }
    Ws count(nullptr);
    CovPlan p;
    plan_cov(count, n, m, form, prec, p);
    LN_TRY(check_ws(ws, wsb, count.off));
    Ws w(ws);
    plan_cov(w, n, m, form, prec, p);
    if (stats) {
        p.mean = stats;
        p.ss = stats + m;
    }

    EpiParams e{};
    e.mode = EPI_SYM;
    e.M = e.N = m;
    e.C = out;
    e.ldc = ldo;
    e.fill = LN_FILL_FULL;
    e.sym_kind = corr ? SYM_CORR : SYM_SCALE;
    e.alpha = (float)(1.0 / (double)(n - 1));
    e.rs = p.rs;

    if (form == LN_FORM_PLAIN) {
        LN_TRY(plain_col_stats(n, m, X, ldx, p.mean, p.ss, st));
        LN_TRY(stats_derive(m, p.mean, p.ss, nullptr, nullptr, p.rs, st));
        return plain_cov(n, m, X, ldx, p.mean, e, st);
    }
    LN_TRY(zero_streamk_flags(p.split, st));
    // covariance centres with the means only; correlation, and a call that
    // returns the statistics, also need the second pass
    if (corr || stats) LN_TRY(col_stats(n, m, X, ldx, p.mean, p.ss, p.hi, p.lo, p.rs, p.partials, st));
    else LN_TRY(col_mean(n, m, X, ldx, p.mean, p.hi, p.lo, p.partials, st));
    if (!tensor_prec(prec)) {
        SimtOperands op{};
        op.A[0] = op.A[1] = X;
        op.B[0] = op.B[1] = X;
        op.lda[0] = op.lda[1] = ldx;
        op.ldb[0] = op.ldb[1] = ldx;
        op.a_t = 1;
        op.b_t = 0;
        op.nseg = 1;
        op.a_off_hi = op.b_off_hi = p.hi;
        op.a_off_lo = op.b_off_lo = p.lo;
        return simt_contract(m, m, n, op, e, st);
    }
    const int P = prec_terms(prec);
    PackSrc ps{X, ldx, 1, m, n, p.hi, p.lo, p.pack, p.prt, p.kt};
    ps.tf32 = is_tf32(prec);
    LN_TRY(pack_operand(ps, P, st));
    UmmaProblem pb{};
    pb.seg[0] = {p.pack, p.pack};
    pb.nseg = 1;
    pb.kt = p.kt;
    pb.x_kt = pb.y_kt = p.kt;
    pb.mt = p.mt;
    pb.nt = (int)ceil_div(p.mt * 128, p.bn);
    pb.bn = p.bn;
    pb.sym = 1;
    pb.chunk_kt = tune_chunk_kt();
    pb.tf32 = is_tf32(prec);
    apply_split(pb, p.split);
    pb.epi = e;
    return umma_contract(pb, P, st);
}

// ------------------------------------------------------------------ SYRK / SYR2K
struct SymPlan {
    char *pa = nullptr, *pb = nullptr;
    int mt = 0, kt = 0;
    int bn = 128, prt = 0;  // symmetric tile width, packed 128-row tiles
    SplitPlan split;
};

void plan_sym(Ws &w, bool two, int n, int k, ln_form form, ln_precision prec, SymPlan &p) {
    if (form != LN_FORM_INTERNALIZED || !tensor_prec(prec)) return;
    p.mt = (int)ceil_div(n, PK_ROWS);
    p.kt = (int)ceil_div(k, PK_K);
    const int ktot = (two ? 2 : 1) * p.kt;
    p.bn = umma_sym_tile_n(prec_terms(prec), p.mt, ktot);
    p.prt = sym_packed_rt(p.mt, p.bn);
    p.pa = w.take<char>(packed_bytes(p.prt, p.kt, prec_terms(prec)));
    if (two) p.pb = w.take<char>(packed_bytes(p.prt, p.kt, prec_terms(prec)));
    plan_split(w, sym_tiles(p.mt, p.bn), ktot, p.bn, p.split);
}

ln_status run_sym(bool two, ln_fill fill, int n, int k, float alpha, const float *A, int lda, const float *B, int ldb,
                  float beta, float *C, int ldc, void *ws, size_t wsb, ln_form form, ln_precision prec,
                  cudaStream_t st) {
    LN_TRY(check_dims({n, k}));
    LN_TRY(check_form(form, prec));
    if (fill != LN_FILL_FULL && fill != LN_FILL_LOWER && fill != LN_FILL_UPPER)
        return fail(LN_ERR_INVALID_VALUE, "unknown fill %d", (int)fill);
    if (n == 0) return LN_SUCCESS;
    if (!C || (k > 0 && (!A || (two && !B)))) return fail(LN_ERR_INVALID_VALUE, "NULL operand");
    if (ldc < n || (k > 0 && (lda < k || (two && ldb < k))))
        return fail(LN_ERR_INVALID_VALUE, "leading dimension too small");
    Span sc = mspan(C, n, n, ldc);
    if (overlap(sc, mspan(A, n, k, lda)) || (two && overlap(sc, mspan(B, n, k, ldb))))
        return fail(LN_ERR_ALIASING, "C overlaps an input");
    if (k == 0) return sym_fill_zero_k(n, fill, beta, C, ldc, st);
    Ws count(nullptr);
    SymPlan p;
    plan_sym(count, two, n, k, form, prec, p);
    LN_TRY(check_ws(ws, wsb, count.off));
    Ws w(ws);
    plan_sym(w, two, n, k, form, prec, p);

    EpiParams e{};
    e.mode = EPI_SYM;
    e.M = e.N = n;
    e.alpha = alpha;
    e.beta = beta;
    e.C = C;
    e.ldc = ldc;
    e.fill = fill;
    e.sym_kind = SYM_AXPBY;
    if (form == LN_FORM_PLAIN) return plain_sym(n, k, A, lda, two ? B : nullptr, ldb, e, st);
    if (!tensor_prec(prec)) {
        SimtOperands op{};
        op.a_t = 0;
        op.b_t = 1;
        op.nseg = two ? 2 : 1;
        op.A[0] = A;
        op.lda[0] = lda;
        op.B[0] = two ? B : A;
        op.ldb[0] = two ? ldb : lda;
        op.A[1] = op.B[0];
        op.lda[1] = op.ldb[0];
        op.B[1] = A;
        op.ldb[1] = lda;
        return simt_contract(n, n, k, op, e, st);
    }
    const int P = prec_terms(prec);
    PackSrc ps[2] = {{A, lda, 0, n, k, nullptr, nullptr, p.pa, p.prt, p.kt},
                     {B, ldb, 0, n, k, nullptr, nullptr, p.pb, p.prt, p.kt}};
    for (PackSrc &q : ps) q.tf32 = is_tf32(prec);
    LN_TRY(zero_streamk_flags(p.split, st));
    LN_TRY(pack_operands(ps, two ? 2 : 1, P, st));
    UmmaProblem pb{};
    if (two) {
        pb.seg[0] = {p.pa, p.pb};
        pb.seg[1] = {p.pb, p.pa};
        pb.nseg = 2;
    } else {
        pb.seg[0] = {p.pa, p.pa};
        pb.nseg = 1;
    }
    pb.kt = p.kt;
    pb.x_kt = pb.y_kt = p.kt;
    pb.mt = p.mt;
    pb.nt = (int)ceil_div(p.mt * 128, p.bn);
    pb.bn = p.bn;
    pb.sym = 1;
    pb.chunk_kt = tune_chunk_kt();
    pb.tf32 = is_tf32(prec);
    apply_split(pb, p.split);
    pb.epi = e;
    return umma_contract(pb, P, st);
}

// ------------------------------------------------------------------ batched
struct BatchPlan {
    UmmaProblem *probs = nullptr;
    int *tile_prefix = nullptr;
    long long *pack_off = nullptr;
    int *pack_prefix = nullptr;
    int *order = nullptr;
    int *tile_owner = nullptr;
    int *queue = nullptr;
    char *pack = nullptr;
    long long total_tiles = 0, total_pack_tiles = 0;
    int max_n = 0;
};

ln_status validate_batch(bool two, int count, const ln_sym_desc *h, BatchPlan &bp) {
    if (count < 0 || count > (1 << 20)) return fail(LN_ERR_INVALID_VALUE, "batch count %d out of range", count);
    if (count > 0 && !h) return fail(LN_ERR_INVALID_VALUE, "NULL host descriptor array");
    std::vector<Span> outs, ins;
    outs.reserve(count);
    for (int i = 0; i < count; ++i) {
        const ln_sym_desc &d = h[i];
        if (d.n < 0 || d.k < 0 || d.n > MAX_DIM || d.k > MAX_DIM)
            return fail(LN_ERR_INVALID_VALUE, "instance %d: size out of range", i);
        if (d.n == 0) continue;
        if (!d.C || (d.k > 0 && (!d.A || (two && !d.B))))
            return fail(LN_ERR_INVALID_VALUE, "instance %d: NULL operand", i);
        if (d.ldc < d.n || (d.k > 0 && (d.lda < d.k || (two && d.ldb < d.k))))
            return fail(LN_ERR_INVALID_VALUE, "instance %d: leading dimension too small", i);
        outs.push_back(mspan(d.C, d.n, d.n, d.ldc));
        ins.push_back(mspan(d.A, d.n, d.k, d.lda));
        if (two) ins.push_back(mspan(d.B, d.n, d.k, d.ldb));
        long long t = ceil_div(d.n, PK_ROWS);
        bp.total_tiles += t * (t + 1) / 2;
        bp.total_pack_tiles += t * ceil_div(d.k, PK_K) * (two ? 2 : 1);
        bp.max_n = std::max(bp.max_n, d.n);
    }
    auto by_addr = [](const Span &a, const Span &b) { return a.p < b.p; };
    std::sort(outs.begin(), outs.end(), by_addr);
    for (size_t i = 1; i < outs.size(); ++i)
        if (overlap(outs[i - 1], outs[i])) return fail(LN_ERR_ALIASING, "two instances' outputs overlap");
    std::sort(ins.begin(), ins.end(), by_addr);
    for (const Span &o : outs) {  // binary search the inputs around each output
        auto it = std::lower_bound(ins.begin(), ins.end(), o, by_addr);
        for (auto jt = (it == ins.begin() ? it : it - 1); jt != ins.end() && jt->p < (const char *)o.p + o.bytes; ++jt)
            if (overlap(o, *jt)) return fail(LN_ERR_ALIASING, "an instance's output overlaps an input");
        // inputs that start before o and reach into it
        for (auto jt = ins.begin(); jt != it; ++jt)
            if (overlap(o, *jt)) return fail(LN_ERR_ALIASING, "an instance's output overlaps an input");
    }
    if (bp.total_tiles > 0x7fffffffLL || bp.total_pack_tiles > 0x7fffffffLL)
        return fail(LN_ERR_INVALID_VALUE, "batch too large");
    return LN_SUCCESS;
}

size_t batch_pack_bytes(bool two, int count, const ln_sym_desc *h, int P) {
    size_t b = 0;
    for (int i = 0; i < count; ++i) {
        if (h[i].n == 0) continue;
        size_t one = packed_bytes(ceil_div(h[i].n, PK_ROWS), ceil_div(h[i].k, PK_K), P);
        b += one * (two ? 2 : 1);
    }
    return b;
}

void plan_batch(Ws &w, bool two, int count, const ln_sym_desc *h, ln_form form, ln_precision prec, BatchPlan &bp) {
    if (form != LN_FORM_INTERNALIZED) return;
    bp.tile_prefix = w.take<int>(sizeof(int) * (count + 1));
    if (!tensor_prec(prec)) return;
    bp.probs = w.take<UmmaProblem>(sizeof(UmmaProblem) * (size_t)std::max(count, 1));
    bp.pack_off = w.take<long long>(sizeof(long long) * 2 * (size_t)std::max(count, 1));
    bp.pack_prefix = w.take<int>(sizeof(int) * (count + 1));
    bp.order = w.take<int>(sizeof(int) * (size_t)std::max(count, 1));
    bp.tile_owner = w.take<int>(sizeof(int) * (size_t)std::max<long long>(bp.total_tiles, 1));
    bp.queue = w.take<int>(sizeof(int));
    bp.pack = w.take<char>(batch_pack_bytes(two, count, h, prec_terms(prec)));
}

ln_status run_batch(bool two, ln_fill fill, int count, const ln_sym_desc *h, const ln_sym_desc *d, float alpha,
                    float beta, void *ws, size_t wsb, ln_form form, ln_precision prec, cudaStream_t st) {
    LN_TRY(check_form(form, prec));
    if (fill != LN_FILL_FULL && fill != LN_FILL_LOWER && fill != LN_FILL_UPPER)
        return fail(LN_ERR_INVALID_VALUE, "unknown fill %d", (int)fill);
    BatchPlan bp;
    LN_TRY(validate_batch(two, count, h, bp));
    if (count == 0 || bp.max_n == 0) return LN_SUCCESS;
    if (!d) return fail(LN_ERR_INVALID_VALUE, "NULL device descriptor array");
    for (int i = 0; i < count; ++i)
        if (h[i].n > 0 && h[i].k == 0) {
            // k == 0 instances only scale C; not worth a special path in the batched kernels
            return fail(LN_ERR_UNSUPPORTED, "batched call with an instance of k == 0 (instance %d)", i);
        }
    Ws count_ws(nullptr);
    BatchPlan tmp = bp;
    plan_batch(count_ws, two, count, h, form, prec, tmp);
    LN_TRY(check_ws(ws, wsb, count_ws.off));
    Ws w(ws);
    plan_batch(w, two, count, h, form, prec, bp);
    if (form == LN_FORM_PLAIN) return plain_sym_batched(two, count, d, bp.max_n, fill, alpha, beta, st);
    if (!tensor_prec(prec)) {
        LN_TRY(simt_sym_batched_prefix(count, d, bp.tile_prefix, st));
        const long long tiles = simt_sym_batched_tiles(count, h);
        if (tiles > 0x7fffffffLL) return fail(LN_ERR_INVALID_VALUE, "batch too large");
        return simt_sym_batched(two, count, d, bp.tile_prefix, (int)tiles, fill, alpha, beta, st);
    }
    const int P = prec_terms(prec), tf = is_tf32(prec) ? 1 : 0;
    LN_TRY(sym_batched_plan(two, count, d, fill, alpha, beta, bp.probs, bp.tile_prefix, bp.tile_owner, bp.pack_off,
                            bp.pack_prefix, bp.order, bp.pack, P, tf, st));
    LN_TRY(sym_batched_pack(two, count, d, bp.pack_off, bp.pack_prefix, bp.order, (int)bp.total_pack_tiles, bp.pack,
                            P, tf, st));
    return umma_contract_batched(bp.probs, bp.tile_prefix, bp.tile_owner, (int)bp.total_tiles, bp.queue,
                                 mma_terms(prec), tf, st);
}

// ------------------------------------------------------------------ backward
struct ChainBwdPlan {
    float *BC = nullptr, *GCt = nullptr, *T = nullptr;
    ContractPlan c;  // sized for the largest of the contractions, reused in stream order
    SplitArea split;
    char *px2 = nullptr;  // the same again for the branch that may run on a second stream
    SplitArea split2;
};

void plan_chain_bwd(Ws &w, int ni, int nj, int nk, int nl, ln_form form, ln_precision prec, ChainBwdPlan &p) {
    p.BC = w.take<float>(sizeof(float) * (size_t)nk * nl);
    p.GCt = w.take<float>(sizeof(float) * (size_t)ni * nj);
    p.T = w.take<float>(sizeof(float) * (size_t)ni * nj);
    if (form == LN_FORM_INTERNALIZED && tensor_prec(prec)) {
        // contractions (M, N, K): BC (nk,nl,nj), dA (ni,nk,nl), GCt (ni,nj,nl), dB (nk,nj,ni), T (ni,nj,nk), dC (nj,nl,ni)
        const int P = prec_terms(prec);
        size_t best = 0;
        int dims[6][3] = {{nk, nl, nj}, {ni, nk, nl}, {ni, nj, nl}, {nk, nj, ni}, {ni, nj, nk}, {nj, nl, ni}};
        for (auto &d : dims) {
            ContractPlan g;
            contract_geometry(d[0], d[1], d[2], P, g);
            best = std::max(best, contract_pack_bytes(g, P));
        }
        p.c.px = w.take<char>(best);
        plan_split_area(w, dims, 6, P, p.split);
        p.px2 = w.take<char>(best);
        plan_split_area(w, dims, 6, P, p.split2);
    }
}

// Work items (output tiles x K slices) of one tensor-core contraction, the
// number of persistent CTAs it launches at most.
long long contract_work(int M, int N, int K, int P) {
    ContractPlan g;
    contract_geometry(M, N, K, P, g);
    const long long t = (long long)g.mt * g.nt;
    return t * umma_ksplit(t, g.kt);
}

ln_status contract_into(int M, int N, int K, Operand a, Operand b, const EpiParams &e, ln_form form, ln_precision prec,
                        char *pack_area, const SplitArea &split, cudaStream_t st) {
    ContractPlan cp;
    if (form == LN_FORM_INTERNALIZED && tensor_prec(prec)) {
        const int P = prec_terms(prec);
        contract_geometry(M, N, K, P, cp);
        cp.px = pack_area;
        cp.py = pack_area + align_up(packed_bytes(cp.mt, cp.kt, P), 256);
        cp.split.ksplit = umma_ksplit((long long)cp.mt * cp.nt, cp.kt);
        if (cp.split.ksplit > 1) {  // the area was planned for these dimensions
            cp.split.part = split.part;
            cp.split.cnt = split.cnt;
        }
    }
    return run_contract(M, N, K, a, b, e, form, prec, cp, st);
}

// E = A B and F = C D recomputed; dE = Gb F^T, dF = E^T Gb; then the four
// factor gradients. Contractions (M, N, K) in execution order:
constexpr int MM3_BWD_N = 8;
void mm3_bwd_dims(int ni, int nj, int nk, int nl, int nm, int (*d)[3]) {
    const int dims[MM3_BWD_N][3] = {{ni, nj, nk}, {nj, nl, nm}, {ni, nj, nl}, {nj, nl, ni},
                                    {ni, nk, nj}, {nk, nj, ni}, {nj, nm, nl}, {nm, nl, nj}};
    for (int i = 0; i < MM3_BWD_N; ++i)
        for (int q = 0; q < 3; ++q) d[i][q] = dims[i][q];
}

struct Mm3BwdPlan {
    float *E = nullptr, *F = nullptr, *dE = nullptr, *dF = nullptr;
    char *pack = nullptr;
    SplitArea split;
    char *pack2 = nullptr;  // the same again for the half that may run on a second stream
    SplitArea split2;
};

void plan_3mm_bwd(Ws &w, int ni, int nj, int nk, int nl, int nm, ln_form form, ln_precision prec, Mm3BwdPlan &p) {
    p.E = w.take<float>(sizeof(float) * (size_t)ni * nj);
    p.F = w.take<float>(sizeof(float) * (size_t)nj * nl);
    p.dE = w.take<float>(sizeof(float) * (size_t)ni * nj);
    p.dF = w.take<float>(sizeof(float) * (size_t)nj * nl);
    if (form == LN_FORM_INTERNALIZED && tensor_prec(prec)) {
        const int P = prec_terms(prec);
        int dims[MM3_BWD_N][3];
        mm3_bwd_dims(ni, nj, nk, nl, nm, dims);
        size_t best = 0;
        for (auto &d : dims) {
            ContractPlan g;
            contract_geometry(d[0], d[1], d[2], P, g);
            best = std::max(best, contract_pack_bytes(g, P));
        }
        p.pack = w.take<char>(best);
        plan_split_area(w, dims, MM3_BWD_N, P, p.split);
        p.pack2 = w.take<char>(best);
        plan_split_area(w, dims, MM3_BWD_N, P, p.split2);
    }
}

struct CovBwdPlan {
    double *mean = nullptr, *ss = nullptr, *partials = nullptr;
    float *hi = nullptr, *lo = nullptr, *rs = nullptr;
    float *Z = nullptr, *Ws_ = nullptr, *dZ = nullptr;
    char *pack = nullptr;
    SplitArea split;
};

void plan_cov_bwd(Ws &w, bool corr, int n, int m, ln_form form, ln_precision prec, CovBwdPlan &p) {
    p.mean = w.take<double>(sizeof(double) * m);
    p.ss = w.take<double>(sizeof(double) * m);
    p.hi = w.take<float>(sizeof(float) * m);
    p.lo = w.take<float>(sizeof(float) * m);
    p.rs = w.take<float>(sizeof(float) * m);
    p.partials = w.take<double>(std::max(col_stats_partials_bytes(n, m), corr_bwd_partials_bytes(n, m)));
    p.Z = w.take<float>(sizeof(float) * (size_t)n * m);
    p.Ws_ = w.take<float>(sizeof(float) * (size_t)m * m);
    if (corr) p.dZ = w.take<float>(sizeof(float) * (size_t)n * m);
    if (form == LN_FORM_INTERNALIZED && tensor_prec(prec)) {
        const int P = prec_terms(prec);
        ContractPlan g;
        contract_geometry(n, m, m, P, g);
        p.pack = w.take<char>(contract_pack_bytes(g, P));
        const int dims[1][3] = {{n, m, m}};
        plan_split_area(w, dims, 1, P, p.split);
    }
}

ln_status run_cov_bwd(bool corr, int n, int m, const float *X, int ldx, const float *W, int ldw, const double *stats,
                      float *dX, int lddx, void *ws, size_t wsb, ln_form form, ln_precision prec, cudaStream_t st) {
    LN_TRY(check_dims({n, m}));
    LN_TRY(check_form(form, prec));
    if (m == 0 || n == 0) return LN_SUCCESS;
    if (n < 2) return fail(LN_ERR_INVALID_VALUE, "nsamples >= 2 required (got %d)", n);
    if (!X || !W || !dX) return fail(LN_ERR_INVALID_VALUE, "NULL operand");
    if (ldx < m || ldw < m || lddx < m) return fail(LN_ERR_INVALID_VALUE, "leading dimension too small");
    Span so = mspan(dX, n, m, lddx);
    if (overlap(so, mspan(X, n, m, ldx)) || overlap(so, mspan(W, m, m, ldw)) ||
        (stats && overlap(so, {stats, sizeof(double) * 2 * (size_t)m})))
        return fail(LN_ERR_ALIASING, "dX overlaps an input");
    Ws count(nullptr);
    CovBwdPlan p;
    plan_cov_bwd(count, corr, n, m, form, prec, p);
    LN_TRY(check_ws(ws, wsb, count.off));
    Ws w(ws);
    plan_cov_bwd(w, corr, n, m, form, prec, p);

    if (stats) {
        LN_TRY(stats_derive(m, stats, stats + m, p.hi, p.lo, p.rs, st));
    } else if (form == LN_FORM_PLAIN) {
        LN_TRY(plain_col_stats(n, m, X, ldx, p.mean, p.ss, st));
        LN_TRY(stats_derive(m, p.mean, p.ss, p.hi, p.lo, p.rs, st));
    } else {
        LN_TRY(col_stats(n, m, X, ldx, p.mean, p.ss, p.hi, p.lo, p.rs, p.partials, st));
    }
    // Z = Xc (covariance) or Xc * diag(1/s) (correlation), recomputed from X
    LN_TRY(center_matrix(n, m, X, ldx, p.hi, p.lo, corr ? p.rs : nullptr, p.Z, m, st));
    LN_TRY(symmetrize_weights(m, W, ldw, corr ? 1.0f : (float)(1.0 / (double)(n - 1)), corr ? 1 : 0, p.Ws_, st));
    Operand z{p.Z, m, 0}, wsop{p.Ws_, m, 0};
    if (!corr) return contract_into(n, m, m, z, wsop, epi_store(n, m, 1.0f, dX, lddx), form, prec, p.pack, p.split, st);
    LN_TRY(contract_into(n, m, m, z, wsop, epi_store(n, m, 1.0f, p.dZ, m), form, prec, p.pack, p.split, st));
    return corr_bwd_finish(n, m, p.Z, m, p.dZ, m, p.rs, dX, lddx, p.partials, st);
}

}  // namespace

}  // namespace ln

// ====================================================================== C ABI
using namespace ln;

extern "C" {

const char *ln_get_last_error(void) { return g_msg; }

const char *ln_status_string(ln_status s) {
    switch (s) {
        case LN_SUCCESS: return "LN_SUCCESS";
        case LN_ERR_INVALID_VALUE: return "LN_ERR_INVALID_VALUE";
        case LN_ERR_ALIASING: return "LN_ERR_ALIASING";
        case LN_ERR_MISALIGNED: return "LN_ERR_MISALIGNED";
        case LN_ERR_UNSUPPORTED: return "LN_ERR_UNSUPPORTED";
        case LN_ERR_CUDA: return "LN_ERR_CUDA";
        case LN_ERR_TIMEOUT: return "LN_ERR_TIMEOUT";
        case LN_ERR_WORKSPACE: return "LN_ERR_WORKSPACE";
    }
    return "LN_UNKNOWN_STATUS";
}

int ln_version(void) { return 100; }

long long ln_launch_count(void) { return g_launches.load(); }

ln_status ln_set_tuning(const char *key, int value) {
    clear_error();
    if (!key) return fail(LN_ERR_INVALID_VALUE, "NULL key");
    if (strcmp(key, "chunk_kt") == 0) {
        if (value != 1 && value != 2) return fail(LN_ERR_INVALID_VALUE, "chunk_kt must be 1 or 2 (got %d)", value);
        g_chunk_kt.store(value);
        return LN_SUCCESS;
    }
    if (strcmp(key, "tile_n") == 0) {
        if (value != 0 && value != 128 && value != 256)
            return fail(LN_ERR_INVALID_VALUE, "tile_n must be 0 (automatic), 128 or 256 (got %d)", value);
        g_tile_n.store(value);
        return LN_SUCCESS;
    }
    if (strcmp(key, "split_k") == 0) {
        if (value != 0 && value != 1) return fail(LN_ERR_INVALID_VALUE, "split_k must be 0 or 1 (got %d)", value);
        g_split_k.store(value);
        return LN_SUCCESS;
    }
    if (strcmp(key, "simt_exact") == 0) {
        if (value != 0 && value != 1) return fail(LN_ERR_INVALID_VALUE, "simt_exact must be 0 or 1 (got %d)", value);
        g_simt_exact.store(value);
        return LN_SUCCESS;
    }
    if (strcmp(key, "stage_beta") == 0) {
        if (value != 0 && value != 1) return fail(LN_ERR_INVALID_VALUE, "stage_beta must be 0 or 1 (got %d)", value);
        g_stage_beta.store(value);
        return LN_SUCCESS;
    }
    if (strcmp(key, "simt_tile") == 0) {
        if (value != 0 && value != 64 && value != 128)
            return fail(LN_ERR_INVALID_VALUE, "simt_tile must be 0 (automatic), 64 or 128 (got %d)", value);
        g_simt_tile.store(value);
        return LN_SUCCESS;
    }
    if (strcmp(key, "stage_out") == 0) {
        if (value != 0 && value != 1) return fail(LN_ERR_INVALID_VALUE, "stage_out must be 0 or 1 (got %d)", value);
        g_stage_out.store(value);
        return LN_SUCCESS;
    }
    if (strcmp(key, "sym_wide") == 0) {
        if (value < 0 || value > 2) return fail(LN_ERR_INVALID_VALUE, "sym_wide must be 0, 1 or 2 (got %d)", value);
        g_sym_wide.store(value);
        return LN_SUCCESS;
    }
    if (strcmp(key, "pair") == 0) {
        if (value < 0 || value > 2) return fail(LN_ERR_INVALID_VALUE, "pair must be 0, 1 or 2 (got %d)", value);
        g_pair.store(value);
        return LN_SUCCESS;
    }
    if (strcmp(key, "stream_k") == 0) {
        if (value < 0 || value > 2) return fail(LN_ERR_INVALID_VALUE, "stream_k must be 0, 1 or 2 (got %d)", value);
        g_stream_k.store(value);
        return LN_SUCCESS;
    }
    if (strcmp(key, "gs_rows") == 0) {
        if (value != 2 && value != 4) return fail(LN_ERR_INVALID_VALUE, "gs_rows must be 2 or 4 (got %d)", value);
        g_gs_rows.store(value);
        return LN_SUCCESS;
    }
    if (strcmp(key, "pack_threads") == 0) {
        if (value != 512 && value != 1024)
            return fail(LN_ERR_INVALID_VALUE, "pack_threads must be 512 or 1024 (got %d)", value);
        g_pack_threads.store(value);
        return LN_SUCCESS;
    }
    return fail(LN_ERR_INVALID_VALUE, "unknown tuning key '%s'", key);
}

ln_status ln_get_tuning(const char *key, int *value) {
    clear_error();
    if (!key || !value) return fail(LN_ERR_INVALID_VALUE, "NULL argument");
    if (strcmp(key, "chunk_kt") == 0) *value = g_chunk_kt.load();
    else if (strcmp(key, "tile_n") == 0) *value = g_tile_n.load();
    else if (strcmp(key, "pack_threads") == 0) *value = g_pack_threads.load();
    else if (strcmp(key, "split_k") == 0) *value = g_split_k.load();
    else if (strcmp(key, "gs_rows") == 0) *value = g_gs_rows.load();
    else if (strcmp(key, "stream_k") == 0) *value = g_stream_k.load();
    else if (strcmp(key, "pair") == 0) *value = g_pair.load();
    else if (strcmp(key, "stage_beta") == 0) *value = g_stage_beta.load();
    else if (strcmp(key, "stage_out") == 0) *value = g_stage_out.load();
    else if (strcmp(key, "simt_tile") == 0) *value = g_simt_tile.load();
    else if (strcmp(key, "sym_wide") == 0) *value = g_sym_wide.load();
    else if (strcmp(key, "simt_exact") == 0) *value = g_simt_exact.load();
    else return fail(LN_ERR_INVALID_VALUE, "unknown tuning key '%s'", key);
    return LN_SUCCESS;
}

ln_status ln_timing_enable(int on) {
    clear_error();
    if (on < 0 || on > 2) return fail(LN_ERR_INVALID_VALUE, "timing mode must be 0, 1 or 2 (got %d)", on);
    close_span();
    g_timing.mode = on;
    return LN_SUCCESS;
}

ln_status ln_timing_read(const char *family, double *total_ms, int *launches) {
    clear_error();
    if (!family || !total_ms || !launches) return fail(LN_ERR_INVALID_VALUE, "NULL argument");
    int f = -1;
    for (int i = 0; i < FAM_COUNT; ++i)
        if (strcmp(family, kFamilies[i]) == 0) f = i;
    if (f < 0) return fail(LN_ERR_INVALID_VALUE, "unknown kernel family '%s'", family);
    double total = 0.0;
    int n = 0;
    close_span();
    for (auto &r : g_timing.pending[f]) {
        LN_CUDA_TRY(cudaEventSynchronize(r.stop));
        float ms = 0.0f;
        LN_CUDA_TRY(cudaEventElapsedTime(&ms, r.start, r.stop));
        total += ms;
        n += r.launches;
        g_timing.pool.push_back(r);
    }
    g_timing.pending[f].clear();
    *total_ms = total;
    *launches = n;
    return LN_SUCCESS;
}

ln_status ln_stream_check(void *stream) {
    clear_error();
    cudaError_t e = cudaStreamSynchronize(S(stream));
    if (e != cudaSuccess) return fail(LN_ERR_CUDA, "stream error: %s", cudaGetErrorString(e));
    int v = 0;
    LN_TRY(umma_read_error(&v));
    if (v) return fail(LN_ERR_TIMEOUT, "a bounded device wait ran out (roles 0x%x)", v);
    return LN_SUCCESS;
}

// ------------------------------------------------------------------ GEMM
ln_status ln_gemm_workspace_size(int M, int N, int K, ln_form form, ln_precision prec, size_t *bytes) {
    clear_error();
    LN_TRY(check_dims({M, N, K}));
    LN_TRY(check_form(form, prec));
    if (!bytes) return fail(LN_ERR_INVALID_VALUE, "NULL bytes");
    Ws w(nullptr);
    ContractPlan cp;
    plan_contract(w, M, N, K, form, prec, cp);
    *bytes = w.off;
    return LN_SUCCESS;
}

ln_status ln_gemm(int M, int N, int K, float alpha, const float *A, int lda, const float *B, int ldb, float beta,
                  float *C, int ldc, void *ws, size_t wsb, ln_form form, ln_precision prec, void *stream) {
    clear_error();
    LN_TRY(check_dims({M, N, K}));
    LN_TRY(check_form(form, prec));
    if (M == 0 || N == 0) return LN_SUCCESS;
    if (!C || (K > 0 && (!A || !B))) return fail(LN_ERR_INVALID_VALUE, "NULL operand");
    if (ldc < N || (K > 0 && (lda < K || ldb < N))) return fail(LN_ERR_INVALID_VALUE, "leading dimension too small");
    Span sc = mspan(C, M, N, ldc);
    if (overlap(sc, mspan(A, M, K, lda)) || overlap(sc, mspan(B, K, N, ldb)))
        return fail(LN_ERR_ALIASING, "C overlaps A or B");
    if (K == 0) return scale_matrix(M, N, beta, C, ldc, S(stream));
    Ws count(nullptr);
    ContractPlan cp;
    plan_contract(count, M, N, K, form, prec, cp);
    LN_TRY(check_ws(ws, wsb, count.off));
    Ws w(ws);
    plan_contract(w, M, N, K, form, prec, cp);
    return run_contract(M, N, K, {A, lda, 0}, {B, ldb, 0}, epi_gemm(M, N, alpha, beta, C, ldc), form, prec, cp,
                        S(stream));
}

// ------------------------------------------------------------------ chain
ln_status ln_gemm_chain_workspace_size(int ni, int nj, int nk, int nl, ln_form form, ln_precision prec,
                                       size_t *bytes) {
    clear_error();
    LN_TRY(check_dims({ni, nj, nk, nl}));
    LN_TRY(check_form(form, prec));
    if (!bytes) return fail(LN_ERR_INVALID_VALUE, "NULL bytes");
    Ws w(nullptr);
    ChainPlan p;
    plan_chain(w, ni, nj, nk, nl, form, prec, p);
    *bytes = w.off;
    return LN_SUCCESS;
}

ln_status ln_gemm_chain(int ni, int nj, int nk, int nl, float alpha, const float *A, const float *B, const float *C,
                        float beta, const float *D, float *E, float *F, void *ws, size_t wsb, ln_form form,
                        ln_precision prec, void *stream) {
    clear_error();
    LN_TRY(check_dims({ni, nj, nk, nl}));
    LN_TRY(check_form(form, prec));
    if (ni == 0 || nl == 0) return LN_SUCCESS;
    if (!E || !F || (nk > 0 && nj > 0 && (!A || !B || !C)) || (beta != 0.0f && !D))
        return fail(LN_ERR_INVALID_VALUE, "NULL operand");
    Span se = mspan(E, ni, nl, nl), sf = mspan(F, ni, nl, nl);
    Span ins[4] = {mspan(A, ni, nk, nk), mspan(B, nk, nj, nj), mspan(C, nj, nl, nl),
                   mspan(beta != 0.0f ? D : nullptr, ni, nl, nl)};
    if (overlap(se, sf)) return fail(LN_ERR_ALIASING, "E overlaps F");
    for (const Span &s : ins)
        if (overlap(se, s) || overlap(sf, s)) return fail(LN_ERR_ALIASING, "E or F overlaps an input");
    // operands may live in host memory the GPU can reach (see device_view)
    LN_TRY(device_view(A, &A, "A"));
    LN_TRY(device_view(B, &B, "B"));
    LN_TRY(device_view(C, &C, "C"));
    LN_TRY(device_view(D, &D, "D"));
    LN_TRY(device_view(E, &E, "E"));
    LN_TRY(device_view(F, &F, "F"));
    cudaStream_t st = S(stream);
    EpiParams ef{};
    ef.mode = EPI_EF;
    ef.M = ni;
    ef.N = nl;
    ef.alpha = alpha;
    ef.beta = beta;
    ef.D = D;
    ef.E = E;
    ef.F = F;
    ef.ld_ef = nl;
    if (nk == 0 || nj == 0)  // T = 0, so E = 0 and F = beta * D
        return plain_gemm(ni, nl, 0, nullptr, 0, 0, nullptr, 0, 0, ef, st);
    Ws count(nullptr);
    ChainPlan p;
    plan_chain(count, ni, nj, nk, nl, form, prec, p);
    LN_TRY(check_ws(ws, wsb, count.off));
    Ws w(ws);
    plan_chain(w, ni, nj, nk, nl, form, prec, p);
    if (p.T) {
        ContractPlan none;
        LN_TRY(run_contract(ni, nj, nk, {A, nk, 0}, {B, nj, 0}, epi_store(ni, nj, 1.0f, p.T, nj), form, prec, none, st));
        return run_contract(ni, nl, nj, {p.T, nj, 0}, {C, nl, 0}, ef, form, prec, none, st);
    }
    const int P = prec_terms(prec);
    PackSrc ps[3] = {{A, nk, 0, ni, nk, nullptr, nullptr, p.pa, p.g1.mt, p.g1.kt},
                     {B, nj, 1, nj, nk, nullptr, nullptr, p.pb, p.g1.yrt, p.g1.kt},
                     {C, nl, 1, nl, nj, nullptr, nullptr, p.pc, p.g2.yrt, p.g2.kt}};
    for (PackSrc &q : ps) q.tf32 = is_tf32(prec);
    // C is packed by the first contraction's spare CTAs when it has fewer
    // output tiles than SMs (and no stream-K, which gives every SM mainloop
    // work), else here with A and B
    PackMulti side;
    const bool try_side = p.g1.bn == 256 && !p.s1.streamk && make_pack_multi(ps + 2, 1, side) &&
                          pack_stream_eligible(side);
    LN_TRY(zero_streamk_flags(p.s1, st));
    LN_TRY(zero_streamk_flags(p.s2, st));
    LN_TRY(pack_operands(ps, try_side ? 2 : 3, P, st));
    UmmaProblem g1{};
    g1.seg[0] = {p.pa, p.pb};
    g1.nseg = 1;
    g1.kt = p.g1.kt;
    g1.x_kt = g1.y_kt = p.g1.kt;
    g1.mt = p.g1.mt;
    g1.nt = p.g1.nt;
    g1.chunk_kt = tune_chunk_kt();
    g1.tf32 = is_tf32(prec);
    g1.inject_timeout = inject_timeout_requested();
    g1.epi.mode = EPI_PACK;
    g1.epi.M = ni;
    g1.epi.N = nj;
    g1.epi.pack = p.pt;
    g1.epi.pack_kt = p.ktT;
    apply_split(g1, p.s1);
    g1.bn = p.g1.bn;
    bool side_done = false;
    SpanHold hold;  // GEMM2 follows GEMM1 on this stream with programmatic overlap
    LN_TRY(umma_contract(g1, P, st, try_side ? &side : nullptr, &side_done));
    if (try_side && !side_done) LN_TRY(pack_operands(ps + 2, 1, P, st));
    UmmaProblem g2{};
    g2.seg[0] = {p.pt, p.pc};
    g2.nseg = 1;
    g2.kt = p.g2.kt;
    g2.x_kt = p.ktT;
    g2.y_kt = p.g2.kt;
    g2.mt = p.g2.mt;
    g2.nt = p.g2.nt;
    g2.chunk_kt = tune_chunk_kt();
    g2.tf32 = is_tf32(prec);
    g2.inject_timeout = g1.inject_timeout;
    apply_split(g2, p.s2);
    g2.bn = p.g2.bn;
    g2.epi = ef;
    return umma_contract(g2, P, st);
}

// ------------------------------------------------------------------ 3mm
ln_status ln_3mm_workspace_size(int ni, int nj, int nk, int nl, int nm, ln_form form, ln_precision prec,
                                size_t *bytes) {
    clear_error();
    LN_TRY(check_dims({ni, nj, nk, nl, nm}));
    LN_TRY(check_form(form, prec));
    if (!bytes) return fail(LN_ERR_INVALID_VALUE, "NULL bytes");
    Ws w(nullptr);
    Mm3Plan p;
    plan_3mm(w, ni, nj, nk, nl, nm, form, prec, p);
    *bytes = w.off;
    return LN_SUCCESS;
}

ln_status ln_3mm(int ni, int nj, int nk, int nl, int nm, const float *A, const float *B, const float *C,
                 const float *D, float *G, void *ws, size_t wsb, ln_form form, ln_precision prec, void *stream) {
    clear_error();
    LN_TRY(check_dims({ni, nj, nk, nl, nm}));
    LN_TRY(check_form(form, prec));
    if (ni == 0 || nl == 0) return LN_SUCCESS;
    const bool zero = nj == 0 || nk == 0 || nm == 0;  // E or F is empty: G = 0
    if (!G || (!zero && (!A || !B || !C || !D))) return fail(LN_ERR_INVALID_VALUE, "NULL operand");
    const Span sg = mspan(G, ni, nl, nl);
    const Span ins[4] = {mspan(A, ni, nk, nk), mspan(B, nk, nj, nj), mspan(C, nj, nm, nm), mspan(D, nm, nl, nl)};
    for (const Span &x : ins)
        if (!zero && overlap(sg, x)) return fail(LN_ERR_ALIASING, "G overlaps an input");
    LN_TRY(device_view(A, &A, "A"));
    LN_TRY(device_view(B, &B, "B"));
    LN_TRY(device_view(C, &C, "C"));
    LN_TRY(device_view(D, &D, "D"));
    LN_TRY(device_view(G, &G, "G"));
    cudaStream_t st = S(stream);
    const EpiParams eg = epi_store(ni, nl, 1.0f, G, nl);
    if (zero) return plain_gemm(ni, nl, 0, nullptr, 0, 0, nullptr, 0, 0, eg, st);
    Ws count(nullptr);
    Mm3Plan p;
    plan_3mm(count, ni, nj, nk, nl, nm, form, prec, p);
    LN_TRY(check_ws(ws, wsb, count.off));
    Ws w(ws);
    plan_3mm(w, ni, nj, nk, nl, nm, form, prec, p);
    if (p.E) {
        ContractPlan none;
        LN_TRY(run_contract(ni, nj, nk, {A, nk, 0}, {B, nj, 0}, epi_store(ni, nj, 1.0f, p.E, nj), form, prec, none,
                            st));
        LN_TRY(run_contract(nj, nl, nm, {C, nm, 0}, {D, nl, 0}, epi_store(nj, nl, 1.0f, p.F, nl), form, prec, none,
                            st));
        return run_contract(ni, nl, nj, {p.E, nj, 0}, {p.F, nl, 0}, eg, form, prec, none, st);
    }
    const int P = prec_terms(prec);
    // E = A B: rows of A, columns of B (B^T K-major); F^T = D^T C^T: rows of
    // D^T (D transposed), columns of C^T = rows of C (K = nm contiguous)
    PackSrc ps[4] = {{A, nk, 0, ni, nk, nullptr, nullptr, p.pa, p.gE.mt, p.gE.kt},
                     {B, nj, 1, nj, nk, nullptr, nullptr, p.pb, p.gE.yrt, p.gE.kt},
                     {D, nl, 1, nl, nm, nullptr, nullptr, p.pd, p.gF.mt, p.gF.kt},
                     {C, nm, 0, nj, nm, nullptr, nullptr, p.pc, p.gF.yrt, p.gF.kt}};
    for (PackSrc &q : ps) q.tf32 = is_tf32(prec);
    PackMulti side;
    const bool try_side = p.gE.bn == 256 && !p.sE.streamk && make_pack_multi(ps + 2, 2, side) &&
                          pack_stream_eligible(side);
    LN_TRY(zero_streamk_flags(p.sE, st));
    LN_TRY(zero_streamk_flags(p.sF, st));
    LN_TRY(zero_streamk_flags(p.sG, st));
    LN_TRY(pack_operands(ps, try_side ? 2 : 4, P, st));
    UmmaProblem gE{};
    gE.seg[0] = {p.pa, p.pb};
    gE.nseg = 1;
    gE.kt = p.gE.kt;
    gE.x_kt = gE.y_kt = p.gE.kt;
    gE.mt = p.gE.mt;
    gE.nt = p.gE.nt;
    gE.chunk_kt = tune_chunk_kt();
    gE.tf32 = is_tf32(prec);
    gE.inject_timeout = inject_timeout_requested();
    apply_split(gE, p.sE);
    gE.bn = p.gE.bn;
    gE.epi.mode = EPI_PACK;
    gE.epi.M = ni;
    gE.epi.N = nj;
    gE.epi.pack = p.pe;
    gE.epi.pack_kt = p.ktE;
    UmmaProblem gF{};
    gF.seg[0] = {p.pd, p.pc};
    gF.nseg = 1;
    gF.kt = p.gF.kt;
    gF.x_kt = gF.y_kt = p.gF.kt;
    gF.mt = p.gF.mt;
    gF.nt = p.gF.nt;
    gF.chunk_kt = tune_chunk_kt();
    gF.tf32 = is_tf32(prec);
    gF.inject_timeout = gE.inject_timeout;
    apply_split(gF, p.sF);
    gF.bn = p.gF.bn;
    gF.epi.mode = EPI_PACK;
    gF.epi.M = nl;
    gF.epi.N = nj;
    gF.epi.pack = p.pf;
    gF.epi.pack_kt = p.ktF;
    // E and F are independent: when both fit on the GPU at once (one
    // persistent CTA per work item) F runs on a second stream beside E, then
    // without stream-K (a stream-K launch needs all its CTAs on the GPU at once)
    const long long wE = (long long)gE.mt * gE.nt * (gE.ksplit > 1 ? gE.ksplit : 1);
    const long long wF = (long long)gF.mt * gF.nt * (gF.ksplit > 1 ? gF.ksplit : 1);
    SideStream *ss = (!try_side && wE + wF <= sm_count()) ? side_stream(st) : nullptr;
    if (ss) gE.streamk = gF.streamk = 0;
    if (ss) {
        LN_CUDA_TRY(cudaEventRecord(ss->fork, st));
        LN_CUDA_TRY(cudaStreamWaitEvent(ss->s, ss->fork, 0));
        const ln_status sf = umma_contract(gF, P, ss->s);
        LN_CUDA_TRY(cudaEventRecord(ss->join, ss->s));  // joined below even if F failed to launch
        LN_TRY(umma_contract(gE, P, st));
        LN_CUDA_TRY(cudaStreamWaitEvent(st, ss->join, 0));
        LN_TRY(sf);
    } else {
        bool side_done = false;
        LN_TRY(umma_contract(gE, P, st, try_side ? &side : nullptr, &side_done));
        if (try_side && !side_done) LN_TRY(pack_operands(ps + 2, 2, P, st));
        LN_TRY(umma_contract(gF, P, st));
    }
    if (p.rowsF > p.gF.mt)  // row tiles of F^T that G reads but no product writes
        LN_CUDA_TRY(cudaMemsetAsync(p.pf + packed_bytes(p.gF.mt, p.ktF, P), 0,
                                    packed_bytes(p.rowsF - p.gF.mt, p.ktF, P), st));
    UmmaProblem gG{};
    gG.seg[0] = {p.pe, p.pf};
    gG.nseg = 1;
    gG.kt = p.gG.kt;
    gG.x_kt = p.ktE;
    gG.y_kt = p.ktF;
    gG.mt = p.gG.mt;
    gG.nt = p.gG.nt;
    gG.chunk_kt = tune_chunk_kt();
    gG.tf32 = is_tf32(prec);
    gG.inject_timeout = gE.inject_timeout;
    apply_split(gG, p.sG);
    gG.bn = p.gG.bn;
    gG.epi = eg;
    return umma_contract(gG, P, st);
}

ln_status ln_3mm_bwd_workspace_size(int ni, int nj, int nk, int nl, int nm, ln_form form, ln_precision prec,
                                    size_t *bytes) {
    clear_error();
    LN_TRY(check_dims({ni, nj, nk, nl, nm}));
    LN_TRY(check_form(form, prec));
    if (!bytes) return fail(LN_ERR_INVALID_VALUE, "NULL bytes");
    Ws w(nullptr);
    Mm3BwdPlan p;
    plan_3mm_bwd(w, ni, nj, nk, nl, nm, form, prec, p);
    *bytes = w.off;
    return LN_SUCCESS;
}

ln_status ln_3mm_bwd(int ni, int nj, int nk, int nl, int nm, const float *A, const float *B, const float *C,
                     const float *D, const float *Gb, float *dA, float *dB, float *dC, float *dD, void *ws,
                     size_t wsb, ln_form form, ln_precision prec, void *stream) {
    clear_error();
    LN_TRY(check_dims({ni, nj, nk, nl, nm}));
    LN_TRY(check_form(form, prec));
    if (!A || !B || !C || !D || !Gb || !dA || !dB || !dC || !dD) return fail(LN_ERR_INVALID_VALUE, "NULL operand");
    const Span outs[4] = {mspan(dA, ni, nk, nk), mspan(dB, nk, nj, nj), mspan(dC, nj, nm, nm), mspan(dD, nm, nl, nl)};
    const Span ins[5] = {mspan(A, ni, nk, nk), mspan(B, nk, nj, nj), mspan(C, nj, nm, nm), mspan(D, nm, nl, nl),
                         mspan(Gb, ni, nl, nl)};
    for (int i = 0; i < 4; ++i) {
        for (int j = i + 1; j < 4; ++j)
            if (overlap(outs[i], outs[j])) return fail(LN_ERR_ALIASING, "gradient outputs overlap");
        for (const Span &x : ins)
            if (overlap(outs[i], x)) return fail(LN_ERR_ALIASING, "a gradient output overlaps an input");
    }
    Ws count(nullptr);
    Mm3BwdPlan p;
    plan_3mm_bwd(count, ni, nj, nk, nl, nm, form, prec, p);
    LN_TRY(check_ws(ws, wsb, count.off));
    Ws w(ws);
    plan_3mm_bwd(w, ni, nj, nk, nl, nm, form, prec, p);
    cudaStream_t st = S(stream);
    // Operand {p, ld, t}: t = 1 reads the stored matrix transposed. Two halves:
    // E = A B, then (with F) dE = Gb F^T, dA = dE B^T, dB = A^T dE; and
    // F = C D, then (with E) dF = E^T Gb, dC = dF D^T, dD = C^T dF.
    auto prod_E = [&](char *pk, const SplitArea &sa, cudaStream_t s) {
        return contract_into(ni, nj, nk, {A, nk, 0}, {B, nj, 0}, epi_store(ni, nj, 1.0f, p.E, nj), form, prec, pk, sa,
                             s);
    };
    auto prod_F = [&](char *pk, const SplitArea &sa, cudaStream_t s) {
        return contract_into(nj, nl, nm, {C, nm, 0}, {D, nl, 0}, epi_store(nj, nl, 1.0f, p.F, nl), form, prec, pk, sa,
                             s);
    };
    auto grads_AB = [&](char *pk, const SplitArea &sa, cudaStream_t s) -> ln_status {
        LN_TRY(contract_into(ni, nj, nl, {Gb, nl, 0}, {p.F, nl, 1}, epi_store(ni, nj, 1.0f, p.dE, nj), form, prec, pk,
                             sa, s));
        LN_TRY(contract_into(ni, nk, nj, {p.dE, nj, 0}, {B, nj, 1}, epi_store(ni, nk, 1.0f, dA, nk), form, prec, pk,
                             sa, s));
        return contract_into(nk, nj, ni, {A, nk, 1}, {p.dE, nj, 0}, epi_store(nk, nj, 1.0f, dB, nj), form, prec, pk,
                             sa, s);
    };
    auto grads_CD = [&](char *pk, const SplitArea &sa, cudaStream_t s) -> ln_status {
        LN_TRY(contract_into(nj, nl, ni, {p.E, nj, 1}, {Gb, nl, 0}, epi_store(nj, nl, 1.0f, p.dF, nl), form, prec, pk,
                             sa, s));
        LN_TRY(contract_into(nj, nm, nl, {p.dF, nl, 0}, {D, nl, 1}, epi_store(nj, nm, 1.0f, dC, nm), form, prec, pk,
                             sa, s));
        return contract_into(nm, nl, nj, {C, nm, 1}, {p.dF, nl, 0}, epi_store(nm, nl, 1.0f, dD, nl), form, prec, pk,
                             sa, s);
    };
    // the two halves side by side when each pair of concurrent contractions fits on the GPU
    SideStream *ss = nullptr;
    if (p.pack2) {
        const int P = prec_terms(prec);
        int d[MM3_BWD_N][3];
        mm3_bwd_dims(ni, nj, nk, nl, nm, d);
        auto wk = [&](int i) { return contract_work(d[i][0], d[i][1], d[i][2], P); };
        const long long sms = sm_count();
        // pairs in execution order: (E, F), (dE, dF), (dA, dC), (dB, dD)
        if (wk(0) + wk(1) <= sms && wk(2) + wk(3) <= sms && wk(4) + wk(6) <= sms && wk(5) + wk(7) <= sms)
            ss = side_stream(st);
    }
    if (!ss) {
        LN_TRY(prod_E(p.pack, p.split, st));
        LN_TRY(prod_F(p.pack, p.split, st));
        LN_TRY(grads_AB(p.pack, p.split, st));
        return grads_CD(p.pack, p.split, st);
    }
    LN_CUDA_TRY(cudaEventRecord(ss->fork, st));
    LN_CUDA_TRY(cudaStreamWaitEvent(ss->s, ss->fork, 0));
    ln_status sb = prod_F(p.pack2, p.split2, ss->s);
    LN_CUDA_TRY(cudaEventRecord(ss->mid_b, ss->s));  // F written
    ln_status sa = prod_E(p.pack, p.split, st);
    LN_CUDA_TRY(cudaEventRecord(ss->mid_a, st));  // E written
    LN_CUDA_TRY(cudaStreamWaitEvent(ss->s, ss->mid_a, 0));
    if (sb == LN_SUCCESS) sb = grads_CD(p.pack2, p.split2, ss->s);
    LN_CUDA_TRY(cudaEventRecord(ss->join, ss->s));
    LN_CUDA_TRY(cudaStreamWaitEvent(st, ss->mid_b, 0));
    if (sa == LN_SUCCESS) sa = grads_AB(p.pack, p.split, st);
    LN_CUDA_TRY(cudaStreamWaitEvent(st, ss->join, 0));  // joined whatever either half returned
    LN_TRY(sb);
    return sa;
}

// ------------------------------------------------------------------ statistics, covariance, correlation
ln_status ln_col_stats_workspace_size(int nsamples, int nfeat, ln_form form, size_t *bytes) {
    clear_error();
    LN_TRY(check_dims({nsamples, nfeat}));
    LN_TRY(check_form(form, LN_PREC_FP32));
    if (!bytes) return fail(LN_ERR_INVALID_VALUE, "NULL bytes");
    *bytes = form == LN_FORM_INTERNALIZED ? align_up(col_stats_partials_bytes(nsamples, nfeat), 256) : 0;
    return LN_SUCCESS;
}

ln_status ln_col_stats(int nsamples, int nfeat, const float *X, int ldx, double *mean, double *ss, void *ws,
                       size_t wsb, ln_form form, void *stream) {
    clear_error();
    LN_TRY(check_dims({nsamples, nfeat}));
    LN_TRY(check_form(form, LN_PREC_FP32));
    if (nfeat == 0) return LN_SUCCESS;
    if (nsamples < 1) return fail(LN_ERR_INVALID_VALUE, "nsamples >= 1 required");
    if (!X || !mean || !ss) return fail(LN_ERR_INVALID_VALUE, "NULL operand");
    if (ldx < nfeat) return fail(LN_ERR_INVALID_VALUE, "ldx smaller than nfeat");
    Span sx = mspan(X, nsamples, nfeat, ldx);
    Span sm = {mean, sizeof(double) * (size_t)nfeat}, sq = {ss, sizeof(double) * (size_t)nfeat};
    if (overlap(sm, sx) || overlap(sq, sx) || overlap(sm, sq)) return fail(LN_ERR_ALIASING, "outputs overlap");
    if (form == LN_FORM_PLAIN) return plain_col_stats(nsamples, nfeat, X, ldx, mean, ss, S(stream));
    LN_TRY(check_ws(ws, wsb, align_up(col_stats_partials_bytes(nsamples, nfeat), 256)));
    return col_stats(nsamples, nfeat, X, ldx, mean, ss, nullptr, nullptr, nullptr, static_cast<double *>(ws),
                     S(stream));
}

ln_status ln_covariance_workspace_size(int nsamples, int nfeat, ln_form form, ln_precision prec, size_t *bytes) {
    clear_error();
    LN_TRY(check_dims({nsamples, nfeat}));
    LN_TRY(check_form(form, prec));
    if (!bytes) return fail(LN_ERR_INVALID_VALUE, "NULL bytes");
    Ws w(nullptr);
    CovPlan p;
    plan_cov(w, nsamples, nfeat, form, prec, p);
    *bytes = w.off;
    return LN_SUCCESS;
}

ln_status ln_covariance(int nsamples, int nfeat, const float *X, int ldx, float *cov, int ldcov, void *ws, size_t wsb,
                        ln_form form, ln_precision prec, void *stream) {
    clear_error();
    return run_cov(false, nsamples, nfeat, X, ldx, cov, ldcov, nullptr, ws, wsb, form, prec, S(stream));
}

ln_status ln_correlation(int nsamples, int nfeat, const float *X, int ldx, float *corr, int ldcorr, void *ws,
                         size_t wsb, ln_form form, ln_precision prec, void *stream) {
    clear_error();
    return run_cov(true, nsamples, nfeat, X, ldx, corr, ldcorr, nullptr, ws, wsb, form, prec, S(stream));
}

ln_status ln_covariance_fwd(int nsamples, int nfeat, const float *X, int ldx, float *cov, int ldcov, double *stats,
                            void *ws, size_t wsb, ln_form form, ln_precision prec, void *stream) {
    clear_error();
    if (!stats) return fail(LN_ERR_INVALID_VALUE, "NULL statistics");
    return run_cov(false, nsamples, nfeat, X, ldx, cov, ldcov, stats, ws, wsb, form, prec, S(stream));
}

ln_status ln_correlation_fwd(int nsamples, int nfeat, const float *X, int ldx, float *corr, int ldcorr,
                             double *stats, void *ws, size_t wsb, ln_form form, ln_precision prec, void *stream) {
    clear_error();
    if (!stats) return fail(LN_ERR_INVALID_VALUE, "NULL statistics");
    return run_cov(true, nsamples, nfeat, X, ldx, corr, ldcorr, stats, ws, wsb, form, prec, S(stream));
}

// ------------------------------------------------------------------ SYRK / SYR2K
ln_status ln_syrk_workspace_size(int n, int k, ln_form form, ln_precision prec, size_t *bytes) {
    clear_error();
    LN_TRY(check_dims({n, k}));
    LN_TRY(check_form(form, prec));
    if (!bytes) return fail(LN_ERR_INVALID_VALUE, "NULL bytes");
    Ws w(nullptr);
    SymPlan p;
    plan_sym(w, false, n, k, form, prec, p);
    *bytes = w.off;
    return LN_SUCCESS;
}

ln_status ln_syr2k_workspace_size(int n, int k, ln_form form, ln_precision prec, size_t *bytes) {
    clear_error();
    LN_TRY(check_dims({n, k}));
    LN_TRY(check_form(form, prec));
    if (!bytes) return fail(LN_ERR_INVALID_VALUE, "NULL bytes");
    Ws w(nullptr);
    SymPlan p;
    plan_sym(w, true, n, k, form, prec, p);
    *bytes = w.off;
    return LN_SUCCESS;
}

ln_status ln_syrk(ln_fill fill, int n, int k, float alpha, const float *A, int lda, float beta, float *C, int ldc,
                  void *ws, size_t wsb, ln_form form, ln_precision prec, void *stream) {
    clear_error();
    return run_sym(false, fill, n, k, alpha, A, lda, nullptr, 0, beta, C, ldc, ws, wsb, form, prec, S(stream));
}

ln_status ln_syr2k(ln_fill fill, int n, int k, float alpha, const float *A, int lda, const float *B, int ldb,
                   float beta, float *C, int ldc, void *ws, size_t wsb, ln_form form, ln_precision prec,
                   void *stream) {
    clear_error();
    return run_sym(true, fill, n, k, alpha, A, lda, B, ldb, beta, C, ldc, ws, wsb, form, prec, S(stream));
}

// ------------------------------------------------------------------ batched
static ln_status batched_ws(bool two, int count, const ln_sym_desc *h, ln_form form, ln_precision prec,
                            size_t *bytes) {
    clear_error();
    LN_TRY(check_form(form, prec));
    if (!bytes) return fail(LN_ERR_INVALID_VALUE, "NULL bytes");
    BatchPlan bp;
    LN_TRY(validate_batch(two, count, h, bp));
    Ws w(nullptr);
    plan_batch(w, two, count, h, form, prec, bp);
    *bytes = w.off;
    return LN_SUCCESS;
}

ln_status ln_syrk_batched_workspace_size(int count, const ln_sym_desc *h, ln_form form, ln_precision prec,
                                         size_t *bytes) {
    return batched_ws(false, count, h, form, prec, bytes);
}

ln_status ln_syr2k_batched_workspace_size(int count, const ln_sym_desc *h, ln_form form, ln_precision prec,
                                          size_t *bytes) {
    return batched_ws(true, count, h, form, prec, bytes);
}

ln_status ln_syrk_batched(ln_fill fill, int count, const ln_sym_desc *h, const ln_sym_desc *d, float alpha, float beta,
                          void *ws, size_t wsb, ln_form form, ln_precision prec, void *stream) {
    clear_error();
    return run_batch(false, fill, count, h, d, alpha, beta, ws, wsb, form, prec, S(stream));
}

ln_status ln_syr2k_batched(ln_fill fill, int count, const ln_sym_desc *h, const ln_sym_desc *d, float alpha,
                           float beta, void *ws, size_t wsb, ln_form form, ln_precision prec, void *stream) {
    clear_error();
    return run_batch(true, fill, count, h, d, alpha, beta, ws, wsb, form, prec, S(stream));
}

// ------------------------------------------------------------------ backward
ln_status ln_gemm_chain_bwd_workspace_size(int ni, int nj, int nk, int nl, ln_form form, ln_precision prec,
                                           size_t *bytes) {
    clear_error();
    LN_TRY(check_dims({ni, nj, nk, nl}));
    LN_TRY(check_form(form, prec));
    if (!bytes) return fail(LN_ERR_INVALID_VALUE, "NULL bytes");
    Ws w(nullptr);
    ChainBwdPlan p;
    plan_chain_bwd(w, ni, nj, nk, nl, form, prec, p);
    *bytes = w.off;
    return LN_SUCCESS;
}

ln_status ln_gemm_chain_bwd(int ni, int nj, int nk, int nl, const float *A, const float *B, const float *C,
                            const float *G, float *dA, float *dB, float *dC, void *ws, size_t wsb, ln_form form,
                            ln_precision prec, void *stream) {
    clear_error();
    LN_TRY(check_dims({ni, nj, nk, nl}));
    LN_TRY(check_form(form, prec));
    if (!A || !B || !C || !G || !dA || !dB || !dC) return fail(LN_ERR_INVALID_VALUE, "NULL operand");
    Span outs[3] = {mspan(dA, ni, nk, nk), mspan(dB, nk, nj, nj), mspan(dC, nj, nl, nl)};
    Span ins[4] = {mspan(A, ni, nk, nk), mspan(B, nk, nj, nj), mspan(C, nj, nl, nl), mspan(G, ni, nl, nl)};
    for (int i = 0; i < 3; ++i) {
        for (int j = i + 1; j < 3; ++j)
            if (overlap(outs[i], outs[j])) return fail(LN_ERR_ALIASING, "gradient outputs overlap");
        for (const Span &s : ins)
            if (overlap(outs[i], s)) return fail(LN_ERR_ALIASING, "a gradient output overlaps an input");
    }
    Ws count(nullptr);
    ChainBwdPlan p;
    plan_chain_bwd(count, ni, nj, nk, nl, form, prec, p);
    LN_TRY(check_ws(ws, wsb, count.off));
    Ws w(ws);
    plan_chain_bwd(w, ni, nj, nk, nl, form, prec, p);
    cudaStream_t st = S(stream);
    char *pk = p.c.px;
    // three independent branches: BC = B C (nk x nl), dA = G BC^T;
    // GCt = G C^T (ni x nj), dB = A^T GCt; T = A B (ni x nj), dC = T^T G.
    // The six contractions (M, N, K):
    auto c_T = [&](char *a, const SplitArea &sa, cudaStream_t s) {
        return contract_into(ni, nj, nk, {A, nk, 0}, {B, nj, 0}, epi_store(ni, nj, 1.0f, p.T, nj), form, prec, a, sa,
                             s);
    };
    auto c_dC = [&](char *a, const SplitArea &sa, cudaStream_t s) {
        return contract_into(nj, nl, ni, {p.T, nj, 1}, {G, nl, 0}, epi_store(nj, nl, 1.0f, dC, nl), form, prec, a, sa,
                             s);
    };
    auto c_BC = [&](char *a, const SplitArea &sa, cudaStream_t s) {
        return contract_into(nk, nl, nj, {B, nj, 0}, {C, nl, 0}, epi_store(nk, nl, 1.0f, p.BC, nl), form, prec, a, sa,
                             s);
    };
    auto c_dA = [&](char *a, const SplitArea &sa, cudaStream_t s) {
        return contract_into(ni, nk, nl, {G, nl, 0}, {p.BC, nl, 1}, epi_store(ni, nk, 1.0f, dA, nk), form, prec, a, sa,
                             s);
    };
    auto c_GCt = [&](char *a, const SplitArea &sa, cudaStream_t s) {
        return contract_into(ni, nj, nl, {G, nl, 0}, {C, nl, 1}, epi_store(ni, nj, 1.0f, p.GCt, nj), form, prec, a, sa,
                             s);
    };
    auto c_dB = [&](char *a, const SplitArea &sa, cudaStream_t s) {
        return contract_into(nk, nj, ni, {A, nk, 1}, {p.GCt, nj, 0}, epi_store(nk, nj, 1.0f, dB, nj), form, prec, a, sa,
                             s);
    };
    // When pairs of them fit on the GPU side by side, they run as three rounds
    // on two streams -- (T | GCt), (BC | dB), (dA | dC), dC waiting for T by an
    // event -- so the longest chain is three contractions, not four; the second
    // stream has its own pack and split areas.
    SideStream *ss = nullptr;
    if (p.px2) {
        const int P = prec_terms(prec);
        const long long sms = sm_count();
        if (contract_work(ni, nj, nk, P) + contract_work(ni, nj, nl, P) <= sms &&
            contract_work(nk, nl, nj, P) + contract_work(nk, nj, ni, P) <= sms &&
            contract_work(ni, nk, nl, P) + contract_work(nj, nl, ni, P) <= sms)
            ss = side_stream(st);
    }
    if (!ss) {
        LN_TRY(c_BC(pk, p.split, st));
        LN_TRY(c_dA(pk, p.split, st));
        LN_TRY(c_T(pk, p.split, st));
        LN_TRY(c_dC(pk, p.split, st));
        LN_TRY(c_GCt(pk, p.split, st));
        return c_dB(pk, p.split, st);
    }
    LN_CUDA_TRY(cudaEventRecord(ss->fork, st));
    LN_CUDA_TRY(cudaStreamWaitEvent(ss->s, ss->fork, 0));
    // main stream: T, then BC, dA; second stream: GCt, dB, then dC once T is done
    ln_status sa = c_T(pk, p.split, st);
    if (sa == LN_SUCCESS) sa = cudaEventRecord(ss->mid_a, st) == cudaSuccess ? LN_SUCCESS : fail(LN_ERR_CUDA, "event");
    ln_status sb = c_GCt(p.px2, p.split2, ss->s);
    if (sb == LN_SUCCESS) sb = c_dB(p.px2, p.split2, ss->s);
    if (sb == LN_SUCCESS && sa == LN_SUCCESS)
        sb = cudaStreamWaitEvent(ss->s, ss->mid_a, 0) == cudaSuccess ? LN_SUCCESS : fail(LN_ERR_CUDA, "event wait");
    if (sb == LN_SUCCESS && sa == LN_SUCCESS) sb = c_dC(p.px2, p.split2, ss->s);
    if (sa == LN_SUCCESS) sa = c_BC(pk, p.split, st);
    if (sa == LN_SUCCESS) sa = c_dA(pk, p.split, st);
    LN_CUDA_TRY(cudaEventRecord(ss->join, ss->s));
    LN_CUDA_TRY(cudaStreamWaitEvent(st, ss->join, 0));  // joined whatever either branch returned
    LN_TRY(sb);
    return sa;
}

ln_status ln_covariance_bwd_workspace_size(int nsamples, int nfeat, ln_form form, ln_precision prec, size_t *bytes) {
    clear_error();
    LN_TRY(check_dims({nsamples, nfeat}));
    LN_TRY(check_form(form, prec));
    if (!bytes) return fail(LN_ERR_INVALID_VALUE, "NULL bytes");
    Ws w(nullptr);
    CovBwdPlan p;
    plan_cov_bwd(w, true, nsamples, nfeat, form, prec, p);  // the correlation plan covers both
    *bytes = w.off;
    return LN_SUCCESS;
}

ln_status ln_covariance_bwd(int nsamples, int nfeat, const float *X, int ldx, const float *W, int ldw,
                            const double *stats, float *dX, int lddx, void *ws, size_t wsb, ln_form form,
                            ln_precision prec, void *stream) {
    clear_error();
    return run_cov_bwd(false, nsamples, nfeat, X, ldx, W, ldw, stats, dX, lddx, ws, wsb, form, prec, S(stream));
}

ln_status ln_correlation_bwd(int nsamples, int nfeat, const float *X, int ldx, const float *W, int ldw,
                             const double *stats, float *dX, int lddx, void *ws, size_t wsb, ln_form form,
                             ln_precision prec, void *stream) {
    clear_error();
    return run_cov_bwd(true, nsamples, nfeat, X, ldx, W, ldw, stats, dX, lddx, ws, wsb, form, prec, S(stream));
}

ln_status ln_gramschmidt(int m, int n, const float *A, int lda, float *Q, int ldq, float *R, int ldr, ln_form form,
                         void *stream) {
    clear_error();
    LN_TRY(check_dims({m, n}));
    LN_TRY(check_form(form, LN_PREC_FP32));
    if (n == 0) return LN_SUCCESS;
    if (!R || (m > 0 && (!A || !Q))) return fail(LN_ERR_INVALID_VALUE, "NULL operand");
    if (lda < n || ldq < n || ldr < n) return fail(LN_ERR_INVALID_VALUE, "a leading dimension is smaller than n");
    const bool in_place = m > 0 && A == Q && lda == ldq;
    const Span sa = mspan(A, m, n, lda), sq = mspan(Q, m, n, ldq), sr = mspan(R, n, n, ldr);
    if (!in_place && overlap(sa, sq))
        return fail(LN_ERR_ALIASING, "A and Q overlap (only A == Q with lda == ldq, in place, is allowed)");
    if (overlap(sr, sa) || overlap(sr, sq)) return fail(LN_ERR_ALIASING, "R overlaps A or Q");
    LN_TRY(device_view(R, &R, "R"));
    if (m > 0) {
        LN_TRY(device_view(A, &A, "A"));
        LN_TRY(device_view(Q, &Q, "Q"));
    }
    cudaStream_t st = S(stream);
    if (m > 0 && !in_place)
        LN_CUDA_TRY(cudaMemcpy2DAsync(Q, (size_t)ldq * 4, A, (size_t)lda * 4, (size_t)n * 4, (size_t)m,
                                      cudaMemcpyDefault, st));
    return form == LN_FORM_PLAIN ? gs_plain(m, n, Q, ldq, R, ldr, st) : gs_blocked(m, n, Q, ldq, R, ldr, st);
}

}  // extern "C"
