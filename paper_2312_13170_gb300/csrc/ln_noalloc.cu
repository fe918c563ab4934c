// ln_covariance_noalloc: the covariance of ln_covariance (internalized form,
// exact-FP32 tiled contraction over FP64 column statistics) for callers that
// cannot allocate device memory -- for example code running where cudaMalloc
// is forbidden or would break an allocation budget, such as inside a custom
// allocator, a memory-capped sandbox or a real-time loop that must not call
// into the allocator. Its scratch lives in one fixed device array below
// instead of a caller-provided workspace.
//
// The array is a file-scope __device__ variable, so every GPU that loads the
// library holds it (8 MiB) until the process exits. Host code cannot use the
// array's name as a device address; the first call on each device looks the
// address up with cudaGetSymbolAddress (with that device current) and keeps it.
// That first call should therefore happen before any CUDA graph capture.
//
// All calls on a device share the one array: calls whose kernels overlap on
// the GPU (different streams without ordering) race on it. Each call writes
// every scratch value it reads before reading it, so nothing left by an
// earlier call needs clearing.
#include "ln_internal.h"

namespace ln {

constexpr size_t NOALLOC_SCRATCH_BYTES = (size_t)8 << 20;

static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

namespace {

void *g_scratch_addr[64] = {nullptr};

// Byte offsets of the scratch pieces for an n x m problem (each 256-aligned).
struct NoallocLayout {
    size_t mean, ss, hi, lo, rs, partials, total;
};

NoallocLayout noalloc_layout(int n, int m) {
    NoallocLayout L{};
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t at = off;
        off = align_up(off + bytes, 256);
        return at;
    };
    L.mean = take(sizeof(double) * (size_t)m);
    L.ss = take(sizeof(double) * (size_t)m);
    L.hi = take(sizeof(float) * (size_t)m);
    L.lo = take(sizeof(float) * (size_t)m);
    L.rs = take(sizeof(float) * (size_t)m);
    L.partials = take(col_stats_partials_bytes(n, m));
    L.total = off;
    return L;
}

}  // namespace

}  // namespace ln

using namespace ln;

extern "C" ln_status ln_covariance_noalloc(int nsamples, int nfeat, const float *X, int ldx, float *cov, int ldcov,
                                           void *stream) {
    clear_error();
    if (nsamples < 0 || nfeat < 0) return fail(LN_ERR_INVALID_VALUE, "negative size");
    if (nfeat == 0) return LN_SUCCESS;
    if (nsamples < 2) return fail(LN_ERR_INVALID_VALUE, "covariance needs nsamples >= 2 (got %d)", nsamples);
    if (!X || !cov) return fail(LN_ERR_INVALID_VALUE, "NULL X or output");
    if (ldx < nfeat || ldcov < nfeat) return fail(LN_ERR_INVALID_VALUE, "leading dimension smaller than nfeat");
    const uintptr_t x0 = reinterpret_cast<uintptr_t>(X), c0 = reinterpret_cast<uintptr_t>(cov);
    const uintptr_t x1 = x0 + (((size_t)nsamples - 1) * ldx + nfeat) * sizeof(float);
    const uintptr_t c1 = c0 + (((size_t)nfeat - 1) * ldcov + nfeat) * sizeof(float);
    if (x0 < c1 && c0 < x1) return fail(LN_ERR_ALIASING, "output overlaps X");
    const NoallocLayout L = noalloc_layout(nsamples, nfeat);
    if (L.total > NOALLOC_SCRATCH_BYTES)
        return fail(LN_ERR_INVALID_VALUE,
                    "ln_covariance_noalloc needs %zu bytes of scratch for %d x %d, more than its fixed %zu bytes "
                    "(about 40*nfeat + 8*nfeat*ceil(nsamples/r) bytes, r = 64 to 256 rows per reduction block); "
                    "use ln_covariance with a workspace",
                    L.total, nsamples, nfeat, NOALLOC_SCRATCH_BYTES);
    int dev = 0;
    LN_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return fail(LN_ERR_UNSUPPORTED, "device ordinal %d out of range", dev);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        LN_CUDA_TRY(cudaGetSymbolAddress(&p, g_noalloc_scratch));
        g_scratch_addr[dev] = p;
    }
    char *base = static_cast<char *>(g_scratch_addr[dev]);
    double *mean = reinterpret_cast<double *>(base + L.mean);
    double *ss = reinterpret_cast<double *>(base + L.ss);
    float *hi = reinterpret_cast<float *>(base + L.hi);
    float *lo = reinterpret_cast<float *>(base + L.lo);
    float *rs = reinterpret_cast<float *>(base + L.rs);
    double *partials = reinterpret_cast<double *>(base + L.partials);
    cudaStream_t st = static_cast<cudaStream_t>(stream);

    ln_status s = col_stats(nsamples, nfeat, X, ldx, mean, ss, hi, lo, rs, partials, st);
    if (s != LN_SUCCESS) return s;
    EpiParams e{};
    e.mode = EPI_SYM;
    e.M = e.N = nfeat;
    e.C = cov;
    e.ldc = ldcov;
    e.fill = LN_FILL_FULL;
    e.sym_kind = SYM_SCALE;
    e.alpha = (float)(1.0 / (double)(nsamples - 1));
    SimtOperands op{};
    op.A[0] = op.A[1] = X;
    op.B[0] = op.B[1] = X;
    op.lda[0] = op.lda[1] = ldx;
    op.ldb[0] = op.ldb[1] = ldx;
    op.a_t = 1;
    op.b_t = 0;
    op.nseg = 1;
    op.a_off_hi = op.b_off_hi = hi;
    op.a_off_lo = op.b_off_lo = lo;
    return simt_contract(nfeat, nfeat, nsamples, op, e, st);
}
