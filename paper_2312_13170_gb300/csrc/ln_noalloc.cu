// ln_covariance_noalloc: the covariance of ln_covariance (internalized form,
// exact-FP32 tiled contraction centred by FP64 column means) for callers that
// cannot allocate device memory -- for example code running where cudaMalloc
// is forbidden or would break an allocation budget, such as inside a custom
// allocator, a memory-capped sandbox or a real-time loop that must not call
// into the allocator. Its scratch lives in one fixed device array below
// instead of a caller-provided workspace.
//
// The array is a file-scope __device__ variable, so every GPU that loads the
// library holds it (8 MiB) until the process exits. Host code cannot use the
// array's name as a device address: a call outside stream capture looks the
// address up with cudaGetSymbolAddress (with the call's device current) and
// remembers it per device; a call during capture uses the remembered address,
// so a device's first call must come before any capture on it, and after a
// cudaDeviceReset the first call must again come outside capture (the reset
// can move the array).
//
// All calls on a device share the one array: calls whose kernels overlap on
// the GPU (different streams without ordering) race on it. Each call writes
// every scratch value it reads before reading it, so nothing left by an
// earlier call needs clearing.
#include <mutex>

#include "ln_internal.h"
#include "ln_stats.h"

namespace ln {

constexpr size_t NOALLOC_SCRATCH_BYTES = (size_t)8 << 20;

static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

namespace {

std::mutex g_scratch_mu;
void *g_scratch_addr[64] = {nullptr};

// Byte offsets of the scratch pieces for an n x m problem (each 256-aligned):
// the FP64 column means, the FP32 centring pair (hi, lo) and the per-block
// partial sums of the mean pass.
struct NoallocLayout {
    size_t mean, hi, lo, partials, total;
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
    L.hi = take(sizeof(float) * (size_t)m);
    L.lo = take(sizeof(float) * (size_t)m);
    L.partials = take(col_stats_partials_bytes(n, m));
    L.total = off;
    return L;
}

// The array's device address on the current device (see the file comment).
ln_status scratch_address(cudaStream_t st, char **out) {
    int dev = 0;
    LN_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return fail(LN_ERR_UNSUPPORTED, "device ordinal %d out of range", dev);
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    LN_CUDA_TRY(cudaStreamIsCapturing(st, &cs));
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (cs == cudaStreamCaptureStatusNone) {
        void *p = nullptr;
        LN_CUDA_TRY(cudaGetSymbolAddress(&p, g_noalloc_scratch));
        g_scratch_addr[dev] = p;
    } else if (!g_scratch_addr[dev]) {
        return fail(LN_ERR_UNSUPPORTED,
                    "ln_covariance_noalloc: the first call on a device must come before stream capture");
    }
    *out = static_cast<char *>(g_scratch_addr[dev]);
    return LN_SUCCESS;
}

}  // namespace

}  // namespace ln

using namespace ln;

extern "C" ln_status ln_covariance_noalloc(int nsamples, int nfeat, const float *X, int ldx, float *cov, int ldcov,
                                           void *stream) {
    clear_error();
    ln_status s = check_dims({nsamples, nfeat});
    if (s != LN_SUCCESS) return s;
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
                    "(at most 16*nfeat + 8*nfeat*ceil(nsamples/r) + 1024 bytes, r = 256, 128 or 64 rows per "
                    "reduction block); use ln_covariance with a workspace",
                    L.total, nsamples, nfeat, NOALLOC_SCRATCH_BYTES);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    char *base = nullptr;
    s = scratch_address(st, &base);
    if (s != LN_SUCCESS) return s;
    double *mean = reinterpret_cast<double *>(base + L.mean);
    float *hi = reinterpret_cast<float *>(base + L.hi);
    float *lo = reinterpret_cast<float *>(base + L.lo);
    double *partials = reinterpret_cast<double *>(base + L.partials);

    // the mean pass of ln_covariance's internalized form: the same partial sums
    // and reduction, so the centring pair and the result are the same
    s = col_mean(nsamples, nfeat, X, ldx, mean, hi, lo, partials, st);
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
