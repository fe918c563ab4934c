/*
 * libloopnest — GB300 (sm_103a) kernels for the loop nests that loop
 * internalization and array-reduction detection speed up
 * ("Experiences Building an MLIR-based SYCL Compiler", arXiv 2312.13170):
 * GEMM, a chain of two GEMMs (polybench 2mm), three chained products
 * (polybench 3mm), covariance, correlation, SYRK and SYR2K (single and
 * batched), modified Gram-Schmidt QR, plus the vector-Jacobian products of the
 * chain, 3mm, covariance and correlation. Around them: tuning knobs
 * (ln_set_tuning), launch counting and CUDA-event timing (ln_timing_*), and
 * peak probes that measure this device's tensor-core, FFMA and copy rates
 * (ln_peak_probe).
 *
 * Every operation exists in two forms:
 *   LN_FORM_PLAIN        one thread per output element, reading global memory
 *                        in its inner loop with a register accumulator: the
 *                        loop nest of paper Sec. VI-C, Listing 5, after the
 *                        array-reduction detection of Sec. VI-B.
 *   LN_FORM_INTERNALIZED the inner loop's operands are staged in on-chip
 *                        memory tile by tile, as loop internalization does
 *                        with work-group local memory (Sec. VI-C, Listing 6):
 *                        with LN_PREC_FP32 a shared-memory tiled FP32 SIMT
 *                        kernel; with a tensor-core precision, operands are
 *                        split into BF16 or TF32 terms, packed in tcgen05
 *                        operand tiles, copied into shared memory by the
 *                        bulk-copy (TMA) engine and multiplied by
 *                        tcgen05.mma into TMEM accumulators.
 *
 * Conventions shared by every entry point
 *  - Matrices are FP32, row-major; ld* are leading dimensions in elements
 *    (ld >= number of columns). Sizes are int; negative sizes or ld < columns
 *    give LN_ERR_INVALID_VALUE. A size of 0 makes the call a no-op (GEMM with
 *    K = 0 scales C by beta).
 *  - Every pointer argument that names an array (inputs, outputs, workspace)
 *    is a DEVICE pointer unless the comment says "host". The caller owns all
 *    memory and the stream; the library never allocates device memory.
 *  - `stream` is a cudaStream_t (NULL = the legacy default stream). Calls are
 *    asynchronous: the returned status covers argument validation and kernel
 *    launch only. Errors raised on the device (a bounded wait that ran out)
 *    are reported by ln_stream_check() after the work has finished.
 *  - beta == 0 means the input C (or D) is never read, so NaN/Inf there is not
 *    propagated (BLAS convention).
 *  - Outputs must not overlap any input, except where the comment allows
 *    in-place C: overlapping ranges give LN_ERR_ALIASING. This is the
 *    no-alias guarantee that the paper's alias analysis proves before it
 *    transforms a loop (Sec. V-A, Sec. VI-A), checked here at run time.
 *  - Internalized tensor-core calls need a workspace of at least the size the
 *    matching *_workspace_size function returns (256-byte aligned device
 *    memory); too small a workspace gives LN_ERR_WORKSPACE. Plain and FP32
 *    SIMT calls need none except where noted (workspace may then be NULL).
 *  - On any error the call launches nothing and ln_get_last_error() returns a
 *    message for the calling thread.
 */
#ifndef LOOPNEST_H
#define LOOPNEST_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    LN_SUCCESS = 0,
    LN_ERR_INVALID_VALUE = 1, /* bad size, leading dimension, enum or NULL pointer */
    LN_ERR_ALIASING = 2,      /* an output range overlaps an input range */
    LN_ERR_MISALIGNED = 3,    /* the workspace pointer is not 256-byte aligned; data
                                 pointers of any alignment are accepted (unaligned
                                 rows take the slower copy paths), so no other
                                 argument returns this code */
    LN_ERR_UNSUPPORTED = 4,   /* form/precision combination not available */
    LN_ERR_CUDA = 5,          /* a CUDA runtime call or launch failed */
    LN_ERR_TIMEOUT = 6,       /* a bounded device wait ran out (ln_stream_check) */
    LN_ERR_WORKSPACE = 7      /* workspace missing or smaller than required */
} ln_status;

typedef enum { LN_FORM_PLAIN = 0, LN_FORM_INTERNALIZED = 1 } ln_form;

/*
 * Arithmetic of the contraction. FP32 is exact-FP32 FFMA (both forms). The
 * others run on tcgen05 tensor cores with FP32 accumulation (internalized form
 * only): BF16 = one product of BF16-rounded operands; 3XBF16 = each operand
 * split x = hi + lo into two BF16 terms, products hi*hi + hi*lo + lo*hi;
 * 6XBF16 = three BF16 terms (hi + mid + lo), the six products whose order is
 * at least 2^-16. TF32 = one product of TF32-rounded operands (10-bit
 * mantissa, round to nearest, ties away from zero); 3XTF32 = x = hi + lo in
 * two TF32 terms, products hi*hi + hi*lo + lo*hi, on the tensor cores' TF32
 * path (half the BF16 rate per product). FP32, 3XBF16, 6XBF16 and 3XTF32
 * meet a 1e-5 relative Frobenius error against exact arithmetic on the shipped
 * workloads; BF16 and TF32 do not.
 */
typedef enum {
    LN_PREC_FP32 = 0,
    LN_PREC_BF16 = 1,
    LN_PREC_3XBF16 = 2,
    LN_PREC_6XBF16 = 3,
    LN_PREC_TF32 = 4,
    LN_PREC_3XTF32 = 5
} ln_precision;

/* Triangle of a symmetric output (SYRK/SYR2K): LOWER/UPPER read and write only
 * that triangle of C; FULL computes the lower triangle from C's lower triangle
 * and writes each value to both (i,j) and (j,i). */
typedef enum { LN_FILL_FULL = 0, LN_FILL_LOWER = 1, LN_FILL_UPPER = 2 } ln_fill;

/* Message for the last failed call on this host thread ("" if none). */
const char *ln_get_last_error(void);
/* Static name of a status code. */
const char *ln_status_string(ln_status s);
/* Library version as major*10000 + minor*100 + patch. */
int ln_version(void);

/*
 * Wait for `stream`, then read and clear the library's device error word.
 * Returns LN_ERR_TIMEOUT if a kernel on this device gave up a bounded wait
 * since the last check, LN_ERR_CUDA if the stream reports a CUDA error, else
 * LN_SUCCESS.
 */
ln_status ln_stream_check(void *stream);

/*
 * Launch accounting for benchmarks and profiling. ln_launch_count() is the
 * number of kernels this library has launched in the process (always
 * counted). While timing is enabled, every launch of a kernel family is
 * bracketed by CUDA events recorded on the stream it is launched on;
 * ln_timing_read() waits for those events and returns the total time in
 * milliseconds and the number of launches of one family since the last read
 * (families: "umma" = tcgen05 contraction, "pack" = split-and-pack,
 * "simt" = FP32 tiled contraction, "plain" = one-thread-per-output kernels,
 * "stats" = column statistics and element-wise helpers). Launches captured
 * into a CUDA graph get external event-record nodes, so their times are those
 * of the latest replay of the graph (read after replaying each captured graph
 * once). Enabling and reading must not happen during capture. Not thread-safe.
 * ln_timing_enable(on): 0 off; 1 one event pair per launch; 2 spans: launches
 * of one family that the library issues back to back on one stream with
 * programmatic launch overlap (the two contractions of ln_gemm_chain's
 * tensor-core path) share one event pair, so that no event node sits between
 * them, and count as that many launches (an event between two such launches
 * delays the second until the first has finished, a few microseconds more
 * per launch); every other launch keeps its own pair. Other values:
 * LN_ERR_INVALID_VALUE.
 */
long long ln_launch_count(void);
ln_status ln_timing_enable(int on);
ln_status ln_timing_read(const char *family, double *total_ms /*host*/, int *launches /*host*/);

/*
 * Peak probes: the roofline denominators measured on this device. The paper
 * has no counterpart (its evaluation reports speedups, not fractions of a
 * peak); these exist so that a kernel's achieved rate can be set against what
 * the same GPU does on a loop that does nothing but that one kind of work.
 * Each call launches one kernel on `stream` and returns at once; *work
 * receives the algorithmic work of that launch (flops, or bytes read plus
 * bytes written), which the caller divides by the launch's CUDA-event time.
 *   LN_PEAK_MMA_BF16, LN_PEAK_MMA_TF32: one CTA per SM issues 4 * iters
 *     tcgen05.mma (M = 128, N = 256, K = 16 BF16 or 8 TF32 elements) on
 *     operand tiles resident in its shared memory, accumulating in TMEM.
 *     dst: a device word (4 bytes, bytes >= 4) that the call zeroes and the
 *     kernel sets to 1 if its bounded wait for the MMAs (2 s) ran out.
 *     iters in [1, 2^20].
 *   LN_PEAK_FFMA: 8 CTAs of 256 threads per SM, each thread 128 * iters FP32
 *     FFMAs in 8 independent chains; dst: a 4-byte device sink (never
 *     written for these inputs); iters in [1, 2^20].
 *   LN_PEAK_COPY: dst[0, bytes) = src[0, bytes) with 16-byte loads and
 *     stores; both 16-byte aligned, bytes a positive multiple of 16, the
 *     ranges disjoint (LN_ERR_ALIASING otherwise); iters unused.
 * Bad arguments give LN_ERR_INVALID_VALUE before anything is launched.
 */
typedef enum { LN_PEAK_MMA_BF16 = 0, LN_PEAK_MMA_TF32 = 1, LN_PEAK_FFMA = 2, LN_PEAK_COPY = 3 } ln_peak_kind;
ln_status ln_peak_probe(int kind, long long iters, const void *src, void *dst, long long bytes,
                        double *work /*host*/, void *stream);

/*
 * Tuning knobs of the tensor-core engine, process-wide (the autotuner in the
 * Python package picks them per problem class). Keys:
 *   "chunk_kt" 1 or 2 (default 2): k tiles of 64 accumulated in tensor memory
 *              before the partial sum is added to an FP32 running sum; 1 is
 *              more accurate, 2 faster;
 *   "tile_n"   0, 128 or 256 (default 0 = automatic: 256, or 128 when
 *              256-wide tiles would fill at most half the SMs): output tile
 *              width of general (non-symmetric) contractions with one or two
 *              split terms;
 *   "pack_threads" 512 or 1024 (default 512): threads per CTA of the
 *              split-and-pack stream;
 *   "split_k"  0 or 1 (default 0): split the K range of tensor-core
 *              contractions whose output tiles fill less than half the GPU
 *              (slices exchange FP32 partial sums through the workspace; the
 *              last slice of a tile to finish adds them in slice order);
 *   "pair"     0, 1 or 2 (default 1): CTA pairs for single tensor-core
 *              contractions with at least two row tiles: clusters of two
 *              CTAs compute vertically adjacent output tiles with
 *              tcgen05.mma.cta_group::2, each holding its own rows of A and
 *              half of the shared column tile of B; 1 pairs 256-wide general
 *              tiles of the split precisions (3XBF16, 3XTF32), 2 also
 *              single-pass BF16 and TF32 (measured slower paired) and, with
 *              BF16 operands, every other tile width and symmetric outputs
 *              (measured slower on 128-wide tiles), 0 none; results are
 *              bit-identical;
 *   "simt_exact" 0 or 1 (default 1): the FP32 tiled form launches its EXACT
 *              instance (no bounds predicates, 16-byte epilogue accesses) when
 *              M, N are multiples of its tile width, K of 8, and every operand
 *              and output row is 16-byte aligned; 0 always takes the general
 *              instance; results are bit-identical;
 *   "simt_tile" 0, 64 or 128 (default 0): the CTA output tile of the FP32
 *              tiled form; 0 takes 64 when the problem has at most as many
 *              128-wide tiles as the device has SMs and at most twice as many
 *              64-wide tiles, else 128;
 *              both give the same exact-FP32 sums in the same k order;
 *   "stage_beta" 0 or 1 (default 1): the last 256-wide tile of each CTA of
 *              a general tensor-core contraction with beta != 0 copies its
 *              block of D (chain) or C (GEMM) into the operand stages once its
 *              MMAs are done, so the epilogue stores E at once and reads D or
 *              C from shared memory;
 *   "stage_out" 0 or 1 (default 1): the last 256-wide tile of each CTA of a
 *              contraction with the packing epilogue (the chain's T, 3mm's E
 *              and F) builds its packed output in the freed operand stages and
 *              writes it with bulk copies (4 KiB per warp, block and term)
 *              instead of 16-byte stores from registers; results are
 *              bit-identical;
 *   "sym_wide" 0, 1 or 2 (default 0): output tiles of 128 x 256 instead of
 *              128 x 128 over the lower triangle of single symmetric
 *              contractions (covariance, correlation, SYRK/SYR2K); 2 takes them
 *              where they fill at most half the SMs and so take stream-K
 *              (deep problems such as covariance of 8192 samples), 1 always
 *              (one or two split terms), 0 never (measured faster on the
 *              shipped workloads); results are bit-identical on integer inputs;
 *   "stream_k" 0, 1 or 2 (default 2): stream-K for single tensor-core
 *              contractions with fewer output tiles than SMs (covariance,
 *              correlation, SYRK/SYR2K and the general contractions that do
 *              not run beside another one): the tiles' k ranges are split
 *              evenly over one CTA per SM; a tile spread over several CTAs
 *              gets their FP32 partial sums through the workspace, added in
 *              k order by the CTA that holds its first k tile; 1 applies it
 *              to every such contraction with at least 4 k tiles per SM,
 *              2 only to those that also fill at most half the SMs and have
 *              at least 32 k tiles of 64 (where it measured faster), 0 never;
 *   "gs_rows"  2 or 4 (default 4): rows of the matrix each thread holds in
 *              registers in the internalized Gram-Schmidt panel kernel when
 *              512 < m <= 1024 (512 or 256 threads per panel CTA).
 * A knob changes the workspace size of later calls: set it before the
 * *_workspace_size query of a call, not between the query and the call.
 * Unknown keys or values give LN_ERR_INVALID_VALUE. Not for use while kernels
 * of this library are being enqueued from other host threads.
 */
ln_status ln_set_tuning(const char *key, int value);
ln_status ln_get_tuning(const char *key, int *value /*host*/);

/*
 * GEMM, polybench form (paper Sec. VI-C, Listings 5-6; Sec. VIII "GEMM"):
 *   C[i][j] = alpha * sum_k A[i][k] * B[k][j] + beta * C[i][j]
 * A is M x K (lda), B is K x N (ldb), C is M x N (ldc), in place.
 */
ln_status ln_gemm_workspace_size(int M, int N, int K, ln_form form, ln_precision prec, size_t *bytes /*host*/);
ln_status ln_gemm(int M, int N, int K, float alpha, const float *A, int lda, const float *B, int ldb,
                  float beta, float *C, int ldc, void *workspace, size_t workspace_bytes, ln_form form,
                  ln_precision prec, void *stream);

/*
 * Chained product (polybench 2mm, Sec. VIII):
 *   T = A * B;  E = T * C;  F = alpha * E + beta * D
 * A is ni x nk, B is nk x nj, C is nj x nl, D/E/F are ni x nl; all contiguous
 * (ld = columns). T lives in the workspace (FP32 for FP32 forms; as packed
 * BF16 split terms for tensor-core forms), so every form needs a workspace.
 * D may be NULL when beta == 0. E and F must not overlap each other or inputs.
 * A, B, C, D, E and F may be device memory or host memory the GPU can reach:
 * pinned (page-locked or registered) host buffers are read and written by the
 * kernels through their device mapping, over the host link, without staging
 * copies; pageable host memory is accepted only where the device reports
 * coherent pageable access (cudaDevAttrPageableMemoryAccess), otherwise the
 * call returns LN_ERR_INVALID_VALUE before launching anything. The workspace
 * must be device memory.
 */
ln_status ln_gemm_chain_workspace_size(int ni, int nj, int nk, int nl, ln_form form, ln_precision prec,
                                       size_t *bytes /*host*/);
ln_status ln_gemm_chain(int ni, int nj, int nk, int nl, float alpha, const float *A, const float *B,
                        const float *C, float beta, const float *D, float *E, float *F, void *workspace,
                        size_t workspace_bytes, ln_form form, ln_precision prec, void *stream);

/*
 * Three chained products (polybench 3mm, Sec. VIII):
 *   E = A * B;  F = C * D;  G = E * F
 * A is ni x nk, B is nk x nj, C is nj x nm, D is nm x nl, G is ni x nl; all
 * contiguous (ld = columns). E (ni x nj) and F (nj x nl) live in the
 * workspace: in FP32 for FP32 forms; for tensor-core forms E is written by its
 * product's epilogue directly as the packed BF16 row operand of G, and F (as
 * F^T = D^T C^T) as the packed column operand, so neither exists in FP32.
 * G must not overlap an input. A, B, C, D and G may be host memory the GPU
 * can reach, as for ln_gemm_chain. Sizes of 0 are allowed (G = 0 when
 * nj, nk or nm is 0). Tensor-core forms whose E and F products fit on the GPU
 * together run F on a second stream of the library. That stream is one per
 * host thread and device, created on first use outside graph capture (a call
 * made while `stream` is capturing and before that first use stays on
 * `stream`). It is ordered after `stream` by an event and joined back before
 * G, so the call stays stream-ordered on `stream`.
 */
ln_status ln_3mm_workspace_size(int ni, int nj, int nk, int nl, int nm, ln_form form, ln_precision prec,
                                size_t *bytes /*host*/);
ln_status ln_3mm(int ni, int nj, int nk, int nl, int nm, const float *A, const float *B, const float *C,
                 const float *D, float *G, void *workspace, size_t workspace_bytes, ln_form form, ln_precision prec,
                 void *stream);

/*
 * Column statistics of a data matrix X (nsamples x nfeat, ldx), the array
 * reductions of polybench covariance/correlation (Sec. VI-B, Sec. VIII), two
 * passes: mean[j] = sum_s X[s][j] / n; ss[j] = sum_s (X[s][j] - mean[j])^2.
 * mean and ss are FP64 device arrays of nfeat elements (nsamples >= 1). The
 * internalized form needs a workspace for its per-block partial sums; the
 * plain form needs none. Both forms accumulate in FP64.
 */
ln_status ln_col_stats_workspace_size(int nsamples, int nfeat, ln_form form, size_t *bytes /*host*/);
ln_status ln_col_stats(int nsamples, int nfeat, const float *X, int ldx, double *mean, double *ss,
                       void *workspace, size_t workspace_bytes, ln_form form, void *stream);

/*
 * Covariance (polybench covariance, Sec. VIII): with Xc = X - 1 mean^T,
 *   cov[i][j] = sum_s Xc[s][i] * Xc[s][j] / (nsamples - 1)      (nsamples >= 2)
 * The full symmetric nfeat x nfeat matrix is written.
 * Correlation (polybench correlation): corr[i][j] = sum_s Xc[s][i] Xc[s][j] /
 * (sqrt(ss_i) sqrt(ss_j)) for i != j, corr[i][i] = 1 exactly, and 0 off the
 * diagonal for a zero-variance column. Both need a workspace (the FP64
 * column statistics; packed operands for tensor-core forms).
 */
ln_status ln_covariance_workspace_size(int nsamples, int nfeat, ln_form form, ln_precision prec,
                                       size_t *bytes /*host*/);
ln_status ln_covariance(int nsamples, int nfeat, const float *X, int ldx, float *cov, int ldcov,
                        void *workspace, size_t workspace_bytes, ln_form form, ln_precision prec,
                        void *stream);
ln_status ln_correlation(int nsamples, int nfeat, const float *X, int ldx, float *corr, int ldcorr,
                         void *workspace, size_t workspace_bytes, ln_form form, ln_precision prec,
                         void *stream);

/*
 * Forward calls that also keep the adjoint's saved state: the same result as
 * ln_covariance / ln_correlation (bit for bit: the same kernels in the same
 * order), and `stats` (device, 8-byte aligned, 2*nfeat doubles, not
 * overlapping X or the output) receives the FP64 column means then the sums
 * of squared deviations from them, as ln_col_stats computes them -- the
 * `stats` that ln_covariance_bwd / ln_correlation_bwd take. The statistics
 * are written straight into `stats`, so a forward-backward pair runs the
 * statistics passes once. The covariance's internalized form adds the second
 * (squared deviations) pass that ln_covariance skips. Workspace: as
 * ln_covariance_workspace_size. NULL stats gives LN_ERR_INVALID_VALUE.
 */
ln_status ln_covariance_fwd(int nsamples, int nfeat, const float *X, int ldx, float *cov, int ldcov, double *stats,
                            void *workspace, size_t workspace_bytes, ln_form form, ln_precision prec,
                            void *stream);
ln_status ln_correlation_fwd(int nsamples, int nfeat, const float *X, int ldx, float *corr, int ldcorr,
                             double *stats, void *workspace, size_t workspace_bytes, ln_form form,
                             ln_precision prec, void *stream);

/*
 * Covariance for callers that cannot allocate device memory (code that runs
 * where cudaMalloc is not allowed or would exceed a fixed memory budget, such
 * as inside an allocator, a memory-capped sandbox or a loop that must never
 * enter the allocator). The paper has no counterpart to this entry point; it
 * computes exactly what ln_covariance computes with LN_FORM_INTERNALIZED and
 * LN_PREC_FP32, but takes no workspace: its scratch (the FP64 column
 * means, their FP32 centring pair and per-block partial sums) is one fixed
 * 8 MiB device array in the library, held on every GPU that loads the library
 * until the process exits. The scratch of an nsamples x nfeat call is at most
 * 16*nfeat + 8*nfeat*ceil(nsamples/r) + 1024 bytes, r the rows per reduction
 * block (256, 128 or 64: the largest that still gives about 600 blocks of 128
 * columns); sizes whose scratch exceeds 8 MiB, and sizes outside [0, 2^22],
 * give LN_ERR_INVALID_VALUE with a message and launch nothing.
 * The array's device address is looked up (cudaGetSymbolAddress, under a
 * lock) on each call and remembered per device (a cudaDeviceReset can move
 * the array; the next lookup finds it); where the stream's state does not
 * allow the lookup, the remembered address is used, and with none remembered
 * the call gives LN_ERR_UNSUPPORTED and launches nothing. All calls share the
 * array, so calls whose kernels may overlap on the GPU (unordered streams)
 * race; calls in one stream are safe. X, cov and stream as in ln_covariance.
 */
ln_status ln_covariance_noalloc(int nsamples, int nfeat, const float *X, int ldx, float *cov, int ldcov,
                                void *stream);

/*
 * SYRK (polybench syrk, Sec. VIII): on the triangle chosen by `fill`,
 *   C[i][j] = alpha * sum_k A[i][k] * A[j][k] + beta * C[i][j]       A: n x k
 * SYR2K (polybench syr2k): C[i][j] = alpha * sum_k (A[i][k] B[j][k] +
 * B[i][k] A[j][k]) + beta * C[i][j]; A and B are n x k. C is n x n, in place.
 */
ln_status ln_syrk_workspace_size(int n, int k, ln_form form, ln_precision prec, size_t *bytes /*host*/);
ln_status ln_syrk(ln_fill fill, int n, int k, float alpha, const float *A, int lda, float beta, float *C,
                  int ldc, void *workspace, size_t workspace_bytes, ln_form form, ln_precision prec,
                  void *stream);
ln_status ln_syr2k_workspace_size(int n, int k, ln_form form, ln_precision prec, size_t *bytes /*host*/);
ln_status ln_syr2k(ln_fill fill, int n, int k, float alpha, const float *A, int lda, const float *B, int ldb,
                   float beta, float *C, int ldc, void *workspace, size_t workspace_bytes, ln_form form,
                   ln_precision prec, void *stream);

/*
 * Batched SYRK / SYR2K over instances of uneven sizes in one persistent
 * launch fed by a device-side tile queue (polybench syrk/syr2k, Sec. VIII,
 * batched). Each instance i is described by descs[i]; B/ldb are ignored by
 * SYRK. `h_descs` (host) and `d_descs` (device) must hold the same `count`
 * descriptors: the host copy sizes the launch and is validated, the device
 * copy is what the kernels read (so a captured CUDA graph may be replayed
 * after the caller rewrites d_descs with instances of the same sizes).
 * The same alpha, beta and fill apply to every instance. Instances' outputs
 * must not overlap each other or any input.
 */
typedef struct {
    int n, k;
    const float *A;
    int lda;
    const float *B;
    int ldb;
    float *C;
    int ldc;
} ln_sym_desc;

ln_status ln_syrk_batched_workspace_size(int count, const ln_sym_desc *h_descs /*host*/, ln_form form,
                                         ln_precision prec, size_t *bytes /*host*/);
ln_status ln_syrk_batched(ln_fill fill, int count, const ln_sym_desc *h_descs /*host*/,
                          const ln_sym_desc *d_descs, float alpha, float beta, void *workspace,
                          size_t workspace_bytes, ln_form form, ln_precision prec, void *stream);
ln_status ln_syr2k_batched_workspace_size(int count, const ln_sym_desc *h_descs /*host*/, ln_form form,
                                          ln_precision prec, size_t *bytes /*host*/);
ln_status ln_syr2k_batched(ln_fill fill, int count, const ln_sym_desc *h_descs /*host*/,
                           const ln_sym_desc *d_descs, float alpha, float beta, void *workspace,
                           size_t workspace_bytes, ln_form form, ln_precision prec, void *stream);

/*
 * Gram-Schmidt QR (polybench gramschmidt, paper Sec. VIII; the kernel whose
 * candidate loop lies in a divergent region, Sec. VI-C): modified
 * Gram-Schmidt on A (m x n, lda), column by column in the benchmark's order,
 *   R[k][k] = ||w_k||,  Q[:,k] = w_k / R[k][k],
 *   R[k][j] = Q[:,k] . w_j,  w_j -= R[k][j] Q[:,k]   (j > k),
 * with w the working columns (initially A). Outputs: Q (m x n, ldq) with
 * orthonormal columns when A has full column rank, and R (n x n, ldr) upper
 * triangular with R[k][k] >= 0 and zeros below the diagonal. A column whose
 * norm is exactly zero gives R[k][k] = 0, a zero column of Q and a zero row
 * of R. Arithmetic is FP32 (LN_PREC_FP32 only; the forward error of Q grows
 * with the condition number of A, as for any Gram-Schmidt).
 *
 * LN_FORM_PLAIN runs the benchmark's three kernels per column (3n launches:
 * a single work-item computes the norm, one work-item per row scales, one
 * per later column projects). LN_FORM_INTERNALIZED factorises 32-column
 * panels in one CTA each (rows held in registers for m <= 1024, in shared
 * memory or L2 above) and applies each panel to the later columns in a
 * second kernel (2 ceil(n/32) launches). No workspace: Q is the working
 * array. A == Q with lda == ldq factorises in place (A is overwritten, as in
 * the benchmark); otherwise Q must not overlap A, and R overlaps neither.
 * Pointers are device memory, or pinned/managed host memory the GPU can reach
 * (slow: every column step crosses the host link). Stream-ordered.
 */
ln_status ln_gramschmidt(int m, int n, const float *A, int lda, float *Q, int ldq, float *R, int ldr, ln_form form,
                         void *stream);

/*
 * Adjoint of 3mm (ln_3mm), G = (A B)(C D): given Gb = dL/dG (ni x nl), writes
 * dA = Gb (C D)^T B^T, dB = A^T Gb (C D)^T, dC = (A B)^T Gb D^T and
 * dD = C^T (A B)^T Gb (E = A B and F = C D are recomputed in the workspace).
 * Shapes as in ln_3mm; every matrix contiguous; gradient outputs must not
 * overlap each other or an input.
 * Tensor-core forms run the two halves (E, dE, dA, dB and F, dF, dC, dD) on
 * `stream` and the library's second stream when their contractions fit on
 * the GPU side by side (stream rules as for ln_3mm).
 */
ln_status ln_3mm_bwd_workspace_size(int ni, int nj, int nk, int nl, int nm, ln_form form, ln_precision prec,
                                    size_t *bytes /*host*/);
ln_status ln_3mm_bwd(int ni, int nj, int nk, int nl, int nm, const float *A, const float *B, const float *C,
                     const float *D, const float *Gb, float *dA, float *dB, float *dC, float *dD, void *workspace,
                     size_t workspace_bytes, ln_form form, ln_precision prec, void *stream);

/*
 * Vector-Jacobian products (hand-written adjoints).
 *
 * Chain: for E = (A*B)*C and an upstream gradient G = dL/dE (ni x nl),
 *   dA = G (B C)^T,  dB = A^T G C^T,  dC = (A B)^T G.
 * All contiguous; dA/dB/dC must not overlap the inputs or each other. In the
 * tensor-core forms the dB branch (G C^T, then dB) may run on the library's
 * second stream. That happens when its contractions fit on the GPU beside
 * those of the other branches, and the stream rules are those of ln_3mm. The
 * call stays stream-ordered on `stream`.
 *
 * Covariance: for an upstream gradient W = dL/dcov (nfeat x nfeat, ldw),
 *   dX = Xc (W + W^T) / (nsamples - 1).
 * Correlation: with s_j = sqrt(ss_j), Z = Xc diag(1/s), W' = W with a zero
 * diagonal: dZ = Z (W' + W'^T); dXc_j = (dZ_j - Z_j (Z_j . dZ_j)) / s_j;
 * dX = dXc - 1 (1^T dXc) / nsamples.
 * `stats` (nullable) holds 2*nfeat doubles, mean then ss, from a forward call
 * (ln_covariance_fwd, ln_correlation_fwd or ln_col_stats), read in place;
 * when NULL they are recomputed from X. The centred matrix is
 * always recomputed from X rather than stored.
 */
ln_status ln_gemm_chain_bwd_workspace_size(int ni, int nj, int nk, int nl, ln_form form, ln_precision prec,
                                           size_t *bytes /*host*/);
ln_status ln_gemm_chain_bwd(int ni, int nj, int nk, int nl, const float *A, const float *B, const float *C,
                            const float *G, float *dA, float *dB, float *dC, void *workspace,
                            size_t workspace_bytes, ln_form form, ln_precision prec, void *stream);
ln_status ln_covariance_bwd_workspace_size(int nsamples, int nfeat, ln_form form, ln_precision prec,
                                           size_t *bytes /*host*/);
ln_status ln_covariance_bwd(int nsamples, int nfeat, const float *X, int ldx, const float *W, int ldw,
                            const double *stats, float *dX, int lddx, void *workspace, size_t workspace_bytes,
                            ln_form form, ln_precision prec, void *stream);
ln_status ln_correlation_bwd(int nsamples, int nfeat, const float *X, int ldx, const float *W, int ldw,
                             const double *stats, float *dX, int lddx, void *workspace,
                             size_t workspace_bytes, ln_form form, ln_precision prec, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* LOOPNEST_H */
