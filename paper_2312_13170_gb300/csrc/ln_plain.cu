// Plain form of every loop nest: one thread per output element, the inner
// loop reading its operands straight from global memory, the sum held in a
// register and stored once. This is the kernel of paper Sec. VI-C, Listing 5
// after the array-reduction detection of Sec. VI-B (no local-memory tiles).
#include "ln_epilogue.cuh"
#include "ln_internal.h"

namespace ln {

// acc(i,j) = sum_k A[i*sai + k*sak] * B[k*sbk + j*sbj]; j runs along threadIdx.x
// so that row-major B and the output are accessed contiguously by a warp.
__global__ void k_plain_gemm(int M, int N, int K, const float *__restrict__ A, long long sai, long long sak,
                             const float *__restrict__ B, long long sbk, long long sbj, EpiParams epi) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    int i = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= M || j >= N) return;
    const float *a = A + (long long)i * sai;
    const float *b = B + (long long)j * sbj;
    float acc = 0.0f;
    for (int k = 0; k < K; ++k) acc = fmaf(a[(long long)k * sak], b[(long long)k * sbk], acc);
    epi_store(epi, i, j, acc);
}

ln_status plain_gemm(int M, int N, int K, const float *A, long long sai, long long sak, const float *B,
                     long long sbk, long long sbj, const EpiParams &epi, cudaStream_t st) {
    dim3 block(32, 8);
    dim3 grid((unsigned)ceil_div(N, 32), (unsigned)ceil_div(M, 8));
    { LaunchScope ls_(FAM_PLAIN, st); k_plain_gemm<<<grid, block, 0, st>>>(M, N, K, A, sai, sak, B, sbk, sbj, epi); }
    return check_launch("plain gemm");
}

// One thread per column: the two passes of the column statistics in FP64.
__global__ void k_plain_col_stats(int n, int m, const float *__restrict__ X, long long ldx, double *mean,
                                  double *ss) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= m) return;
    double s = 0.0;
    for (int r = 0; r < n; ++r) s += (double)X[(long long)r * ldx + j];
    double mu = s / (double)n;
    double q = 0.0;
    for (int r = 0; r < n; ++r) {
        double d = (double)X[(long long)r * ldx + j] - mu;
        q = fma(d, d, q);
    }
    mean[j] = mu;
    ss[j] = q;
}

ln_status plain_col_stats(int n, int m, const float *X, long long ldx, double *mean, double *ss, cudaStream_t st) {
    { LaunchScope ls_(FAM_PLAIN, st); k_plain_col_stats<<<(unsigned)ceil_div(m, 128), 128, 0, st>>>(n, m, X, ldx, mean, ss); }
    return check_launch("plain column statistics");
}

// One thread per lower-triangle output (i >= j) of Xc^T Xc, centring each
// operand on the fly with the FP64 mean split into two floats.
__global__ void k_plain_cov(int n, int m, const float *__restrict__ X, long long ldx, const double *__restrict__ mean,
                            EpiParams epi) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    int i = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= m || j >= m || i < j) return;
    float hi_i = (float)mean[i], lo_i = (float)(mean[i] - (double)hi_i);
    float hi_j = (float)mean[j], lo_j = (float)(mean[j] - (double)hi_j);
    float acc = 0.0f;
    for (int r = 0; r < n; ++r) {
        const float *x = X + (long long)r * ldx;
        float xi = (x[i] - hi_i) - lo_i;
        float xj = (x[j] - hi_j) - lo_j;
        acc = fmaf(xi, xj, acc);
    }
    epi_store(epi, i, j, acc);
}

ln_status plain_cov(int n, int m, const float *X, long long ldx, const double *mean, const EpiParams &epi,
                    cudaStream_t st) {
    dim3 block(32, 8);
    dim3 grid((unsigned)ceil_div(m, 32), (unsigned)ceil_div(m, 8));
    { LaunchScope ls_(FAM_PLAIN, st); k_plain_cov<<<grid, block, 0, st>>>(n, m, X, ldx, mean, epi); }
    return check_launch("plain covariance");
}

// One thread per lower-triangle output of SYRK (B == nullptr) or SYR2K.
__global__ void k_plain_sym(int n, int k, const float *__restrict__ A, long long lda, const float *__restrict__ B,
                            long long ldb, EpiParams epi) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    int i = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= n || j >= n || i < j) return;
    const float *ai = A + (long long)i * lda, *aj = A + (long long)j * lda;
    float acc = 0.0f;
    if (B == nullptr) {
        for (int q = 0; q < k; ++q) acc = fmaf(ai[q], aj[q], acc);
    } else {
        const float *bi = B + (long long)i * ldb, *bj = B + (long long)j * ldb;
        for (int q = 0; q < k; ++q) acc = fmaf(bi[q], aj[q], fmaf(ai[q], bj[q], acc));
    }
    epi_store(epi, i, j, acc);
}

ln_status plain_sym(int n, int k, const float *A, long long lda, const float *B, long long ldb, const EpiParams &epi,
                    cudaStream_t st) {
    dim3 block(32, 8);
    dim3 grid((unsigned)ceil_div(n, 32), (unsigned)ceil_div(n, 8));
    { LaunchScope ls_(FAM_PLAIN, st); k_plain_sym<<<grid, block, 0, st>>>(n, k, A, lda, B, ldb, epi); }
    return check_launch("plain syrk/syr2k");
}

// Batched plain SYRK/SYR2K: blockIdx.z selects the instance.
__global__ void k_plain_sym_batched(int is_syr2k, const ln_sym_desc *__restrict__ descs, int fill, float alpha,
                                    float beta) {
    const ln_sym_desc d = descs[blockIdx.z];
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    int i = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= d.n || j >= d.n || i < j) return;
    const float *ai = d.A + (long long)i * d.lda, *aj = d.A + (long long)j * d.lda;
    float acc = 0.0f;
    if (!is_syr2k) {
        for (int q = 0; q < d.k; ++q) acc = fmaf(ai[q], aj[q], acc);
    } else {
        const float *bi = d.B + (long long)i * d.ldb, *bj = d.B + (long long)j * d.ldb;
        for (int q = 0; q < d.k; ++q) acc = fmaf(bi[q], aj[q], fmaf(ai[q], bj[q], acc));
    }
    EpiParams e{};
    e.mode = EPI_SYM;
    e.M = e.N = d.n;
    e.alpha = alpha;
    e.beta = beta;
    e.C = d.C;
    e.ldc = d.ldc;
    e.fill = fill;
    e.sym_kind = SYM_AXPBY;
    epi_store(e, i, j, acc);
}

ln_status plain_sym_batched(int is_syr2k, int count, const ln_sym_desc *d_descs, int max_n, int fill, float alpha,
                            float beta, cudaStream_t st) {
    dim3 block(32, 8);
    dim3 grid((unsigned)ceil_div(max_n, 32), (unsigned)ceil_div(max_n, 8), (unsigned)count);
    { LaunchScope ls_(FAM_PLAIN, st); k_plain_sym_batched<<<grid, block, 0, st>>>(is_syr2k, d_descs, fill, alpha, beta); }
    return check_launch("plain batched syrk/syr2k");
}

}  // namespace ln
