// Column statistics and the small element-wise / column-wise kernels around
// the contractions (centring, weight symmetrisation, the correlation adjoint).
//
// The column mean and sum of squared deviations are the array reductions of
// polybench covariance/correlation (paper Sec. VI-B, Sec. VIII). Internalized
// form: each CTA reduces a 128-column x 256-row block with coalesced 128-bit
// loads, accumulating in registers (compensated FP32 pairs, see
// k_col_partial), combines its 8 row groups in shared memory in FP64 and
// writes one FP64 partial per column; a second kernel adds the partials in a
// fixed order (deterministic, no atomics). Two passes: the mean first, then
// the squared deviations from it.
#include "ln_internal.h"

namespace ln {

namespace {

inline unsigned rows_grid(long long rows) { return (unsigned)(rows < 65535 ? rows : 65535); }

constexpr int SC = 128;  // columns per CTA (32 threads x float4)
constexpr int SR = 256;  // rows per CTA

__device__ __forceinline__ float4 ld4_guard(const float *row, int c, int m, bool vec) {
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (vec && c + 3 < m) return __ldg(reinterpret_cast<const float4 *>(row + c));
    if (c + 0 < m) v.x = __ldg(row + c + 0);
    if (c + 1 < m) v.y = __ldg(row + c + 1);
    if (c + 2 < m) v.z = __ldg(row + c + 2);
    if (c + 3 < m) v.w = __ldg(row + c + 3);
    return v;
}

// s + t == a + b exactly (Knuth's error-free sum; no reassociation is allowed
// because the library is compiled without fast-math).
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &t) {
    s = a + b;
    const float bp = s - a;
    t = (a - (s - bp)) + (b - bp);
}

// pass 0: partial sums of X; pass 1: partial sums of (X - mean)^2.
// Each thread keeps its running sums as unevaluated FP32 pairs (hi + lo, hi
// accumulating with error-free sums whose errors gather in lo). In pass 1 the
// FP64 mean is split as mh + ml (two floats); the deviation from mh,
// d = x - mh, is formed exactly as a pair and the thread accumulates S1 = sum d
// and S2 = sum d^2 (squares carry their exact FMA residual). Its share of the
// squared deviations from the FP64 mean then follows in FP64 as
// S2 - 2 ml S1 + cnt ml^2, so ml never enters a product of small numbers.
// The pairs are widened to FP64 for the combination across threads and
// blocks. GB300 issues FP64 at a small fraction of its FP32 rate, so native
// FP64 per element made this bandwidth-bound pass compute-bound; the pairs
// keep FP64-level accuracy at FP32 speed.
template <int PASS>
__global__ __launch_bounds__(256) void k_col_partial(int n, int m, const float *__restrict__ X, long long ldx,
                                                     const double *__restrict__ mean, double *partials) {
    __shared__ double red[8][SC];
    const int cx = threadIdx.x & 31, ry = threadIdx.x >> 5;
    const int c = blockIdx.x * SC + cx * 4;
    const int r0 = blockIdx.y * SR;
    const bool vec = ((reinterpret_cast<uintptr_t>(X) & 15) == 0) && ((ldx & 3) == 0);
    float mh[4] = {0, 0, 0, 0};
    double ml[4] = {0, 0, 0, 0};
    if (PASS == 1) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const double mu = (c + q < m) ? mean[c + q] : 0.0;
            mh[q] = (float)mu;
            ml[q] = mu - (double)mh[q];
        }
    }
    float h1[4] = {0, 0, 0, 0}, l1[4] = {0, 0, 0, 0};  // sum x (pass 0) or sum d (pass 1)
    float h2[4] = {0, 0, 0, 0}, l2[4] = {0, 0, 0, 0};  // sum d^2 (pass 1)
    int cnt = 0;
    const int r1 = min(n, r0 + SR);
#pragma unroll 4
    for (int r = r0 + ry; r < r1; r += 8) {
        float4 v = ld4_guard(X + (long long)r * ldx, c, m, vec);
        float x[4] = {v.x, v.y, v.z, v.w};
        ++cnt;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            float s, t;
            if (PASS == 0) {
                two_sum(h1[q], x[q], s, t);
                h1[q] = s;
                l1[q] += t;
            } else {
                float dh, dl;
                two_sum(x[q], -mh[q], dh, dl);
                two_sum(h1[q], dh, s, t);
                h1[q] = s;
                l1[q] += t + dl;
                const float p = dh * dh;
                const float pe = fmaf(dh, dh, -p) + (2.0f * dh + dl) * dl;
                two_sum(h2[q], p, s, t);
                h2[q] = s;
                l2[q] += t + pe;
            }
        }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const double s1 = (double)h1[q] + (double)l1[q];
        if (PASS == 0) {
            red[ry][cx * 4 + q] = s1;
        } else {
            const double s2 = (double)h2[q] + (double)l2[q];
            red[ry][cx * 4 + q] = s2 - 2.0 * ml[q] * s1 + (double)cnt * ml[q] * ml[q];
        }
    }
    __syncthreads();
    if (threadIdx.x < SC) {
        int col = blockIdx.x * SC + threadIdx.x;
        double s = 0.0;
#pragma unroll
        for (int g = 0; g < 8; ++g) s += red[g][threadIdx.x];
        if (col < m) partials[(long long)blockIdx.y * m + col] = s;
    }
}

template <int PASS>
__global__ void k_col_final(int n, int m, int nchunks, const double *__restrict__ partials, double *out) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= m) return;
    double s = 0.0;
    for (int ch = 0; ch < nchunks; ++ch) s += partials[(long long)ch * m + j];
    out[j] = (PASS == 0) ? s / (double)n : s;
}

__global__ void k_derive(int m, const double *__restrict__ mean, const double *__restrict__ ss, float *off_hi,
                         float *off_lo, float *rs) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= m) return;
    if (off_hi) {
        double mu = mean[j];
        float h = (float)mu;
        off_hi[j] = h;
        off_lo[j] = (float)(mu - (double)h);
    }
    if (rs) {
        double q = ss[j];
        rs[j] = (q > 0.0) ? (float)(1.0 / sqrt(q)) : 0.0f;
    }
}

__global__ void k_scale(int M, int N, float beta, float *C, long long ldc) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= N) return;
    for (int i = blockIdx.y; i < M; i += gridDim.y) {
        float *c = C + (long long)i * ldc + j;
        *c = (beta == 0.0f) ? 0.0f : beta * *c;
    }
}

__global__ void k_sym_scale(int n, int fill, float beta, float *C, long long ldc) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    for (int i = blockIdx.y; i < n; i += gridDim.y) {
        if (i < j) continue;
        long long lo = (long long)i * ldc + j, up = (long long)j * ldc + i;
        long long src = (fill == LN_FILL_UPPER) ? up : lo;
        float v = (beta == 0.0f) ? 0.0f : beta * C[src];
        if (fill == LN_FILL_FULL) {
            C[lo] = v;
            C[up] = v;
        } else {
            C[src] = v;
        }
    }
}

__global__ void k_center(int n, int m, const float *__restrict__ X, long long ldx, const float *__restrict__ hi,
                         const float *__restrict__ lo, const float *__restrict__ rs, float *Y, long long ldy) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= m) return;
    for (int r = blockIdx.y; r < n; r += gridDim.y) {
        float v = (X[(long long)r * ldx + j] - hi[j]) - lo[j];
        if (rs) v *= rs[j];
        Y[(long long)r * ldy + j] = v;
    }
}

__global__ void k_symw(int m, const float *__restrict__ W, long long ldw, float scale, int zero_diag, float *Ws) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= m) return;
    for (int i = blockIdx.y; i < m; i += gridDim.y) {
        float v = scale * (W[(long long)i * ldw + j] + W[(long long)j * ldw + i]);
        if (zero_diag && i == j) v = 0.0f;
        Ws[(long long)i * m + j] = v;
    }
}

// Partial column sums of Z .* dZ (PASS 0) or of dX (PASS 1) over 128-row chunks.
template <int PASS>
__global__ __launch_bounds__(256) void k_pair_partial(int n, int m, const float *__restrict__ Z, long long ldz,
                                                      const float *__restrict__ dZ, long long lddz,
                                                      double *partials) {
    __shared__ double red[8][SC];
    const int cx = threadIdx.x & 31, ry = threadIdx.x >> 5;
    const int r0 = blockIdx.y * SR;
    double acc[4] = {0, 0, 0, 0};
    for (int r = r0 + ry; r < min(n, r0 + SR); r += 8) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            int c = blockIdx.x * SC + cx * 4 + q;
            if (c < m) {
                float a = Z[(long long)r * ldz + c];
                acc[q] += (PASS == 0) ? (double)a * (double)dZ[(long long)r * lddz + c] : (double)a;
            }
        }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) red[ry][cx * 4 + q] = acc[q];
    __syncthreads();
    if (threadIdx.x < SC) {
        int col = blockIdx.x * SC + threadIdx.x;
        double s = 0.0;
#pragma unroll
        for (int g = 0; g < 8; ++g) s += red[g][threadIdx.x];
        if (col < m) partials[(long long)blockIdx.y * m + col] = s;
    }
}

__global__ void k_sum_partials(int m, int nchunks, const double *__restrict__ partials, double *out) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= m) return;
    double s = 0.0;
    for (int ch = 0; ch < nchunks; ++ch) s += partials[(long long)ch * m + j];
    out[j] = s;
}

// dX = (dZ - Z * dot) * rs   (the adjoint of the column normalisation)
__global__ void k_corr_dxc(int n, int m, const float *__restrict__ Z, long long ldz, const float *__restrict__ dZ,
                           long long lddz, const double *__restrict__ dot, const float *__restrict__ rs, float *dX,
                           long long lddx) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= m) return;
    const float d = (float)dot[j], s = rs[j];
    for (int r = blockIdx.y; r < n; r += gridDim.y) {
        float z = Z[(long long)r * ldz + j];
        float g = dZ[(long long)r * lddz + j];
        dX[(long long)r * lddx + j] = (g - z * d) * s;
    }
}

// dX -= colsum / n   (the adjoint of the centring)
__global__ void k_sub_colmean(int n, int m, const double *__restrict__ colsum, float *dX, long long lddx) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= m) return;
    const float c = (float)(colsum[j] / (double)n);
    for (int r = blockIdx.y; r < n; r += gridDim.y) dX[(long long)r * lddx + j] -= c;
}

}  // namespace

size_t col_stats_partials_bytes(int n, int m) { return sizeof(double) * (size_t)ceil_div(n, SR) * (size_t)m; }

ln_status col_stats(int n, int m, const float *X, long long ldx, double *mean, double *ss, float *off_hi,
                    float *off_lo, float *rs, double *partials, cudaStream_t st) {
    const int nch = (int)ceil_div(n, SR);
    dim3 grid((unsigned)ceil_div(m, SC), (unsigned)nch);
    { LaunchScope ls_(FAM_STATS, st); k_col_partial<0><<<grid, 256, 0, st>>>(n, m, X, ldx, nullptr, partials); }
    { LaunchScope ls_(FAM_STATS, st); k_col_final<0><<<(unsigned)ceil_div(m, 256), 256, 0, st>>>(n, m, nch, partials, mean); }
    { LaunchScope ls_(FAM_STATS, st); k_col_partial<1><<<grid, 256, 0, st>>>(n, m, X, ldx, mean, partials); }
    { LaunchScope ls_(FAM_STATS, st); k_col_final<1><<<(unsigned)ceil_div(m, 256), 256, 0, st>>>(n, m, nch, partials, ss); }
    if (off_hi || rs) {
        LaunchScope ls_(FAM_STATS, st);
        k_derive<<<(unsigned)ceil_div(m, 256), 256, 0, st>>>(m, mean, ss, off_hi, off_lo, rs);
    }
    return check_launch("column statistics");
}

ln_status stats_derive(int m, const double *mean, const double *ss, float *off_hi, float *off_lo, float *rs,
                       cudaStream_t st) {
    { LaunchScope ls_(FAM_STATS, st); k_derive<<<(unsigned)ceil_div(m, 256), 256, 0, st>>>(m, mean, ss, off_hi, off_lo, rs); }
    return check_launch("statistics derive");
}

ln_status scale_matrix(int M, int N, float beta, float *C, long long ldc, cudaStream_t st) {
    if (M == 0 || N == 0) return LN_SUCCESS;
    { LaunchScope ls_(FAM_STATS, st); k_scale<<<dim3((unsigned)ceil_div(N, 256), rows_grid(M)), 256, 0, st>>>(M, N, beta, C, ldc); }
    return check_launch("scale");
}

ln_status sym_fill_zero_k(int n, int fill, float beta, float *C, long long ldc, cudaStream_t st) {
    if (n == 0) return LN_SUCCESS;
    { LaunchScope ls_(FAM_STATS, st); k_sym_scale<<<dim3((unsigned)ceil_div(n, 256), rows_grid(n)), 256, 0, st>>>(n, fill, beta, C, ldc); }
    return check_launch("symmetric scale");
}

ln_status center_matrix(int n, int m, const float *X, long long ldx, const float *off_hi, const float *off_lo,
                        const float *rs, float *Y, long long ldy, cudaStream_t st) {
    { LaunchScope ls_(FAM_STATS, st); k_center<<<dim3((unsigned)ceil_div(m, 256), rows_grid(n)), 256, 0, st>>>(n, m, X, ldx, off_hi, off_lo, rs, Y, ldy); }
    return check_launch("centre");
}

ln_status symmetrize_weights(int m, const float *W, long long ldw, float scale, int zero_diag, float *Ws,
                             cudaStream_t st) {
    { LaunchScope ls_(FAM_STATS, st); k_symw<<<dim3((unsigned)ceil_div(m, 256), rows_grid(m)), 256, 0, st>>>(m, W, ldw, scale, zero_diag, Ws); }
    return check_launch("symmetrise weights");
}

size_t corr_bwd_partials_bytes(int n, int m) {
    return sizeof(double) * ((size_t)ceil_div(n, SR) * (size_t)m + 2 * (size_t)m);
}

ln_status corr_bwd_finish(int n, int m, const float *Z, long long ldz, const float *dZ, long long lddz,
                          const float *rs, float *dX, long long lddx, double *partials, cudaStream_t st) {
    const int nch = (int)ceil_div(n, SR);
    double *dot = partials + (size_t)nch * m;
    double *colsum = dot + m;
    dim3 grid((unsigned)ceil_div(m, SC), (unsigned)nch);
    dim3 g2((unsigned)ceil_div(m, 256), rows_grid(n));
    { LaunchScope ls_(FAM_STATS, st); k_pair_partial<0><<<grid, 256, 0, st>>>(n, m, Z, ldz, dZ, lddz, partials); }
    { LaunchScope ls_(FAM_STATS, st); k_sum_partials<<<(unsigned)ceil_div(m, 256), 256, 0, st>>>(m, nch, partials, dot); }
    { LaunchScope ls_(FAM_STATS, st); k_corr_dxc<<<g2, 256, 0, st>>>(n, m, Z, ldz, dZ, lddz, dot, rs, dX, lddx); }
    { LaunchScope ls_(FAM_STATS, st); k_pair_partial<1><<<grid, 256, 0, st>>>(n, m, dX, lddx, nullptr, 0, partials); }
    { LaunchScope ls_(FAM_STATS, st); k_sum_partials<<<(unsigned)ceil_div(m, 256), 256, 0, st>>>(m, nch, partials, colsum); }
    { LaunchScope ls_(FAM_STATS, st); k_sub_colmean<<<g2, 256, 0, st>>>(n, m, colsum, dX, lddx); }
    return check_launch("correlation adjoint");
}

}  // namespace ln
