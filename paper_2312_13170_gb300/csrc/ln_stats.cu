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
#include "ln_async.cuh"
#include "ln_internal.h"
#include "ln_launch.h"
#include "ln_stats.h"

#define LN_TRY_STATUS(expr)            \
    do {                               \
        const ln_status s_ = (expr);   \
        if (s_ != LN_SUCCESS) return s_; \
    } while (0)

namespace ln {

namespace {

inline unsigned rows_grid(long long rows) { return (unsigned)(rows < 65535 ? rows : 65535); }

constexpr int SC = 128;  // columns per CTA (32 threads x float4)
constexpr int EW_ROWS = 32;  // rows per CTA of the element-wise kernels

// Rows per CTA of the column reductions: the largest of 256, 128, 64 that
// still gives about four CTAs per SM of a 152-SM GPU (a fixed target, so that
// workspace sizes do not depend on the device).
int stats_rows(int n, int m) {
    const long long colb = ceil_div(m, SC);
    for (int sr = 256; sr > 64; sr >>= 1)
        if (colb * ceil_div(n, sr) >= 608) return sr;
    return 64;
}

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
// d = x - mh, is formed exactly as a pair (dh, dl) and the thread accumulates
// sum d^2 (the square of the pair, carrying its exact FMA residual). Because
// the deviations from the mean sum to zero, sum (x - mean)^2 =
// sum (x - mh)^2 - n ml^2; the final kernel subtracts n ml^2 once per column.
// The pairs are widened to FP64 for the combination across threads and
// blocks. GB300 issues FP64 at a small fraction of its FP32 rate, so native
// FP64 per element made this bandwidth-bound pass compute-bound; the pairs
// keep FP64-level accuracy at FP32 speed.
template <int PASS>
__global__ __launch_bounds__(256) void k_col_partial(int n, int m, const float *__restrict__ X, long long ldx,
                                                     const double *__restrict__ mean, double *partials, int sr) {
    __shared__ float red_h[8][SC], red_l[8][SC];
    const int cx = threadIdx.x & 31, ry = threadIdx.x >> 5;
    const int c = blockIdx.x * SC + cx * 4;
    const int r0 = blockIdx.y * sr;
    pdl_wait();  // X and the mean may come from the preceding launch
    pdl_trigger();
    const bool vec = ((reinterpret_cast<uintptr_t>(X) & 15) == 0) && ((ldx & 3) == 0);
    float mh[4] = {0, 0, 0, 0};
    if (PASS == 1) {
#pragma unroll
        for (int q = 0; q < 4; ++q) mh[q] = (c + q < m) ? (float)mean[c + q] : 0.0f;
    }
    float h[4] = {0, 0, 0, 0}, l[4] = {0, 0, 0, 0};  // sum x (pass 0) or sum d^2 (pass 1)
    const int r1 = min(n, r0 + sr);
#pragma unroll 8
    for (int r = r0 + ry; r < r1; r += 8) {
        float4 v = ld4_guard(X + (long long)r * ldx, c, m, vec);
        float x[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            float s, t;
            if (PASS == 0) {
                two_sum(h[q], x[q], s, t);
                h[q] = s;
                l[q] += t;
            } else {
                float dh, dl;
                two_sum(x[q], -mh[q], dh, dl);
                const float p = dh * dh;
                const float pe = fmaf(dh, dh, -p) + (2.0f * dh + dl) * dl;
                two_sum(h[q], p, s, t);
                h[q] = s;
                l[q] += t + pe;
            }
        }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        red_h[ry][cx * 4 + q] = h[q];
        red_l[ry][cx * 4 + q] = l[q];
    }
    __syncthreads();
    // the 8 row groups' pairs combine in FP32 with the same error-free sum (FP64
    // is a narrow pipe on this GPU); one FP64 value per column leaves the CTA
    if (threadIdx.x < SC) {
        const int col = blockIdx.x * SC + threadIdx.x;
        float H = red_h[0][threadIdx.x], L = red_l[0][threadIdx.x];
#pragma unroll
        for (int g = 1; g < 8; ++g) {
            float s, t;
            two_sum(H, red_h[g][threadIdx.x], s, t);
            H = s;
            L += t + red_l[g][threadIdx.x];
        }
        if (col < m) partials[(long long)blockIdx.y * m + col] = (double)H + (double)L;
    }
}

// Sum of each column's chunk partials, 8 threads per column (strided over the
// chunks, coalesced across columns) combined in a fixed order. PASS 0 writes
// the mean; PASS 1 writes the sum of squared deviations and, on request, the
// centring pair (hi + lo = mean) and 1/sqrt(ss) (0 for a zero-variance column).
template <int PASS>
__global__ __launch_bounds__(256) void k_col_final(int n, int m, int nchunks, const double *__restrict__ partials,
                                                   const double *__restrict__ mean, double *out, float *off_hi,
                                                   float *off_lo, float *rs) {
    __shared__ double red[8][32];
    const int cx = threadIdx.x & 31, g = threadIdx.x >> 5;
    const int j = blockIdx.x * 32 + cx;
    pdl_wait();  // the partial sums come from the preceding launch
    pdl_trigger();
    double s = 0.0;
    if (j < m)
        for (int ch = g; ch < nchunks; ch += 8) s += partials[(long long)ch * m + j];
    red[g][cx] = s;
    __syncthreads();
    if (g != 0 || j >= m) return;
#pragma unroll
    for (int k = 1; k < 8; ++k) s += red[k][cx];
    if (PASS == 0) {
        const double mu = s / (double)n;
        out[j] = mu;
        if (off_hi) {  // centring pair from the mean (mean-only statistics)
            const float h = (float)mu;
            off_hi[j] = h;
            off_lo[j] = (float)(mu - (double)h);
        }
        return;
    }
    const double mu = mean[j];
    const float h = (float)mu;
    const double ml = mu - (double)h;
    double q = s - (double)n * ml * ml;
    if (q < 0.0) q = 0.0;
    out[j] = q;
    if (off_hi) {
        off_hi[j] = h;
        off_lo[j] = (float)ml;
    }
    if (rs) rs[j] = (q > 0.0) ? (float)(1.0 / sqrt(q)) : 0.0f;
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

// Element-wise kernels: a CTA of 64 x 4 threads covers 256 columns x EW_ROWS
// rows, each thread 4 consecutive columns (one 16-byte access when the rows
// are 16-byte aligned) of every fourth row.
__device__ __forceinline__ void ld4(const float *row, int c, int m, bool vec, float (&v)[4]) {
    if (vec && c + 3 < m) {
        const float4 x = __ldg(reinterpret_cast<const float4 *>(row + c));
        v[0] = x.x; v[1] = x.y; v[2] = x.z; v[3] = x.w;
        return;
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) v[q] = (c + q < m) ? __ldg(row + c + q) : 0.0f;
}
__device__ __forceinline__ void st4(float *row, int c, int m, bool vec, const float (&v)[4]) {
    if (vec && c + 3 < m) {
        *reinterpret_cast<float4 *>(row + c) = make_float4(v[0], v[1], v[2], v[3]);
        return;
    }
#pragma unroll
    for (int q = 0; q < 4; ++q)
        if (c + q < m) row[c + q] = v[q];
}

// Y = (X - (hi + lo)) * rs, column-wise offsets and scales (rs optional)
__global__ __launch_bounds__(256) void k_center(int n, int m, const float *__restrict__ X, long long ldx,
                                                const float *__restrict__ hi, const float *__restrict__ lo,
                                                const float *__restrict__ rs, float *Y, long long ldy, int vec) {
    const int c = (blockIdx.x * 64 + threadIdx.x) * 4;
    if (c >= m) return;
    float h[4], l[4], sc[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const bool in = c + q < m;
        h[q] = in ? hi[c + q] : 0.0f;
        l[q] = in ? lo[c + q] : 0.0f;
        sc[q] = (in && rs) ? rs[c + q] : 1.0f;
    }
    const int r0 = blockIdx.y * EW_ROWS, r1 = min(n, r0 + EW_ROWS);
    for (int r = r0 + threadIdx.y; r < r1; r += 4) {
        float v[4];
        ld4(X + (long long)r * ldx, c, m, vec != 0, v);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            v[q] = (v[q] - h[q]) - l[q];
            if (rs) v[q] *= sc[q];
        }
        st4(Y + (long long)r * ldy, c, m, vec != 0, v);
    }
}

// Ws = scale * (W + W^T) (diagonal zeroed on request), through a 32 x 32
// shared-memory tile so that both W reads are coalesced.
__global__ __launch_bounds__(256) void k_symw(int m, const float *__restrict__ W, long long ldw, float scale,
                                              int zero_diag, float *Ws) {
    __shared__ float t[32][33];
    const int bi = blockIdx.y * 32, bj = blockIdx.x * 32, tx = threadIdx.x, ty = threadIdx.y;
    for (int k = ty; k < 32; k += 8) {  // t[k][tx] = W[bj + k][bi + tx]
        const int r = bj + k, c = bi + tx;
        t[k][tx] = (r < m && c < m) ? W[(long long)r * ldw + c] : 0.0f;
    }
    __syncthreads();
    for (int k = ty; k < 32; k += 8) {
        const int i = bi + k, j = bj + tx;
        if (i < m && j < m) {
            float v = scale * (W[(long long)i * ldw + j] + t[tx][k]);  // W[j][i] = t[j - bj][i - bi]
            if (zero_diag && i == j) v = 0.0f;
            Ws[(long long)i * m + j] = v;
        }
    }
}

// Per-column partial sums over a chunk of rows, for the correlation adjoint:
// S0 = sum Z.*dZ, S1 = sum dZ, S2 = sum Z, each kept per thread as a
// compensated FP32 pair (products carry their exact FMA residual) and
// combined across the CTA in FP64. partials = [3][nchunks][m].
__global__ __launch_bounds__(256) void k_corr_cols(int n, int m, const float *__restrict__ Z, long long ldz,
                                                   const float *__restrict__ dZ, long long lddz, double *partials,
                                                   int sr, int nch) {
    __shared__ double red[3][8][SC];
    const int cx = threadIdx.x & 31, ry = threadIdx.x >> 5;
    const int c = blockIdx.x * SC + cx * 4;
    const int r0 = blockIdx.y * sr, r1 = min(n, r0 + sr);
    const bool vz = ((reinterpret_cast<uintptr_t>(Z) & 15) == 0) && ((ldz & 3) == 0);
    const bool vd = ((reinterpret_cast<uintptr_t>(dZ) & 15) == 0) && ((lddz & 3) == 0);
    float h[3][4] = {}, l[3][4] = {};
#pragma unroll 2
    for (int r = r0 + ry; r < r1; r += 8) {
        float z[4], g[4];
        ld4(Z + (long long)r * ldz, c, m, vz, z);
        ld4(dZ + (long long)r * lddz, c, m, vd, g);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            float s, t;
            const float p = z[q] * g[q], pe = fmaf(z[q], g[q], -p);
            two_sum(h[0][q], p, s, t);
            h[0][q] = s;
            l[0][q] += t + pe;
            two_sum(h[1][q], g[q], s, t);
            h[1][q] = s;
            l[1][q] += t;
            two_sum(h[2][q], z[q], s, t);
            h[2][q] = s;
            l[2][q] += t;
        }
    }
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int q = 0; q < 4; ++q) red[k][ry][cx * 4 + q] = (double)h[k][q] + (double)l[k][q];
    __syncthreads();
    if (threadIdx.x < SC) {
        const int col = blockIdx.x * SC + threadIdx.x;
        if (col < m) {
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                double s = 0.0;
#pragma unroll
                for (int gi = 0; gi < 8; ++gi) s += red[k][gi][threadIdx.x];
                partials[((long long)k * nch + blockIdx.y) * m + col] = s;
            }
        }
    }
}

// d_j = sum_r Z dZ and the column mean of dXc = (dZ - Z d) rs, which is
// rs_j (sum dZ - d_j sum Z) / n (the adjoint of the centring subtracts it).
// Column sums of the three partial-sum sets: a CTA takes 32 columns (lane =
// column, coalesced), its 8 warps take every 8th row chunk, and the warps'
// sums are added in warp order (deterministic).
__global__ __launch_bounds__(256) void k_corr_cols_final(int n, int m, int nch, const double *__restrict__ partials,
                                                         const float *__restrict__ rs, float *d, float *cmean) {
    __shared__ double red[3][8][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int j = blockIdx.x * 32 + lane;
    double s0 = 0.0, s1 = 0.0, s2 = 0.0;
    if (j < m) {
#pragma unroll 4
        for (int ch = w; ch < nch; ch += 8) {
            s0 += partials[(long long)ch * m + j];
            s1 += partials[((long long)nch + ch) * m + j];
            s2 += partials[(2LL * nch + ch) * m + j];
        }
    }
    red[0][w][lane] = s0;
    red[1][w][lane] = s1;
    red[2][w][lane] = s2;
    __syncthreads();
    if (w == 0 && j < m) {
        double t0 = 0.0, t1 = 0.0, t2 = 0.0;
#pragma unroll
        for (int g = 0; g < 8; ++g) {
            t0 += red[0][g][lane];
            t1 += red[1][g][lane];
            t2 += red[2][g][lane];
        }
        d[j] = (float)t0;
        cmean[j] = (float)((double)rs[j] * (t1 - t0 * t2) / (double)n);
    }
}

// dX = (dZ - Z * d) * rs - cmean
__global__ __launch_bounds__(256) void k_corr_dx(int n, int m, const float *__restrict__ Z, long long ldz,
                                                 const float *__restrict__ dZ, long long lddz,
                                                 const float *__restrict__ d, const float *__restrict__ rs,
                                                 const float *__restrict__ cmean, float *dX, long long lddx, int vec) {
    const int c = (blockIdx.x * 64 + threadIdx.x) * 4;
    if (c >= m) return;
    float dd[4], sc[4], cm[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const bool in = c + q < m;
        dd[q] = in ? d[c + q] : 0.0f;
        sc[q] = in ? rs[c + q] : 0.0f;
        cm[q] = in ? cmean[c + q] : 0.0f;
    }
    const int r0 = blockIdx.y * EW_ROWS, r1 = min(n, r0 + EW_ROWS);
    for (int r = r0 + threadIdx.y; r < r1; r += 4) {
        float z[4], g[4];
        ld4(Z + (long long)r * ldz, c, m, vec != 0, z);
        ld4(dZ + (long long)r * lddz, c, m, vec != 0, g);
#pragma unroll
        for (int q = 0; q < 4; ++q) g[q] = fmaf(-z[q], dd[q], g[q]) * sc[q] - cm[q];
        st4(dX + (long long)r * lddx, c, m, vec != 0, g);
    }
}

}  // namespace

size_t col_stats_partials_bytes(int n, int m) {
    return sizeof(double) * (size_t)ceil_div(n, stats_rows(n, m)) * (size_t)m;
}

ln_status col_stats(int n, int m, const float *X, long long ldx, double *mean, double *ss, float *off_hi,
                    float *off_lo, float *rs, double *partials, cudaStream_t st) {
    const int sr = stats_rows(n, m);
    const int nch = (int)ceil_div(n, sr);
    dim3 grid((unsigned)ceil_div(m, SC), (unsigned)nch);
    const unsigned gf = (unsigned)ceil_div(m, 32);
    const double *no_mean = nullptr;
    float *no_f = nullptr;
    {
        LaunchScope ls_(FAM_STATS, st);
        LN_TRY_STATUS(pdl_launch(k_col_partial<0>, grid, dim3(256), 0, st, "column statistics", n, m, X, ldx, no_mean,
                                 partials, sr));
    }
    {
        LaunchScope ls_(FAM_STATS, st);
        LN_TRY_STATUS(pdl_launch(k_col_final<0>, dim3(gf), dim3(256), 0, st, "column statistics", n, m, nch,
                                 (const double *)partials, no_mean, mean, no_f, no_f, no_f));
    }
    {
        LaunchScope ls_(FAM_STATS, st);
        LN_TRY_STATUS(pdl_launch(k_col_partial<1>, grid, dim3(256), 0, st, "column statistics", n, m, X, ldx,
                                 (const double *)mean, partials, sr));
    }
    {
        LaunchScope ls_(FAM_STATS, st);
        LN_TRY_STATUS(pdl_launch(k_col_final<1>, dim3(gf), dim3(256), 0, st, "column statistics", n, m, nch,
                                 (const double *)partials, (const double *)mean, ss, off_hi, off_lo, rs));
    }
    return LN_SUCCESS;
}

ln_status col_mean(int n, int m, const float *X, long long ldx, double *mean, float *off_hi, float *off_lo,
                   double *partials, cudaStream_t st) {
    const int sr = stats_rows(n, m);
    const int nch = (int)ceil_div(n, sr);
    dim3 grid((unsigned)ceil_div(m, SC), (unsigned)nch);
    const unsigned gf = (unsigned)ceil_div(m, 32);
    const double *no_mean = nullptr;
    float *no_f = nullptr;
    {
        LaunchScope ls_(FAM_STATS, st);
        LN_TRY_STATUS(pdl_launch(k_col_partial<0>, grid, dim3(256), 0, st, "column means", n, m, X, ldx, no_mean,
                                 partials, sr));
    }
    {
        LaunchScope ls_(FAM_STATS, st);
        LN_TRY_STATUS(pdl_launch(k_col_final<0>, dim3(gf), dim3(256), 0, st, "column means", n, m, nch,
                                 (const double *)partials, no_mean, mean, off_hi, off_lo, no_f));
    }
    return LN_SUCCESS;
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

namespace {
bool rows16(const void *p, long long ld) { return ((reinterpret_cast<uintptr_t>(p) & 15) == 0) && ((ld & 3) == 0); }
dim3 ew_grid(int n, int m) { return dim3((unsigned)ceil_div(m, 256), (unsigned)ceil_div(n, EW_ROWS)); }
}  // namespace

ln_status center_matrix(int n, int m, const float *X, long long ldx, const float *off_hi, const float *off_lo,
                        const float *rs, float *Y, long long ldy, cudaStream_t st) {
    if (n == 0 || m == 0) return LN_SUCCESS;
    if (ceil_div(n, EW_ROWS) > 65535) return fail(LN_ERR_INVALID_VALUE, "too many rows to centre (%d)", n);
    const int vec = rows16(X, ldx) && rows16(Y, ldy);
    {
        LaunchScope ls_(FAM_STATS, st);
        k_center<<<ew_grid(n, m), dim3(64, 4), 0, st>>>(n, m, X, ldx, off_hi, off_lo, rs, Y, ldy, vec);
    }
    return check_launch("centre");
}

ln_status symmetrize_weights(int m, const float *W, long long ldw, float scale, int zero_diag, float *Ws,
                             cudaStream_t st) {
    if (m == 0) return LN_SUCCESS;
    if (ceil_div(m, 32) > 65535) return fail(LN_ERR_INVALID_VALUE, "weights too large to symmetrise (%d)", m);
    const unsigned g = (unsigned)ceil_div(m, 32);
    { LaunchScope ls_(FAM_STATS, st); k_symw<<<dim3(g, g), dim3(32, 8), 0, st>>>(m, W, ldw, scale, zero_diag, Ws); }
    return check_launch("symmetrise weights");
}

size_t corr_bwd_partials_bytes(int n, int m) {
    return sizeof(double) * (3 * (size_t)ceil_div(n, stats_rows(n, m)) * (size_t)m + (size_t)m);
}

ln_status corr_bwd_finish(int n, int m, const float *Z, long long ldz, const float *dZ, long long lddz,
                          const float *rs, float *dX, long long lddx, double *partials, cudaStream_t st) {
    if (n == 0 || m == 0) return LN_SUCCESS;
    if (ceil_div(n, EW_ROWS) > 65535) return fail(LN_ERR_INVALID_VALUE, "too many rows (%d)", n);
    const int sr = stats_rows(n, m);
    const int nch = (int)ceil_div(n, sr);
    float *d = reinterpret_cast<float *>(partials + 3 * (size_t)nch * m);
    float *cmean = d + m;
    const int vec = rows16(Z, ldz) && rows16(dZ, lddz) && rows16(dX, lddx);
    {
        LaunchScope ls_(FAM_STATS, st);
        k_corr_cols<<<dim3((unsigned)ceil_div(m, SC), (unsigned)nch), 256, 0, st>>>(n, m, Z, ldz, dZ, lddz, partials,
                                                                                 sr, nch);
    }
    {
        LaunchScope ls_(FAM_STATS, st);
        k_corr_cols_final<<<(unsigned)ceil_div(m, 32), 256, 0, st>>>(n, m, nch, partials, rs, d, cmean);
    }
    {
        LaunchScope ls_(FAM_STATS, st);
        k_corr_dx<<<ew_grid(n, m), dim3(64, 4), 0, st>>>(n, m, Z, ldz, dZ, lddz, d, rs, cmean, dX, lddx, vec);
    }
    return check_launch("correlation adjoint");
}

}  // namespace ln
