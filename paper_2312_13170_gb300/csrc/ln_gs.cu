// Gram-Schmidt QR (polybench gramschmidt, paper Sec. VIII), modified
// Gram-Schmidt on an m x n FP32 matrix held in Q (overwritten by the
// orthonormal factor), with R (n x n) upper triangular.
//
// Plain form: the benchmark's structure, three kernels per column k -- a
// single work-item sums the column's squares (the divergent region of Sec.
// VI-C and Sec. VIII that keeps loop internalization from this kernel), one
// work-item per row scales the column, and one work-item per later column j
// forms R[k][j] and removes the projection from column j.
//
// Internalized form: the same computation restructured so that every loop
// runs in CTA-uniform control flow. Columns are taken in panels of 32. One
// CTA factorises a panel with its rows held in registers (or, for tall
// matrices, in shared memory or L2), one CTA-wide reduction per column:
// the column's squared norm and its dot products with the panel's later
// columns come out of the same reduction, and each R[k][j] is that dot
// product divided by R[k][k] -- the projection onto the normalised column
// that MGS takes, up to rounding. A second kernel then applies the panel to
// every later column (R block = Q_p^T W, W -= Q_p R block). In exact
// arithmetic this block form gives MGS's Q and R; between panels it is MGS,
// inside the trailing update it projects against the panel's columns at once.
//
// Reading where the benchmark would divide by zero: a column whose norm is
// exactly zero gets R[k][k] = 0, a zero column of Q and R[k][j] = 0.
#include <cuda_runtime.h>

#include <cstdint>

#include "ln_async.cuh"
#include "ln_gs.h"
#include "ln_internal.h"
#include "ln_launch.h"

#define LN_TRY_LAUNCH(what)                      \
    do {                                         \
        ln_status s_ = ::ln::check_launch(what); \
        if (s_ != LN_SUCCESS) return s_;         \
    } while (0)

namespace ln {

namespace {

constexpr int GS_BW = 32;    // panel width (columns)
constexpr int GS_CB = 8;     // later columns per CTA of the trailing update
constexpr int GS_UNT = 256;  // threads of the trailing update
constexpr int GS_PAD = 33;   // shared-memory row stride of a panel held in shared memory
constexpr int GS_TS = 36;    // row stride (floats) of the register-resident panel's tile

__device__ __forceinline__ void cp_async16(void *dst, const void *src, int src_bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
                 "l"(src), "r"(src_bytes)
                 : "memory");
}

// ------------------------------------------------------------------ plain form
__global__ void k_gs_norm(int m, int k, const float *Q, long long ldq, float *R, long long ldr) {
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    float s = 0.f;
    for (int i = 0; i < m; ++i) {
        const float x = Q[(long long)i * ldq + k];
        s = fmaf(x, x, s);
    }
    R[(long long)k * ldr + k] = __fsqrt_rn(s);
}

__global__ void k_gs_scale(int m, int k, float *Q, long long ldq, const float *R, long long ldr) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    const float r = R[(long long)k * ldr + k];
    float *q = Q + (long long)i * ldq + k;
    *q = r > 0.f ? __fdiv_rn(*q, r) : 0.f;
}

__global__ void k_gs_project(int m, int n, int k, float *Q, long long ldq, float *R, long long ldr) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    if (j < k) {  // strictly lower triangle of R
        R[(long long)k * ldr + j] = 0.f;
        return;
    }
    if (j == k) return;
    float s = 0.f;
    for (int i = 0; i < m; ++i) s = fmaf(Q[(long long)i * ldq + k], Q[(long long)i * ldq + j], s);
    R[(long long)k * ldr + j] = s;
    for (int i = 0; i < m; ++i) {
        float *w = Q + (long long)i * ldq + j;
        *w = fmaf(-Q[(long long)i * ldq + k], s, *w);
    }
}

// ------------------------------------------------------------------ panel factorisation
// Transpose-reduce of WD values over the warp followed by a butterfly over
// the remaining lane bits: afterwards v[0] of lane l is the warp's total for
// index l % WD (WD - 1 + log2(32 / WD) shuffles).
template <int WD>
__device__ __forceinline__ void warp_reduce_cols(float (&v)[WD], int lane) {
#pragma unroll
    for (int o = WD / 2; o >= 1; o >>= 1) {
        const bool up = (lane & o) != 0;
#pragma unroll
        for (int i = 0; i < o; ++i) {
            const float send = up ? v[i] : v[i + o];
            const float keep = up ? v[i + o] : v[i];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
        }
    }
#pragma unroll
    for (int o = WD; o < 32; o <<= 1) v[0] += __shfl_xor_sync(0xffffffffu, v[0], o);
}

// One column step's reduction. v holds this thread's partial sums of
// x_c * x_j (j >= c) over its rows. Returns R[k][k] (k = p0 + c); writes the
// panel's row k of R (k <= j < p0 + bw) and leaves R[k][p0 + j] for j > c in
// this warp's row of rcs. Every warp sums the per-warp totals in the same
// order, so all threads see bit-identical coefficients. One __syncthreads;
// `red` is double-buffered by column parity, which makes that the only one.
template <int NW>
__device__ __forceinline__ float gs_reduce(float (&v)[32], int c, int bw, int p0, float *R, long long ldr,
                                           float (*red)[NW][32], float (*rcs)[32]) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    warp_reduce_cols<32>(v, lane);
    float(*rb)[32] = red[c & 1];
    rb[warp][lane] = v[0];
    __syncthreads();
    float tot = 0.f;
#pragma unroll
    for (int q = 0; q < NW; ++q) tot += rb[q][lane];
    const float r = __fsqrt_rn(__shfl_sync(0xffffffffu, tot, c));
    const float rc = r > 0.f ? __fdiv_rn(tot, r) : 0.f;
    if (warp == 0 && lane >= c && lane < bw) R[(long long)(p0 + c) * ldr + p0 + lane] = lane == c ? r : rc;
    rcs[warp][lane] = rc;
    __syncwarp();
    return r;
}

// One column step of the register-resident panel. w holds this thread's
// rows as 16 pairs of slots; the current column k = p0 + c sits in slot PH
// (= c & 1) and slot j holds column k - PH + j; slots >= WD are zero, and in
// a PH = 1 step slot 0 holds the previous, finished column. The squared norm
// and the dot products with the later columns come out of one CTA-wide
// reduction (packed FP32x2 multiply-adds, then warp_reduce_cols and one
// barrier); the normalised column goes to column c of the shared-memory tile
// and the later columns lose their projection. After a PH = 1 step every
// pair moves down one place, so the next column is again in slot 0 and every
// register index is a constant.
template <int S, int NT, int WD, int PH>
__device__ __forceinline__ void gs_reg_step(float2 (&w)[S][GS_BW / 2], int c, int bw, int p0, float *tile,
                                            float *R, long long ldr, float (*red)[NT / 32][32], float (*rcs)[32]) {
    constexpr int NW = NT / 32, NP = WD / 2;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    float2 v2[NP];
#pragma unroll
    for (int p = 0; p < NP; ++p) v2[p] = make_float2(0.f, 0.f);
#pragma unroll
    for (int s = 0; s < S; ++s) {
        const float x = PH ? w[s][0].y : w[s][0].x;
        const float2 x2 = make_float2(x, x);
        if (PH == 0) v2[0] = __ffma2_rn(x2, w[s][0], v2[0]);
        else v2[0].y = fmaf(x, x, v2[0].y);
#pragma unroll
        for (int p = 1; p < NP; ++p) v2[p] = __ffma2_rn(x2, w[s][p], v2[p]);
    }
    float v[WD];
#pragma unroll
    for (int p = 0; p < NP; ++p) {
        v[2 * p] = v2[p].x;
        v[2 * p + 1] = v2[p].y;
    }
    warp_reduce_cols<WD>(v, lane);  // lane l: the warp's total for slot l % WD
    float(*rb)[32] = red[c & 1];
    rb[warp][lane] = v[0];
    __syncthreads();
    float part[NW];
#pragma unroll
    for (int q = 0; q < NW; ++q) part[q] = rb[q][lane];
#pragma unroll
    for (int h = 1; h < NW; h <<= 1)  // fixed pairwise tree: the same in every warp
#pragma unroll
        for (int q = 0; q + h < NW; q += 2 * h) part[q] += part[q + h];
    const float tot = part[0];
    const float nrm2 = __shfl_sync(0xffffffffu, tot, PH);
    // hardware reciprocal square root (a few ulps; the norm is nrm2 * inv)
    const float inv = nrm2 > 0.f ? rsqrtf(nrm2) : 0.f;
    const float r = nrm2 * inv;
    const float rc = tot * inv;  // R[k][k + l - PH] for slot l > PH
    if (warp == 0 && lane >= PH && lane < WD && c + lane - PH < bw)
        R[(long long)(p0 + c) * ldr + p0 + c + lane - PH] = lane == PH ? r : rc;
    rcs[warp][lane] = -rc;
    __syncwarp();
    float nr[WD];
    const float4 *r4 = reinterpret_cast<const float4 *>(rcs[warp]);
#pragma unroll
    for (int g = 0; g < WD / 4; ++g) {
        const float4 t = r4[g];
        nr[4 * g] = t.x;
        nr[4 * g + 1] = t.y;
        nr[4 * g + 2] = t.z;
        nr[4 * g + 3] = t.w;
    }
#pragma unroll
    for (int s = 0; s < S; ++s) {
        const float q = (PH ? w[s][0].y : w[s][0].x) * inv;
        tile[(tid + s * NT) * GS_TS + c] = q;
        const float2 q2 = make_float2(q, q);
        if (PH == 0) {
            w[s][0].y = fmaf(nr[1], q, w[s][0].y);
#pragma unroll
            for (int p = 1; p < NP; ++p) w[s][p] = __ffma2_rn(make_float2(nr[2 * p], nr[2 * p + 1]), q2, w[s][p]);
        } else {
#pragma unroll
            for (int p = 1; p < NP; ++p)
                w[s][p - 1] = __ffma2_rn(make_float2(nr[2 * p], nr[2 * p + 1]), q2, w[s][p]);
            w[s][NP - 1] = make_float2(0.f, 0.f);
        }
    }
}

template <int S, int NT, int PH>
__device__ __forceinline__ void gs_reg_step_any(float2 (&w)[S][GS_BW / 2], int c, int bw, int p0, float *tile,
                                                float *R, long long ldr, float (*red)[NT / 32][32],
                                                float (*rcs)[32]) {
    const int need = PH + bw - c;  // slots the step must cover
    if (need > 16) gs_reg_step<S, NT, 32, PH>(w, c, bw, p0, tile, R, ldr, red, rcs);
    else if (need > 8) gs_reg_step<S, NT, 16, PH>(w, c, bw, p0, tile, R, ldr, red, rcs);
    else gs_reg_step<S, NT, 8, PH>(w, c, bw, p0, tile, R, ldr, red, rcs);
}

// Panel of up to 32 columns, rows in registers: thread t holds rows t + s*NT
// (s < S). The panel comes into a row-major shared-memory tile (row stride
// GS_TS) by 16-byte asynchronous copies (plain loads when rows are not
// 16-byte aligned), goes to registers, and the normalised columns go back to
// the tile and out to Q with 16-byte stores.
template <int S, int NT>
__host__ __device__ constexpr size_t gs_panel_smem() {
    return (size_t)S * NT * GS_TS * sizeof(float);
}

template <int S, int NT>
__global__ void __launch_bounds__(NT, 1)
    k_gs_panel_reg(int m, int p0, int bw, float *Q, long long ldq, float *R, long long ldr, int vec) {
    extern __shared__ __align__(16) float tile[];
    __shared__ float red[2][NT / 32][32];
    __shared__ __align__(16) float rcs[NT / 32][32];
    const int tid = threadIdx.x;
    // launched programmatically after the previous update: Q only after it has completed
    pdl_wait();
    pdl_trigger();
    if (vec) {
#pragma unroll 8
        for (int it = 0; it < S * 8; ++it) {
            const int e = tid + it * NT, i = e / 8, k = e % 8;
            const int valid = i < m ? min(max(bw - 4 * k, 0), 4) : 0;
            const float *src = valid ? Q + (long long)i * ldq + p0 + 4 * k : Q;
            cp_async16(tile + i * GS_TS + 4 * k, src, 4 * valid);
        }
        asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;" ::: "memory");
    } else {
#pragma unroll 32
        for (int it = 0; it < S * GS_BW; ++it) {
            const int e = tid + it * NT, i = e / GS_BW, j = e % GS_BW;
            tile[i * GS_TS + j] = (i < m && j < bw) ? Q[(long long)i * ldq + p0 + j] : 0.f;
        }
    }
    __syncthreads();
    float2 w[S][GS_BW / 2];
#pragma unroll
    for (int s = 0; s < S; ++s) {
        const float4 *row = reinterpret_cast<const float4 *>(tile + (tid + s * NT) * GS_TS);
#pragma unroll
        for (int g = 0; g < GS_BW / 4; ++g) {
            const float4 t = row[g];
            w[s][2 * g] = make_float2(t.x, t.y);
            w[s][2 * g + 1] = make_float2(t.z, t.w);
        }
    }
    // between the two barriers each thread reads and rewrites only its own rows of the tile
    for (int c = 0; c < bw; ++c) {
        if (c & 1) gs_reg_step_any<S, NT, 1>(w, c, bw, p0, tile, R, ldr, red, rcs);
        else gs_reg_step_any<S, NT, 0>(w, c, bw, p0, tile, R, ldr, red, rcs);
    }
    __syncthreads();
#pragma unroll 8
    for (int it = 0; it < S * 8; ++it) {
        const int e = tid + it * NT, i = e / 8, k = e % 8;
        if (i >= m || 4 * k >= bw) continue;
        const float4 t = *reinterpret_cast<const float4 *>(tile + i * GS_TS + 4 * k);
        float *dst = Q + (long long)i * ldq + p0 + 4 * k;
        if (vec && 4 * k + 4 <= bw) {
            *reinterpret_cast<float4 *>(dst) = t;
        } else {
            const float tv[4] = {t.x, t.y, t.z, t.w};
            for (int q = 0; q < 4 && 4 * k + q < bw; ++q) dst[q] = tv[q];
        }
    }
}

// Panel of up to 32 columns for matrices taller than the register-resident
// kernel takes: the rows live in shared memory (stride GS_PAD) when they fit,
// else in Q itself (L2), and each column step re-reads the rows it needs.
template <int NT>
__global__ void __launch_bounds__(NT, 1)
    k_gs_panel_mem(int m, int p0, int bw, float *Q, long long ldq, float *R, long long ldr, int in_smem) {
    constexpr int NW = NT / 32;
    extern __shared__ __align__(16) float pan[];
    __shared__ float red[2][NW][32];
    __shared__ __align__(16) float rcs[NW][32];
    const int tid = threadIdx.x, warp = tid >> 5;
    pdl_wait();
    pdl_trigger();
    float *P = Q + p0;
    long long ldp = ldq;
    if (in_smem) {
        for (long long e = tid; e < (long long)m * GS_BW; e += NT) {
            const int i = (int)(e / GS_BW), j = (int)(e % GS_BW);
            pan[(long long)i * GS_PAD + j] = j < bw ? Q[(long long)i * ldq + p0 + j] : 0.f;
        }
        __syncthreads();
        P = pan;
        ldp = GS_PAD;
    }
    for (int c = 0; c < bw; ++c) {
        float v[GS_BW];
#pragma unroll
        for (int j = 0; j < GS_BW; ++j) v[j] = 0.f;
        for (int i = tid; i < m; i += NT) {
            const float *row = P + (long long)i * ldp;
            const float x = row[c];
#pragma unroll
            for (int j = 0; j < GS_BW; ++j)
                if (j >= c && j < bw) v[j] = fmaf(x, row[j], v[j]);
        }
        const float r = gs_reduce<NW>(v, c, bw, p0, R, ldr, red, rcs);
        float rr[GS_BW];
#pragma unroll
        for (int j = 0; j < GS_BW; ++j) rr[j] = rcs[warp][j];
        for (int i = tid; i < m; i += NT) {
            float *row = P + (long long)i * ldp;
            const float q = r > 0.f ? __fdiv_rn(row[c], r) : 0.f;
            row[c] = q;
#pragma unroll
            for (int j = 0; j < GS_BW; ++j)
                if (j > c && j < bw) row[j] = fmaf(-rr[j], q, row[j]);
        }
    }
    if (in_smem) {
        __syncthreads();
        for (long long e = tid; e < (long long)m * GS_BW; e += NT) {
            const int i = (int)(e / GS_BW), j = (int)(e % GS_BW);
            if (j < bw) Q[(long long)i * ldq + p0 + j] = pan[(long long)i * GS_PAD + j];
        }
    }
}

// ------------------------------------------------------------------ trailing update
constexpr int GS_URC = 1024;  // rows per staged chunk of the trailing update
constexpr int GS_QP = 36;     // shared-memory row stride (floats) of staged panel rows

__host__ __device__ constexpr size_t gs_update_smem(int m) {
    return (size_t)(m < GS_URC ? m : GS_URC) * (GS_QP + GS_CB) * sizeof(float);
}

// Stage rows i0 .. i0+nr-1 of the panel (32 floats each, stride GS_QP) and of
// this CTA's ncols later columns (GS_CB floats each, zero beyond ncols) into
// shared memory. vec: every row start is 16-byte aligned (asynchronous
// 16-byte copies); otherwise plain loads.
__device__ __forceinline__ void gs_stage(const float *Q, long long ldq, int p0, int j0, int ncols, int i0, int nr,
                                         float *Qs, float *Ws, bool vec) {
    const int tid = threadIdx.x;
    if (vec) {
        for (int e = tid; e < nr * 10; e += GS_UNT) {
            const int i = e / 10, k = e % 10;
            const float *row = Q + (long long)(i0 + i) * ldq;
            if (k < 8) {
                cp_async16(Qs + i * GS_QP + 4 * k, row + p0 + 4 * k, 16);
            } else {
                const int h = k - 8, valid = ncols - 4 * h;
                const int bytes = valid >= 4 ? 16 : (valid > 0 ? 4 * valid : 0);
                cp_async16(Ws + i * GS_CB + 4 * h, row + j0 + (bytes ? 4 * h : 0), bytes);
            }
        }
        asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;" ::: "memory");
    } else {
        for (int e = tid; e < nr * (GS_BW + GS_CB); e += GS_UNT) {
            const int i = e / (GS_BW + GS_CB), k = e % (GS_BW + GS_CB);
            const float *row = Q + (long long)(i0 + i) * ldq;
            if (k < GS_BW) Qs[i * GS_QP + k] = row[p0 + k];
            else Ws[i * GS_CB + k - GS_BW] = k - GS_BW < ncols ? row[j0 + k - GS_BW] : 0.f;
        }
    }
    __syncthreads();
}

// Apply the factorised panel (columns p0 .. p0+31 of Q, orthonormal) to the
// later columns j >= p1: R[p0 + a][j] = sum_i Q[i][p0 + a] W[i][j], then
// W[i][j] -= sum_a Q[i][p0 + a] R[p0 + a][j]. CTA b takes GS_CB columns from
// p1 + b*GS_CB; the panel rows and those columns are staged in shared memory
// (GS_URC rows at a time), and thread (g, jj) walks rows g, g + NG, ... of
// column jj.
__global__ void __launch_bounds__(GS_UNT, 1)
    k_gs_update(int m, int n, int p0, int p1, float *Q, long long ldq, float *R, long long ldr, int vec) {
    constexpr int NG = GS_UNT / GS_CB;
    extern __shared__ __align__(16) float gs_sm[];
    __shared__ float red[NG][GS_CB][GS_PAD];
    __shared__ float Rs[GS_BW][GS_CB];
    float *Qs = gs_sm;
    float *Ws = gs_sm + (m < GS_URC ? m : GS_URC) * GS_QP;
    const int tid = threadIdx.x, g = tid / GS_CB, jj = tid % GS_CB;
    const int j0 = p1 + blockIdx.x * GS_CB, j = j0 + jj;
    const int ncols = min(GS_CB, n - j0);
    // launched programmatically after the panel: its Q and R only after it has completed
    pdl_wait();
    pdl_trigger();
    float2 acc[GS_BW / 2];
#pragma unroll
    for (int a = 0; a < GS_BW / 2; ++a) acc[a] = make_float2(0.f, 0.f);
    for (int i0 = 0; i0 < m; i0 += GS_URC) {
        const int nr = min(GS_URC, m - i0);
        if (i0 > 0) __syncthreads();  // the previous chunk is no longer read
        gs_stage(Q, ldq, p0, j0, ncols, i0, nr, Qs, Ws, vec != 0);
#pragma unroll 2
        for (int i = g; i < nr; i += NG) {
            const float4 *q4 = reinterpret_cast<const float4 *>(Qs + i * GS_QP);
            const float x = Ws[i * GS_CB + jj];
            const float2 x2 = make_float2(x, x);
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const float4 t = q4[k];
                acc[2 * k] = __ffma2_rn(make_float2(t.x, t.y), x2, acc[2 * k]);
                acc[2 * k + 1] = __ffma2_rn(make_float2(t.z, t.w), x2, acc[2 * k + 1]);
            }
        }
    }
#pragma unroll
    for (int a = 0; a < GS_BW / 2; ++a) {
        red[g][jj][2 * a] = acc[a].x;
        red[g][jj][2 * a + 1] = acc[a].y;
    }
    __syncthreads();
    for (int o = tid; o < GS_BW * GS_CB; o += GS_UNT) {
        const int a = o / GS_CB, cc = o % GS_CB;
        float s = 0.f;
#pragma unroll 8
        for (int h = 0; h < NG; ++h) s += red[h][cc][a];
        Rs[a][cc] = s;
        if (cc < ncols) R[(long long)(p0 + a) * ldr + j0 + cc] = s;
    }
    __syncthreads();
    float2 rr[GS_BW / 2];
#pragma unroll
    for (int a = 0; a < GS_BW / 2; ++a) rr[a] = make_float2(Rs[2 * a][jj], Rs[2 * a + 1][jj]);
    // the last staged chunk is still in shared memory: walk the chunks backwards
    for (int i0 = ((m - 1) / GS_URC) * GS_URC; i0 >= 0; i0 -= GS_URC) {
        const int nr = min(GS_URC, m - i0);
        if (i0 + GS_URC < m) {
            __syncthreads();
            gs_stage(Q, ldq, p0, j0, ncols, i0, nr, Qs, Ws, vec != 0);
        }
        if (jj < ncols) {
#pragma unroll 2
            for (int i = g; i < nr; i += NG) {
                const float4 *q4 = reinterpret_cast<const float4 *>(Qs + i * GS_QP);
                // sum_a Q[i][a] R[a][j] as four interleaved partial sums (even/odd a, two halves)
                float2 s0 = make_float2(0.f, 0.f), s1 = make_float2(0.f, 0.f);
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    const float4 t = q4[k];
                    if (k < 4) {
                        s0 = __ffma2_rn(make_float2(t.x, t.y), rr[2 * k], s0);
                        s0 = __ffma2_rn(make_float2(t.z, t.w), rr[2 * k + 1], s0);
                    } else {
                        s1 = __ffma2_rn(make_float2(t.x, t.y), rr[2 * k], s1);
                        s1 = __ffma2_rn(make_float2(t.z, t.w), rr[2 * k + 1], s1);
                    }
                }
                const float s = (s0.x + s0.y) + (s1.x + s1.y);
                Q[(long long)(i0 + i) * ldq + j] = Ws[i * GS_CB + jj] - s;
            }
        }
    }
}

constexpr int GS_MEM_NT = 512;

}  // namespace

// ------------------------------------------------------------------ launchers
ln_status gs_plain(int m, int n, float *Q, long long ldq, float *R, long long ldr, cudaStream_t st) {
    for (int k = 0; k < n; ++k) {
        {
            LaunchScope ls_(FAM_PLAIN, st);
            k_gs_norm<<<1, 32, 0, st>>>(m, k, Q, ldq, R, ldr);
        }
        LN_TRY_LAUNCH("k_gs_norm");
        if (m > 0) {
            {
                LaunchScope ls_(FAM_PLAIN, st);
                k_gs_scale<<<(unsigned)ceil_div(m, 256), 256, 0, st>>>(m, k, Q, ldq, R, ldr);
            }
            LN_TRY_LAUNCH("k_gs_scale");
        }
        {
            LaunchScope ls_(FAM_PLAIN, st);
            k_gs_project<<<(unsigned)ceil_div(n, 256), 256, 0, st>>>(m, n, k, Q, ldq, R, ldr);
        }
        LN_TRY_LAUNCH("k_gs_project");
    }
    return LN_SUCCESS;
}

ln_status gs_blocked(int m, int n, float *Q, long long ldq, float *R, long long ldr, cudaStream_t st) {
    if (n == 0) return LN_SUCCESS;
    // the kernels write R on and above the diagonal; zero the whole of it first
    LN_CUDA_TRY(cudaMemset2DAsync(R, (size_t)ldr * 4, 0, (size_t)n * 4, (size_t)n, st));
    if (m == 0) return LN_SUCCESS;
    const int vec = (reinterpret_cast<uintptr_t>(Q) % 16 == 0 && ldq % 4 == 0) ? 1 : 0;
    // tall panels: shared memory when the 33-float rows fit beside the static arrays
    const size_t mem_bytes = (size_t)m * GS_PAD * sizeof(float);
    const int in_smem = (m > 1024 && mem_bytes <= 200 * 1024) ? 1 : 0;
    if (in_smem)
        LN_CUDA_TRY(cudaFuncSetAttribute(k_gs_panel_mem<GS_MEM_NT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)mem_bytes));
    LN_CUDA_TRY(cudaFuncSetAttribute(k_gs_update, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)gs_update_smem(m)));
    LN_CUDA_TRY(cudaFuncSetAttribute(k_gs_panel_reg<2, 256>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)gs_panel_smem<2, 256>()));
    LN_CUDA_TRY(cudaFuncSetAttribute(k_gs_panel_reg<2, 512>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)gs_panel_smem<2, 512>()));
    LN_CUDA_TRY(cudaFuncSetAttribute(k_gs_panel_reg<4, 256>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)gs_panel_smem<4, 256>()));
    const int rows = tune_gs_rows();
    for (int p0 = 0; p0 < n; p0 += GS_BW) {
        const int bw = n - p0 < GS_BW ? n - p0 : GS_BW;
        {
            LaunchScope ls_(FAM_SIMT, st);
            ln_status ps;
            if (m <= 512)
                ps = pdl_launch(k_gs_panel_reg<2, 256>, 1, 256, gs_panel_smem<2, 256>(), st, "k_gs_panel", m, p0, bw, Q,
                               ldq, R, ldr, vec);
            else if (m <= 1024 && rows == 2)
                ps = pdl_launch(k_gs_panel_reg<2, 512>, 1, 512, gs_panel_smem<2, 512>(), st, "k_gs_panel", m, p0, bw, Q,
                               ldq, R, ldr, vec);
            else if (m <= 1024)
                ps = pdl_launch(k_gs_panel_reg<4, 256>, 1, 256, gs_panel_smem<4, 256>(), st, "k_gs_panel", m, p0, bw, Q,
                               ldq, R, ldr, vec);
            else
                ps = pdl_launch(k_gs_panel_mem<GS_MEM_NT>, 1, GS_MEM_NT, in_smem ? mem_bytes : 0, st, "k_gs_panel", m,
                               p0, bw, Q, ldq, R, ldr, in_smem);
            if (ps != LN_SUCCESS) return ps;
        }
        const int p1 = p0 + bw;
        if (p1 < n) {
            LaunchScope ls_(FAM_SIMT, st);
            const ln_status us = pdl_launch(k_gs_update, (unsigned)ceil_div(n - p1, GS_CB), GS_UNT, gs_update_smem(m), st,
                                           "k_gs_update", m, n, p0, p1, Q, ldq, R, ldr, vec);
            if (us != LN_SUCCESS) return us;
        }
    }
    return LN_SUCCESS;
}

}  // namespace ln
