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

#include "ln_gs.h"
#include "ln_internal.h"

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

// Zero the strictly lower part of the panel's rows of R (columns < k).
__device__ __forceinline__ void gs_zero_lower(int p0, int bw, float *R, long long ldr, int nt) {
    for (int c = 0; c < bw; ++c)
        for (int j = threadIdx.x; j < p0 + c; j += nt) R[(long long)(p0 + c) * ldr + j] = 0.f;
}

// One column step of the register-resident panel. Slot 0 of w holds the
// current column k = p0 + c of this thread's rows, slot j the column k + j;
// slots >= WD are zero. The squared norm and the dot products with the later
// columns come out of one CTA-wide reduction; the normalised column goes to
// column c of the shared-memory tile qs (column-major, stride S*NT + 1) and
// the later columns, after removing their projection, move down one slot, so
// the next column is again in slot 0 and every register index is a constant.
template <int S, int NT, int WD>
__device__ __forceinline__ void gs_reg_step(float (&w)[S][GS_BW], int c, int bw, int p0, float *qs, float *R,
                                            long long ldr, float (*red)[NT / 32][32], float (*rcs)[32]) {
    constexpr int NW = NT / 32;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    float v[WD];
#pragma unroll
    for (int j = 0; j < WD; ++j) v[j] = 0.f;
#pragma unroll
    for (int s = 0; s < S; ++s) {
        const float x = w[s][0];
#pragma unroll
        for (int j = 0; j < WD; ++j) v[j] = fmaf(x, w[s][j], v[j]);
    }
    warp_reduce_cols<WD>(v, lane);
    float(*rb)[32] = red[c & 1];
    rb[warp][lane] = v[0];
    __syncthreads();
    float tot = 0.f;
#pragma unroll
    for (int q = 0; q < NW; ++q) tot += rb[q][lane];
    const float r = __fsqrt_rn(__shfl_sync(0xffffffffu, tot, 0));
    const float inv = r > 0.f ? __frcp_rn(r) : 0.f;
    const float rc = tot * inv;  // R[k][k + lane % WD] for lane % WD > 0
    if (warp == 0 && lane < WD && c + lane < bw) R[(long long)(p0 + c) * ldr + p0 + c + lane] = lane == 0 ? r : rc;
    rcs[warp][lane] = rc;
    __syncwarp();
    float rr[WD];
    const float4 *r4 = reinterpret_cast<const float4 *>(rcs[warp]);
#pragma unroll
    for (int g = 0; g < WD / 4; ++g) {
        const float4 t = r4[g];
        rr[4 * g] = t.x;
        rr[4 * g + 1] = t.y;
        rr[4 * g + 2] = t.z;
        rr[4 * g + 3] = t.w;
    }
#pragma unroll
    for (int s = 0; s < S; ++s) {
        const float q = w[s][0] * inv;
        qs[c * (S * NT + 1) + tid + s * NT] = q;
#pragma unroll
        for (int j = 1; j < WD; ++j) w[s][j - 1] = fmaf(-rr[j], q, w[s][j]);
        w[s][WD - 1] = 0.f;
    }
}

// Panel of up to 32 columns, rows in registers: thread t holds rows t + s*NT
// (s < S). The panel goes from Q to registers and back through a
// column-major shared-memory tile (coalesced global accesses both ways). The
// column loop is a runtime loop over gs_reg_step; the step's width drops to
// 16 and then 8 slots once that many columns remain.
template <int S, int NT>
__host__ __device__ constexpr size_t gs_panel_smem() {
    return (size_t)GS_BW * (S * NT + 1) * sizeof(float);
}

template <int S, int NT>
__global__ void __launch_bounds__(NT, 1)
    k_gs_panel_reg(int m, int p0, int bw, float *Q, long long ldq, float *R, long long ldr) {
    constexpr int LD = S * NT + 1;  // column stride of the tile
    extern __shared__ __align__(16) float qs[];
    __shared__ float red[2][NT / 32][32];
    __shared__ __align__(16) float rcs[NT / 32][32];
    const int tid = threadIdx.x;
    // S * 32 loads per thread, unrolled so that many are in flight at once
#pragma unroll 32
    for (int it = 0; it < S * GS_BW; ++it) {
        const int e = tid + it * NT, i = e / GS_BW, j = e % GS_BW;
        qs[j * LD + i] = (i < m && j < bw) ? Q[(long long)i * ldq + p0 + j] : 0.f;
    }
    __syncthreads();
    float w[S][GS_BW];
#pragma unroll
    for (int s = 0; s < S; ++s)
#pragma unroll
        for (int j = 0; j < GS_BW; ++j) w[s][j] = qs[j * LD + tid + s * NT];
    // between the two barriers each thread reads and rewrites only its own rows of the tile
    int c = 0;
    for (; c < bw && bw - c > 16; ++c) gs_reg_step<S, NT, 32>(w, c, bw, p0, qs, R, ldr, red, rcs);
    for (; c < bw && bw - c > 8; ++c) gs_reg_step<S, NT, 16>(w, c, bw, p0, qs, R, ldr, red, rcs);
    for (; c < bw; ++c) gs_reg_step<S, NT, 8>(w, c, bw, p0, qs, R, ldr, red, rcs);
    __syncthreads();
#pragma unroll 8
    for (int it = 0; it < S * GS_BW; ++it) {
        const int e = tid + it * NT, i = e / GS_BW, j = e % GS_BW;
        if (i < m && j < bw) Q[(long long)i * ldq + p0 + j] = qs[j * LD + i];
    }
    gs_zero_lower(p0, bw, R, ldr, NT);
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
    gs_zero_lower(p0, bw, R, ldr, NT);
}

// ------------------------------------------------------------------ trailing update
constexpr int GS_URC = 1024;  // rows per staged chunk of the trailing update
constexpr int GS_QP = 36;     // shared-memory row stride (floats) of staged panel rows

__host__ __device__ constexpr size_t gs_update_smem(int m) {
    return (size_t)(m < GS_URC ? m : GS_URC) * (GS_QP + GS_CB) * sizeof(float);
}

__device__ __forceinline__ void cp_async16(void *dst, const void *src, int src_bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
                 "l"(src), "r"(src_bytes)
                 : "memory");
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
    float acc[GS_BW];
#pragma unroll
    for (int a = 0; a < GS_BW; ++a) acc[a] = 0.f;
    for (int i0 = 0; i0 < m; i0 += GS_URC) {
        const int nr = min(GS_URC, m - i0);
        if (i0 > 0) __syncthreads();  // the previous chunk is no longer read
        gs_stage(Q, ldq, p0, j0, ncols, i0, nr, Qs, Ws, vec != 0);
        for (int i = g; i < nr; i += NG) {
            const float4 *q4 = reinterpret_cast<const float4 *>(Qs + i * GS_QP);
            const float x = Ws[i * GS_CB + jj];
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const float4 t = q4[k];
                acc[4 * k] = fmaf(t.x, x, acc[4 * k]);
                acc[4 * k + 1] = fmaf(t.y, x, acc[4 * k + 1]);
                acc[4 * k + 2] = fmaf(t.z, x, acc[4 * k + 2]);
                acc[4 * k + 3] = fmaf(t.w, x, acc[4 * k + 3]);
            }
        }
    }
#pragma unroll
    for (int a = 0; a < GS_BW; ++a) red[g][jj][a] = acc[a];
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
    float rr[GS_BW];
#pragma unroll
    for (int a = 0; a < GS_BW; ++a) rr[a] = Rs[a][jj];
    // the last staged chunk is still in shared memory: walk the chunks backwards
    for (int i0 = ((m - 1) / GS_URC) * GS_URC; i0 >= 0; i0 -= GS_URC) {
        const int nr = min(GS_URC, m - i0);
        if (i0 + GS_URC < m) {
            __syncthreads();
            gs_stage(Q, ldq, p0, j0, ncols, i0, nr, Qs, Ws, vec != 0);
        }
        if (jj < ncols) {
            for (int i = g; i < nr; i += NG) {
                const float4 *q4 = reinterpret_cast<const float4 *>(Qs + i * GS_QP);
                float s = 0.f;
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    const float4 t = q4[k];
                    s = fmaf(t.x, rr[4 * k], s);
                    s = fmaf(t.y, rr[4 * k + 1], s);
                    s = fmaf(t.z, rr[4 * k + 2], s);
                    s = fmaf(t.w, rr[4 * k + 3], s);
                }
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
    if (m == 0) {
        LN_CUDA_TRY(cudaMemset2DAsync(R, (size_t)ldr * 4, 0, (size_t)n * 4, (size_t)n, st));
        return LN_SUCCESS;
    }
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
            if (m <= 512)
                k_gs_panel_reg<2, 256><<<1, 256, gs_panel_smem<2, 256>(), st>>>(m, p0, bw, Q, ldq, R, ldr);
            else if (m <= 1024 && rows == 2)
                k_gs_panel_reg<2, 512><<<1, 512, gs_panel_smem<2, 512>(), st>>>(m, p0, bw, Q, ldq, R, ldr);
            else if (m <= 1024)
                k_gs_panel_reg<4, 256><<<1, 256, gs_panel_smem<4, 256>(), st>>>(m, p0, bw, Q, ldq, R, ldr);
            else
                k_gs_panel_mem<GS_MEM_NT><<<1, GS_MEM_NT, in_smem ? mem_bytes : 0, st>>>(m, p0, bw, Q, ldq, R, ldr,
                                                                                      in_smem);
        }
        LN_TRY_LAUNCH("k_gs_panel");
        const int p1 = p0 + bw;
        if (p1 < n) {
            {
                LaunchScope ls_(FAM_SIMT, st);
                k_gs_update<<<(unsigned)ceil_div(n - p1, GS_CB), GS_UNT, gs_update_smem(m), st>>>(m, n, p0, p1, Q, ldq,
                                                                                                R, ldr, vec);
            }
            LN_TRY_LAUNCH("k_gs_update");
        }
    }
    return LN_SUCCESS;
}

}  // namespace ln
