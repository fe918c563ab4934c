// Internalized FP32 form: the work-group tiling of loop internalization
// (paper Sec. VI-C, Listing 6) mapped to a CTA. Each CTA owns a 128 x 128
// output tile; the inner k loop is tiled by 8, and each k-tile of both
// operands is prefetched from global memory (coalesced 128-bit loads where
// the layout allows) into shared memory, double-buffered so that one barrier
// per k-tile separates the prefetch of the next tile from the use of the
// current one. Each thread accumulates an 8 x 8 register block in exact FP32
// FFMA and stores it once (Sec. VI-B).
#include "ln_epilogue.cuh"
#include "ln_internal.h"

namespace ln {

namespace {

constexpr int TB = 128;  // output tile edge
constexpr int TK = 8;    // k-tile depth
constexpr int PADW = TB + 4;

struct TileCtx {
    const float *A, *B;
    long long lda, ldb;
    int M, N, K;
    int i0, j0;
    bool a_vec, b_vec;  // 16-byte loads legal (aligned base, ld % 4 == 0)
    const float *a_hi, *a_lo, *b_hi, *b_lo;
};

// Four consecutive elements of row `row` starting at column `col` of a
// row-major (rows x cols) matrix, zero outside the matrix.
__device__ __forceinline__ float4 load4(const float *p, long long ld, int row, int col, int rows, int cols, bool vec) {
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (row >= rows) return v;
    const float *q = p + (long long)row * ld + col;
    if (vec && col + 3 < cols) return __ldg(reinterpret_cast<const float4 *>(q));
    if (col + 0 < cols) v.x = __ldg(q + 0);
    if (col + 1 < cols) v.y = __ldg(q + 1);
    if (col + 2 < cols) v.z = __ldg(q + 2);
    if (col + 3 < cols) v.w = __ldg(q + 3);
    return v;
}

template <int AT, int BT>
__device__ __forceinline__ void fetch(const TileCtx &c, int k0, int tid, float4 &ra, float4 &rb) {
    if (AT == 0) {  // A[i][k]: 128 rows x 8 k, two float4 per row
        ra = load4(c.A, c.lda, c.i0 + (tid >> 1), k0 + (tid & 1) * 4, c.M, c.K, c.a_vec);
        if (c.a_hi) {
            int i = c.i0 + (tid >> 1);
            if (i < c.M) {
                float h = c.a_hi[i], l = c.a_lo[i];
                int kk = k0 + (tid & 1) * 4;
                if (kk + 0 < c.K) ra.x = (ra.x - h) - l;
                if (kk + 1 < c.K) ra.y = (ra.y - h) - l;
                if (kk + 2 < c.K) ra.z = (ra.z - h) - l;
                if (kk + 3 < c.K) ra.w = (ra.w - h) - l;
            }
        }
    } else {  // A[k][i]: 8 k-rows x 128 i
        int kk = k0 + (tid >> 5), i = c.i0 + (tid & 31) * 4;
        ra = load4(c.A, c.lda, kk, i, c.K, c.M, c.a_vec);
        if (c.a_hi && kk < c.K) {
            if (i + 0 < c.M) ra.x = (ra.x - c.a_hi[i + 0]) - c.a_lo[i + 0];
            if (i + 1 < c.M) ra.y = (ra.y - c.a_hi[i + 1]) - c.a_lo[i + 1];
            if (i + 2 < c.M) ra.z = (ra.z - c.a_hi[i + 2]) - c.a_lo[i + 2];
            if (i + 3 < c.M) ra.w = (ra.w - c.a_hi[i + 3]) - c.a_lo[i + 3];
        }
    }
    if (BT == 0) {  // B[k][j]: 8 k-rows x 128 j
        int kk = k0 + (tid >> 5), j = c.j0 + (tid & 31) * 4;
        rb = load4(c.B, c.ldb, kk, j, c.K, c.N, c.b_vec);
        if (c.b_hi && kk < c.K) {
            if (j + 0 < c.N) rb.x = (rb.x - c.b_hi[j + 0]) - c.b_lo[j + 0];
            if (j + 1 < c.N) rb.y = (rb.y - c.b_hi[j + 1]) - c.b_lo[j + 1];
            if (j + 2 < c.N) rb.z = (rb.z - c.b_hi[j + 2]) - c.b_lo[j + 2];
            if (j + 3 < c.N) rb.w = (rb.w - c.b_hi[j + 3]) - c.b_lo[j + 3];
        }
    } else {  // B[j][k]: 128 rows x 8 k
        rb = load4(c.B, c.ldb, c.j0 + (tid >> 1), k0 + (tid & 1) * 4, c.N, c.K, c.b_vec);
        if (c.b_hi) {
            int j = c.j0 + (tid >> 1);
            if (j < c.N) {
                float h = c.b_hi[j], l = c.b_lo[j];
                int kk = k0 + (tid & 1) * 4;
                if (kk + 0 < c.K) rb.x = (rb.x - h) - l;
                if (kk + 1 < c.K) rb.y = (rb.y - h) - l;
                if (kk + 2 < c.K) rb.z = (rb.z - h) - l;
                if (kk + 3 < c.K) rb.w = (rb.w - h) - l;
            }
        }
    }
}

template <int AT, int BT>
__device__ __forceinline__ void stash(float (*As)[PADW], float (*Bs)[PADW], int tid, const float4 &ra,
                                      const float4 &rb) {
    if (AT == 0) {
        int i = tid >> 1, k = (tid & 1) * 4;
        As[k + 0][i] = ra.x;
        As[k + 1][i] = ra.y;
        As[k + 2][i] = ra.z;
        As[k + 3][i] = ra.w;
    } else {
        *reinterpret_cast<float4 *>(&As[tid >> 5][(tid & 31) * 4]) = ra;
    }
    if (BT == 0) {
        *reinterpret_cast<float4 *>(&Bs[tid >> 5][(tid & 31) * 4]) = rb;
    } else {
        int j = tid >> 1, k = (tid & 1) * 4;
        Bs[k + 0][j] = rb.x;
        Bs[k + 1][j] = rb.y;
        Bs[k + 2][j] = rb.z;
        Bs[k + 3][j] = rb.w;
    }
}

__device__ __forceinline__ bool vec_ok(const float *p, long long ld) {
    return ((reinterpret_cast<uintptr_t>(p) & 15) == 0) && ((ld & 3) == 0);
}

// One 128 x 128 output tile at (i0, j0) over nseg segments of K.
template <int AT, int BT>
__device__ void simt_tile(int M, int N, int K, const SimtOperands &op, const EpiParams &epi, int i0, int j0) {
    __shared__ __align__(16) float As[2][TK][PADW];
    __shared__ __align__(16) float Bs[2][TK][PADW];
    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    float acc[8][8];
#pragma unroll
    for (int r = 0; r < 8; ++r)
#pragma unroll
        for (int q = 0; q < 8; ++q) acc[r][q] = 0.0f;

    const int kt = (K + TK - 1) / TK;
    const int total = kt * op.nseg;
    TileCtx c;
    c.M = M;
    c.N = N;
    c.K = K;
    c.i0 = i0;
    c.j0 = j0;
    c.a_hi = op.a_off_hi;
    c.a_lo = op.a_off_lo;
    c.b_hi = op.b_off_hi;
    c.b_lo = op.b_off_lo;

    float4 ra, rb;
    if (total > 0) {
        c.A = op.A[0];
        c.B = op.B[0];
        c.lda = op.lda[0];
        c.ldb = op.ldb[0];
        c.a_vec = vec_ok(c.A, c.lda);
        c.b_vec = vec_ok(c.B, c.ldb);
        fetch<AT, BT>(c, 0, tid, ra, rb);
        stash<AT, BT>(As[0], Bs[0], tid, ra, rb);
    }
    __syncthreads();
    for (int it = 0; it < total; ++it) {
        const int buf = it & 1;
        const bool more = it + 1 < total;
        if (more) {
            const bool seg1 = (it + 1) >= kt;
            c.A = seg1 ? op.A[1] : op.A[0];
            c.B = seg1 ? op.B[1] : op.B[0];
            c.lda = seg1 ? op.lda[1] : op.lda[0];
            c.ldb = seg1 ? op.ldb[1] : op.ldb[0];
            c.a_vec = vec_ok(c.A, c.lda);
            c.b_vec = vec_ok(c.B, c.ldb);
            fetch<AT, BT>(c, ((it + 1) % kt) * TK, tid, ra, rb);
        }
#pragma unroll
        for (int kk = 0; kk < TK; ++kk) {
            float4 a0 = *reinterpret_cast<const float4 *>(&As[buf][kk][ty * 4]);
            float4 a1 = *reinterpret_cast<const float4 *>(&As[buf][kk][64 + ty * 4]);
            float4 b0 = *reinterpret_cast<const float4 *>(&Bs[buf][kk][tx * 4]);
            float4 b1 = *reinterpret_cast<const float4 *>(&Bs[buf][kk][64 + tx * 4]);
            float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
            float b[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
            for (int r = 0; r < 8; ++r)
#pragma unroll
                for (int q = 0; q < 8; ++q) acc[r][q] = fmaf(a[r], b[q], acc[r][q]);
        }
        if (more) stash<AT, BT>(As[buf ^ 1], Bs[buf ^ 1], tid, ra, rb);
        __syncthreads();
    }
    // per row: issue the row's eight epilogue loads, then its stores
#pragma unroll
    for (int r = 0; r < 8; ++r) {
        const int i = i0 + (r < 4 ? ty * 4 + r : 64 + ty * 4 + (r - 4));
        float2 g[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) g[q] = epi_load(epi, i, j0 + (q < 4 ? tx * 4 + q : 64 + tx * 4 + (q - 4)));
#pragma unroll
        for (int q = 0; q < 8; ++q) epi_apply(epi, i, j0 + (q < 4 ? tx * 4 + q : 64 + tx * 4 + (q - 4)), acc[r][q], g[q]);
    }
}

__device__ __forceinline__ void tri_tile(int t, int &ti, int &tj) {
    int r = (int)((sqrtf(8.0f * (float)t + 1.0f) - 1.0f) * 0.5f);
    while ((r + 1) * (r + 2) / 2 <= t) ++r;
    while (r * (r + 1) / 2 > t) --r;
    ti = r;
    tj = t - r * (r + 1) / 2;
}

template <int AT, int BT>
__global__ __launch_bounds__(256, 2) void k_simt(int M, int N, int K, SimtOperands op, EpiParams epi, int sym) {
    int ti, tj;
    if (sym) {
        tri_tile(blockIdx.x, ti, tj);
    } else {
        ti = blockIdx.y;
        tj = blockIdx.x;
    }
    simt_tile<AT, BT>(M, N, K, op, epi, ti * TB, tj * TB);
}

// Batched SYRK/SYR2K: a flat grid over every instance's lower-triangle tiles.
__global__ __launch_bounds__(256, 2) void k_simt_sym_batched(int is_syr2k, const ln_sym_desc *__restrict__ descs,
                                                          const int *__restrict__ prefix, int count, int fill,
                                                          float alpha, float beta) {
    int t = blockIdx.x;
    int lo = 0, hi = count - 1;
    while (lo < hi) {  // last instance whose prefix <= t
        int mid = (lo + hi + 1) >> 1;
        if (prefix[mid] <= t) lo = mid;
        else hi = mid - 1;
    }
    const ln_sym_desc d = descs[lo];
    int ti, tj;
    tri_tile(t - prefix[lo], ti, tj);
    SimtOperands op{};
    op.a_t = 0;
    op.b_t = 1;
    op.nseg = is_syr2k ? 2 : 1;
    op.A[0] = d.A;
    op.lda[0] = d.lda;
    op.B[0] = is_syr2k ? d.B : d.A;
    op.ldb[0] = is_syr2k ? d.ldb : d.lda;
    op.A[1] = op.B[0];
    op.lda[1] = op.ldb[0];
    op.B[1] = d.A;
    op.ldb[1] = d.lda;
    EpiParams e{};
    e.mode = EPI_SYM;
    e.M = e.N = d.n;
    e.alpha = alpha;
    e.beta = beta;
    e.C = d.C;
    e.ldc = d.ldc;
    e.fill = fill;
    e.sym_kind = SYM_AXPBY;
    simt_tile<0, 1>(d.n, d.n, d.k, op, e, ti * TB, tj * TB);
}

__global__ void k_sym_prefix(int count, const ln_sym_desc *__restrict__ descs, int *prefix) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    int acc = 0;
    for (int i = 0; i < count; ++i) {
        prefix[i] = acc;
        int t = (descs[i].n + TB - 1) / TB;
        acc += t * (t + 1) / 2;
    }
    prefix[count] = acc;
}

}  // namespace

ln_status simt_contract(int M, int N, int K, const SimtOperands &op, const EpiParams &epi, cudaStream_t st) {
    const bool sym = epi.mode == EPI_SYM;
    dim3 grid;
    if (sym) {
        long long t = ceil_div(M, TB);
        grid = dim3((unsigned)(t * (t + 1) / 2));
    } else {
        grid = dim3((unsigned)ceil_div(N, TB), (unsigned)ceil_div(M, TB));
    }
    LaunchScope ls_(FAM_SIMT, st);
    if (op.a_t == 0 && op.b_t == 0) k_simt<0, 0><<<grid, 256, 0, st>>>(M, N, K, op, epi, sym);
    else if (op.a_t == 0 && op.b_t == 1) k_simt<0, 1><<<grid, 256, 0, st>>>(M, N, K, op, epi, sym);
    else if (op.a_t == 1 && op.b_t == 0) k_simt<1, 0><<<grid, 256, 0, st>>>(M, N, K, op, epi, sym);
    else k_simt<1, 1><<<grid, 256, 0, st>>>(M, N, K, op, epi, sym);
    return check_launch("fp32 tiled contraction");
}

ln_status simt_sym_batched_prefix(int count, const ln_sym_desc *d_descs, int *d_tile_prefix, cudaStream_t st) {
    { LaunchScope ls_(FAM_SIMT, st); k_sym_prefix<<<1, 32, 0, st>>>(count, d_descs, d_tile_prefix); }
    return check_launch("batched tile prefix");
}

ln_status simt_sym_batched(int is_syr2k, int count, const ln_sym_desc *d_descs, const int *d_tile_prefix,
                           int total_tiles, int fill, float alpha, float beta, cudaStream_t st) {
    { LaunchScope ls_(FAM_SIMT, st); k_simt_sym_batched<<<(unsigned)total_tiles, 256, 0, st>>>(is_syr2k, d_descs, d_tile_prefix, count, fill, alpha,
                                                              beta); }
    return check_launch("fp32 tiled batched syrk/syr2k");
}

}  // namespace ln
