// Internalized FP32 form: the work-group tiling of loop internalization
// (paper Sec. VI-C, Listing 6) mapped to a CTA. Each CTA owns a TB x TB output
// tile (TB = 128, or 64 for problems whose 128-wide tiles would leave SMs idle
// while their 64-wide tiles fit two to an SM); the inner k loop is tiled by TK
// (16 at TB = 128, 8 at 64), and each k-tile of both operands is copied from global memory into shared memory by
// 16-byte cp.async copies (4-byte ones, or zero fill, at ragged or unaligned
// edges) into a ring of NST stages (3 at TB = 128, 4 at 64), so that NST - 1
// k-tiles are in flight while one is consumed and a single barrier per k-tile
// orders the ring. Each thread accumulates an 8 x 8
// (TB = 128) or 4 x 4 (TB = 64) register block in exact FP32 FFMA and stores it
// once (Sec. VI-B).
//
// Constant propagation (the analogue of the paper's host-device constant
// propagation, Sec. VII): when the host sees that the problem divides into
// whole tiles and k-tiles and that every operand row is 16-byte aligned, it
// launches the EXACT instance, in which those facts are compile-time
// constants: no bounds predicates in the copies or the epilogue, and 16-byte
// epilogue accesses.
#include <type_traits>

#include "ln_async.cuh"
#include "ln_epilogue.cuh"
#include "ln_internal.h"

namespace ln {

int tune_simt_exact();  // ln_api.cu: the "simt_exact" knob
int tune_simt_tile();   // ln_api.cu: the "simt_tile" knob (0 automatic, 64, 128)

namespace {

constexpr int PADT = 4;   // row padding of k-major tiles ([TK][TB + PADT])
template <int TB>
constexpr int tk_of() { return TB == 128 ? 16 : 8; }  // k-tile depth
template <int TB>
constexpr int nst_of() { return TB == 128 ? 3 : 4; }  // ring stages

// Shared-memory extent (floats) of one operand tile: k-major ([TK][TB + PADT],
// rows of the operand's contiguous index) or k-contiguous ([TB][TK + 4]: 48-byte
// rows), both filled by 16-byte copies. k-major tiles are read 4 consecutive
// rows (columns) at a time; k-contiguous ones 4 consecutive k at a time, by
// lanes whose rows are one address per half-warp (A: rows follow ty) or
// consecutive (B: columns tx + 16 q), so that no read has bank conflicts.
template <int TB, int KMAJ>
struct TileShape {
    static constexpr int TK = tk_of<TB>();
    static constexpr bool KMAJOR = KMAJ;  // 1: element (k, x) at [k][x]; 0: at [x][k]
    static constexpr int LD = KMAJOR ? TB + PADT : TK + 4;
    static constexpr int FLOATS = KMAJOR ? TK * LD : TB * LD;
    static constexpr bool V16 = true;
};

__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src, bool ok) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(ok ? 16 : 0) : "memory");
}
__device__ __forceinline__ void cp_async4(uint32_t dst, const void *src, bool ok) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(dst), "l"(src), "r"(ok ? 4 : 0) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

__device__ __forceinline__ bool vec_ok(const float *p, long long ld) {
    return ((reinterpret_cast<uintptr_t>(p) & 15) == 0) && ((ld & 3) == 0);
}

// Copies the 16-byte chunk (r, c .. c + 3) of a row-major rows x cols matrix
// (leading dimension ld) to shared address dst; elements outside the matrix
// are zero. vec: 16-byte copies are legal for whole chunks.
// V16: the shared-memory destination takes 16-byte copies; else four 4-byte
// ones at dst, dst + dstep, dst + 2 dstep, dst + 3 dstep (bytes).
template <bool EXACT, bool V16>
__device__ __forceinline__ void copy_chunk(uint32_t dst, uint32_t dstep, const float *p, long long ld, int r, int c,
                                           int rows, int cols, bool vec) {
    if (V16 && EXACT) {
        cp_async16(dst, p + (long long)r * ld + c, true);
        return;
    }
    const bool inr = EXACT || r < rows;
    const float *q = p + (long long)r * ld + c;
    if (V16) {
        if (!inr || c >= cols) {
            cp_async16(dst, p, false);
            return;
        }
        if (vec && c + 3 < cols) {
            cp_async16(dst, q, true);
            return;
        }
    }
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        const bool ok = inr && (EXACT || c + e < cols);
        cp_async4(dst + dstep * e, ok ? q + e : p, ok);
    }
}

// Operand roles: op A is M x K (AT = 0: A[i][k], AT = 1: A[k][i]); op B is
// K x N (BT = 0: B[k][j], BT = 1: B[j][k]). In shared memory A is k-major when
// AT = 1 (its rows are k), B k-major when BT = 0.
template <int AT, int BT, int TB, bool EXACT>
struct Simt {
    using SA = TileShape<TB, AT>;      // A k-major iff AT == 1
    using SB = TileShape<TB, 1 - BT>;  // B k-major iff BT == 0
    static constexpr int TK = tk_of<TB>();
    static constexpr int NST = nst_of<TB>();
    static constexpr int STAGE = SA::FLOATS + SB::FLOATS;
    static constexpr int SMEM = NST * STAGE * 4;  // dynamic shared memory (bytes)
    // k values per read of a k-contiguous tile: 4 (16-byte reads), or 2 when both
    // operands are k-contiguous, so that the held values fit two CTAs per SM
    static constexpr int KG = (AT == 0 && BT == 1) ? 2 : 4;
    static constexpr int R = TB / 16;  // rows (and columns) per thread: 8 or 4
    static constexpr int CHUNKS = TK * TB / 4;  // 16-byte chunks per operand per k-tile

    struct Ctx {
        const float *A, *B;
        long long lda, ldb;
        bool avec, bvec;
    };

    __device__ static Ctx seg_ctx(const SimtOperands &op, int sg) {
        // selects, not a runtime index into the parameter block (which would
        // copy it to local memory)
        Ctx c;
        c.A = sg ? op.A[1] : op.A[0];
        c.B = sg ? op.B[1] : op.B[0];
        c.lda = sg ? op.lda[1] : op.lda[0];
        c.ldb = sg ? op.ldb[1] : op.ldb[0];
        c.avec = vec_ok(c.A, c.lda);
        c.bvec = vec_ok(c.B, c.ldb);
        return c;
    }

    // chunk `id` of an operand tile: (row, col) in the operand's storage and the
    // shared-memory float offset it goes to (its four elements are consecutive
    // in both)
    __device__ static void chunk_a(int id, int i0, int k0, int &r, int &c, int &off) {
        if (AT) {  // A[k][i]: rows k, cols i
            const int k = id / (TB / 4), x = (id % (TB / 4)) * 4;
            r = k0 + k;
            c = i0 + x;
            off = k * SA::LD + x;
        } else {  // A[i][k]: rows i, cols k
            const int x = id / (TK / 4), k = (id % (TK / 4)) * 4;
            r = i0 + x;
            c = k0 + k;
            off = x * SA::LD + k;
        }
    }
    __device__ static void chunk_b(int id, int j0, int k0, int &r, int &c, int &off) {
        if (BT == 0) {  // B[k][j]: rows k, cols j
            const int k = id / (TB / 4), x = (id % (TB / 4)) * 4;
            r = k0 + k;
            c = j0 + x;
            off = k * SB::LD + x;
        } else {  // B[j][k]: rows j, cols k
            const int x = id / (TK / 4), k = (id % (TK / 4)) * 4;
            r = j0 + x;
            c = k0 + k;
            off = x * SB::LD + k;
        }
    }

    // Issue the copies of flattened k-tile q (segment q / kt) into stage `buf`.
    __device__ static void issue(float *sm, int buf, int q, int kt, const SimtOperands &op, int M, int N, int K,
                                 int i0, int j0, int tid) {
        const Ctx c = seg_ctx(op, q / kt);
        const int k0 = (q % kt) * TK;
        float *sa = sm + buf * STAGE, *sb = sa + SA::FLOATS;
        for (int id = tid; id < 2 * CHUNKS; id += 256) {
            int r, col, off;
            if (id < CHUNKS) {
                chunk_a(id, i0, k0, r, col, off);
                copy_chunk<EXACT, SA::V16>(saddr(sa + off), 4, c.A, c.lda, r, col, AT ? K : M, AT ? M : K, c.avec);
            } else {
                chunk_b(id - CHUNKS, j0, k0, r, col, off);
                copy_chunk<EXACT, SB::V16>(saddr(sb + off), 4, c.B, c.ldb, r, col, BT ? N : K, BT ? K : N, c.bvec);
            }
        }
    }

    // Centring (covariance: v = (x - hi) - lo per column of the data matrix)
    // of the chunks this thread copied into stage `buf`. Only the k-major
    // layouts carry offsets (the data matrix is A[k][i] and B[k][j]); a thread's
    // chunks keep their columns from k-tile to k-tile, so their offsets were
    // read once into ha/la (A) and hb/lb (B). Elements outside the matrix stay 0.
    __device__ static void centre(float *sm, int buf, int q, int kt, int K, int i0, int j0, int tid, int M, int N,
                                  const float4 &ha, const float4 &la, const float4 &hb, const float4 &lb, bool offa,
                                  bool offb) {
        const int k0 = (q % kt) * TK;
        float *sa = sm + buf * STAGE, *sb = sa + SA::FLOATS;
        for (int id = tid; id < 2 * CHUNKS; id += 256) {
            const bool isa = id < CHUNKS;
            if (isa ? !offa : !offb) continue;
            int r, col, off;
            if (isa) chunk_a(id, i0, k0, r, col, off);
            else chunk_b(id - CHUNKS, j0, k0, r, col, off);
            if (r >= K) continue;
            float *v = (isa ? sa : sb) + off;
            const float4 h = isa ? ha : hb, l = isa ? la : lb;
            const int cols = isa ? M : N;
            if (col + 0 < cols) v[0] = (v[0] - h.x) - l.x;
            if (col + 1 < cols) v[1] = (v[1] - h.y) - l.y;
            if (col + 2 < cols) v[2] = (v[2] - h.z) - l.z;
            if (col + 3 < cols) v[3] = (v[3] - h.w) - l.w;
        }
    }

    // this thread's centring offsets of chunk `id`'s four columns (zero outside)
    __device__ static float4 offsets4(const float *off, int x0, int n) {
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (!off) return v;
        if (x0 + 0 < n) v.x = off[x0 + 0];
        if (x0 + 1 < n) v.y = off[x0 + 1];
        if (x0 + 2 < n) v.z = off[x0 + 2];
        if (x0 + 3 < n) v.w = off[x0 + 3];
        return v;
    }

    __device__ static float comp(const float4 &v, int i) { return i == 0 ? v.x : i == 1 ? v.y : i == 2 ? v.z : v.w; }
    __device__ static float comp(const float2 &v, int i) { return i == 0 ? v.x : v.y; }

    // output row of this thread's accumulator row r, and column of its column q
    __device__ static int row_of(int r, int ty) { return (r / 4) * (TB / 2) + ty * 4 + r % 4; }
    __device__ static int col_of(int q, int tx) { return BT ? tx + 16 * q : (q / 4) * (TB / 2) + tx * 4 + q % 4; }

    __device__ static void tile(int M, int N, int K, const SimtOperands &op, const EpiParams &epi, int i0, int j0) {
        extern __shared__ __align__(16) float sm[];
        const int tid = threadIdx.x;
        const int tx = tid & 15, ty = tid >> 4;
        float acc[R][R];
#pragma unroll
        for (int r = 0; r < R; ++r)
#pragma unroll
            for (int q = 0; q < R; ++q) acc[r][q] = 0.0f;
        const int kt = (K + TK - 1) / TK;
        const int nkt = kt * op.nseg;
        // centring offsets: only the k-major layouts (covariance's A[k][i], B[k][j]) take them
        const bool offa = AT == 1 && op.a_off_hi, offb = BT == 0 && op.b_off_hi;
        float4 ha{}, la{}, hb{}, lb{};
        if (offa || offb) {
            // this thread's chunks (ids tid, tid + 256, ... over A then B) keep their
            // columns x = (id % (TB / 4)) * 4 in every k-tile
            for (int id = tid; id < 2 * CHUNKS; id += 256) {
                const int x = (id < CHUNKS ? i0 : j0) + ((id % CHUNKS) % (TB / 4)) * 4;
                if (id < CHUNKS && offa) ha = offsets4(op.a_off_hi, x, M), la = offsets4(op.a_off_lo, x, M);
                if (id >= CHUNKS && offb) hb = offsets4(op.b_off_hi, x, N), lb = offsets4(op.b_off_lo, x, N);
            }
        }

#pragma unroll
        for (int s = 0; s < NST - 1; ++s) {
            if (s < nkt) issue(sm, s, s, kt, op, M, N, K, i0, j0, tid);
            cp_commit();
        }
        for (int it = 0; it < nkt; ++it) {
            const int buf = it % NST;
            if constexpr (NST == 4) cp_wait<2>();  // this thread's copies of k-tile it have landed
            else cp_wait<1>();
            if (offa || offb) centre(sm, buf, it, kt, K, i0, j0, tid, M, N, ha, la, hb, lb, offa, offb);
            __syncthreads();  // every thread's copies of k-tile it; stage (it - 1) % NST is free
            if (it + NST - 1 < nkt) issue(sm, (it + NST - 1) % NST, it + NST - 1, kt, op, M, N, K, i0, j0, tid);
            cp_commit();
            const float *sa = sm + buf * STAGE, *sb = sa + SA::FLOATS;
#pragma unroll
            for (int kq = 0; kq < TK; kq += KG) {
                // k-contiguous tiles: KG consecutive k of a row (column) per read
                using VK = typename std::conditional<KG == 4, float4, float2>::type;
                VK a4[AT ? 1 : R], b4[BT ? R : 1];
                if (!AT) {
#pragma unroll
                    for (int r = 0; r < R; ++r) a4[r] = *reinterpret_cast<const VK *>(sa + row_of(r, ty) * SA::LD + kq);
                }
                if (BT) {
#pragma unroll
                    for (int q = 0; q < R; ++q) b4[q] = *reinterpret_cast<const VK *>(sb + col_of(q, tx) * SB::LD + kq);
                }
#pragma unroll
                for (int k4 = 0; k4 < KG; ++k4) {
                    const int kk = kq + k4;
                    float a[R], b[R];
                    if (AT) {  // k-major: four consecutive rows per 16-byte read
#pragma unroll
                        for (int h = 0; h < R / 4; ++h) {
                            const float4 v = *reinterpret_cast<const float4 *>(sa + kk * SA::LD + row_of(4 * h, ty));
                            a[4 * h] = v.x, a[4 * h + 1] = v.y, a[4 * h + 2] = v.z, a[4 * h + 3] = v.w;
                        }
                    } else {
#pragma unroll
                        for (int r = 0; r < R; ++r) a[r] = comp(a4[r], k4);
                    }
                    if (BT == 0) {
#pragma unroll
                        for (int h = 0; h < R / 4; ++h) {
                            const float4 v = *reinterpret_cast<const float4 *>(sb + kk * SB::LD + col_of(4 * h, tx));
                            b[4 * h] = v.x, b[4 * h + 1] = v.y, b[4 * h + 2] = v.z, b[4 * h + 3] = v.w;
                        }
                    } else {
#pragma unroll
                        for (int q = 0; q < R; ++q) b[q] = comp(b4[q], k4);
                    }
#pragma unroll
                    for (int r = 0; r < R; ++r)
#pragma unroll
                        for (int q = 0; q < R; ++q) acc[r][q] = fmaf(a[r], b[q], acc[r][q]);
                }
            }
        }
        cp_wait<0>();
        epilogue(epi, i0, j0, tx, ty, acc);
        static_assert(NST == 3 || NST == 4, "ring depth");
    }

    // Row r of this thread's block is output row i0 + row_of(r), column q is
    // j0 + col_of(q): four consecutive columns per group unless B is k-contiguous.
    __device__ static void epilogue(const EpiParams &epi, int i0, int j0, int tx, int ty, float (&acc)[R][R]) {
        if (EXACT && BT == 0 && (epi.mode == EPI_GEMM || epi.mode == EPI_STORE || epi.mode == EPI_EF)) {
            // whole tile inside the output, rows 16-byte aligned: four columns per access
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int i = i0 + row_of(r, ty);
#pragma unroll
                for (int h = 0; h < R / 4; ++h) {
                    const int j = j0 + col_of(4 * h, tx);
                    const float4 v = make_float4(acc[r][4 * h], acc[r][4 * h + 1], acc[r][4 * h + 2], acc[r][4 * h + 3]);
                    if (epi.mode == EPI_EF) {
                        const long long o = (long long)i * epi.ld_ef + j;
                        *reinterpret_cast<float4 *>(epi.E + o) = v;
                        float4 f = make_float4(epi.alpha * v.x, epi.alpha * v.y, epi.alpha * v.z, epi.alpha * v.w);
                        if (epi.beta != 0.0f) {
                            const float4 d = *reinterpret_cast<const float4 *>(epi.D + o);
                            f.x = fmaf(epi.beta, d.x, f.x), f.y = fmaf(epi.beta, d.y, f.y);
                            f.z = fmaf(epi.beta, d.z, f.z), f.w = fmaf(epi.beta, d.w, f.w);
                        }
                        *reinterpret_cast<float4 *>(epi.F + o) = f;
                    } else {
                        float *c = epi.C + (long long)i * epi.ldc + j;
                        float4 f = make_float4(epi.alpha * v.x, epi.alpha * v.y, epi.alpha * v.z, epi.alpha * v.w);
                        if (epi.mode == EPI_GEMM && epi.beta != 0.0f) {
                            const float4 d = *reinterpret_cast<const float4 *>(c);
                            f.x = fmaf(epi.beta, d.x, f.x), f.y = fmaf(epi.beta, d.y, f.y);
                            f.z = fmaf(epi.beta, d.z, f.z), f.w = fmaf(epi.beta, d.w, f.w);
                        }
                        *reinterpret_cast<float4 *>(c) = f;
                    }
                }
            }
            return;
        }
        // per row: issue the row's epilogue loads, then its stores
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int i = i0 + row_of(r, ty);
            float2 g[R];
#pragma unroll
            for (int q = 0; q < R; ++q) g[q] = epi_load(epi, i, j0 + col_of(q, tx));
#pragma unroll
            for (int q = 0; q < R; ++q) epi_apply(epi, i, j0 + col_of(q, tx), acc[r][q], g[q]);
        }
    }
};

__device__ __forceinline__ void tri_tile(int t, int &ti, int &tj) {
    int r = (int)((sqrtf(8.0f * (float)t + 1.0f) - 1.0f) * 0.5f);
    while ((r + 1) * (r + 2) / 2 <= t) ++r;
    while (r * (r + 1) / 2 > t) --r;
    ti = r;
    tj = t - r * (r + 1) / 2;
}

// Two CTAs of 256 threads per SM (at most 128 registers a thread).
template <int AT, int BT, int TB>
constexpr int simt_min_blocks() { return 2; }

template <int AT, int BT, int TB, bool EXACT>
__global__ __launch_bounds__(256, simt_min_blocks<AT, BT, TB>()) void k_simt(int M, int N, int K, SimtOperands op, EpiParams epi, int sym) {
    int ti, tj;
    if (sym) {
        tri_tile(blockIdx.x, ti, tj);
    } else {
        ti = blockIdx.y;
        tj = blockIdx.x;
    }
    Simt<AT, BT, TB, EXACT>::tile(M, N, K, op, epi, ti * TB, tj * TB);
}

// Batched SYRK/SYR2K: a flat grid over every instance's lower-triangle tiles.
constexpr int TB_BATCH = 128;
__global__ __launch_bounds__(256, simt_min_blocks<0, 1, TB_BATCH>()) void k_simt_sym_batched(int is_syr2k, const ln_sym_desc *__restrict__ descs,
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
    Simt<0, 1, TB_BATCH, false>::tile(d.n, d.n, d.k, op, e, ti * TB_BATCH, tj * TB_BATCH);
}

__global__ void k_sym_prefix(int count, const ln_sym_desc *__restrict__ descs, int *prefix) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    int acc = 0;
    for (int i = 0; i < count; ++i) {
        prefix[i] = acc;
        int t = (descs[i].n + TB_BATCH - 1) / TB_BATCH;
        acc += t * (t + 1) / 2;
    }
    prefix[count] = acc;
}

bool host_vec(const void *p, long long ld) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0 && (ld & 3) == 0; }

// The facts the EXACT instance takes as constants, checked on the host.
bool exact_ok(int M, int N, int K, int TB, const SimtOperands &op, const EpiParams &e) {
    const int tk = TB == 128 ? tk_of<128>() : tk_of<64>();
    if (M % TB || N % TB || K % tk || K == 0) return false;
    for (int s = 0; s < op.nseg; ++s)
        if (!host_vec(op.A[s], op.lda[s]) || !host_vec(op.B[s], op.ldb[s])) return false;
    switch (e.mode) {
        case EPI_GEMM:
        case EPI_STORE: return host_vec(e.C, e.ldc);
        case EPI_EF: return host_vec(e.E, e.ld_ef) && host_vec(e.F, e.ld_ef) && (e.beta == 0.0f || host_vec(e.D, e.ld_ef));
        default: return true;  // symmetric outputs keep the element-wise epilogue
    }
}

// The dynamic shared-memory opt-in of a kernel, once per device (so that
// nothing but launches happens while a caller captures a graph).
template <class F>
ln_status smem_optin(F kern, int bytes, bool (&done)[64]) {
    int dev = 0;
    LN_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64 || !done[dev]) {
        LN_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
        if (dev >= 0 && dev < 64) done[dev] = true;
    }
    return LN_SUCCESS;
}

template <int AT, int BT, int TB, bool EXACT>
ln_status launch_one(dim3 grid, int M, int N, int K, const SimtOperands &op, const EpiParams &epi, int sym,
                     cudaStream_t st) {
    static bool done[64] = {false};
    auto kern = k_simt<AT, BT, TB, EXACT>;
    constexpr int smem = Simt<AT, BT, TB, EXACT>::SMEM;
    ln_status s = smem_optin(kern, smem, done);
    if (s != LN_SUCCESS) return s;
    kern<<<grid, 256, smem, st>>>(M, N, K, op, epi, sym);
    return LN_SUCCESS;
}

template <int AT, int BT, int TB>
ln_status launch_simt(dim3 grid, int M, int N, int K, const SimtOperands &op, const EpiParams &epi, int sym,
                      bool exact, cudaStream_t st) {
    return exact ? launch_one<AT, BT, TB, true>(grid, M, N, K, op, epi, sym, st)
                 : launch_one<AT, BT, TB, false>(grid, M, N, K, op, epi, sym, st);
}

template <int TB>
ln_status launch_simt_tb(dim3 grid, int M, int N, int K, const SimtOperands &op, const EpiParams &epi, int sym,
                         bool exact, cudaStream_t st) {
    if (op.a_t == 0 && op.b_t == 0) return launch_simt<0, 0, TB>(grid, M, N, K, op, epi, sym, exact, st);
    if (op.a_t == 0 && op.b_t == 1) return launch_simt<0, 1, TB>(grid, M, N, K, op, epi, sym, exact, st);
    if (op.a_t == 1 && op.b_t == 0) return launch_simt<1, 0, TB>(grid, M, N, K, op, epi, sym, exact, st);
    return launch_simt<1, 1, TB>(grid, M, N, K, op, epi, sym, exact, st);
}

}  // namespace

ln_status simt_contract(int M, int N, int K, const SimtOperands &op, const EpiParams &epi, cudaStream_t st) {
    const bool sym = epi.mode == EPI_SYM;
    // 64-wide tiles when the 128-wide ones leave SMs idle (one tile per SM at
    // most) and the 64-wide ones still fit two to an SM; otherwise the 8 x 8
    // register blocks of the 128-wide tiles do more FFMAs per shared load
    auto tiles_of = [&](int tb) {
        const long long t = ceil_div(M, tb);
        return sym ? t * (t + 1) / 2 : t * ceil_div(N, tb);
    };
    const int knob = tune_simt_tile();
    const long long sms = sm_count();
    const int TB = knob == 64 || knob == 128 ? knob
                                             : (tiles_of(128) <= sms && tiles_of(64) <= 2 * sms ? 64 : 128);
    dim3 grid;
    if (sym) {
        grid = dim3((unsigned)tiles_of(TB));
    } else {
        grid = dim3((unsigned)ceil_div(N, TB), (unsigned)ceil_div(M, TB));
    }
    const bool exact = tune_simt_exact() && exact_ok(M, N, K, TB, op, epi);
    ln_status s;
    {
        LaunchScope ls_(FAM_SIMT, st);
        s = TB == 64 ? launch_simt_tb<64>(grid, M, N, K, op, epi, sym, exact, st)
                     : launch_simt_tb<128>(grid, M, N, K, op, epi, sym, exact, st);
    }
    if (s != LN_SUCCESS) return s;
    return check_launch("fp32 tiled contraction");
}

long long simt_sym_batched_tiles(int count, const ln_sym_desc *h) {
    long long total = 0;
    for (int i = 0; i < count; ++i) {
        const long long t = ceil_div(h[i].n, TB_BATCH);
        total += t * (t + 1) / 2;
    }
    return total;
}

ln_status simt_sym_batched_prefix(int count, const ln_sym_desc *d_descs, int *d_tile_prefix, cudaStream_t st) {
    { LaunchScope ls_(FAM_SIMT, st); k_sym_prefix<<<1, 32, 0, st>>>(count, d_descs, d_tile_prefix); }
    return check_launch("batched tile prefix");
}

ln_status simt_sym_batched(int is_syr2k, int count, const ln_sym_desc *d_descs, const int *d_tile_prefix,
                           int total_tiles, int fill, float alpha, float beta, cudaStream_t st) {
    static bool done[64] = {false};
    constexpr int smem = Simt<0, 1, TB_BATCH, false>::SMEM;
    ln_status s = smem_optin(k_simt_sym_batched, smem, done);
    if (s != LN_SUCCESS) return s;
    {
        LaunchScope ls_(FAM_SIMT, st);
        k_simt_sym_batched<<<(unsigned)total_tiles, 256, smem, st>>>(is_syr2k, d_descs, d_tile_prefix, count, fill,
                                                                    alpha, beta);
    }
    return check_launch("fp32 tiled batched syrk/syr2k");
}

}  // namespace ln
