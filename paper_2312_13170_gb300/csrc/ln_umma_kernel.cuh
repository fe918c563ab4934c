// Internalized tensor-core form: loop internalization (paper Sec. VI-C,
// Listing 6) on sm_103a. The work-group tile becomes a 128 x BN CTA output
// tile (BN = 256 for general contractions, 128 for symmetric ones); the "prefetch one tile of each operand into local memory, barrier,
// inner loop over the tile, barrier" sequence becomes a ring of shared-memory
// stages filled by the bulk-copy (TMA) engine and guarded by mbarriers, and
// the inner loop over the tile becomes tcgen05.mma instructions accumulating
// in tensor memory (TMEM), stored once per tile (Sec. VI-B).
//
// Operands arrive pre-split into BF16 terms and pre-packed in the tensor
// core's K-major 128-byte-swizzled layout (ln_pack.cu), so each stage is a
// couple of contiguous bulk copies. The kernel is persistent: one CTA per SM
// takes output tiles from a static stride or from a device-side queue (an
// atomic counter), and double-buffers its TMEM accumulator so that the
// epilogue of one tile overlaps the MMAs of the next.
//
// Warp roles: warp 0 issues bulk copies, warp 1 allocates TMEM and issues
// MMAs (one lane each), BN/32 epilogue warps from warp EPI0 on read the
// accumulator back with tcgen05.ld (each warp owns the 32 TMEM lanes = output
// rows its warp index may access, and 128 of the tile's columns) and run the
// shared epilogue. With BN = 256 the epilogue is two whole warpgroups that
// take registers from warpgroup 0 with setmaxnreg.
//
// Accumulation precision: the tensor core's FP32 accumulation into TMEM loses
// accuracy in proportion to the number of accumulation steps, so every
// UMMA_CHUNK_KT k tiles the partial sum moves to a fresh TMEM buffer and the
// epilogue warps add it, with round-to-nearest FP32 adds, into a running sum
// kept in registers (128 values per thread).
//
// Every mbarrier wait is bounded by the global timer: a wait that runs out
// sets the CTA's abort flag and the library's device error word, every role
// leaves its loop, in-flight copies and MMAs are waited for (again bounded),
// TMEM is freed and the kernel returns. ln_stream_check() reports it.
#pragma once

#include "ln_async.cuh"
#include "ln_epilogue.cuh"
#include "ln_internal.h"
#include "ln_pack_stream.cuh"
#include "ln_split.cuh"

namespace ln {

namespace {

// Device error word of the translation unit that includes this header (each
// tcgen05 translation unit has its own; umma_read_error reads them all).
__device__ int g_umma_error;

constexpr int BM = 128;
constexpr int SCHED = 4;
constexpr int MAX_NACC = 4;
constexpr int TMEM_COLS = 512;
constexpr int MAX_STAGES = 8;
constexpr unsigned long long WAIT_NS = 2000000000ull;  // 2 s per wait
constexpr int CTL_BYTES = 2048;
constexpr int SMEM_BUDGET = 227 * 1024;

enum : int { ERR_PRODUCER = 1, ERR_MMA = 2, ERR_EPILOGUE = 4, ERR_DRAIN = 8 };

// One scheduled tile: the producer resolves it once (tile index -> problem,
// row tile, column tile) and, for batched launches, copies the problem's
// descriptor into shared memory; the MMA and epilogue roles read the slot and
// release it (sempty) when they have finished the tile.
struct SchedSlot {
    int t, mi, ni, ks;  // work item (stream-K: output tile; pairs: pair tile), row tile, column tile, k slice
    int qa, qb;         // k tiles [qa, qb) of the flattened nseg * kt range this item covers
    int ghost;          // pairs: this CTA's tile lies outside the output (or above the diagonal):
                        // it only copies and releases its share of the pair's stages
    int dsmem;          // the CTA's last tile: once its MMAs are done the producer copies the tile's
                        // block of the beta input (D or C) into the freed stage memory (dfull);
                        // packing epilogue: the tile's packed output is built there and bulk-stored
    UmmaProblem prob;
};

// Stream-K decomposition (UmmaProblem::streamk): the tiles x ktot k-tile units
// of a single problem, in tile-major order, are split evenly over the G CTAs of
// the launch; CTA c covers units [sk_start(c), sk_start(c + 1)).
__device__ __forceinline__ long long sk_start(int c, long long units, int G) { return (long long)c * units / G; }

// Bounded wait until the int at f is non-zero (acquire, GPU scope).
__device__ __forceinline__ int ld_acquire(const int *f) {
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(f) : "memory");
    return v;
}

// k tiles [qa, qb) of slice ks of a problem's nseg * kt flattened k range
__device__ __forceinline__ void slice_range(const UmmaProblem &p, int ks, int &qa, int &qb) {
    const int ktot = p.nseg * p.kt;
    if (p.ksplit <= 1) {
        qa = 0;
        qb = ktot;
        return;
    }
    const int per = (ktot + p.ksplit - 1) / p.ksplit;
    qa = ks * per;
    qb = qa + per < ktot ? qa + per : ktot;
}

struct Ctl {
    uint64_t full[MAX_STAGES];
    uint64_t empty[MAX_STAGES];
    uint64_t pfull[MAX_STAGES];  // CTA pairs, leader: the peer's stage is full (relayed by the peer)
    uint64_t tfull[MAX_NACC];
    uint64_t tempty[MAX_NACC];
    uint64_t sfull[SCHED];
    uint64_t sempty[SCHED];
    uint64_t drain;
    uint64_t dfull;  // the beta-input block of a dsmem tile is in the stage memory
    uint32_t tmem_base;
    volatile int abort;
    SchedSlot slot[SCHED];
};
static_assert(sizeof(Ctl) <= CTL_BYTES, "control block too large");

// ---------------------------------------------------------------- PTX wrappers
// (mbarrier, bulk-copy and timer wrappers are in ln_async.cuh)

// Bounded wait for the phase of `b` with the given parity. With honor_abort,
// returns false as soon as another role has aborted. A waiter that may wait
// long (epilogue, producer) passes sleep_ns > 0: after a few polls it sleeps
// between polls, so it does not take issue slots from the MMA-issuing thread
// that shares its SM sub-partition; the MMA thread polls without sleeping.
__device__ bool wait_phase(Ctl *ctl, uint64_t *b, uint32_t parity, int who, bool honor_abort = true,
                           unsigned sleep_ns = 0) {
    if (mbar_try_wait(b, parity)) return true;
    const unsigned long long t0 = gtimer();
    for (uint32_t n = 1;; ++n) {
        if (mbar_try_wait(b, parity)) return true;
        if (sleep_ns && n > 4) __nanosleep(sleep_ns);
        if ((n & 31) == 0) {
            if (honor_abort && ctl->abort) return false;
            if (gtimer() - t0 > WAIT_NS) {
                ctl->abort = 1;
                atomicOr(&g_umma_error, who);
                return false;
            }
        }
    }
}

// wait_phase with cluster-scope acquire, for barriers that the peer CTA of a
// pair arrives on
__device__ bool wait_phase_cl(Ctl *ctl, uint64_t *b, uint32_t parity, int who) {
    auto probe = [&]() {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(saddr(b)), "r"(parity)
            : "memory");
        return ok != 0;
    };
    if (probe()) return true;
    const unsigned long long t0 = gtimer();
    for (uint32_t n = 1;; ++n) {
        if (probe()) return true;
        if ((n & 31) == 0) {
            if (ctl->abort) return false;
            if (gtimer() - t0 > WAIT_NS) {
                ctl->abort = 1;
                atomicOr(&g_umma_error, who);
                return false;
            }
        }
    }
}

// Arrival (release, cluster scope) on the mbarrier at bar's offset in CTA
// `cta` of this cluster.
__device__ __forceinline__ void mbar_arrive_remote(uint64_t *bar, uint32_t cta) {
    uint32_t remote;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(remote) : "r"(saddr(bar)), "r"(cta));
    asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(remote) : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor of a K-major operand with 128-byte swizzle:
// 8-row groups 1024 bytes apart, descriptor version 1, swizzle mode 2.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t addr) {
    uint64_t d = (uint64_t)((addr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1 << 16;
    d |= (uint64_t)(1024 >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}

// Instruction descriptor: BF16 x BF16 -> FP32, both operands K-major, M x N.
__host__ __device__ constexpr uint32_t idesc_bf16(int n, int m = BM) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

template <int BN>
__device__ __forceinline__ void umma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc_bf16(BN)), "r"(acc)
        : "memory");
}
// CTA pair, issued by the leader: M = 256 (128 rows in each CTA's shared
// memory and tensor memory), N = BN with each CTA holding BN / 2 rows of B.
template <int BN>
__device__ __forceinline__ void umma_bf16_pair(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc_bf16(BN, 2 * BM)), "r"(acc)
        : "memory");
}
// TF32 operands (kind::tf32, K = 8 per instruction: the same 32 bytes of each
// 128-byte row as a BF16 K = 16 step, so the descriptors advance alike). The
// instruction descriptor differs from the BF16 one only in the A and B format
// fields (TF32 = 2).
__host__ __device__ constexpr uint32_t idesc_tf32(int n, int m = BM) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}
template <int BN>
__device__ __forceinline__ void umma_tf32(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc_tf32(BN)), "r"(acc)
        : "memory");
}
template <int BN>
__device__ __forceinline__ void umma_tf32_pair(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::2.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc_tf32(BN, 2 * BM)), "r"(acc)
        : "memory");
}
// completion of the pair's MMAs, signalled on the mbarrier at bar's offset in both CTAs
__device__ __forceinline__ void umma_commit_pair_mc(uint64_t *bar) {
    asm volatile(
        "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(
            saddr(bar)),
        "h"((uint16_t)0x3)
        : "memory");
}
__device__ __forceinline__ void umma_commit_pair(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(saddr(bar))
                 : "memory");
}
__device__ __forceinline__ void umma_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(saddr(bar))
                 : "memory");
}
// Pair tile T of a CTA pair -> this CTA's (row tile, column tile), and whether
// that tile is a ghost. General problems: row-tile pairs (2p, 2p + 1) times the
// nt column tiles. Symmetric problems: row-tile pair p with the column tiles
// 0 .. min(2p + 1, mt - 1); the tile of row 2p and column 2p + 1 lies above the
// diagonal.
__device__ __forceinline__ void pair_tile(const UmmaProblem &p, int T, int rank, int &mi, int &ni, int &ghost) {
    int pr;
    if (p.sym) {
        pr = (int)((sqrtf(4.0f * (float)T + 1.0f) - 1.0f) * 0.5f);
        while ((pr + 1) * (pr + 2) <= T) ++pr;
        while (pr * (pr + 1) > T) --pr;
        ni = T - pr * (pr + 1);
    } else {
        pr = T / p.nt;
        ni = T - pr * p.nt;
    }
    mi = 2 * pr + rank;
    ghost = mi >= p.mt || (p.sym && ni > mi);
}

// 32 lanes x 16 consecutive columns, without the wait: r is valid only after
// tmem_wait() and tmem_after_wait(r).
__device__ __forceinline__ void tmem_ld16_async(uint32_t taddr, uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
// Ties registers written by tcgen05.ld to a point after tmem_wait(): the empty
// volatile statements cannot move above the wait, and every later use reads
// the value they "produce".
__device__ __forceinline__ void tmem_after_wait(uint32_t (&r)[16]) {
#pragma unroll
    for (int q = 0; q < 16; ++q) asm volatile("" : "+r"(r[q]));
}

// ---------------------------------------------------------------- tile scheduling
__device__ __forceinline__ void tri_tile(int t, int &ti, int &tj) {
    int r = (int)((sqrtf(8.0f * (float)t + 1.0f) - 1.0f) * 0.5f);
    while ((r + 1) * (r + 2) / 2 <= t) ++r;
    while (r * (r + 1) / 2 > t) --r;
    ti = r;
    tj = t - r * (r + 1) / 2;
}

// Lower-triangle tiles of 128 rows x 256 columns: row tile mi holds column
// tiles 0 .. mi / 2 (those with a column <= some row of the tile), so row
// tiles 2q and 2q + 1 hold q + 1 each and tiles 0 .. q(q + 1) - 1 cover row
// tiles below 2q.
__device__ __forceinline__ void tri_tile_wide(int t, int &ti, int &tj) {
    int q = (int)((sqrtf(4.0f * (float)t + 1.0f) - 1.0f) * 0.5f);
    while ((q + 1) * (q + 2) <= t) ++q;
    while (q * (q + 1) > t) --q;
    if (t < (q + 1) * (q + 1)) {
        ti = 2 * q;
        tj = t - q * (q + 1);
    } else {
        ti = 2 * q + 1;
        tj = t - (q + 1) * (q + 1);
    }
}

struct TileRef {
    const UmmaProblem *p;
    int mi, ni;
};

// Tile index -> (problem, row tile, column tile). Batched launches look the
// problem up in the tile -> instance map the planning kernel wrote.
template <int BATCHED, int BN = 128>
__device__ __forceinline__ TileRef resolve(int t, const UmmaProblem *single, const UmmaProblem *probs,
                                           const int *prefix, const int *owner) {
    TileRef r;
    int local = t;
    if (BATCHED) {
        const int i = __ldg(owner + t);
        r.p = probs + i;
        local = t - __ldg(prefix + i);
    } else {
        r.p = single;
    }
    if (r.p->sym) {
        if constexpr (BN == 256) tri_tile_wide(local, r.mi, r.ni);
        else tri_tile(local, r.mi, r.ni);
    } else {
        r.mi = local / r.p->nt;
        r.ni = local - r.mi * r.p->nt;
    }
    return r;
}

__device__ __forceinline__ void prefetch_l2(const void *p) {
    asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

template <int P>
struct Products;
template <>
struct Products<1> {
    static constexpr int n = 1;
    __device__ static int a(int i) { return 0; }
    __device__ static int b(int i) { return 0; }
};
template <>
struct Products<2> {  // hi*hi + hi*lo + lo*hi
    static constexpr int n = 3;
    __device__ static int a(int i) { return i == 2 ? 1 : 0; }
    __device__ static int b(int i) { return i == 1 ? 1 : 0; }
};
template <>
struct Products<3> {  // the six products of order >= 2^-16
    static constexpr int n = 6;
    __device__ static int a(int i) { return (i == 2 || i == 3) ? 1 : (i == 5 ? 2 : 0); }
    __device__ static int b(int i) { return (i == 1 || i == 3) ? 1 : (i == 4 ? 2 : 0); }
};

// Tile configuration: BN columns per CTA tile, P split terms per operand.
//  shared memory per stage: A (P x 16 KiB) + B (P x BN/128 x 16 KiB), B term q
//  at q * BN/128 * 16 KiB with its two 128-row halves 16 KiB apart;
//  TMEM: NACC = 512 / BN accumulator buffers of BN columns.
// EPW: columns per epilogue warp (128, or 64 for symmetric outputs, whose
// element-wise epilogue is latency-bound and gains from twice the warps).
template <int P, int BN, int EPW = 128, int PAIR = 0>
struct Cfg {
    static constexpr int NEPI = 4 * BN / EPW;  // epilogue warps: 4 (one per TMEM lane quarter) per EPW columns
    // first epilogue warp: eight epilogue warps make two whole warpgroups
    // (warpgroup 0 = producer, MMA issuer and two idle warps), so that
    // setmaxnreg can move registers from warpgroup 0 to the epilogue, which
    // does not fit in the 168 registers a thread of a 12-warp CTA gets at
    // launch
    static constexpr int EPI0 = NEPI == 8 ? 4 : 2;
    static constexpr int NTHREADS = 32 * (EPI0 + NEPI);
    static constexpr bool REG_SPLIT = NEPI == 8;
    static constexpr int REG_LAUNCH = ((65536 / NTHREADS) & ~7) > 255 ? 255 : ((65536 / NTHREADS) & ~7);
    static constexpr int REG_LO = 64;
    static constexpr int REG_HI = ((REG_LAUNCH * NTHREADS - 128 * REG_LO) / (32 * NEPI)) & ~7;
    static constexpr int NACC = TMEM_COLS / BN;
    static constexpr int HALVES = BN / 128;
    static constexpr int A_BYTES = P * PK_TILE_BYTES;
    // CTA pairs: each CTA holds BN / 2 rows of every B term (BN * 64 bytes)
    static constexpr int BH_BYTES = BN * 64;
    static constexpr int B_BYTES = PAIR ? P * BH_BYTES : P * HALVES * PK_TILE_BYTES;
    static constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
    static constexpr int SCRATCH_BYTES = NEPI * 32 * 32 * 4;  // one 32 x 32 FP32 block per epilogue warp
    // 1 KiB of slack lets the kernel align the control block and stages to 1 KiB
    static constexpr int STAGES_RAW = (SMEM_BUDGET - 1024 - CTL_BYTES - SCRATCH_BYTES) / STAGE_BYTES;
    static constexpr int STAGES = STAGES_RAW > MAX_STAGES ? MAX_STAGES : STAGES_RAW;
    static constexpr int SMEM = 1024 + CTL_BYTES + STAGES * STAGE_BYTES + SCRATCH_BYTES;
    static constexpr int NLD = (BN == 128 && EPW == 128) ? 4 : 2;  // tcgen05.ld (x16) in flight per wait
    // a tile's FP32 block of the beta input fits in the stage memory; staged for
    // 256-wide tiles only (on 128-wide ones, loading it after the mainloop
    // measured slower than the epilogue's own loads)
    static constexpr bool DSMEM_OK = BN == 256 && BM * BN * 4 <= STAGES * STAGE_BYTES;
    // the packed image of a 256-wide tile (BN / 64 blocks of P terms) fits in the stage memory
    static constexpr bool POUT_OK = BN == 256 && (BN / PK_K) * P * PK_TILE_BYTES <= STAGES * STAGE_BYTES;
    static_assert((EPW == 64 || EPW == 128) && NEPI <= 8, "epilogue width");
    static_assert(NACC <= MAX_NACC && STAGES >= 2, "tile configuration does not fit");
    static_assert(!REG_SPLIT || (128 * REG_LO + 32 * NEPI * REG_HI <= REG_LAUNCH * NTHREADS && REG_HI <= 256 &&
                                 NTHREADS == 128 + 32 * NEPI),
                  "register split exceeds the launch allocation");
    // input stages of the pack stream that spare CTAs run in this shared memory
    static constexpr int SIDE_NOUT = SMEM - 1024 - 3 * P * PK_TILE_BYTES >= 4 * PS_IN_BYTES ? 3 : 2;
    static constexpr int SIDE_NS_RAW = (SMEM - 1024 - SIDE_NOUT * P * PK_TILE_BYTES) / PS_IN_BYTES;
    static constexpr int SIDE_NS = SIDE_NS_RAW > PS_MAX_STAGES ? PS_MAX_STAGES : SIDE_NS_RAW;
    // spare CTAs can pack the next contraction's operand: wide packing-epilogue kernels
    static constexpr bool SIDE_OK = BN == 256 && NTHREADS >= 256 && SIDE_NS >= 2;
};

// ---------------------------------------------------------------- epilogue of one 32 x 32 chunk
__device__ __forceinline__ void epi_chunk(const EpiParams &e, int row, int col0, const float *v) {
    if (row >= e.M) return;
    const bool full_cols = col0 + 31 < e.N;
    if (full_cols && (e.mode == EPI_GEMM || e.mode == EPI_STORE)) {
        float *c = e.C + (long long)row * e.ldc + col0;
        if (((reinterpret_cast<uintptr_t>(c) & 15) == 0)) {
#pragma unroll
            for (int q = 0; q < 32; q += 4) {
                float4 o;
                o.x = e.alpha * v[q + 0];
                o.y = e.alpha * v[q + 1];
                o.z = e.alpha * v[q + 2];
                o.w = e.alpha * v[q + 3];
                if (e.mode == EPI_GEMM && e.beta != 0.0f) {
                    float4 ci = *reinterpret_cast<const float4 *>(c + q);
                    o.x = fmaf(e.beta, ci.x, o.x);
                    o.y = fmaf(e.beta, ci.y, o.y);
                    o.z = fmaf(e.beta, ci.z, o.z);
                    o.w = fmaf(e.beta, ci.w, o.w);
                }
                *reinterpret_cast<float4 *>(c + q) = o;
            }
            return;
        }
    }
    if (full_cols && e.mode == EPI_EF) {
        const long long o = (long long)row * e.ld_ef + col0;
        if (((reinterpret_cast<uintptr_t>(e.E + o) & 15) == 0) && ((reinterpret_cast<uintptr_t>(e.F + o) & 15) == 0) &&
            (e.beta == 0.0f || (reinterpret_cast<uintptr_t>(e.D + o) & 15) == 0)) {
#pragma unroll
            for (int q = 0; q < 32; q += 4) {
                float4 ev = make_float4(v[q], v[q + 1], v[q + 2], v[q + 3]);
                *reinterpret_cast<float4 *>(e.E + o + q) = ev;
                float4 f;
                f.x = e.alpha * ev.x;
                f.y = e.alpha * ev.y;
                f.z = e.alpha * ev.z;
                f.w = e.alpha * ev.w;
                if (e.beta != 0.0f) {
                    float4 d = *reinterpret_cast<const float4 *>(e.D + o + q);
                    f.x = fmaf(e.beta, d.x, f.x);
                    f.y = fmaf(e.beta, d.y, f.y);
                    f.z = fmaf(e.beta, d.z, f.z);
                    f.w = fmaf(e.beta, d.w, f.w);
                }
                *reinterpret_cast<float4 *>(e.F + o + q) = f;
            }
            return;
        }
    }
#pragma unroll
    for (int q = 0; q < 32; ++q) epi_store(e, row, col0 + q, v[q]);
}

// ---------------------------------------------------------------- symmetric epilogue of one 32-column chunk
// Row `row`, columns col0..col0+31 of a lower-triangle tile. All loads the
// chunk needs (C for alpha*acc + beta*C, rs for correlation) are issued before
// any store, so a thread waits for one memory latency per chunk rather than
// one per element. The lower triangle is written along the row (float4 when
// aligned); the mirrored upper triangle is written column by column, where the
// 32 lanes (consecutive rows) make each store one contiguous 128-byte run.
__device__ __forceinline__ void epi_sym32(const EpiParams &e, int row, int col0, const float *v, bool diag) {
    if (row >= e.M) return;
    bool ok[32];
#pragma unroll
    for (int q = 0; q < 32; ++q) ok[q] = (col0 + q < e.N) && (!diag || col0 + q <= row);
    const bool dense = !diag && col0 + 31 < e.N;
    float val[32];
    if (e.sym_kind == SYM_CORR) {
        const float ri = e.rs[row];
        float rj[32];
        if (dense && ((reinterpret_cast<uintptr_t>(e.rs + col0) & 15) == 0)) {
#pragma unroll
            for (int q = 0; q < 32; q += 4) {
                float4 t = *reinterpret_cast<const float4 *>(e.rs + col0 + q);
                rj[q] = t.x;
                rj[q + 1] = t.y;
                rj[q + 2] = t.z;
                rj[q + 3] = t.w;
            }
        } else {
#pragma unroll
            for (int q = 0; q < 32; ++q) rj[q] = ok[q] ? e.rs[col0 + q] : 0.0f;
        }
#pragma unroll
        for (int q = 0; q < 32; ++q) val[q] = (col0 + q == row) ? 1.0f : v[q] * ri * rj[q];
    } else if (e.sym_kind == SYM_SCALE || e.beta == 0.0f) {
#pragma unroll
        for (int q = 0; q < 32; ++q) val[q] = e.alpha * v[q];
    } else {
        float c[32];
        if (e.fill == LN_FILL_UPPER) {
#pragma unroll
            for (int q = 0; q < 32; ++q) c[q] = ok[q] ? e.C[(long long)(col0 + q) * e.ldc + row] : 0.0f;
        } else {
            const float *src = e.C + (long long)row * e.ldc + col0;
            if (dense && ((reinterpret_cast<uintptr_t>(src) & 15) == 0)) {
#pragma unroll
                for (int q = 0; q < 32; q += 4) {
                    float4 t = *reinterpret_cast<const float4 *>(src + q);
                    c[q] = t.x;
                    c[q + 1] = t.y;
                    c[q + 2] = t.z;
                    c[q + 3] = t.w;
                }
            } else {
#pragma unroll
                for (int q = 0; q < 32; ++q) c[q] = ok[q] ? src[q] : 0.0f;
            }
        }
#pragma unroll
        for (int q = 0; q < 32; ++q) val[q] = fmaf(e.beta, c[q], e.alpha * v[q]);
    }
    const bool write_lower = !(e.sym_kind == SYM_AXPBY && e.fill == LN_FILL_UPPER);
    const bool write_upper = !(e.sym_kind == SYM_AXPBY && e.fill == LN_FILL_LOWER);
    if (write_lower) {
        float *dst = e.C + (long long)row * e.ldc + col0;
        if (dense && ((reinterpret_cast<uintptr_t>(dst) & 15) == 0)) {
#pragma unroll
            for (int q = 0; q < 32; q += 4)
                *reinterpret_cast<float4 *>(dst + q) = make_float4(val[q], val[q + 1], val[q + 2], val[q + 3]);
        } else {
#pragma unroll
            for (int q = 0; q < 32; ++q)
                if (ok[q]) dst[q] = val[q];
        }
    }
    if (write_upper) {
#pragma unroll
        for (int q = 0; q < 32; ++q)
            if (ok[q] && (col0 + q != row || !write_lower)) e.C[(long long)(col0 + q) * e.ldc + row] = val[q];
    }
}

// Epilogue kinds, a template parameter so that each instantiation carries only
// the store code it needs.
enum : int { EK_PACK = 0, EK_EF = 1, EK_GEMM = 2, EK_SYM = 3 };

// ---------------------------------------------------------------- warp-cooperative 32 x 32 block epilogue
// The accumulator arrives with one output row per lane (TMEM lane = row). Row-
// major global accesses from that layout send 32 separate requests per
// instruction, so stores would be limited by the memory request rate. The warp
// therefore stages its 32 x 32 block in shared memory (16-byte chunks
// XOR-swizzled by row, conflict-free) and reads it back so that lanes
// 8r'..8r'+7 hold one row's 32 consecutive values: with aligned data every
// LDG.128 / STG.128 covers four whole 128-byte row segments. Mirrored
// (transposed) stores of symmetric outputs are contiguous across lanes in the
// row-per-lane layout and are written from it. Ragged edges, diagonal blocks of
// symmetric outputs (only i >= j is produced) and unaligned data are handled
// element by element within the same scheme.
__device__ __forceinline__ bool aligned16(const void *p, long long ld) {
    return ((reinterpret_cast<uintptr_t>(p) & 15) == 0) && ((ld & 3) == 0);
}

template <int EK>
__device__ __forceinline__ bool block_epilogue(const EpiParams &e, float *sc, int wrow0, int c0, const float *v,
                                               int lane) {
    if (wrow0 + 31 >= e.M || c0 + 31 >= e.N) return false;
    if (EK == EK_EF) {
        if (!aligned16(e.E, e.ld_ef) || !aligned16(e.F, e.ld_ef) || (e.beta != 0.0f && !aligned16(e.D, e.ld_ef)))
            return false;
    } else if (!aligned16(e.C, e.ldc)) {
        return false;
    }
    // stage: lane = row, 8 chunks of 4 values, chunk k of row r at (k ^ (r & 7))
#pragma unroll
    for (int k = 0; k < 8; ++k)
        *reinterpret_cast<float4 *>(sc + lane * 32 + ((k ^ (lane & 7)) << 2)) =
            make_float4(v[4 * k], v[4 * k + 1], v[4 * k + 2], v[4 * k + 3]);
    __syncwarp();
    const int ch = lane & 7;  // this lane's 16-byte chunk of a row
    const int col = c0 + ch * 4;
    const bool need_in = (EK == EK_GEMM || EK == EK_EF) && e.beta != 0.0f;
    const float *src = EK == EK_EF ? e.D : e.C;
    const long long lds = EK == EK_EF ? e.ld_ef : e.ldc;
    // every load of the block (C or D) first, one latency per block; E does not
    // wait for them
    float4 in[8];
    if (need_in) {
#pragma unroll
        for (int h = 0; h < 8; ++h) {
            const int r = h * 4 + (lane >> 3);
            in[h] = *reinterpret_cast<const float4 *>(src + (long long)(wrow0 + r) * lds + col);
        }
    }
    if (EK == EK_EF) {
#pragma unroll
        for (int h = 0; h < 8; ++h) {
            const int r = h * 4 + (lane >> 3);
            *reinterpret_cast<float4 *>(e.E + (long long)(wrow0 + r) * e.ld_ef + col) =
                *reinterpret_cast<const float4 *>(sc + r * 32 + ((ch ^ (r & 7)) << 2));
        }
    }
#pragma unroll
    for (int h = 0; h < 8; ++h) {
        const int r = h * 4 + (lane >> 3);
        const float4 o = *reinterpret_cast<const float4 *>(sc + r * 32 + ((ch ^ (r & 7)) << 2));
        float4 f = make_float4(e.alpha * o.x, e.alpha * o.y, e.alpha * o.z, e.alpha * o.w);
        if (need_in) {
            f.x = fmaf(e.beta, in[h].x, f.x);
            f.y = fmaf(e.beta, in[h].y, f.y);
            f.z = fmaf(e.beta, in[h].z, f.z);
            f.w = fmaf(e.beta, in[h].w, f.w);
        }
        float *dst = EK == EK_EF ? e.F + (long long)(wrow0 + r) * e.ld_ef + col : e.C + (long long)(wrow0 + r) * e.ldc + col;
        *reinterpret_cast<float4 *>(dst) = f;
    }
    __syncwarp();
    return true;
}

// The same block layout for a tile whose beta input sits in shared memory
// (SchedSlot::dsmem): E alone, then F = alpha * acc + beta * D (EK_EF) or
// C = alpha * acc + beta * C (EK_GEMM) with D or C read from `ds` (the warp's
// rows of the staged block, row pitch `pitch` floats). The tile is wholly
// inside the output and its rows 16-byte aligned (checked when it was staged).
__device__ __forceinline__ void block_stage(float *sc, const float *v, int lane) {
#pragma unroll
    for (int k = 0; k < 8; ++k)
        *reinterpret_cast<float4 *>(sc + lane * 32 + ((k ^ (lane & 7)) << 2)) =
            make_float4(v[4 * k], v[4 * k + 1], v[4 * k + 2], v[4 * k + 3]);
    __syncwarp();
}

__device__ __forceinline__ void block_store_e(const EpiParams &e, float *sc, int wrow0, int c0, const float *v,
                                              int lane) {
    block_stage(sc, v, lane);
    const int ch = lane & 7;
#pragma unroll
    for (int h = 0; h < 8; ++h) {
        const int r = h * 4 + (lane >> 3);
        *reinterpret_cast<float4 *>(e.E + (long long)(wrow0 + r) * e.ld_ef + c0 + ch * 4) =
            *reinterpret_cast<const float4 *>(sc + r * 32 + ((ch ^ (r & 7)) << 2));
    }
    __syncwarp();
}

template <int EK>
__device__ __forceinline__ void block_store_f(const EpiParams &e, float *sc, int wrow0, int c0, const float *v,
                                              int lane, const float *ds, int pitch) {
    block_stage(sc, v, lane);
    const int ch = lane & 7;
#pragma unroll
    for (int h = 0; h < 8; ++h) {
        const int r = h * 4 + (lane >> 3);
        const float4 o = *reinterpret_cast<const float4 *>(sc + r * 32 + ((ch ^ (r & 7)) << 2));
        const float4 d = *reinterpret_cast<const float4 *>(ds + (size_t)r * pitch + ch * 4);
        float4 f;
        f.x = fmaf(e.beta, d.x, e.alpha * o.x);
        f.y = fmaf(e.beta, d.y, e.alpha * o.y);
        f.z = fmaf(e.beta, d.z, e.alpha * o.z);
        f.w = fmaf(e.beta, d.w, e.alpha * o.w);
        float *dst = EK == EK_EF ? e.F + (long long)(wrow0 + r) * e.ld_ef + c0 + ch * 4
                                 : e.C + (long long)(wrow0 + r) * e.ldc + c0 + ch * 4;
        *reinterpret_cast<float4 *>(dst) = f;
    }
    __syncwarp();
}

// ---------------------------------------------------------------- the kernel
// Grid: tile_ctas CTAs take output tiles (static stride tile_ctas, or the
// queue); CTAs from tile_ctas on (only launched for single problems with the
// packing epilogue, see Cfg::SIDE_OK) run the pack stream over `side`, the
// operand of the next contraction, on SMs that have no output tile.
// The MMAs of one k tile (every split product, K / 16 steps each) into the
// accumulator d; `first` starts the accumulation (no add to d's old value).
template <class C, class PR, int BN, bool PAIR, bool TF>
__device__ __forceinline__ void issue_ktile(uint32_t d, uint32_t a0, uint32_t b0, bool first) {
#pragma unroll
    for (int pr = 0; pr < PR::n; ++pr) {
#pragma unroll
        for (int ks = 0; ks < PK_K / 16; ++ks) {
            const uint64_t ad = sw128_desc(a0 + PR::a(pr) * PK_TILE_BYTES + ks * 32);
            const uint32_t acc_in = (!first || pr || ks) ? 1u : 0u;
            if constexpr (PAIR) {
                const uint64_t bd = sw128_desc(b0 + PR::b(pr) * C::BH_BYTES + ks * 32);
                if constexpr (TF) umma_tf32_pair<BN>(d, ad, bd, acc_in);
                else umma_bf16_pair<BN>(d, ad, bd, acc_in);
            } else {
                const uint64_t bd = sw128_desc(b0 + PR::b(pr) * C::HALVES * PK_TILE_BYTES + ks * 32);
                if constexpr (TF) umma_tf32<BN>(d, ad, bd, acc_in);
                else umma_bf16<BN>(d, ad, bd, acc_in);
            }
        }
    }
}

// Columns per epilogue warp: 64 for 128-wide symmetric tiles (their
// element-wise epilogue is latency-bound and gains from twice the warps), 128
// otherwise (eight warps at most).
template <int EK, int BN>
constexpr int epi_width() { return EK == EK_SYM && BN == 128 ? 64 : 128; }

// TF: TF32 operands (kind::tf32, 32-K tiles, TF32 packing epilogue). A
// template parameter so that the BF16 instantiations carry no TF32 code (a
// runtime choice enlarged the issue loop and slowed the BF16 kernels).
template <int P, int BN, int BATCHED, int EK, int PAIR = 0, int TF = 0>
__global__ __launch_bounds__(Cfg<P, BN, epi_width<EK, BN>(), PAIR>::NTHREADS, 1) void k_umma(const __grid_constant__ UmmaProblem single,
                                                                  const UmmaProblem *__restrict__ probs,
                                                                  const int *__restrict__ prefix,
                                                                  const int *__restrict__ owner, int total_tiles,
                                                                  int *queue, const __grid_constant__ PackMulti side,
                                                                  int tile_ctas) {
    using C = Cfg<P, BN, epi_width<EK, BN>(), PAIR>;
    constexpr int EPW = epi_width<EK, BN>();
    using PR = Products<P>;
    static_assert(!PAIR || !BATCHED, "CTA pairs take single problems");
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    // 1024-byte alignment of the stage area is required by the 128-byte swizzle.
    const uint32_t raw = saddr(smem_raw);
    const uint32_t pad = ((raw + 1023u) & ~1023u) - raw;
    if constexpr (EK == EK_PACK && !BATCHED && C::SIDE_OK && !TF) {
        if ((int)blockIdx.x >= tile_ctas) {
            pdl_wait();
            pdl_trigger();
            if (threadIdx.x < 256)
                pack_stream<P, 256, false>(side, (int)blockIdx.x - tile_ctas, (int)gridDim.x - tile_ctas,
                                           smem_raw + pad, C::SIDE_NS, C::SIDE_NOUT);
            return;
        }
    }
    Ctl *ctl = reinterpret_cast<Ctl *>(smem_raw + pad);
    const uint32_t stage0 = raw + pad + CTL_BYTES;
    float *const scratch = reinterpret_cast<float *>(smem_raw + pad + CTL_BYTES + C::STAGES * C::STAGE_BYTES);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    // CTA pairs (PAIR): the leader (rank 0) issues the pair's MMAs; its tensor
    // memory buffers are released by both CTAs' epilogue warps
    constexpr bool pair = PAIR != 0;
    const int rank = pair ? (int)cluster_rank() : 0;
    if (threadIdx.x == 0) {
        for (int s = 0; s < C::STAGES; ++s) {
            mbar_init(&ctl->full[s], 1);
            mbar_init(&ctl->empty[s], 1);
            mbar_init(&ctl->pfull[s], 1);
        }
        for (int b = 0; b < C::NACC; ++b) {
            mbar_init(&ctl->tfull[b], 1);
            mbar_init(&ctl->tempty[b], pair ? 2 * C::NEPI : C::NEPI);
        }
        for (int s = 0; s < SCHED; ++s) {
            mbar_init(&ctl->sfull[s], 1);
            mbar_init(&ctl->sempty[s], 1 + C::NEPI);
        }
        mbar_init(&ctl->drain, 1);
        mbar_init(&ctl->dfull, 1);
        ctl->abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 1) {
        if constexpr (pair) {
            // allocated collectively by one warp of each CTA of the pair: the same
            // columns in both CTAs' tensor memory
            asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                             saddr(&ctl->tmem_base)),
                         "r"(TMEM_COLS)
                         : "memory");
            asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
        } else {
            asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                             saddr(&ctl->tmem_base)),
                         "r"(TMEM_COLS)
                         : "memory");
            asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
        }
    }
    tc_fence_before();
    __syncthreads();
    // the peer copies into this CTA's stages and arrives on its barriers only
    // after both CTAs have initialised theirs
    if (pair) cluster_sync();
    tc_fence_after();
    const uint32_t tmem = ctl->tmem_base;
    // everything above touched only shared memory and TMEM: with a programmatic
    // launch it overlapped the previous kernel; global memory only from here on
    pdl_wait();
    pdl_trigger();
    // Each warpgroup changes its register count at the top of its own branch
    // (the role code is then allocated under that count); the host checked that
    // the launch allocation covers the split.
    if (warp < C::EPI0) {
    if constexpr (C::REG_SPLIT) asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(C::REG_LO));
    if (warp == 0) {
        // ------------------------------------------------------------ producer
        if (lane == 0) {
            int it = 0, sidx = 0;
            bool dsm_issued = false;
            int next = pair ? (int)blockIdx.x >> 1 : (int)blockIdx.x;
            const int stride = pair ? tile_ctas >> 1 : tile_ctas;
            const bool sk = !BATCHED && single.streamk;
            const int sk_ktot = single.nseg * single.kt;
            const long long sk_units = (long long)total_tiles * sk_ktot;
            long long sk_u = sk ? sk_start(blockIdx.x, sk_units, tile_ctas) : 0;
            const long long sk_end = sk ? sk_start(blockIdx.x + 1, sk_units, tile_ctas) : 0;
            for (;;) {
                int t, qa = 0, qb = 0;
                if (sk) {
                    if (sk_u < sk_end) {
                        t = (int)(sk_u / sk_ktot);
                        qa = (int)(sk_u - (long long)t * sk_ktot);
                        qb = (int)(sk_end - sk_u < sk_ktot - qa ? qa + (sk_end - sk_u) : sk_ktot);
                        sk_u += qb - qa;
                    } else {
                        t = -1;
                    }
                } else if (queue) {
                    t = atomicAdd(queue, 1);
                } else {
                    t = next;
                    next += stride;
                }
                if (t >= total_tiles) t = -1;
                const int s = sidx % SCHED;
                if (!wait_phase(ctl, &ctl->sempty[s], ((sidx / SCHED) & 1) ^ 1, ERR_PRODUCER, true, 64)) break;
                SchedSlot &sl = ctl->slot[s];
                TileRef tr{&single, 0, 0};
                const int ksplit = (!BATCHED && !sk && single.ksplit > 1) ? single.ksplit : 1;
                sl.ghost = 0;
                if (t >= 0 && pair) {
                    pair_tile(single, t, rank, tr.mi, tr.ni, sl.ghost);
                    sl.prob = single;
                    sl.mi = tr.mi;
                    sl.ni = tr.ni;
                    sl.ks = 0;
                    slice_range(single, 0, qa, qb);
                    sl.qa = qa;
                    sl.qb = qb;
                } else if (t >= 0) {
                    tr = resolve<BATCHED, BN>(t / ksplit, &single, probs, prefix, owner);
                    sl.prob = *tr.p;  // roles read the problem from shared memory, not from registers
                    sl.mi = tr.mi;
                    sl.ni = tr.ni;
                    sl.ks = t - (t / ksplit) * ksplit;
                    if (!sk) slice_range(*tr.p, sl.ks, qa, qb);
                    sl.qa = qa;
                    sl.qb = qb;
                }
                sl.dsmem = 0;
                if constexpr (EK == EK_PACK && !BATCHED && !TF && C::POUT_OK) {
                    // the last tile of a statically scheduled CTA: no later copy reuses the stages
                    sl.dsmem = single.stage_out && t >= 0 && !queue && !sk && ksplit <= 1 && next >= total_tiles &&
                               !sl.ghost;
                }
                if constexpr ((EK == EK_EF || EK == EK_GEMM) && !BATCHED && C::DSMEM_OK) {
                    // the last tile of a statically scheduled CTA, wholly inside an aligned output
                    const EpiParams &e = single.epi;
                    const float *src = EK == EK_EF ? e.D : e.C;
                    const long long ld = EK == EK_EF ? e.ld_ef : e.ldc;
                    sl.dsmem = single.stage_beta && t >= 0 && !queue && !sk && ksplit <= 1 && next >= total_tiles &&
                               !sl.ghost &&
                               e.beta != 0.0f && tr.mi * BM + BM <= e.M && tr.ni * BN + BN <= e.N && aligned16(src, ld);
                }
                sl.t = t;
                mbar_arrive(&ctl->sfull[s]);
                ++sidx;
                if (t < 0) break;
                const UmmaProblem &pb = *tr.p;
                if (pb.inject_timeout) break;  // nothing arrives on full[]: the MMA wait runs out
                const bool ghost = sl.ghost;
                bool ok = true;
                {
                    for (int q = qa; q < qb; ++q) {
                        const int sg = q / pb.kt, kt = q - sg * pb.kt;
                        const char *xb = pb.seg[sg].X + (size_t)tr.mi * pb.x_kt * C::A_BYTES;
                        const int st = it % C::STAGES;
                        if (!wait_phase(ctl, &ctl->empty[st], ((it / C::STAGES) & 1) ^ 1, ERR_PRODUCER, true, 32)) {
                            ok = false;
                            break;
                        }
                        const uint32_t dst = stage0 + st * C::STAGE_BYTES;
                        if constexpr (pair) {
                            // own rows of A; this CTA's BN / 2 rows of every B term
                            mbar_expect_tx(&ctl->full[st], ghost ? C::B_BYTES : C::STAGE_BYTES);
                            if (!ghost) bulk_g2s(dst, xb + (size_t)kt * C::A_BYTES, C::A_BYTES, &ctl->full[st]);
                            const int brt = BN == 256 ? tr.ni * 2 + rank : tr.ni;  // packed 128-row tile of B
                            const uint32_t boff = BN == 256 ? 0u : (uint32_t)rank * C::BH_BYTES;
                            const char *yb = pb.seg[sg].Y + ((size_t)brt * pb.y_kt + kt) * C::A_BYTES + boff;
#pragma unroll
                            for (int q = 0; q < P; ++q)
                                bulk_g2s(dst + C::A_BYTES + q * C::BH_BYTES, yb + q * PK_TILE_BYTES, C::BH_BYTES,
                                         &ctl->full[st]);
                            ++it;
                            continue;
                        }
                        mbar_expect_tx(&ctl->full[st], C::STAGE_BYTES);
                        bulk_g2s(dst, xb + (size_t)kt * C::A_BYTES, C::A_BYTES, &ctl->full[st]);
                        if (C::HALVES == 1) {
                            const char *yb = pb.seg[sg].Y + ((size_t)tr.ni * pb.y_kt + kt) * C::A_BYTES;
                            bulk_g2s(dst + C::A_BYTES, yb, C::A_BYTES, &ctl->full[st]);
                        } else {
#pragma unroll
                            for (int h = 0; h < C::HALVES; ++h) {
                                const char *yb =
                                    pb.seg[sg].Y + ((size_t)(tr.ni * C::HALVES + h) * pb.y_kt + kt) * C::A_BYTES;
#pragma unroll
                                for (int q = 0; q < P; ++q)
                                    bulk_g2s(dst + C::A_BYTES + (q * C::HALVES + h) * PK_TILE_BYTES,
                                             yb + q * PK_TILE_BYTES, PK_TILE_BYTES, &ctl->full[st]);
                            }
                        }
                        ++it;
                    }
                }
                if (!ok) break;
                if constexpr ((EK == EK_EF || EK == EK_GEMM) && !BATCHED && C::DSMEM_OK) {
                    if (sl.dsmem) {
                        // every stage has been read by the MMAs (its empty phase completed):
                        // the stage memory now takes the tile's rows of D (or C)
                        for (int j = (it > C::STAGES ? it - C::STAGES : 0); j < it && ok; ++j)
                            ok = wait_phase(ctl, &ctl->empty[j % C::STAGES], (j / C::STAGES) & 1, ERR_PRODUCER, true,
                                            32);
                        if (!ok) break;
                        const EpiParams &e = pb.epi;
                        const float *src = EK == EK_EF ? e.D : e.C;
                        const long long ld = EK == EK_EF ? e.ld_ef : e.ldc;
                        const float *row0 = src + (long long)tr.mi * BM * ld + (long long)tr.ni * BN;
                        mbar_expect_tx(&ctl->dfull, BM * BN * 4);
                        for (int r = 0; r < BM; ++r) bulk_g2s(stage0 + r * BN * 4, row0 + r * ld, BN * 4, &ctl->dfull);
                        dsm_issued = true;
                    }
                }
            }
            // wait for this CTA's copies still in flight
            for (int j = (it > C::STAGES ? it - C::STAGES : 0); j < it; ++j)
                wait_phase(ctl, &ctl->full[j % C::STAGES], (j / C::STAGES) & 1, ERR_DRAIN, false, 256);
            if (dsm_issued) wait_phase(ctl, &ctl->dfull, 0, ERR_DRAIN, false, 256);
        }
    } else if (warp == 1) {
        // ------------------------------------------------------------ MMA issuer
        if (lane == 0) {
            int it = 0, sidx = 0, acc = 0;
            for (;;) {
                const int s = sidx % SCHED;
                if (!wait_phase(ctl, &ctl->sfull[s], (sidx / SCHED) & 1, ERR_MMA)) break;
                const SchedSlot &sl = ctl->slot[s];
                ++sidx;
                if (sl.t < 0) break;
                const UmmaProblem &pb = sl.prob;
                const int qa = sl.qa, qb = sl.qb;
                const int ck = pb.chunk_kt > 0 ? pb.chunk_kt : (qb - qa > 0 ? qb - qa : 1);
                bool ok = true;
                if (pair && rank != 0) {
                    // the peer of a pair issues no MMA: it tells the leader when each
                    // of its stages is full
                    for (int q = qa; q < qb; ++q) {
                        const int st = it % C::STAGES;
                        if (!wait_phase(ctl, &ctl->full[st], (it / C::STAGES) & 1, ERR_MMA)) {
                            ok = false;
                            break;
                        }
                        mbar_arrive_remote(&ctl->pfull[st], 0);
                        ++it;
                    }
                    if (!ok) break;
                    mbar_arrive(&ctl->sempty[s]);
                    continue;
                }
                // one TMEM accumulator buffer per chunk of ck k tiles (pairs: the
                // leader computes both CTAs' tiles, ghosts included)
                for (int q0 = qa; q0 < qb && ok; q0 += ck) {
                    const int b = acc % C::NACC;
                    if (!(pair ? wait_phase_cl(ctl, &ctl->tempty[b], ((acc / C::NACC) & 1) ^ 1, ERR_MMA)
                               : wait_phase(ctl, &ctl->tempty[b], ((acc / C::NACC) & 1) ^ 1, ERR_MMA))) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t d = tmem + (uint32_t)(b * BN);
                    const int q1 = q0 + ck < qb ? q0 + ck : qb;
                    for (int q = q0; q < q1; ++q) {
                        const int st = it % C::STAGES;
                        if (!wait_phase(ctl, &ctl->full[st], (it / C::STAGES) & 1, ERR_MMA) ||
                            (pair && !wait_phase_cl(ctl, &ctl->pfull[st], (it / C::STAGES) & 1, ERR_MMA))) {
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                        const uint32_t a0 = stage0 + st * C::STAGE_BYTES;
                        const uint32_t b0 = a0 + C::A_BYTES;
                        issue_ktile<C, PR, BN, pair, TF != 0>(d, a0, b0, q == q0);
                        if constexpr (pair) umma_commit_pair_mc(&ctl->empty[st]);
                        else umma_commit(&ctl->empty[st]);
                        ++it;
                    }
                    if (!ok) break;
                    if constexpr (pair) umma_commit_pair_mc(&ctl->tfull[b]);
                    else umma_commit(&ctl->tfull[b]);
                    ++acc;
                }
                if (!ok) break;
                mbar_arrive(&ctl->sempty[s]);
            }
            // every MMA this thread issued has completed before TMEM is freed
            if constexpr (pair) {
                if (rank == 0) {
                    umma_commit_pair(&ctl->drain);
                    wait_phase(ctl, &ctl->drain, 0, ERR_DRAIN, false, 256);
                }
            } else {
                umma_commit(&ctl->drain);
                wait_phase(ctl, &ctl->drain, 0, ERR_DRAIN, false, 256);
            }
        }
    }
    } else {
        if constexpr (C::REG_SPLIT) asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;" ::"n"(C::REG_HI));
        // ------------------------------------------------------------ epilogue warps
        const int quarter = warp & 3;             // TMEM lanes (= tile rows) this warp may access
        const int half = (warp - C::EPI0) >> 2;  // which EPW of the tile's BN columns
        const int col_base = half * EPW;
        int sidx = 0, acc = 0;
        for (;;) {
            const int s = sidx % SCHED;
            bool ok = wait_phase(ctl, &ctl->sfull[s], (sidx / SCHED) & 1, ERR_EPILOGUE, true, 128);
            if (!__all_sync(0xffffffffu, ok)) break;
            const SchedSlot &sl = ctl->slot[s];
            ++sidx;
            if (sl.t < 0) break;
            if (sl.ghost) {
                // pairs: nothing of this tile is stored; the leader still computed it
                // into this CTA's tensor memory, so each chunk is waited for and
                // released as usual
                const int gck = sl.prob.chunk_kt > 0 ? sl.prob.chunk_kt : (sl.qb - sl.qa > 0 ? sl.qb - sl.qa : 1);
                const int gnch = (sl.qb - sl.qa + gck - 1) / gck;
                for (int c = 0; c < gnch && ok; ++c) {
                    const int b = acc % C::NACC;
                    ok = wait_phase(ctl, &ctl->tfull[b], (acc / C::NACC) & 1, ERR_EPILOGUE, true, 128);
                    ok = __all_sync(0xffffffffu, ok);
                    if (!ok) break;
                    tc_fence_after();
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive_remote(&ctl->tempty[b], 0);
                    ++acc;
                }
                if (!ok) break;
                __syncwarp();
                if (lane == 0) mbar_arrive(&ctl->sempty[s]);
                continue;
            }
            const TileRef tr{nullptr, sl.mi, sl.ni};
            const UmmaProblem &pb = sl.prob;
            const int qa = sl.qa, qb = sl.qb;
            const int ck = pb.chunk_kt > 0 ? pb.chunk_kt : (qb - qa > 0 ? qb - qa : 1);
            const int nch = (qb - qa + ck - 1) / ck;
            {
                // bring the values the final epilogue reads (C or D) towards L2
                // while the tile's MMAs run (prefetching the lines it only
                // writes as well was measured slower: the extra HBM reads cost
                // more than the write misses they avoid)
                const EpiParams &pe = pb.epi;
                const int prow = tr.mi * BM + quarter * 32 + lane;
                const int pcol = tr.ni * BN + col_base;
                if (EK != EK_PACK && pe.beta != 0.0f && prow < pe.M && pcol < pe.N) {
                    if (pe.mode == EPI_GEMM || (pe.mode == EPI_SYM && pe.sym_kind == SYM_AXPBY && pe.fill != LN_FILL_UPPER)) {
                        const float *r0 = pe.C + (long long)prow * pe.ldc + pcol;
#pragma unroll
                        for (int q = 0; q < EPW; q += 32)
                            if (pcol + q < pe.N) prefetch_l2(r0 + q);
                    } else if (pe.mode == EPI_EF) {
                        const float *r0 = pe.D + (long long)prow * pe.ld_ef + pcol;
#pragma unroll
                        for (int q = 0; q < EPW; q += 32)
                            if (pcol + q < pe.N) prefetch_l2(r0 + q);
                    } else if (pe.mode == EPI_SYM && pe.sym_kind == SYM_AXPBY) {
                        const int wrow = tr.mi * BM + quarter * 32;  // the warp's first row (< M here)
#pragma unroll
                        for (int q = 0; q < EPW / 32; ++q) {
                            const int j = pcol + lane * (EPW / 32) + q;
                            if (j < pe.N) prefetch_l2(pe.C + (long long)j * pe.ldc + wrow);
                        }
                    }
                }
            }
            // running FP32 sum of this thread's EPW outputs: each TMEM chunk is
            // added here with round-to-nearest adds
            float sum[EPW];
#pragma unroll
            for (int q = 0; q < EPW; ++q) sum[q] = 0.0f;
            for (int c = 0; c < nch && ok; ++c) {
                const int b = acc % C::NACC;
                ok = wait_phase(ctl, &ctl->tfull[b], (acc / C::NACC) & 1, ERR_EPILOGUE, true, 128);
                ok = __all_sync(0xffffffffu, ok);
                if (!ok) break;
                tc_fence_after();
#pragma unroll
                for (int g0 = 0; g0 < EPW / 16; g0 += C::NLD) {
                    uint32_t r[C::NLD][16];
#pragma unroll
                    for (int j = 0; j < C::NLD; ++j)
                        tmem_ld16_async(tmem + ((uint32_t)(quarter * 32) << 16) +
                                            (uint32_t)(b * BN + col_base + (g0 + j) * 16),
                                        r[j]);
                    tmem_wait();
#pragma unroll
                    for (int j = 0; j < C::NLD; ++j) {
                        tmem_after_wait(r[j]);
#pragma unroll
                        for (int q = 0; q < 16; ++q) sum[(g0 + j) * 16 + q] += __uint_as_float(r[j][q]);
                    }
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) {
                    if constexpr (pair) mbar_arrive_remote(&ctl->tempty[b], 0);  // the leader's buffer
                    else mbar_arrive(&ctl->tempty[b]);
                }
                ++acc;
            }
            if (!ok) break;
            bool last = true;
            if (!BATCHED && pb.streamk && !(qa == 0 && qb == pb.nseg * pb.kt)) {
                // stream-K hand-off. A segment that starts inside the tile (qa > 0)
                // is the first of its CTA's range: it publishes its FP32 sums and
                // takes no epilogue. The segment with k tile 0 comes last in its
                // CTA's range; it adds the later segments' sums, CTA by CTA (k
                // order, so the result does not depend on timing), and runs the
                // tile's epilogue.
                const int ew = warp - C::EPI0;
                constexpr int SLAB = EPW * 32;  // one warp's partial sums
                if (qa > 0) {
                    float *const mine = pb.skpart + ((size_t)blockIdx.x * C::NEPI + ew) * SLAB;
#pragma unroll
                    for (int q = 0; q < EPW; q += 4)
                        *reinterpret_cast<float4 *>(mine + q * 32 + lane * 4) =
                            make_float4(sum[q], sum[q + 1], sum[q + 2], sum[q + 3]);
                    __threadfence();
                    __syncwarp();
                    if (lane == 0) atomicExch(pb.skflag + (size_t)blockIdx.x * C::NEPI + ew, 1);
                    last = false;
                } else {
                    const int ktot = pb.nseg * pb.kt;
                    const long long units = (long long)total_tiles * ktot;
                    const long long tile_end = (long long)(sl.t + 1) * ktot;
                    for (int c2 = blockIdx.x + 1; c2 < tile_ctas && sk_start(c2, units, tile_ctas) < tile_end && ok;
                         ++c2) {
                        const int *f = pb.skflag + (size_t)c2 * C::NEPI + ew;
                        if (lane == 0) {
                            const unsigned long long t0 = gtimer();
                            for (uint32_t n = 0; !ld_acquire(f); ++n) {
                                __nanosleep(64);
                                if ((n & 15) == 15) {
                                    if (ctl->abort) {
                                        ok = false;
                                        break;
                                    }
                                    if (gtimer() - t0 > WAIT_NS) {
                                        ctl->abort = 1;
                                        atomicOr(&g_umma_error, ERR_EPILOGUE);
                                        ok = false;
                                        break;
                                    }
                                }
                            }
                        }
                        ok = __shfl_sync(0xffffffffu, ok, 0);
                        if (!ok) break;
                        __threadfence();
                        const float *src = pb.skpart + ((size_t)c2 * C::NEPI + ew) * SLAB + lane * 4;
#pragma unroll
                        for (int q = 0; q < EPW; q += 4) {
                            const float4 v = __ldcg(reinterpret_cast<const float4 *>(src + q * 32));
                            sum[q] += v.x;
                            sum[q + 1] += v.y;
                            sum[q + 2] += v.z;
                            sum[q + 3] += v.w;
                        }
                    }
                    if (!ok) break;
                }
            } else if (!BATCHED && pb.ksplit > 1) {
                // split-K hand-off: publish this slice's sums, count the arrival;
                // the last slice to arrive adds all slices in slice order
                const int ew = warp - C::EPI0;
                const long long tile = sl.t / pb.ksplit;
                constexpr int SLAB = EPW * 32;  // one warp's partial sums
                float *const base = pb.kpart + (size_t)(tile * pb.ksplit) * C::NEPI * SLAB + (size_t)ew * SLAB;
                float *const mine = base + (size_t)sl.ks * C::NEPI * SLAB;
#pragma unroll
                for (int q = 0; q < EPW; q += 4)
                    *reinterpret_cast<float4 *>(mine + q * 32 + lane * 4) =
                        make_float4(sum[q], sum[q + 1], sum[q + 2], sum[q + 3]);
                __threadfence();
                __syncwarp();
                int old = 0;
                if (lane == 0) old = atomicAdd(pb.kcnt + tile * C::NEPI + ew, 1);
                old = __shfl_sync(0xffffffffu, old, 0);
                last = old == pb.ksplit - 1;
                if (last) {
                    // every slice, this one included, is in kpart: add them in slice order
                    __threadfence();
                    const float *src = base + lane * 4;
#pragma unroll
                    for (int q = 0; q < EPW; q += 4) {
                        float4 a = __ldcg(reinterpret_cast<const float4 *>(src + q * 32));
                        for (int k = 1; k < pb.ksplit; ++k) {
                            const float4 v =
                                __ldcg(reinterpret_cast<const float4 *>(src + (size_t)k * C::NEPI * SLAB + q * 32));
                            a.x += v.x;
                            a.y += v.y;
                            a.z += v.z;
                            a.w += v.w;
                        }
                        sum[q] = a.x;
                        sum[q + 1] = a.y;
                        sum[q + 2] = a.z;
                        sum[q + 3] = a.w;
                    }
                }
            }
            const int rloc = quarter * 32 + lane;
            const int col0 = tr.ni * BN + col_base;
            const EpiParams &e = pb.epi;
            if (!last) {
                // another slice of this tile finishes it
            } else if constexpr (EK == EK_PACK && !TF && C::POUT_OK) {
                // row rloc of M tile mi; column j of the result is k = j of the packed operand
                if (sl.dsmem) {
                    // the tile's packed image in the freed stage memory, [block][term][row][128 B]
                    // as in global memory; each warp then bulk-stores its 32 rows of each
                    // (block, term): 4 KiB, contiguous on both sides
                    char *img = reinterpret_cast<char *>(smem_raw + pad + CTL_BYTES);
                    const int kb0 = col_base / PK_K;  // this warp's first block of the tile
#pragma unroll
                    for (int g = 0; g < EPW / 32; ++g) {
                        char *blk = img + (size_t)(kb0 + g / 2) * P * PK_TILE_BYTES;
#pragma unroll
                        for (int cc = 0; cc < 4; ++cc)
                            store_chunk<P>(blk, rloc, (g & 1) * 4 + cc, &sum[g * 32 + cc * 8]);
                    }
                    fence_proxy_async_smem();
                    __syncwarp();
                    if (lane == 0) {
                        char *gt = e.pack + (size_t)((long long)tr.mi * e.pack_kt + tr.ni * (BN / PK_K)) * P *
                                                PK_TILE_BYTES;
#pragma unroll
                        for (int b = 0; b < EPW / PK_K; ++b)
#pragma unroll
                            for (int q = 0; q < P; ++q) {
                                const size_t off = ((size_t)(kb0 + b) * P + q) * PK_TILE_BYTES + (size_t)quarter * 4096;
                                bulk_s2g(gt + off, saddr(img + off), 4096u);
                            }
                        bulk_commit();
                        bulk_wait<0>();
                    }
                    __syncwarp();
                } else {
#pragma unroll
                    for (int g = 0; g < EPW / 32; ++g) {
                        const int kt = (col0 + g * 32) / PK_K;  // 128 x 64 block of the packed operand
                        char *tile0 = e.pack + (size_t)((long long)tr.mi * e.pack_kt + kt) * P * PK_TILE_BYTES;
#pragma unroll
                        for (int cc = 0; cc < 4; ++cc)
                            store_chunk<P>(tile0, rloc, (g & 1) * 4 + cc, &sum[g * 32 + cc * 8]);
                    }
                }
            } else if constexpr (EK == EK_PACK) {
                // row rloc of M tile mi; column j of the result is k = j of the packed operand
#pragma unroll
                for (int g = 0; g < EPW / 32; ++g) {
                    const int kt = (col0 + g * 32) / PK_K;  // 128 x 64 block of the packed operand
                    if constexpr (TF != 0) {  // blocks of 2P pieces: P TF32 terms of two 32-K tiles
                        char *blk = e.pack + (size_t)((long long)tr.mi * e.pack_kt + kt) * 2 * P * PK_TILE_BYTES;
#pragma unroll
                        for (int cc = 0; cc < 4; ++cc)
                            store_chunk_tf32<P>(blk, rloc, (g & 1) * 4 + cc, &sum[g * 32 + cc * 8]);
                    } else {
                        char *tile0 = e.pack + (size_t)((long long)tr.mi * e.pack_kt + kt) * P * PK_TILE_BYTES;
#pragma unroll
                        for (int cc = 0; cc < 4; ++cc)
                            store_chunk<P>(tile0, rloc, (g & 1) * 4 + cc, &sum[g * 32 + cc * 8]);
                    }
                }
            } else if ((EK == EK_EF || EK == EK_GEMM) && sl.dsmem) {
                // the beta input of this tile arrives in the stage memory (dfull):
                // E first, which does not need it, then F (or C) from it
                float *sc = scratch + (warp - C::EPI0) * 1024;
                const int wrow0 = tr.mi * BM + quarter * 32;
                if constexpr (EK == EK_EF) {
#pragma unroll
                    for (int g = 0; g < EPW / 32; ++g) block_store_e(e, sc, wrow0, col0 + g * 32, &sum[g * 32], lane);
                }
                ok = wait_phase(ctl, &ctl->dfull, 0, ERR_EPILOGUE, true, 128);
                ok = __all_sync(0xffffffffu, ok);
                if (!ok) break;
                const float *ds = reinterpret_cast<const float *>(smem_raw + pad + CTL_BYTES) +
                                  (size_t)(quarter * 32) * BN + col_base;
#pragma unroll
                for (int g = 0; g < EPW / 32; ++g)
                    block_store_f<EK>(e, sc, wrow0, col0 + g * 32, &sum[g * 32], lane, ds + g * 32, BN);
            } else {
                float *sc = scratch + (warp - C::EPI0) * 1024;
                const int wrow0 = tr.mi * BM + quarter * 32;
#pragma unroll
                for (int g = 0; g < EPW / 32; ++g) {
                    if constexpr (EK == EK_SYM) {
                        // chunks reaching above the diagonal (some column > some row
                        // of the warp) keep only their lower-triangle elements
                        const bool diag = col0 + g * 32 + 31 > wrow0;
                        epi_sym32(e, wrow0 + lane, col0 + g * 32, &sum[g * 32], diag);
                    } else {
                        if (!block_epilogue<EK>(e, sc, wrow0, col0 + g * 32, &sum[g * 32], lane))
                            epi_chunk(e, wrow0 + lane, col0 + g * 32, &sum[g * 32]);
                    }
                }
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&ctl->sempty[s]);
        }
    }

    tc_fence_before();
    __syncthreads();
    // neither CTA of a pair leaves while the other may still copy into its
    // stages or arrive on its barriers
    if (pair) cluster_sync();
    if (warp == 1) {
        tc_fence_after();
        __syncwarp();
        if constexpr (pair)
            asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
        else
            asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
    }
}

// With `side` (single problems, packing epilogue, Cfg::SIDE_OK), CTAs beyond
// the tile CTAs pack that operand when enough SMs are free to finish it within
// the contraction's own time; *side_done reports whether they were launched.
template <int P, int BN, int BATCHED, int EK, int PAIR = 0, int TF = 0>
ln_status launch(const UmmaProblem *single, const UmmaProblem *probs, const int *prefix, const int *owner, int total,
                 int *queue, cudaStream_t st, const PackMulti *side = nullptr, bool *side_done = nullptr) {
    using C = Cfg<P, BN, epi_width<EK, BN>(), PAIR>;
    auto kern = k_umma<P, BN, BATCHED, EK, PAIR, TF>;
    // the shared-memory opt-in is set once per device (so nothing but launches
    // happens while a caller captures a graph)
    static bool attr_set[64] = {false};
    int dev = 0;
    LN_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64 || !attr_set[dev]) {
        LN_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM));
        if (dev >= 0 && dev < 64) attr_set[dev] = true;
    }
    if constexpr (C::REG_SPLIT) {
        // setmaxnreg.inc waits until the registers it asks for are free: launch
        // only if the kernel really got the per-thread count the split assumes
        static int regs[64] = {0};
        if (dev < 0 || dev >= 64 || regs[dev] == 0) {
            cudaFuncAttributes fa{};
            LN_CUDA_TRY(cudaFuncGetAttributes(&fa, kern));
            if (dev >= 0 && dev < 64) regs[dev] = fa.numRegs;
            if (fa.numRegs != C::REG_LAUNCH)
                return fail(LN_ERR_UNSUPPORTED, "tcgen05 kernel compiled with %d registers per thread, %d expected",
                            fa.numRegs, C::REG_LAUNCH);
        } else if (regs[dev] != C::REG_LAUNCH) {
            return fail(LN_ERR_UNSUPPORTED, "tcgen05 kernel compiled with %d registers per thread, %d expected",
                        regs[dev], C::REG_LAUNCH);
        }
    }
    const int sms = sm_count();
    const bool sk = single && single->streamk;
    if (sk && (!single->skpart || !single->skflag)) return fail(LN_ERR_INVALID_VALUE, "stream-K without its workspace");
    constexpr bool pair = PAIR != 0;
    if (pair && (!single || !single->pair || sk || single->ksplit > 1))
        return fail(LN_ERR_INVALID_VALUE, "CTA pairs need a single problem without stream-K or split-K");
    // pairs: `total` counts pair tiles, two CTAs each, at most as many pairs as
    // the GPU holds at once (both CTAs of a pair share a GPC)
    int max_pairs = sms / 2;
    if (pair) {
        static int cached[64] = {0};
        if (dev >= 0 && dev < 64 && cached[dev] > 0) {
            max_pairs = cached[dev];
        } else {
            cudaLaunchConfig_t qc{};
            qc.gridDim = dim3((unsigned)(2 * max_pairs));
            qc.blockDim = dim3(C::NTHREADS);
            qc.dynamicSmemBytes = C::SMEM;
            cudaLaunchAttribute qa[1];
            qa[0].id = cudaLaunchAttributeClusterDimension;
            qa[0].val.clusterDim.x = 2;
            qa[0].val.clusterDim.y = 1;
            qa[0].val.clusterDim.z = 1;
            qc.attrs = qa;
            qc.numAttrs = 1;
            int n = 0;
            LN_CUDA_TRY(cudaOccupancyMaxActiveClusters(&n, kern, &qc));
            if (n <= 0) return fail(LN_ERR_UNSUPPORTED, "no cluster of two CTAs of the tcgen05 kernel fits");
            max_pairs = n < sms / 2 ? n : sms / 2;
            if (dev >= 0 && dev < 64) cached[dev] = max_pairs;
        }
    }
    const int tile_ctas = sk ? sms : pair ? 2 * (total < max_pairs ? total : max_pairs) : (total < sms ? total : sms);
    int side_ctas = 0;
    PackMulti none{};
    if (side_done) *side_done = false;
    if constexpr (EK == EK_PACK && !BATCHED && C::SIDE_OK && !TF) {
        if (!sk && side && single && side->prefix[side->count] > 0 && pack_stream_eligible(*side)) {
            // time model: a 128 x BN x 64 MMA step per product at the SM's share of
            // the BF16 peak (~0.33 us at BN = 256) against ~60 GB/s of split
            // traffic (32 KiB in, 32 KiB out per pack tile) for each spare SM
            const int ktot = single->nseg * single->kt;
            const int kslice = single->ksplit > 1 ? (ktot + single->ksplit - 1) / single->ksplit : ktot;
            const double mma_us =
                ceil_div(total, pair ? tile_ctas / 2 : tile_ctas) * (double)kslice * Products<P>::n * 0.33 * (BN / 256.0);
            const int free_sms = pair ? 2 * max_pairs - tile_ctas : sms - tile_ctas;
            const double pack_us =
                free_sms > 0 ? side->prefix[side->count] * 65536.0 / (free_sms * 60e3) : 1e30;
            if (pack_us <= 0.8 * mma_us) side_ctas = free_sms;
        }
    }
    UmmaProblem dummy{};
    {
        LaunchScope ls_(FAM_UMMA, st);
        cudaLaunchConfig_t cfg{};
        cfg.gridDim = dim3((unsigned)(tile_ctas + side_ctas));
        cfg.blockDim = dim3(C::NTHREADS);
        cfg.dynamicSmemBytes = C::SMEM;
        cfg.stream = st;
        cudaLaunchAttribute attr[2];
        attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[0].val.programmaticStreamSerializationAllowed = 1;
        attr[1].id = cudaLaunchAttributeClusterDimension;
        attr[1].val.clusterDim.x = 2;
        attr[1].val.clusterDim.y = 1;
        attr[1].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = pair ? 2 : 1;
        const cudaError_t le = cudaLaunchKernelEx(&cfg, kern, single ? *single : dummy, probs, prefix, owner, total,
                                                  queue, side_ctas ? *side : none, tile_ctas);
        if (le != cudaSuccess) return fail(LN_ERR_CUDA, "tcgen05 contraction launch: %s", cudaGetErrorString(le));
    }
    const ln_status ls = check_launch("tcgen05 contraction");
    if (side_done) *side_done = ls == LN_SUCCESS && side_ctas > 0;
    return ls;
}

}  // namespace

}  // namespace ln
