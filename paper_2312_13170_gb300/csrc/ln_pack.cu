// Split-and-pack: turns an FP32 operand into the BF16 split terms that the
// tcgen05 contraction multiplies, written directly in the tensor core's
// shared-memory operand layout (K-major, 128-byte swizzle; see the packed
// operand description in ln_internal.h).
//
// The split itself is in ln_split.cuh.
//
// Optional centring subtracts a per-row offset given as an FP32 pair
// (hi + lo = the FP64 mean), so the centred value is correct to about one
// FP32 rounding even when the mean is large compared to the spread.
#include "ln_internal.h"
#include "ln_pack_stream.cuh"
#include "ln_split.cuh"

namespace ln {

namespace {

// One 128-row x 64-k tile (all P terms) of the packed operand described by p.
// `s` is a 64 x 129 shared-memory staging block used by the transposed case.
// All global loads of a thread are issued before any split or store.
template <int TRANS, int P, bool TF = false>
__device__ __forceinline__ void pack_tile(const PackSrc &p, int kt, int rt, float (*s)[PK_ROWS + 1]) {
    const int tid = threadIdx.x;
    const int r0 = rt * PK_ROWS, k0 = kt * PK_K;
    char *tile0 = p.dst + (size_t)((long long)rt * p.kt + kt) * P * PK_TILE_BYTES;
    if (TRANS == 0) {
        // thread -> (row r = pass*32 + tid/8, 16-byte chunk c = tid%8): a warp
        // reads 4 rows x 256 contiguous bytes and writes 512 contiguous bytes
        const bool vec = ((reinterpret_cast<uintptr_t>(p.S) & 15) == 0) && ((p.ld & 3) == 0);
        const int c = tid & 7, gk = k0 + c * 8;
        float v[4][8];
#pragma unroll
        for (int pass = 0; pass < 4; ++pass) {
            const int gr = r0 + pass * 32 + (tid >> 3);
#pragma unroll
            for (int q = 0; q < 8; ++q) v[pass][q] = 0.0f;
            if (gr < p.rows) {
                const float *src = p.S + (long long)gr * p.ld + gk;
                if (vec && gk + 7 < p.K) {
                    float4 a = __ldg(reinterpret_cast<const float4 *>(src));
                    float4 b = __ldg(reinterpret_cast<const float4 *>(src + 4));
                    v[pass][0] = a.x; v[pass][1] = a.y; v[pass][2] = a.z; v[pass][3] = a.w;
                    v[pass][4] = b.x; v[pass][5] = b.y; v[pass][6] = b.z; v[pass][7] = b.w;
                } else {
#pragma unroll
                    for (int q = 0; q < 8; ++q)
                        if (gk + q < p.K) v[pass][q] = __ldg(src + q);
                }
            }
        }
#pragma unroll
        for (int pass = 0; pass < 4; ++pass) {
            const int r = pass * 32 + (tid >> 3), gr = r0 + r;
            if (p.off_hi && gr < p.rows) {
                const float h = p.off_hi[gr], l = p.off_lo[gr];
#pragma unroll
                for (int q = 0; q < 8; ++q)
                    if (gk + q < p.K) v[pass][q] = (v[pass][q] - h) - l;
            }
            store_chunk_fmt<P, TF>(tile0, r, c, v[pass]);
        }
    } else {
        // element (r, k) = S[k*ld + r]: stage the 64 x 128 block through shared
        // memory, loading along r (one 512-byte k-row per warp instruction when
        // aligned) and reading back along k.
        const int lane = tid & 31, warp = tid >> 5;
        const bool vec = ((reinterpret_cast<uintptr_t>(p.S) & 15) == 0) && ((p.ld & 3) == 0) &&
                         r0 + PK_ROWS <= p.rows;
        const int rr = lane * 4;
        float4 x[8];
#pragma unroll
        for (int it = 0; it < 8; ++it) {
            const int gk = k0 + warp + 8 * it;
            x[it] = make_float4(0.f, 0.f, 0.f, 0.f);
            if (gk < p.K) {
                const float *src = p.S + (long long)gk * p.ld + r0 + rr;
                if (vec) {
                    x[it] = __ldg(reinterpret_cast<const float4 *>(src));
                } else {
                    if (r0 + rr + 0 < p.rows) x[it].x = __ldg(src + 0);
                    if (r0 + rr + 1 < p.rows) x[it].y = __ldg(src + 1);
                    if (r0 + rr + 2 < p.rows) x[it].z = __ldg(src + 2);
                    if (r0 + rr + 3 < p.rows) x[it].w = __ldg(src + 3);
                }
            }
        }
        float h[4] = {0, 0, 0, 0}, l[4] = {0, 0, 0, 0};
        if (p.off_hi) {
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (r0 + rr + q < p.rows) {
                    h[q] = p.off_hi[r0 + rr + q];
                    l[q] = p.off_lo[r0 + rr + q];
                }
        }
#pragma unroll
        for (int it = 0; it < 8; ++it) {
            const int kk = warp + 8 * it;
            const bool live = k0 + kk < p.K;
            float e[4] = {x[it].x, x[it].y, x[it].z, x[it].w};
            // rotate the four stores by lane/8 so the 32 lanes hit 32 banks
#pragma unroll
            for (int q0 = 0; q0 < 4; ++q0) {
                const int q = (q0 + (lane >> 3)) & 3;
                float val = e[q];
                if (p.off_hi && live && r0 + rr + q < p.rows) val = (val - h[q]) - l[q];
                s[kk][rr + q] = val;
            }
        }
        __syncthreads();
#pragma unroll
        for (int pass = 0; pass < 4; ++pass) {
            const int r = pass * 32 + (tid >> 3), c = tid & 7;
            float v[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) v[q] = s[c * 8 + q][r];
            store_chunk_fmt<P, TF>(tile0, r, c, v);
        }
    }
}

// grid (kt, rt)
// TF: TF32 blocks (PackSrc::tf32); P is then even (two pieces per TF32 term)
template <int TRANS, int P, bool TF>
__global__ __launch_bounds__(256) void k_pack(PackSrc p) {
    __shared__ float s[TRANS ? PK_K : 1][PK_ROWS + 1];
    pack_tile<TRANS, P, TF>(p, blockIdx.x, blockIdx.y, s);
}

// Several operands in one launch: a flat grid over all their tiles.
template <int P, bool TF>
__global__ __launch_bounds__(256) void k_pack_multi(const __grid_constant__ PackMulti m) {
    __shared__ float s[PK_K][PK_ROWS + 1];
    const int t = blockIdx.x;
    int i = 0;
    while (i + 1 < m.count && m.prefix[i + 1] <= t) ++i;
    const PackSrc &p = m.op[i];
    const int local = t - m.prefix[i];
    if (p.trans) pack_tile<1, P, TF>(p, local % p.kt, local / p.kt, s);
    else pack_tile<0, P, TF>(p, local % p.kt, local / p.kt, s);
}

// Persistent bulk-copy pack stream (ln_pack_stream.cuh), one CTA per SM.
template <int P, int NT, bool TF>
__global__ __launch_bounds__(NT, 1) void k_pack_stream(const __grid_constant__ PackMulti m, int ns, int nout) {
    extern __shared__ __align__(128) unsigned char ps_smem[];
    pack_stream<P, NT, TF>(m, blockIdx.x, gridDim.x, ps_smem, ns, nout);
}

// Batched layout, one CTA of 1024 threads: (1) rank instances by decreasing
// work n*n*k (ties by index) so the queue hands out the largest first, keeping
// the weights and the order in shared memory; (2) an exclusive block scan, in
// rank order, of each instance's packed-operand bytes, lower-triangle tiles and
// pack tiles; (3) write every instance's contraction descriptor. Batches of
// more than RANK_MAX instances keep the caller's order.
constexpr int PLAN_THREADS = 1024;
constexpr int RANK_MAX = 8192;

__global__ __launch_bounds__(PLAN_THREADS) void k_batch_plan(int is_syr2k, int count,
                                                             const ln_sym_desc *__restrict__ descs, int *order,
                                                             int fill, float alpha, float beta, UmmaProblem *probs,
                                                             int *tile_prefix, int *tile_owner, long long *pack_off,
                                                             int *pack_prefix, char *pack_base, int terms,
                                                             int chunk_kt_for_kernel, int tf32) {
    __shared__ float w[RANK_MAX];
    __shared__ long long sb[PLAN_THREADS];
    __shared__ int st[PLAN_THREADS], sp[PLAN_THREADS];
    const int tid = threadIdx.x;
    const bool ranked = count <= RANK_MAX;
    if (ranked) {
        for (int i = tid; i < count; i += PLAN_THREADS) {
            const ln_sym_desc d = descs[i];
            w[i] = (float)d.n * (float)d.n * (float)d.k;
        }
        __syncthreads();
        for (int i = tid; i < count; i += PLAN_THREADS) {
            const float wi = w[i];
            int rank = 0;
            for (int j = 0; j < count; ++j) rank += (w[j] > wi) || (w[j] == wi && j < i);
            order[rank] = i;
        }
    } else {
        for (int i = tid; i < count; i += PLAN_THREADS) order[i] = i;
    }
    __syncthreads();
    __threadfence_block();
    // each thread owns a contiguous run of ranks
    const int per = (count + PLAN_THREADS - 1) / PLAN_THREADS;
    const int r0 = tid * per, r1 = min(count, r0 + per);
    long long bytes = 0;
    int tiles = 0, ptiles = 0;
    for (int r = r0; r < r1; ++r) {
        const ln_sym_desc d = descs[order[r]];
        if (d.n <= 0) continue;
        const int mt = (d.n + PK_ROWS - 1) / PK_ROWS;
        const int kt = (d.k + PK_K - 1) / PK_K;
        bytes += (long long)mt * kt * terms * PK_TILE_BYTES * (is_syr2k ? 2 : 1);
        tiles += mt * (mt + 1) / 2;
        ptiles += mt * kt * (is_syr2k ? 2 : 1);
    }
    sb[tid] = bytes;
    st[tid] = tiles;
    sp[tid] = ptiles;
    __syncthreads();
    for (int off = 1; off < PLAN_THREADS; off <<= 1) {  // inclusive Hillis-Steele scan
        long long b2 = tid >= off ? sb[tid - off] : 0;
        int t2 = tid >= off ? st[tid - off] : 0, p2 = tid >= off ? sp[tid - off] : 0;
        __syncthreads();
        sb[tid] += b2;
        st[tid] += t2;
        sp[tid] += p2;
        __syncthreads();
    }
    long long off_b = sb[tid] - bytes;
    int off_t = st[tid] - tiles, off_p = sp[tid] - ptiles;
    for (int r = r0; r < r1; ++r) {
        const ln_sym_desc d = descs[order[r]];
        const int mt = d.n > 0 ? (d.n + PK_ROWS - 1) / PK_ROWS : 0;
        const int kt = (d.k + PK_K - 1) / PK_K;
        const long long one = (long long)mt * kt * terms * PK_TILE_BYTES;
        UmmaProblem p{};
        p.kt = tf32 ? 2 * kt : kt;  // the kernel's k tiles: 32-K tiles for TF32
        p.x_kt = p.y_kt = p.kt;
        p.mt = p.nt = mt;
        p.sym = 1;
        p.chunk_kt = chunk_kt_for_kernel;
        p.tf32 = tf32;
        const char *pa = pack_base + off_b;
        const char *pb = is_syr2k ? pa + one : pa;
        pack_off[2 * r] = off_b;
        pack_off[2 * r + 1] = is_syr2k ? off_b + one : off_b;
        if (is_syr2k) {
            p.seg[0].X = pa;
            p.seg[0].Y = pb;
            p.seg[1].X = pb;
            p.seg[1].Y = pa;
            p.nseg = 2;
        } else {
            p.seg[0].X = pa;
            p.seg[0].Y = pa;
            p.nseg = 1;
        }
        p.epi.mode = EPI_SYM;
        p.epi.M = p.epi.N = d.n;
        p.epi.alpha = alpha;
        p.epi.beta = beta;
        p.epi.C = d.C;
        p.epi.ldc = d.ldc;
        p.epi.fill = fill;
        p.epi.sym_kind = SYM_AXPBY;
        probs[r] = p;
        tile_prefix[r] = off_t;
        pack_prefix[r] = off_p;
        if (d.n > 0) {
            for (int q = 0; q < mt * (mt + 1) / 2; ++q) tile_owner[off_t + q] = r;
            off_b += one * (is_syr2k ? 2 : 1);
            off_t += mt * (mt + 1) / 2;
            off_p += mt * kt * (is_syr2k ? 2 : 1);
        }
    }
    if (tid == PLAN_THREADS - 1) {
        tile_prefix[count] = st[tid];
        pack_prefix[count] = sp[tid];
    }
}

// Packs every instance's operands: a flat grid over all (rank, operand, row
// tile, k tile); each CTA finds its rank by binary search of the prefix sums.
template <int P, bool TF>
__global__ __launch_bounds__(256) void k_pack_batched(int is_syr2k, int count, const ln_sym_desc *__restrict__ descs,
                                                      const long long *__restrict__ pack_off,
                                                      const int *__restrict__ pack_prefix,
                                                      const int *__restrict__ order, char *pack_base) {
    __shared__ float s[1][PK_ROWS + 1];
    const int t = blockIdx.x;
    int lo = 0, hi = count - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (pack_prefix[mid] <= t) lo = mid;
        else hi = mid - 1;
    }
    const ln_sym_desc d = descs[order[lo]];
    const int mt = (d.n + PK_ROWS - 1) / PK_ROWS;
    const int kt = (d.k + PK_K - 1) / PK_K;
    const int local = t - pack_prefix[lo];
    const int operand = local / (mt * kt);
    const int rem = local - operand * mt * kt;
    PackSrc p;
    p.S = operand ? d.B : d.A;
    p.ld = operand ? d.ldb : d.lda;
    p.trans = 0;
    p.rows = d.n;
    p.K = d.k;
    p.off_hi = nullptr;
    p.off_lo = nullptr;
    p.dst = pack_base + pack_off[2 * lo + operand];
    p.rt = mt;
    p.kt = kt;
    p.tf32 = TF;
    pack_tile<0, P, TF>(p, rem % kt, rem / kt, s);
}

}  // namespace

ln_status pack_operand(const PackSrc &p, int terms, cudaStream_t st) {
    if (p.rt <= 0 || p.kt <= 0) return LN_SUCCESS;
    {
        PackMulti m;
        if (make_pack_multi(&p, 1, m) && pack_stream_eligible(m)) return pack_operands(&p, 1, terms, st);
    }
    if (p.rt > 65535) return fail(LN_ERR_INVALID_VALUE, "operand too tall to pack (%d row tiles)", p.rt);
    dim3 grid((unsigned)p.kt, (unsigned)p.rt);
    LaunchScope ls_(FAM_PACK, st);
#define LN_PACK_CASE(T, P, F) \
    if (p.trans == T && terms == P && (p.tf32 != 0) == F) k_pack<T, P, F><<<grid, 256, 0, st>>>(p)
    LN_PACK_CASE(0, 1, false);
    else LN_PACK_CASE(0, 2, false);
    else LN_PACK_CASE(0, 3, false);
    else LN_PACK_CASE(0, 2, true);
    else LN_PACK_CASE(0, 4, true);
    else LN_PACK_CASE(1, 1, false);
    else LN_PACK_CASE(1, 2, false);
    else LN_PACK_CASE(1, 3, false);
    else LN_PACK_CASE(1, 2, true);
    else LN_PACK_CASE(1, 4, true);
    else return fail(LN_ERR_INVALID_VALUE, "unsupported packed format (%d pieces, tf32 %d)", terms, p.tf32);
#undef LN_PACK_CASE
    return check_launch("split-and-pack");
}

bool make_pack_multi(const PackSrc *ps, int count, PackMulti &m) {
    if (count < 1 || count > 4) return false;
    m = PackMulti{};
    m.count = count;
    long long tiles = 0;
    for (int i = 0; i < count; ++i) {
        m.op[i] = ps[i];
        m.prefix[i] = (int)tiles;
        tiles += (long long)ps[i].rt * ps[i].kt;
        if (tiles > 0x7fffffffLL) return false;
    }
    m.prefix[count] = (int)tiles;
    return true;
}

bool pack_stream_eligible(const PackMulti &m) {
    for (int i = 0; i < m.count; ++i) {
        const PackSrc &p = m.op[i];
        if (m.prefix[i + 1] == m.prefix[i]) continue;
        if ((reinterpret_cast<uintptr_t>(p.S) & 15) || (p.ld & 3)) return false;
        if (p.trans ? (p.rows & 3) : (p.K & 3)) return false;
        if (reinterpret_cast<uintptr_t>(p.dst) & 15) return false;
    }
    return true;
}

namespace {

// 4 input stages and 3 output buffers where they fit in 227 KiB (1 and 2
// pieces per block), else 3 and 2
constexpr int stream_stages(int terms) { return terms >= 3 ? 3 : PS_MAX_STAGES; }
constexpr int stream_outs(int terms) { return terms >= 3 ? 2 : 3; }
static_assert(pack_stream_smem(stream_stages(2), stream_outs(2), 2) <= 227 * 1024, "pack stream smem");
static_assert(pack_stream_smem(stream_stages(3), stream_outs(3), 3) <= 227 * 1024, "pack stream smem");
static_assert(pack_stream_smem(stream_stages(4), stream_outs(4), 4) <= 227 * 1024, "pack stream smem");

template <int P, int NT, bool TF>
ln_status launch_pack_stream(const PackMulti &m, cudaStream_t st) {
    const int ns = stream_stages(P), nout = stream_outs(P);
    const int bytes = pack_stream_smem(ns, nout, P);
    // the shared-memory opt-in is set once per device (so nothing but launches
    // happens while a caller captures a graph)
    static bool attr_set[64] = {false};
    int dev = 0;
    LN_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64 || !attr_set[dev]) {
        LN_CUDA_TRY(cudaFuncSetAttribute(k_pack_stream<P, NT, TF>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
        if (dev >= 0 && dev < 64) attr_set[dev] = true;
    }
    const int tiles = m.prefix[m.count];
    const int grid = std::min(tiles, sm_count());
    LaunchScope ls_(FAM_PACK, st);
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(NT);
    cfg.dynamicSmemBytes = (size_t)bytes;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const cudaError_t le = cudaLaunchKernelEx(&cfg, k_pack_stream<P, NT, TF>, m, ns, nout);
    if (le != cudaSuccess) return fail(LN_ERR_CUDA, "split-and-pack stream launch: %s", cudaGetErrorString(le));
    return check_launch("split-and-pack stream");
}

template <int P, bool TF = false>
ln_status launch_pack_stream(const PackMulti &m, cudaStream_t st) {
    return tune_pack_threads() == 1024 ? launch_pack_stream<P, 1024, TF>(m, st) : launch_pack_stream<P, 512, TF>(m, st);
}

}  // namespace

ln_status pack_operands(const PackSrc *ps, int count, int terms, cudaStream_t st) {
    if (count < 1 || count > 4) return fail(LN_ERR_INVALID_VALUE, "pack_operands: bad operand count %d", count);
    PackMulti m;
    if (!make_pack_multi(ps, count, m)) return fail(LN_ERR_INVALID_VALUE, "too many tiles to pack");
    const int tiles = m.prefix[count];
    if (tiles == 0) return LN_SUCCESS;
    const bool tf = m.op[0].tf32 != 0;  // one format per launch
    for (int i = 1; i < count; ++i)
        if ((ps[i].tf32 != 0) != tf) return fail(LN_ERR_INVALID_VALUE, "pack_operands: mixed operand formats");
    if (tf && terms != 2 && terms != 4) return fail(LN_ERR_INVALID_VALUE, "TF32 operand with %d pieces", terms);
    if (pack_stream_eligible(m)) {
        if (tf) return terms == 2 ? launch_pack_stream<2, true>(m, st) : launch_pack_stream<4, true>(m, st);
        switch (terms) {
            case 1: return launch_pack_stream<1>(m, st);
            case 2: return launch_pack_stream<2>(m, st);
            case 3: return launch_pack_stream<3>(m, st);
            default: return fail(LN_ERR_INVALID_VALUE, "unsupported split term count %d", terms);
        }
    }
    LaunchScope ls_(FAM_PACK, st);
    if (tf) {
        if (terms == 2) k_pack_multi<2, true><<<(unsigned)tiles, 256, 0, st>>>(m);
        else k_pack_multi<4, true><<<(unsigned)tiles, 256, 0, st>>>(m);
        return check_launch("split-and-pack (multi)");
    }
    switch (terms) {
        case 1: k_pack_multi<1, false><<<(unsigned)tiles, 256, 0, st>>>(m); break;
        case 2: k_pack_multi<2, false><<<(unsigned)tiles, 256, 0, st>>>(m); break;
        case 3: k_pack_multi<3, false><<<(unsigned)tiles, 256, 0, st>>>(m); break;
        default: return fail(LN_ERR_INVALID_VALUE, "unsupported split term count %d", terms);
    }
    return check_launch("split-and-pack (multi)");
}

ln_status sym_batched_plan(int is_syr2k, int count, const ln_sym_desc *d_descs, int fill, float alpha, float beta,
                           UmmaProblem *d_probs, int *d_tile_prefix, int *d_tile_owner, long long *d_pack_off,
                           int *d_pack_prefix, int *d_order, char *pack_base, int terms, int tf32,
                           cudaStream_t st) {
    LaunchScope ls_(FAM_PACK, st);
    k_batch_plan<<<1, PLAN_THREADS, 0, st>>>(is_syr2k, count, d_descs, d_order, fill, alpha, beta, d_probs,
                                             d_tile_prefix, d_tile_owner, d_pack_off, d_pack_prefix, pack_base, terms,
                                             tune_chunk_kt(), tf32);
    return check_launch("batched plan");
}

ln_status sym_batched_pack(int is_syr2k, int count, const ln_sym_desc *d_descs, const long long *d_pack_off,
                           const int *d_pack_prefix, const int *d_order, int total_pack_tiles, char *pack_base,
                           int terms, int tf32, cudaStream_t st) {
    if (total_pack_tiles == 0) return LN_SUCCESS;
    const bool ok = tf32 ? (terms == 2 || terms == 4) : (terms >= 1 && terms <= 3);
    if (!ok) return fail(LN_ERR_INVALID_VALUE, "unsupported packed format (%d pieces, tf32 %d)", terms, tf32);
#define LN_PACK_BATCHED(P, F)                                                                                   \
    k_pack_batched<P, F><<<total_pack_tiles, 256, 0, st>>>(is_syr2k, count, d_descs, d_pack_off, d_pack_prefix, \
                                                           d_order, pack_base)
    {
        LaunchScope ls_(FAM_PACK, st);
        if (tf32) {
            if (terms == 2) LN_PACK_BATCHED(2, true);
            else LN_PACK_BATCHED(4, true);
        } else {
            switch (terms) {
                case 1: LN_PACK_BATCHED(1, false); break;
                case 2: LN_PACK_BATCHED(2, false); break;
                default: LN_PACK_BATCHED(3, false); break;
            }
        }
    }
#undef LN_PACK_BATCHED
    return check_launch("batched split-and-pack");
}

}  // namespace ln
