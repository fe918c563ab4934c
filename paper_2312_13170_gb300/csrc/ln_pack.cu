// Split-and-pack: turns an FP32 operand into the BF16 split terms that the
// tcgen05 contraction multiplies, written directly in the tensor core's
// shared-memory operand layout (K-major, 128-byte swizzle; see the packed
// operand description in ln_internal.h).
//
// Split: hi = bf16(x), lo = bf16(x - hi) and, for three terms,
// lo2 = bf16((x - hi) - lo), each rounded to nearest even. x - hi is exact in
// FP32, so x = hi + lo + O(2^-16 |x|) with two terms and O(2^-24 |x|) with
// three.
//
// Optional centring subtracts a per-row offset given as an FP32 pair
// (hi + lo = the FP64 mean), so the centred value is correct to about one
// FP32 rounding even when the mean is large compared to the spread.
#include <cuda_bf16.h>

#include "ln_internal.h"

namespace ln {

namespace {

template <int P>
__device__ __forceinline__ void split8(const float (&v)[8], uint4 (&out)[P]) {
    uint32_t w[P][4];
#pragma unroll
    for (int q = 0; q < 8; q += 2) {
        float x0 = v[q], x1 = v[q + 1];
#pragma unroll
        for (int t = 0; t < P; ++t) {
            __nv_bfloat16 h0 = __float2bfloat16_rn(x0), h1 = __float2bfloat16_rn(x1);
            w[t][q / 2] = (uint32_t)__bfloat16_as_ushort(h0) | ((uint32_t)__bfloat16_as_ushort(h1) << 16);
            x0 = x0 - __bfloat162float(h0);
            x1 = x1 - __bfloat162float(h1);
        }
    }
#pragma unroll
    for (int t = 0; t < P; ++t) out[t] = make_uint4(w[t][0], w[t][1], w[t][2], w[t][3]);
}

template <int P>
__device__ __forceinline__ void store_chunk(char *tile0, int r, int c, const float (&v)[8]) {
    uint4 o[P];
    split8<P>(v, o);
    const int off = r * 128 + ((c ^ (r & 7)) << 4);
#pragma unroll
    for (int t = 0; t < P; ++t) *reinterpret_cast<uint4 *>(tile0 + (size_t)t * PK_TILE_BYTES + off) = o[t];
}

// One 128-row x 64-k tile (all P terms) of the packed operand described by p.
// `s` is a 64 x 129 shared-memory staging block used by the transposed case.
template <int TRANS, int P>
__device__ __forceinline__ void pack_tile(const PackSrc &p, int kt, int rt, float (*s)[PK_ROWS + 1]) {
    const int tid = threadIdx.x;
    const int r0 = rt * PK_ROWS, k0 = kt * PK_K;
    char *tile0 = p.dst + (size_t)((long long)rt * p.kt + kt) * P * PK_TILE_BYTES;
    if (TRANS == 0) {
        const bool vec = ((reinterpret_cast<uintptr_t>(p.S) & 15) == 0) && ((p.ld & 3) == 0);
#pragma unroll
        for (int pass = 0; pass < 4; ++pass) {
            const int r = pass * 32 + (tid >> 3), c = tid & 7;
            const int gr = r0 + r, gk = k0 + c * 8;
            float v[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) v[q] = 0.0f;
            if (gr < p.rows) {
                const float *src = p.S + (long long)gr * p.ld + gk;
                if (vec && gk + 7 < p.K) {
                    float4 a = __ldg(reinterpret_cast<const float4 *>(src));
                    float4 b = __ldg(reinterpret_cast<const float4 *>(src + 4));
                    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
                    v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
                } else {
#pragma unroll
                    for (int q = 0; q < 8; ++q)
                        if (gk + q < p.K) v[q] = __ldg(src + q);
                }
                if (p.off_hi) {
                    const float h = p.off_hi[gr], l = p.off_lo[gr];
#pragma unroll
                    for (int q = 0; q < 8; ++q)
                        if (gk + q < p.K) v[q] = (v[q] - h) - l;
                }
            }
            store_chunk<P>(tile0, r, c, v);
        }
    } else {
        // element (r, k) = S[k*ld + r]: stage the 64 x 128 block through shared
        // memory (coalesced along r) and read it back along k.
        const int lane = tid & 31, warp = tid >> 5;
#pragma unroll
        for (int it = 0; it < 8; ++it) {
            const int kk = warp + 8 * it;
            const int gk = k0 + kk;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int rr = lane + 32 * q;
                const int gr = r0 + rr;
                float x = 0.0f;
                if (gk < p.K && gr < p.rows) {
                    x = __ldg(p.S + (long long)gk * p.ld + gr);
                    if (p.off_hi) x = (x - p.off_hi[gr]) - p.off_lo[gr];
                }
                s[kk][rr] = x;
            }
        }
        __syncthreads();
#pragma unroll
        for (int pass = 0; pass < 4; ++pass) {
            const int r = pass * 32 + (tid >> 3), c = tid & 7;
            float v[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) v[q] = s[c * 8 + q][r];
            store_chunk<P>(tile0, r, c, v);
        }
    }
}

// grid (kt, rt)
template <int TRANS, int P>
__global__ __launch_bounds__(256) void k_pack(PackSrc p) {
    __shared__ float s[TRANS ? PK_K : 1][PK_ROWS + 1];
    pack_tile<TRANS, P>(p, blockIdx.x, blockIdx.y, s);
}

// Ranks instances by decreasing work n*n*k (ties by index): order[rank] = i.
__global__ void k_batch_rank(int count, const ln_sym_desc *__restrict__ descs, int *order) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    if (count > 8192) {  // too many to rank by counting; keep the caller's order
        order[i] = i;
        return;
    }
    const ln_sym_desc di = descs[i];
    const double wi = (double)di.n * di.n * di.k;
    int rank = 0;
    for (int j = 0; j < count; ++j) {
        const ln_sym_desc dj = descs[j];
        const double wj = (double)dj.n * dj.n * dj.k;
        rank += (wj > wi) || (wj == wi && j < i);
    }
    order[rank] = i;
}

// Sequential layout in rank order (one thread): packed-operand offsets, tile
// prefix sums and the contraction descriptor of every instance.
__global__ void k_batch_layout(int is_syr2k, int count, const ln_sym_desc *__restrict__ descs, const int *order,
                               int fill, float alpha, float beta, UmmaProblem *probs, int *tile_prefix,
                               long long *pack_off, int *pack_prefix, char *pack_base, int terms) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    long long off = 0;
    int tiles = 0, ptiles = 0;
    for (int r = 0; r < count; ++r) {
        const ln_sym_desc d = descs[order[r]];
        const int mt = (d.n + PK_ROWS - 1) / PK_ROWS;
        const int kt = (d.k + PK_K - 1) / PK_K;
        const long long one = (long long)mt * kt * terms * PK_TILE_BYTES;
        UmmaProblem p{};
        p.kt = kt;
        p.x_kt = p.y_kt = kt;
        p.mt = p.nt = mt;
        p.sym = 1;
        const char *pa = pack_base + off;
        const char *pb = is_syr2k ? pa + one : pa;
        pack_off[2 * r] = off;
        pack_off[2 * r + 1] = is_syr2k ? off + one : off;
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
        tile_prefix[r] = tiles;
        pack_prefix[r] = ptiles;
        if (d.n > 0) {
            off += one * (is_syr2k ? 2 : 1);
            tiles += mt * (mt + 1) / 2;
            ptiles += mt * kt * (is_syr2k ? 2 : 1);
        }
    }
    tile_prefix[count] = tiles;
    pack_prefix[count] = ptiles;
}

// Packs every instance's operands: a flat grid over all (rank, operand, row
// tile, k tile); each CTA finds its rank by binary search of the prefix sums.
template <int P>
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
    pack_tile<0, P>(p, rem % kt, rem / kt, s);
}

}  // namespace

ln_status pack_operand(const PackSrc &p, int terms, cudaStream_t st) {
    if (p.rt <= 0 || p.kt <= 0) return LN_SUCCESS;
    if (p.rt > 65535) return fail(LN_ERR_INVALID_VALUE, "operand too tall to pack (%d row tiles)", p.rt);
    dim3 grid((unsigned)p.kt, (unsigned)p.rt);
    LaunchScope ls_(FAM_PACK, st);
#define LN_PACK_CASE(T, P) \
    if (p.trans == T && terms == P) k_pack<T, P><<<grid, 256, 0, st>>>(p)
    LN_PACK_CASE(0, 1);
    else LN_PACK_CASE(0, 2);
    else LN_PACK_CASE(0, 3);
    else LN_PACK_CASE(1, 1);
    else LN_PACK_CASE(1, 2);
    else LN_PACK_CASE(1, 3);
    else return fail(LN_ERR_INVALID_VALUE, "unsupported split term count %d", terms);
#undef LN_PACK_CASE
    return check_launch("split-and-pack");
}

ln_status sym_batched_plan(int is_syr2k, int count, const ln_sym_desc *d_descs, int fill, float alpha, float beta,
                           UmmaProblem *d_probs, int *d_tile_prefix, long long *d_pack_off, int *d_pack_prefix,
                           int *d_order, char *pack_base, int terms, cudaStream_t st) {
    { LaunchScope ls_(FAM_PACK, st); k_batch_rank<<<(unsigned)ceil_div(count, 256), 256, 0, st>>>(count, d_descs, d_order); }
    { LaunchScope ls_(FAM_PACK, st); k_batch_layout<<<1, 32, 0, st>>>(is_syr2k, count, d_descs, d_order, fill, alpha, beta, d_probs, d_tile_prefix,
                                     d_pack_off, d_pack_prefix, pack_base, terms); }
    return check_launch("batched plan");
}

ln_status sym_batched_pack(int is_syr2k, int count, const ln_sym_desc *d_descs, const long long *d_pack_off,
                           const int *d_pack_prefix, const int *d_order, int total_pack_tiles, char *pack_base,
                           int terms, cudaStream_t st) {
    if (total_pack_tiles == 0) return LN_SUCCESS;
    switch (terms) {
        case 1:
            { LaunchScope ls_(FAM_PACK, st); k_pack_batched<1><<<total_pack_tiles, 256, 0, st>>>(is_syr2k, count, d_descs, d_pack_off, d_pack_prefix,
                                                                d_order, pack_base); }
            break;
        case 2:
            { LaunchScope ls_(FAM_PACK, st); k_pack_batched<2><<<total_pack_tiles, 256, 0, st>>>(is_syr2k, count, d_descs, d_pack_off, d_pack_prefix,
                                                                d_order, pack_base); }
            break;
        case 3:
            { LaunchScope ls_(FAM_PACK, st); k_pack_batched<3><<<total_pack_tiles, 256, 0, st>>>(is_syr2k, count, d_descs, d_pack_off, d_pack_prefix,
                                                                d_order, pack_base); }
            break;
        default: return fail(LN_ERR_INVALID_VALUE, "unsupported split term count %d", terms);
    }
    return check_launch("batched split-and-pack");
}

}  // namespace ln
