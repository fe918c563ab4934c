// Split-and-pack as a persistent stream: a CTA walks its share of the 128-row
// x 64-k tiles of up to four operands, keeping several FP32 source tiles in
// flight with per-thread 16-byte asynchronous copies into a ring of
// shared-memory stages (zero-filled outside the matrix), splits each tile
// into BF16 terms in shared memory (already in the packed K-major,
// 128-byte-swizzled layout), and writes the tile's terms back with a single
// bulk store (they are contiguous in the packed operand). Loads, the split of
// one tile and the store of the previous one overlap.
//
// Used by the split-and-pack kernel and by the spare CTAs of a tcgen05
// contraction that has fewer output tiles than SMs (which pack the operand of
// the next contraction meanwhile).
//
// Requirements (checked on the host by pack_stream_eligible): every source
// 16-byte aligned with ld a multiple of 4; a non-transposed source needs K a
// multiple of 4, a transposed one rows a multiple of 4, so that every row
// segment is a whole number of 16-byte units. Elements outside the logical
// extent are written as zeros. The first NT threads of the CTA (256 or 512)
// take part.
#pragma once

#include "ln_async.cuh"
#include "ln_internal.h"
#include "ln_split.cuh"

namespace ln {

namespace {

constexpr int PS_IN_BYTES = PK_ROWS * PK_K * 4;  // one FP32 source tile, 32 KiB
constexpr int PS_MAX_STAGES = 4;
constexpr int PS_BARRIER = 1;                     // named barrier id

// Shared-memory bytes of a stream with `ns` input stages, `nout` output
// buffers and P split terms.
__host__ __device__ constexpr int pack_stream_smem(int ns, int nout, int P) {
    return ns * PS_IN_BYTES + nout * P * PK_TILE_BYTES;
}

struct PsTile {
    const PackSrc *p;
    int r0, k0, nr, nk;
    size_t dst_off;  // byte offset of the tile's term 0 in p->dst
};

__device__ __forceinline__ PsTile ps_tile(const PackMulti &m, int t, int P) {
    int i = 0;
    while (i + 1 < m.count && m.prefix[i + 1] <= t) ++i;
    PsTile r;
    r.p = &m.op[i];
    const int local = t - m.prefix[i], nkt = r.p->kt;
    // local / nkt from a float estimate (off by at most one below 2^24), then exact
    int rt = (int)__fdividef((float)local, (float)nkt);
    int kt = local - rt * nkt;
    while (kt < 0) {
        --rt;
        kt += nkt;
    }
    while (kt >= nkt) {
        ++rt;
        kt -= nkt;
    }
    r.r0 = rt * PK_ROWS;
    r.k0 = kt * PK_K;
    r.nr = min(max(r.p->rows - r.r0, 0), PK_ROWS);
    r.nk = min(max(r.p->K - r.k0, 0), PK_K);
    r.dst_off = (size_t)((long long)rt * r.p->kt + kt) * P * PK_TILE_BYTES;
    return r;
}

__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src, uint32_t src_bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Every thread copies 2048/NT of the tile's 2048 16-byte units (consecutive
// threads, consecutive units of a row). Non-transposed tiles land as
// [128 r][64 k] (256-byte rows), transposed ones as [64 k][128 r] (512-byte
// rows); units outside the matrix are zero-filled without reading global
// memory.
template <int NT>
__device__ __forceinline__ void ps_issue(const PsTile &tl, float *stage, int tid) {
    const PackSrc &p = *tl.p;
    constexpr int J = 2048 / NT;
    const uint32_t s0 = saddr(stage) + (uint32_t)tid * 16u;
    if (p.trans) {
        const int col = tid & 31, row0 = tid >> 5;  // 32 units per 512-byte row
        const bool cin = col * 4 < tl.nr;
        const float *src = p.S + (long long)(tl.k0 + row0) * p.ld + tl.r0 + col * 4;
#pragma unroll
        for (int j = 0; j < J; ++j) {
            const bool in = cin && row0 + j * (NT / 32) < tl.nk;
            cp_async16(s0 + (uint32_t)(j * NT * 16), in ? src : p.S, in ? 16u : 0u);
            src += (long long)(NT / 32) * p.ld;
        }
    } else {
        const int col = tid & 15, row0 = tid >> 4;  // 16 units per 256-byte row
        const bool cin = col * 4 < tl.nk;
        const float *src = p.S + (long long)(tl.r0 + row0) * p.ld + tl.k0 + col * 4;
#pragma unroll
        for (int j = 0; j < J; ++j) {
            const bool in = cin && row0 + j * (NT / 16) < tl.nr;
            cp_async16(s0 + (uint32_t)(j * NT * 16), in ? src : p.S, in ? 16u : 0u);
            src += (long long)(NT / 16) * p.ld;
        }
    }
}

// Split one staged tile into the P-term packed image at `out`. The staged
// tile is zero outside the matrix, so only centring needs the extent.
template <int P, int NT, bool TF>
__device__ __forceinline__ void ps_split(const PsTile &tl, const float *stage, char *out, int tid) {
    const PackSrc &p = *tl.p;
    const bool centre = p.off_hi != nullptr;
    if (!p.trans) {
        // thread -> (row r, 16-byte chunk c); the two 16-byte halves of a chunk
        // are read in an order that keeps each quarter-warp on 32 banks
        const int c = tid & 7, h1 = (c >> 2) & 1;
#pragma unroll
        for (int pass = 0; pass < 1024 / NT; ++pass) {
            const int r = pass * (NT / 8) + (tid >> 3);
            const float4 *row = reinterpret_cast<const float4 *>(stage + r * PK_K);
            const float4 x = row[c * 2 + h1], y = row[c * 2 + (h1 ^ 1)];
            const float4 a = h1 ? y : x, b = h1 ? x : y;
            float v[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
            if (centre && r < tl.nr) {
                const float h = p.off_hi[tl.r0 + r], l = p.off_lo[tl.r0 + r];
#pragma unroll
                for (int q = 0; q < 8; ++q)
                    if (c * 8 + q < tl.nk) v[q] = (v[q] - h) - l;
            }
            store_chunk_fmt<P, TF>(out, r, c, v);
        }
    } else {
        // warp w builds chunk c = w % 8 of 32 consecutive rows per pass: each
        // scalar read is one 128-byte row segment of the staged [k][r] block
        const int lane = tid & 31, c = (tid >> 5) & 7, g = tid >> 8;
#pragma unroll
        for (int pass = 0; pass < 1024 / NT; ++pass) {
            const int r = (pass * (NT / 256) + g) * 32 + lane;
            float v[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) v[q] = stage[(c * 8 + q) * PK_ROWS + r];
            if (centre && r < tl.nr) {
                const float h = p.off_hi[tl.r0 + r], l = p.off_lo[tl.r0 + r];
#pragma unroll
                for (int q = 0; q < 8; ++q)
                    if (c * 8 + q < tl.nk) v[q] = (v[q] - h) - l;
            }
            store_chunk_fmt<P, TF>(out, r, c, v);
        }
    }
}

// Tiles cta, cta + ncta, ... of m. `smem` holds pack_stream_smem(ns, nout, P)
// bytes (16-byte aligned); ns in [2, PS_MAX_STAGES], nout 2 or 3. Threads >= NT
// must not call this. Every wait is on this thread's own copies (no flag
// written by another agent), so none can outlast the memory system.
// TF: the operands take TF32 blocks (PackSrc::tf32, the same for every operand of m).
template <int P, int NT, bool TF>
__device__ void pack_stream(const PackMulti &m, int cta, int ncta, unsigned char *smem, int ns, int nout) {
    const int tid = threadIdx.x;
    float *stages = reinterpret_cast<float *>(smem);
    char *outs = reinterpret_cast<char *>(smem + ns * PS_IN_BYTES);
    const int total = m.prefix[m.count];
    const int mine = total > cta ? (total - cta + ncta - 1) / ncta : 0;
    if (mine == 0) return;
    // the pack stream's kernel may be launched programmatically: global memory
    // only after the predecessor grid has completed
    pdl_wait();
    pdl_trigger();
    // one commit group per tile slot, empty past the end, so that "all but the
    // newest ns - 1 groups complete" always means "tile i has landed"
    for (int i = 0; i < ns - 1; ++i) {
        if (i < mine) ps_issue<NT>(ps_tile(m, cta + i * ncta, P), stages + i * (PS_IN_BYTES / 4), tid);
        cp_async_commit();
    }
    int so = 0, oo = 0;  // stage and output buffer of tile i
    for (int i = 0; i < mine; ++i) {
        const int ahead = i + ns - 1;
        if (ahead < mine) {
            const int sa = so == 0 ? ns - 1 : so - 1;  // (i + ns - 1) % ns
            ps_issue<NT>(ps_tile(m, cta + ahead * ncta, P), stages + sa * (PS_IN_BYTES / 4), tid);
        }
        cp_async_commit();
        switch (ns) {  // wait_group takes an immediate
            case 2: cp_async_wait<1>(); break;
            case 3: cp_async_wait<2>(); break;
            default: cp_async_wait<3>(); break;
        }
        named_sync(PS_BARRIER, NT);
        const PsTile tl = ps_tile(m, cta + i * ncta, P);
        char *out = outs + oo * P * PK_TILE_BYTES;
        ps_split<P, NT, TF>(tl, stages + so * (PS_IN_BYTES / 4), out, tid);
        fence_proxy_async_smem();
        // every thread is past the split: stage `so` may be refilled, and the
        // output buffer is complete
        named_sync(PS_BARRIER, NT);
        if (tid == 0) {
            bulk_s2g(tl.p->dst + tl.dst_off, saddr(out), (uint32_t)(P * PK_TILE_BYTES));
            bulk_commit();
            // the buffer that tile i + 1 writes last held tile i + 1 - nout, whose
            // store must have read it; the first barrier of the next iteration
            // publishes this wait to the other threads
            if (nout == 3) bulk_wait_read<2>();
            else bulk_wait_read<1>();
        }
        so = so + 1 == ns ? 0 : so + 1;
        oo = oo + 1 == nout ? 0 : oo + 1;
    }
    cp_async_wait<0>();
    if (tid == 0) bulk_wait<0>();
}

}  // namespace

}  // namespace ln
