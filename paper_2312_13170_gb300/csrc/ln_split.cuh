// BF16 (and TF32) split of FP32 values into the packed tensor-core operand layout
// (shared by the split-and-pack kernels and the tcgen05 epilogue that writes
// a packed operand for the next contraction).
//
// Split: hi = bf16(x), lo = bf16(x - hi) and, for three terms,
// lo2 = bf16((x - hi) - lo), each rounded to nearest even. x - hi is exact in
// FP32, so x = hi + lo + O(2^-16 |x|) with two terms and O(2^-24 |x|) with three.
#pragma once

#include <cuda_bf16.h>

#include "ln_internal.h"

namespace ln {

// One cvt.rn.bf16x2.f32 rounds a pair (first value in the low half); a BF16
// value widened to FP32 is its 16 bits shifted to the top, so hi is recovered
// exactly with one shift or mask.
template <int P>
__device__ __forceinline__ void split8(const float *v, uint4 (&out)[P]) {
    uint32_t w[P][4];
#pragma unroll
    for (int q = 0; q < 8; q += 2) {
        float x0 = v[q], x1 = v[q + 1];
#pragma unroll
        for (int t = 0; t < P; ++t) {
            const __nv_bfloat162 h = __floats2bfloat162_rn(x0, x1);
            const uint32_t u = *reinterpret_cast<const uint32_t *>(&h);
            w[t][q / 2] = u;
            if (t + 1 < P) {
                x0 -= __uint_as_float(u << 16);
                x1 -= __uint_as_float(u & 0xffff0000u);
            }
        }
    }
#pragma unroll
    for (int t = 0; t < P; ++t) out[t] = make_uint4(w[t][0], w[t][1], w[t][2], w[t][3]);
}

// Split 8 consecutive k-values of row r (0..127) at 16-byte chunk c (0..7) of
// the tile whose term-0 block starts at tile0; term t lives t * 16 KiB later.
template <int P>
__device__ __forceinline__ void store_chunk(char *tile0, int r, int c, const float *v) {
    uint4 o[P];
    split8<P>(v, o);
    const int off = r * 128 + ((c ^ (r & 7)) << 4);
#pragma unroll
    for (int t = 0; t < P; ++t) *reinterpret_cast<uint4 *>(tile0 + (size_t)t * PK_TILE_BYTES + off) = o[t];
}

// TF32 split: hi = tf32(x), lo = tf32(x - hi), each rounded to nearest (ties
// away from zero) by cvt.rna.tf32.f32, whose result is an FP32 bit pattern
// with the low 13 mantissa bits zero; x - hi is exact in FP32, so
// x = hi + lo + O(2^-22 |x|) with two terms.
__device__ __forceinline__ uint32_t to_tf32(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

// The 8 values of 16-byte BF16 chunk c (k = 8c .. 8c + 7) of row r of a
// 128 x 64 block, as T TF32 terms: they fall in the block's 32-K tile h = c / 4
// (pieces h * T + term), TF32 chunks 2 (c % 4) and 2 (c % 4) + 1 of row r.
template <int T>
__device__ __forceinline__ void store_chunk_tf32(char *block0, int r, int c, const float *v) {
    uint32_t w[T][8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        float x = v[q];
#pragma unroll
        for (int t = 0; t < T; ++t) {
            const uint32_t u = to_tf32(x);
            w[t][q] = u;
            if (t + 1 < T) x -= __uint_as_float(u);
        }
    }
    const int h = c >> 2, c0 = (c & 3) * 2, sw = r & 7;
#pragma unroll
    for (int t = 0; t < T; ++t) {
        char *row = block0 + (size_t)(h * T + t) * PK_TILE_BYTES + r * 128;
        *reinterpret_cast<uint4 *>(row + ((c0 ^ sw) << 4)) = make_uint4(w[t][0], w[t][1], w[t][2], w[t][3]);
        *reinterpret_cast<uint4 *>(row + (((c0 + 1) ^ sw) << 4)) = make_uint4(w[t][4], w[t][5], w[t][6], w[t][7]);
    }
}

// store_chunk for a block of P pieces: P BF16 terms, or (TF) P / 2 TF32 terms
template <int P, bool TF>
__device__ __forceinline__ void store_chunk_fmt(char *block0, int r, int c, const float *v) {
    if constexpr (TF) {
        static_assert(P % 2 == 0, "a TF32 block has two pieces per term");
        store_chunk_tf32<P / 2>(block0, r, c, v);
    } else {
        store_chunk<P>(block0, r, c, v);
    }
}

}  // namespace ln
