// BF16 split of FP32 values into the packed tensor-core operand layout
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

}  // namespace ln
