// Element-wise epilogue shared by the plain, FP32 SIMT and tcgen05 engines.
// The accumulated value of output (i, j) is written exactly once here (the
// single store after the loop that array-reduction detection produces,
// paper Sec. VI-B).
#pragma once

#include "ln_internal.h"

namespace ln {

__device__ __forceinline__ void epi_store(const EpiParams &e, int i, int j, float acc) {
    if (i >= e.M || j >= e.N) return;
    switch (e.mode) {
        case EPI_GEMM: {
            float *c = e.C + (long long)i * e.ldc + j;
            float v = e.alpha * acc;
            if (e.beta != 0.0f) v = fmaf(e.beta, *c, v);
            *c = v;
            break;
        }
        case EPI_STORE: e.C[(long long)i * e.ldc + j] = e.alpha * acc; break;
        case EPI_EF: {
            long long o = (long long)i * e.ld_ef + j;
            e.E[o] = acc;
            float v = e.alpha * acc;
            if (e.beta != 0.0f) v = fmaf(e.beta, e.D[o], v);
            e.F[o] = v;
            break;
        }
        default: {  // EPI_SYM: produced for i >= j only
            if (i < j) return;
            long long lo = (long long)i * e.ldc + j, up = (long long)j * e.ldc + i;
            if (e.sym_kind == SYM_CORR) {
                float v = (i == j) ? 1.0f : acc * e.rs[i] * e.rs[j];
                e.C[lo] = v;
                e.C[up] = v;
            } else if (e.sym_kind == SYM_SCALE) {
                float v = e.alpha * acc;
                e.C[lo] = v;
                e.C[up] = v;
            } else {
                long long src = (e.fill == LN_FILL_UPPER) ? up : lo;
                float v = e.alpha * acc;
                if (e.beta != 0.0f) v = fmaf(e.beta, e.C[src], v);
                if (e.fill == LN_FILL_FULL) {
                    e.C[lo] = v;
                    e.C[up] = v;
                } else {
                    e.C[src] = v;
                }
            }
        }
    }
}

}  // namespace ln
