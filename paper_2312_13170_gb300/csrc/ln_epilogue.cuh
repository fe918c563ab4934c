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

// Two-phase form of epi_store for engines that finish several outputs per
// thread: epi_load fetches what the epilogue of (i, j) reads from memory, so a
// caller can issue the loads of many outputs before any of their stores;
// epi_apply then computes and stores exactly what epi_store would.
__device__ __forceinline__ float2 epi_load(const EpiParams &e, int i, int j) {
    float2 r = make_float2(0.0f, 0.0f);
    if (i >= e.M || j >= e.N) return r;
    switch (e.mode) {
        case EPI_GEMM:
            if (e.beta != 0.0f) r.x = e.C[(long long)i * e.ldc + j];
            break;
        case EPI_EF:
            if (e.beta != 0.0f) r.x = e.D[(long long)i * e.ld_ef + j];
            break;
        case EPI_SYM:
            if (i < j) break;
            if (e.sym_kind == SYM_CORR) {
                r.x = e.rs[i];
                r.y = e.rs[j];
            } else if (e.sym_kind == SYM_AXPBY && e.beta != 0.0f) {
                r.x = e.C[(e.fill == LN_FILL_UPPER) ? (long long)j * e.ldc + i : (long long)i * e.ldc + j];
            }
            break;
        default: break;
    }
    return r;
}

__device__ __forceinline__ void epi_apply(const EpiParams &e, int i, int j, float acc, float2 g) {
    if (i >= e.M || j >= e.N) return;
    switch (e.mode) {
        case EPI_GEMM: {
            float v = e.alpha * acc;
            if (e.beta != 0.0f) v = fmaf(e.beta, g.x, v);
            e.C[(long long)i * e.ldc + j] = v;
            break;
        }
        case EPI_STORE: e.C[(long long)i * e.ldc + j] = e.alpha * acc; break;
        case EPI_EF: {
            long long o = (long long)i * e.ld_ef + j;
            e.E[o] = acc;
            float v = e.alpha * acc;
            if (e.beta != 0.0f) v = fmaf(e.beta, g.x, v);
            e.F[o] = v;
            break;
        }
        default: {
            if (i < j) return;
            long long lo = (long long)i * e.ldc + j, up = (long long)j * e.ldc + i;
            if (e.sym_kind == SYM_CORR) {
                float v = (i == j) ? 1.0f : acc * g.x * g.y;
                e.C[lo] = v;
                e.C[up] = v;
            } else if (e.sym_kind == SYM_SCALE) {
                float v = e.alpha * acc;
                e.C[lo] = v;
                e.C[up] = v;
            } else {
                float v = e.alpha * acc;
                if (e.beta != 0.0f) v = fmaf(e.beta, g.x, v);
                if (e.fill == LN_FILL_FULL) {
                    e.C[lo] = v;
                    e.C[up] = v;
                } else {
                    e.C[(e.fill == LN_FILL_UPPER) ? up : lo] = v;
                }
            }
        }
    }
}

}  // namespace ln
