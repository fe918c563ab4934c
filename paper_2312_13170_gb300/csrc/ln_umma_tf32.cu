// Instantiations of the tcgen05 contraction kernel (ln_umma_kernel.cuh) for
// TF32 operands (tcgen05.mma kind::tf32, LN_PREC_TF32 and LN_PREC_3XTF32):
// general, symmetric and batched problems with one or two TF32 terms, single
// CTAs (no CTA pairs, no spare-CTA packing). Kept apart from the BF16
// instantiations so that those carry no TF32 code.
#include "ln_umma_kernel.cuh"

namespace ln {

namespace {

template <int P, int BN>
ln_status launch_tf32(int ek, const UmmaProblem &p, int total, cudaStream_t st) {
    switch (ek) {
        case EK_PACK: return launch<P, BN, 0, EK_PACK, 0, 1>(&p, nullptr, nullptr, nullptr, total, nullptr, st);
        case EK_EF: return launch<P, BN, 0, EK_EF, 0, 1>(&p, nullptr, nullptr, nullptr, total, nullptr, st);
        default: return launch<P, BN, 0, EK_GEMM, 0, 1>(&p, nullptr, nullptr, nullptr, total, nullptr, st);
    }
}

}  // namespace

ln_status umma_contract_tf32(int ek, const UmmaProblem &p, int terms, int bn, int total, cudaStream_t st) {
    if (bn != 128 && bn != 256) return fail(LN_ERR_INVALID_VALUE, "tile width %d", bn);
    switch (terms) {
        case 1: return bn == 256 ? launch_tf32<1, 256>(ek, p, total, st) : launch_tf32<1, 128>(ek, p, total, st);
        case 2: return bn == 256 ? launch_tf32<2, 256>(ek, p, total, st) : launch_tf32<2, 128>(ek, p, total, st);
        default: return fail(LN_ERR_INVALID_VALUE, "unsupported TF32 term count %d", terms);
    }
}

ln_status umma_contract_sym_tf32(const UmmaProblem &p, int terms, int bn, int total, cudaStream_t st) {
    if (bn == 256) {
        switch (terms) {
            case 1: return launch<1, 256, 0, EK_SYM, 0, 1>(&p, nullptr, nullptr, nullptr, total, nullptr, st);
            case 2: return launch<2, 256, 0, EK_SYM, 0, 1>(&p, nullptr, nullptr, nullptr, total, nullptr, st);
            default: return fail(LN_ERR_INVALID_VALUE, "unsupported TF32 term count %d", terms);
        }
    }
    switch (terms) {
        case 1: return launch<1, 128, 0, EK_SYM, 0, 1>(&p, nullptr, nullptr, nullptr, total, nullptr, st);
        case 2: return launch<2, 128, 0, EK_SYM, 0, 1>(&p, nullptr, nullptr, nullptr, total, nullptr, st);
        default: return fail(LN_ERR_INVALID_VALUE, "unsupported TF32 term count %d", terms);
    }
}

ln_status umma_contract_batched_tf32(const UmmaProblem *d_probs, const int *d_tile_prefix, const int *d_tile_owner,
                                     int total_tiles, int *d_queue, int terms, cudaStream_t st) {
    switch (terms) {
        case 1:
            return launch<1, 128, 1, EK_SYM, 0, 1>(nullptr, d_probs, d_tile_prefix, d_tile_owner, total_tiles, d_queue,
                                                   st);
        case 2:
            return launch<2, 128, 1, EK_SYM, 0, 1>(nullptr, d_probs, d_tile_prefix, d_tile_owner, total_tiles, d_queue,
                                                   st);
        default: return fail(LN_ERR_INVALID_VALUE, "unsupported TF32 term count %d", terms);
    }
}

ln_status umma_read_error_tf32(int *value) {
    int v = 0, zero = 0;
    LN_CUDA_TRY(cudaMemcpyFromSymbol(&v, g_umma_error, sizeof(int)));
    if (v) LN_CUDA_TRY(cudaMemcpyToSymbol(g_umma_error, &zero, sizeof(int)));
    *value = v;
    return LN_SUCCESS;
}

}  // namespace ln
