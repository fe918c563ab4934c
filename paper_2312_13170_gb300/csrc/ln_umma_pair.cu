// Instantiations of the tcgen05 contraction kernel (ln_umma_kernel.cuh) for
// CTA pairs: clusters of two CTAs whose leader issues tcgen05.mma.cta_group::2
// (M = 256), general and symmetric problems.
#include "ln_umma_kernel.cuh"

namespace ln {

namespace {

template <int P, int BN>
ln_status launch_pair(int ek, const UmmaProblem &p, int total, cudaStream_t st, const PackMulti *side,
                      bool *side_done) {
    switch (ek) {
        case EK_PACK:
            return launch<P, BN, 0, EK_PACK, 1>(&p, nullptr, nullptr, nullptr, total, nullptr, st, side, side_done);
        case EK_EF: return launch<P, BN, 0, EK_EF, 1>(&p, nullptr, nullptr, nullptr, total, nullptr, st);
        default: return launch<P, BN, 0, EK_GEMM, 1>(&p, nullptr, nullptr, nullptr, total, nullptr, st);
    }
}

}  // namespace

ln_status umma_contract_pair(int ek, const UmmaProblem &p, int terms, int bn, int total, cudaStream_t st,
                             const PackMulti *side, bool *side_done) {
    const bool wide = bn == 256;
    switch (terms) {
        case 1:
            return wide ? launch_pair<1, 256>(ek, p, total, st, side, side_done)
                        : launch_pair<1, 128>(ek, p, total, st, side, side_done);
        case 2:
            return wide ? launch_pair<2, 256>(ek, p, total, st, side, side_done)
                        : launch_pair<2, 128>(ek, p, total, st, side, side_done);
        case 3: return launch_pair<3, 128>(ek, p, total, st, side, side_done);
        default: return fail(LN_ERR_INVALID_VALUE, "unsupported split term count %d", terms);
    }
}

ln_status umma_contract_sym_pair(const UmmaProblem &p, int terms, int total, cudaStream_t st) {
    switch (terms) {
        case 1: return launch<1, 128, 0, EK_SYM, 1>(&p, nullptr, nullptr, nullptr, total, nullptr, st);
        case 2: return launch<2, 128, 0, EK_SYM, 1>(&p, nullptr, nullptr, nullptr, total, nullptr, st);
        case 3: return launch<3, 128, 0, EK_SYM, 1>(&p, nullptr, nullptr, nullptr, total, nullptr, st);
        default: return fail(LN_ERR_INVALID_VALUE, "unsupported split term count %d", terms);
    }
}

ln_status umma_read_error_pair(int *value) {
    int v = 0, zero = 0;
    LN_CUDA_TRY(cudaMemcpyFromSymbol(&v, g_umma_error, sizeof(int)));
    if (v) LN_CUDA_TRY(cudaMemcpyToSymbol(g_umma_error, &zero, sizeof(int)));
    *value = v;
    return LN_SUCCESS;
}

}  // namespace ln
