// Instantiations of the tcgen05 contraction kernel (ln_umma_kernel.cuh) for
// TF32 operands on CTA pairs: clusters of two CTAs whose leader issues
// tcgen05.mma.cta_group::2.kind::tf32 (M = 256) over 256-wide general tiles,
// each CTA staging its own 128 rows of A and its 128-row half of B. A TF32
// k-tile (32 K, one or two terms of 16 KiB per 128-row block) has the bytes
// of a BF16 one, so the pair's copies and barriers are those of the BF16
// pairs; only the MMA kind differs. Kept apart from the BF16 pairs and the
// unpaired TF32 launches so that neither carries this code.
#include "ln_umma_kernel.cuh"

namespace ln {

namespace {

template <int P>
ln_status launch_tf32_pair(int ek, const UmmaProblem &p, int total, cudaStream_t st) {
    switch (ek) {
        case EK_PACK: return launch<P, 256, 0, EK_PACK, 1, 1>(&p, nullptr, nullptr, nullptr, total, nullptr, st);
        case EK_EF: return launch<P, 256, 0, EK_EF, 1, 1>(&p, nullptr, nullptr, nullptr, total, nullptr, st);
        default: return launch<P, 256, 0, EK_GEMM, 1, 1>(&p, nullptr, nullptr, nullptr, total, nullptr, st);
    }
}

}  // namespace

ln_status umma_contract_tf32_pair(int ek, const UmmaProblem &p, int terms, int total, cudaStream_t st) {
    switch (terms) {
        case 1: return launch_tf32_pair<1>(ek, p, total, st);
        case 2: return launch_tf32_pair<2>(ek, p, total, st);
        default: return fail(LN_ERR_INVALID_VALUE, "unsupported TF32 term count %d", terms);
    }
}

ln_status umma_read_error_tf32_pair(int *value) {
    int v = 0, zero = 0;
    LN_CUDA_TRY(cudaMemcpyFromSymbol(&v, g_umma_error, sizeof(int)));
    if (v) LN_CUDA_TRY(cudaMemcpyToSymbol(g_umma_error, &zero, sizeof(int)));
    *value = v;
    return LN_SUCCESS;
}

}  // namespace ln
