// Instantiations of the tcgen05 contraction kernel (ln_umma_kernel.cuh) for
// symmetric problems (covariance, correlation, SYRK/SYR2K): lower-triangle
// square tiles with mirrored stores, single and batched (device tile queue).
#include <algorithm>

#include "ln_umma_kernel.cuh"

namespace ln {

ln_status umma_contract_sym(const UmmaProblem &p0, int terms, cudaStream_t st) {
    UmmaProblem p = p0;
    p.pair = 0;
    const int bn = p.bn == 256 ? 256 : 128;
    if (bn == 256 && terms > 2) return fail(LN_ERR_INVALID_VALUE, "three split terms need 128-wide tiles");
    long long tiles = sym_tiles(p.mt, bn);
    if (tiles == 0) return LN_SUCCESS;
    if (p.streamk && p.ksplit > 1) return fail(LN_ERR_INVALID_VALUE, "stream-K and split-K together");
    if (p.ksplit > 1) {
        if (!p.kpart || !p.kcnt) return fail(LN_ERR_INVALID_VALUE, "split-K without its workspace");
        LN_CUDA_TRY(cudaMemsetAsync(p.kcnt, 0, umma_split_cnt_bytes(tiles, 128), st));
        tiles *= p.ksplit;
    } else if (bn == 128 && !p.tf32 && tune_pair() == 2 && !p.streamk && p.mt >= 2) {  // slower: opt-in
        // CTA pairs: row-tile pair q covers the column tiles 0 .. min(2q + 1, mt - 1)
        p.pair = 1;
        tiles = 0;
        for (long long q = 0; q < ceil_div(p.mt, 2); ++q) tiles += std::min<long long>(2 * q + 2, p.mt);
    }
    if (tiles > 0x7fffffffLL) return fail(LN_ERR_INVALID_VALUE, "too many output tiles");
    const int total = (int)tiles;
    if (p.tf32) return umma_contract_sym_tf32(p, terms, bn, total, st);
    if (p.pair) return umma_contract_sym_pair(p, terms, total, st);
    if (bn == 256) {  // 128 x 256 lower-triangle tiles (deep problems with stream-K)
        switch (terms) {
            case 1: return launch<1, 256, 0, EK_SYM>(&p, nullptr, nullptr, nullptr, total, nullptr, st);
            case 2: return launch<2, 256, 0, EK_SYM>(&p, nullptr, nullptr, nullptr, total, nullptr, st);
            default: return fail(LN_ERR_INVALID_VALUE, "unsupported split term count %d", terms);
        }
    }
    switch (terms) {
        case 1: return launch<1, 128, 0, EK_SYM>(&p, nullptr, nullptr, nullptr, total, nullptr, st);
        case 2: return launch<2, 128, 0, EK_SYM>(&p, nullptr, nullptr, nullptr, total, nullptr, st);
        case 3: return launch<3, 128, 0, EK_SYM>(&p, nullptr, nullptr, nullptr, total, nullptr, st);
        default: return fail(LN_ERR_INVALID_VALUE, "unsupported split term count %d", terms);
    }
}

ln_status umma_contract_batched(const UmmaProblem *d_probs, const int *d_tile_prefix, const int *d_tile_owner,
                                int total_tiles, int *d_queue, int terms, int tf32, cudaStream_t st) {
    if (total_tiles == 0) return LN_SUCCESS;
    LN_CUDA_TRY(cudaMemsetAsync(d_queue, 0, sizeof(int), st));
    if (tf32) return umma_contract_batched_tf32(d_probs, d_tile_prefix, d_tile_owner, total_tiles, d_queue, terms, st);
    switch (terms) {
        case 1: return launch<1, 128, 1, EK_SYM>(nullptr, d_probs, d_tile_prefix, d_tile_owner, total_tiles, d_queue, st);
        case 2: return launch<2, 128, 1, EK_SYM>(nullptr, d_probs, d_tile_prefix, d_tile_owner, total_tiles, d_queue, st);
        case 3: return launch<3, 128, 1, EK_SYM>(nullptr, d_probs, d_tile_prefix, d_tile_owner, total_tiles, d_queue, st);
        default: return fail(LN_ERR_INVALID_VALUE, "unsupported split term count %d", terms);
    }
}

ln_status umma_read_error_sym(int *value) {
    int v = 0, zero = 0;
    LN_CUDA_TRY(cudaMemcpyFromSymbol(&v, g_umma_error, sizeof(int)));
    if (v) LN_CUDA_TRY(cudaMemcpyToSymbol(g_umma_error, &zero, sizeof(int)));
    *value = v;
    return LN_SUCCESS;
}

}  // namespace ln
