// Instantiations of the tcgen05 contraction kernel (ln_umma_kernel.cuh) for
// general (non-symmetric) problems: packed-operand, E/F and alpha/beta
// epilogues; and the public entry points of the tcgen05 engine.
#include "ln_umma_kernel.cuh"

namespace ln {

namespace {

template <int P, int BN>
ln_status launch_single(int ek, const UmmaProblem &p, int total, cudaStream_t st, const PackMulti *side,
                        bool *side_done) {
    switch (ek) {
        case EK_PACK:
            return launch<P, BN, 0, EK_PACK>(&p, nullptr, nullptr, nullptr, total, nullptr, st, side, side_done);
        case EK_EF: return launch<P, BN, 0, EK_EF>(&p, nullptr, nullptr, nullptr, total, nullptr, st);
        default: return launch<P, BN, 0, EK_GEMM>(&p, nullptr, nullptr, nullptr, total, nullptr, st);
    }
}

int epi_kind(const EpiParams &e) {
    switch (e.mode) {
        case EPI_PACK: return EK_PACK;
        case EPI_EF: return EK_EF;
        case EPI_SYM: return EK_SYM;
        default: return EK_GEMM;
    }
}

}  // namespace

int umma_tile_n(int terms, int sym) { return (!sym && terms <= 2) ? tune_tile_n() : 128; }

ln_status umma_contract(const UmmaProblem &p, int terms, cudaStream_t st, const PackMulti *side, bool *side_done) {
    if (side_done) *side_done = false;
    long long tiles = p.sym ? (long long)p.mt * (p.mt + 1) / 2 : (long long)p.mt * p.nt;
    if (tiles == 0) return LN_SUCCESS;
    if (tiles > 0x7fffffffLL) return fail(LN_ERR_INVALID_VALUE, "too many output tiles");
    const int ek = epi_kind(p.epi);
    if (ek == EK_SYM) {
        if (!p.sym) return fail(LN_ERR_INVALID_VALUE, "symmetric epilogue needs a symmetric problem");
        return umma_contract_sym(p, terms, st);
    }
    if (p.sym) return fail(LN_ERR_INVALID_VALUE, "symmetric problem needs the symmetric epilogue");
    const int total = (int)tiles;
    const bool wide = umma_tile_n(terms, 0) == 256;
    switch (terms) {
        case 1:
            return wide ? launch_single<1, 256>(ek, p, total, st, side, side_done)
                        : launch_single<1, 128>(ek, p, total, st, side, side_done);
        case 2:
            return wide ? launch_single<2, 256>(ek, p, total, st, side, side_done)
                        : launch_single<2, 128>(ek, p, total, st, side, side_done);
        case 3: return launch_single<3, 128>(ek, p, total, st, side, side_done);
        default: return fail(LN_ERR_INVALID_VALUE, "unsupported split term count %d", terms);
    }
}

ln_status umma_read_error_general(int *value) {
    int v = 0, zero = 0;
    LN_CUDA_TRY(cudaMemcpyFromSymbol(&v, g_umma_error, sizeof(int)));
    if (v) LN_CUDA_TRY(cudaMemcpyToSymbol(g_umma_error, &zero, sizeof(int)));
    *value = v;
    return LN_SUCCESS;
}

ln_status umma_read_error(int *value) {
    int a = 0, b = 0;
    ln_status s = umma_read_error_general(&a);
    if (s != LN_SUCCESS) return s;
    s = umma_read_error_sym(&b);
    if (s != LN_SUCCESS) return s;
    *value = a | b;
    return LN_SUCCESS;
}

}  // namespace ln
