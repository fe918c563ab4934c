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

int umma_tile_n(int terms, int sym, long long M, long long N) {
    if (sym || terms == 3) return 128;  // terms: BF16 split terms, or pieces per TF32 block (2, 4)
    const int knob = tune_tile_n();
    if (knob == 128 || knob == 256) return knob;
    const long long wide_tiles = ceil_div(M, 128) * ceil_div(N, 256);
    return 2 * wide_tiles <= sm_count() ? 128 : 256;
}

int umma_sym_tile_n(int terms, long long mt, int ktot) {
    const int knob = tune_sym_wide();
    if (terms == 3 || mt < 2 || knob == 0) return 128;
    if (knob == 1) return 256;
    return umma_streamk(sym_tiles(mt, 256), ktot) ? 256 : 128;
}

int umma_ksplit(long long tiles, int ktot) {
    const int sms = sm_count();
    if (!tune_split_k() || tiles <= 0 || ktot < 8 || 2 * tiles > sms) return 1;
    long long ks = sms / tiles;  // slices per tile that the SMs hold at once
    if (ks > ktot / 4) ks = ktot / 4;
    if (ks > 16) ks = 16;
    if (ks < 2) return 1;
    const int per = (int)((ktot + ks - 1) / ks);
    return (ktot + per - 1) / per;  // no empty slice
}

size_t umma_split_part_bytes(long long tiles, int ksplit, int bn) {
    return ksplit > 1 ? (size_t)tiles * ksplit * (bn / 32) * 4096 * sizeof(float) : 0;
}

// one counter per (tile, epilogue warp); every configuration has at most 8
// epilogue warps (Cfg::NEPI)
size_t umma_split_cnt_bytes(long long tiles, int) { return (size_t)tiles * 8 * sizeof(int); }

int umma_streamk(long long tiles, int ktot) {
    const int sms = sm_count();
    const int knob = tune_stream_k();
    if (!knob || tiles <= 0 || tiles >= sms) return 0;
    // automatic (2): only deep contractions that fill at most half the SMs,
    // where the idle SMs outweigh the partial-sum hand-off
    if (knob == 2 && (2 * tiles > sms || ktot < 32)) return 0;
    return tiles * ktot >= 4LL * sms ? 1 : 0;
}

// one FP32 output tile (128 x bn) of partial sums per CTA
size_t umma_streamk_part_bytes(int bn) { return (size_t)sm_count() * 128 * bn * sizeof(float); }
size_t umma_streamk_flag_bytes() { return (size_t)sm_count() * 8 * sizeof(int); }

ln_status umma_contract(const UmmaProblem &p0, int terms, cudaStream_t st, const PackMulti *side, bool *side_done) {
    if (side_done) *side_done = false;
    UmmaProblem p = p0;
    p.pair = 0;
    p.stage_beta = tune_stage_beta();
    p.stage_out = tune_stage_out();
    if (p.tf32) {
        // TF32 operands: `terms` counts the 16 KiB pieces of a 128 x 64 block
        // (two per TF32 term) and the k-tile counts are in such blocks; the
        // kernel takes the TF32 terms and 32-K tiles. The spare CTAs' pack
        // stream writes BF16 blocks only, so the caller packs a side operand.
        if (terms != 2 && terms != 4) return fail(LN_ERR_INVALID_VALUE, "TF32 operand with %d pieces", terms);
        terms /= 2;
        p.kt *= 2;
        p.x_kt *= 2;
        p.y_kt *= 2;
        side = nullptr;
    }
    long long tiles = p.sym ? (long long)p.mt * (p.mt + 1) / 2 : (long long)p.mt * p.nt;
    if (tiles == 0) return LN_SUCCESS;
    if (tiles > 0x7fffffffLL) return fail(LN_ERR_INVALID_VALUE, "too many output tiles");
    const int ek = epi_kind(p.epi);
    if (ek == EK_SYM) {
        if (!p.sym) return fail(LN_ERR_INVALID_VALUE, "symmetric epilogue needs a symmetric problem");
        return umma_contract_sym(p, terms, st);
    }
    if (p.sym) return fail(LN_ERR_INVALID_VALUE, "symmetric problem needs the symmetric epilogue");
    if (p.streamk && p.ksplit > 1) return fail(LN_ERR_INVALID_VALUE, "stream-K and split-K together");
    if (p.ksplit > 1) {
        if (!p.kpart || !p.kcnt) return fail(LN_ERR_INVALID_VALUE, "split-K without its workspace");
        tiles *= p.ksplit;
        LN_CUDA_TRY(cudaMemsetAsync(p.kcnt, 0, umma_split_cnt_bytes(tiles / p.ksplit, 0), st));
    }
    if (tiles > 0x7fffffffLL) return fail(LN_ERR_INVALID_VALUE, "too many work items");
    // CTA pairs over vertically adjacent tiles ("pair" knob 1: 256-wide tiles of
    // split operands, where they measured faster; with one term a stage holds
    // one product's MMAs, too few to cover the pair's per-stage hand-off;
    // 2: every width and term count, TF32 operands still 256-wide only):
    // `total` counts pair tiles
    const int bn_pair = p.bn > 0 ? p.bn : umma_tile_n(terms, 0, p.epi.M, p.epi.N);
    const bool pair_auto = tune_pair() == 1 && bn_pair == 256 && terms >= 2;
    const bool pair_width = p.tf32 ? bn_pair == 256 && (tune_pair() == 2 || pair_auto)
                                   : tune_pair() == 2 || pair_auto;
    if (pair_width && p.ksplit <= 1 && !p.streamk && p.mt >= 2) {
        p.pair = 1;
        tiles = ceil_div(p.mt, 2) * p.nt;
    }
    const int total = (int)tiles;
    const int bn = p.bn > 0 ? p.bn : umma_tile_n(terms, 0, p.epi.M, p.epi.N);
    if (bn != 128 && bn != 256) return fail(LN_ERR_INVALID_VALUE, "tile width %d", bn);
    if (terms > 2 && bn != 128) return fail(LN_ERR_INVALID_VALUE, "three split terms need 128-wide tiles");
    const bool wide = bn == 256;
    if (p.tf32)
        return p.pair ? umma_contract_tf32_pair(ek, p, terms, total, st) : umma_contract_tf32(ek, p, terms, bn, total, st);
    if (p.pair) return umma_contract_pair(ek, p, terms, bn, total, st, side, side_done);
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
    int a = 0, b = 0, c = 0, d = 0, e = 0;
    ln_status s = umma_read_error_general(&a);
    if (s != LN_SUCCESS) return s;
    s = umma_read_error_sym(&b);
    if (s != LN_SUCCESS) return s;
    s = umma_read_error_pair(&c);
    if (s != LN_SUCCESS) return s;
    s = umma_read_error_tf32(&d);
    if (s != LN_SUCCESS) return s;
    s = umma_read_error_tf32_pair(&e);
    if (s != LN_SUCCESS) return s;
    *value = a | b | c | d | e;
    return LN_SUCCESS;
}

}  // namespace ln
