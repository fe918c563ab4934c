// Internal declarations of libloopnest: error reporting, the epilogue
// description shared by every contraction engine, the packed tensor-core
// operand format, and the host-side launchers of each translation unit.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <initializer_list>

#include "loopnest.h"

namespace ln {

// ------------------------------------------------------------------ errors
ln_status fail(ln_status s, const char *fmt, ...);
void clear_error();

#define LN_CUDA_TRY(expr)                                                                     \
    do {                                                                                      \
        cudaError_t e_ = (expr);                                                              \
        if (e_ != cudaSuccess) return ::ln::fail(LN_ERR_CUDA, "%s: %s", #expr, cudaGetErrorString(e_)); \
    } while (0)

// Check for a launch error right after <<<>>>.
ln_status check_launch(const char *what);

// Every size argument of the C ABI lies in [0, MAX_DIM]; LN_ERR_INVALID_VALUE
// with a message otherwise.
constexpr long long MAX_DIM = 1 << 22;
ln_status check_dims(std::initializer_list<long long> dims);

// Launch accounting (ln_launch_count / ln_timing_*): construct one of these
// right before a kernel launch; it counts the launch and, while timing is
// enabled, records start/stop events around it on the launch stream.
enum Family : int { FAM_UMMA = 0, FAM_PACK, FAM_SIMT, FAM_PLAIN, FAM_STATS, FAM_COUNT };
struct LaunchScope {
    LaunchScope(Family f, cudaStream_t st);
    ~LaunchScope();
    int slot;
    cudaStream_t st;
    Family f;
};

int sm_count();

// ------------------------------------------------------------------ epilogue
// What a contraction engine does with the accumulated value acc(i, j) of the
// logical output element (i, j). Every engine (plain, FP32 SIMT, tcgen05)
// funnels its results through the same description, so the three forms agree
// on alpha/beta, fill and scaling semantics by construction.
enum EpiMode : int {
    EPI_GEMM = 0,  // C[i][j] = alpha*acc + beta*C[i][j]
    EPI_EF = 1,    // E[i][j] = acc; F[i][j] = alpha*acc + beta*D[i][j]
    EPI_SYM = 2,   // symmetric output, see SymKind; only i >= j is produced
    EPI_STORE = 3, // C[i][j] = alpha*acc (no read of C)
    EPI_PACK = 4   // tcgen05 engine only: acc written as split BF16 terms into a packed
                   // operand (rows = i, K = j) for the next contraction
};
enum SymKind : int {
    SYM_AXPBY = 0,  // alpha*acc + beta*C on the requested fill (SYRK/SYR2K)
    SYM_SCALE = 1,  // alpha*acc, full matrix written (covariance, alpha = 1/(n-1))
    SYM_CORR = 2    // acc*rs[i]*rs[j] for i != j, 1 on the diagonal, full matrix
};

struct EpiParams {
    int mode;
    int M, N;  // logical output extent
    float alpha, beta;
    float *C;
    long long ldc;
    const float *D;
    float *E, *F;
    long long ld_ef;
    int fill;      // ln_fill, for EPI_SYM
    int sym_kind;  // SymKind
    const float *rs;
    char *pack;    // EPI_PACK destination and its k-tile pitch
    int pack_kt;
};

// ------------------------------------------------------------------ packed tensor-core operands
// A packed operand holds a logical matrix R (rows x K) as tiles of 128 rows by
// 64 K-elements, each tile one 16 KiB block per BF16 split term, laid out the
// way tcgen05.mma reads a K-major operand with 128-byte swizzling:
//   tile (rt, kt, term) at byte ((rt * KT + kt) * P + term) * 16384,
//   element (r, k) of the tile in row r, 16-byte chunk c = k / 8, stored at
//   chunk position c ^ (r % 8) of that row (128 bytes per row).
// Rows >= rows and k >= K are zero. Because the layout in global memory is the
// layout in shared memory, one bulk copy moves a tile (no tensor map needed).
// TF32 operands (PackSrc::tf32) keep the same 128 x 64 blocks, each holding two
// 32-K tiles of T TF32 terms (P = 2T 16 KiB pieces per block): piece h * T +
// term of block (rt, kt) is 32-K tile 2 kt + h, element (r, k) in 16-byte chunk
// (k mod 32) / 4 of row r at chunk position c ^ (r % 8). So the tiles of a
// TF32 operand are, in order, exactly those of a BF16 operand with 32-K tiles:
// tile (rt, j, term) at ((rt * 2KT + j) * T + term) * 16384.
constexpr int PK_ROWS = 128;
constexpr int PK_K = 64;
constexpr int PK_TILE_BYTES = PK_ROWS * PK_K * 2;

inline long long ceil_div(long long a, long long b) { return (a + b - 1) / b; }
inline size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// 16 KiB pieces per 128 x 64 block of a packed operand (BF16: the split terms;
// TF32: twice the terms, the block holding two 32-K tiles)
inline int prec_terms(ln_precision p) {
    switch (p) {
        case LN_PREC_BF16: return 1;
        case LN_PREC_3XBF16: return 2;
        case LN_PREC_6XBF16: return 3;
        case LN_PREC_TF32: return 2;
        case LN_PREC_3XTF32: return 4;
        default: return 0;
    }
}
inline bool is_tf32(ln_precision p) { return p == LN_PREC_TF32 || p == LN_PREC_3XTF32; }
// split terms the tensor-core products take (the kernel's P)
inline int mma_terms(ln_precision p) { return is_tf32(p) ? prec_terms(p) / 2 : prec_terms(p); }

// bytes of a packed operand with `rt` row tiles and `kt` k tiles
inline size_t packed_bytes(long long rt, long long kt, int terms) {
    return (size_t)(rt * kt * terms) * PK_TILE_BYTES;
}

struct PackSrc {
    const float *S;  // source matrix
    long long ld;
    int trans;       // 0: element (r,k) = S[r*ld+k]; 1: element (r,k) = S[k*ld+r]
    int rows, K;     // logical extent
    const float *off_hi, *off_lo;  // optional per-row centring, v = (x - hi) - lo
    char *dst;       // packed destination
    int rt, kt;      // tile counts of the destination (>= ceil(rows/128), ceil(K/64))
    int tf32;        // TF32 terms (the TF32 block layout above) instead of BF16
};

// Up to four operands packed by one launch: a flat tile index space, operand i
// owning tiles [prefix[i], prefix[i+1]).
struct PackMulti {
    PackSrc op[4];
    int prefix[5];
    int count;
};

// ------------------------------------------------------------------ launchers (one per .cu)
// ln_plain.cu
ln_status plain_gemm(int M, int N, int K, const float *A, long long sai, long long sak, const float *B,
                     long long sbk, long long sbj, const EpiParams &epi, cudaStream_t st);
ln_status plain_col_stats(int n, int m, const float *X, long long ldx, double *mean, double *ss, cudaStream_t st);
ln_status plain_cov(int n, int m, const float *X, long long ldx, const double *mean, const EpiParams &epi,
                    cudaStream_t st);
ln_status plain_sym(int n, int k, const float *A, long long lda, const float *B, long long ldb,
                    const EpiParams &epi, cudaStream_t st);

// ln_simt.cu: FP32 shared-memory tiled contraction
//   acc(i,j) = sum_seg sum_k opA_seg(i,k) * opB_seg(k,j)
//   opA(i,k) = A[i*lda+k] (a_t == 0, A is M x K) or A[k*lda+i] (a_t == 1), minus a_off[i]
//   opB(k,j) = B[k*ldb+j] (b_t == 0, B is K x N) or B[j*ldb+k] (b_t == 1), minus b_off[j]
struct SimtOperands {
    const float *A[2];
    const float *B[2];
    long long lda[2], ldb[2];  // per segment
    int a_t, b_t;
    int nseg;
    const float *a_off_hi, *a_off_lo, *b_off_hi, *b_off_lo;
};
ln_status simt_contract(int M, int N, int K, const SimtOperands &op, const EpiParams &epi, cudaStream_t st);

// ln_stats.cu
// Two-pass column statistics; also writes the centring split (hi, lo) of the
// mean and rs = 1/sqrt(ss) as floats when those pointers are non-null.
ln_status col_stats(int n, int m, const float *X, long long ldx, double *mean, double *ss, float *off_hi,
                    float *off_lo, float *rs, double *partials, cudaStream_t st);
size_t col_stats_partials_bytes(int n, int m);
ln_status stats_derive(int m, const double *mean, const double *ss, float *off_hi, float *off_lo, float *rs,
                       cudaStream_t st);
ln_status scale_matrix(int M, int N, float beta, float *C, long long ldc, cudaStream_t st);
ln_status sym_fill_zero_k(int n, int fill, float beta, float *C, long long ldc, cudaStream_t st);
ln_status center_matrix(int n, int m, const float *X, long long ldx, const float *off_hi, const float *off_lo,
                        const float *rs, float *Y, long long ldy, cudaStream_t st);
ln_status symmetrize_weights(int m, const float *W, long long ldw, float scale, int zero_diag, float *Ws,
                             cudaStream_t st);
ln_status corr_bwd_finish(int n, int m, const float *Z, long long ldz, const float *dZ, long long lddz,
                          const float *rs, float *dX, long long lddx, double *partials, cudaStream_t st);
size_t corr_bwd_partials_bytes(int n, int m);

// ln_pack.cu
ln_status pack_operand(const PackSrc &p, int terms, cudaStream_t st);
// Packs up to four operands in one launch.
ln_status pack_operands(const PackSrc *ps, int count, int terms, cudaStream_t st);
// Fills m for pack_operands' operands; false if count is out of range or the
// tile count overflows.
bool make_pack_multi(const PackSrc *ps, int count, PackMulti &m);
// True if the bulk-copy pack stream can read every operand of m (16-byte
// aligned rows of a whole number of 16-byte units).
bool pack_stream_eligible(const PackMulti &m);
// Process-wide tuning knobs (ln_set_tuning): k tiles per TMEM accumulation
// chunk of the tcgen05 engine (1 or 2; default 2) and the output tile width of
// general tcgen05 contractions (128 or 256; default 256, three-term splits
// always 128).
int tune_chunk_kt();
int tune_tile_n();
int tune_pack_threads();  // threads per CTA of the split-and-pack stream (512 or 1024)
int tune_split_k();       // 1: split the K range of contractions with few output tiles
int tune_stream_k();      // 1: stream-K for general contractions with fewer tiles than SMs
int tune_pair();          // 1: CTA pairs sharing the column operand (UmmaProblem::pair)
int tune_stage_beta();    // UmmaProblem::stage_beta
int tune_stage_out();     // UmmaProblem::stage_out
int tune_sym_wide();      // umma_sym_tile_n: 0 never, 1 always, 2 automatic

// ln_umma.cu: tcgen05 contraction over packed operands
struct UmmaSeg {
    const char *X;  // packed M-side operand (row tiles of 128)
    const char *Y;  // packed N-side operand (row tiles of 128)
};
struct UmmaProblem {
    UmmaSeg seg[2];
    int nseg;
    int kt;          // k tiles per segment
    int x_kt, y_kt;  // k-tile pitch of the packed X and Y buffers
    int mt, nt;      // 128-row tiles on the M side, BN-wide tiles on the N side
    int sym;         // lower-triangle tiles only (mt == nt)
    int chunk_kt;    // k tiles accumulated in TMEM before the partial sum is added (in FP32
                     // registers) to the running sum; <= 0 means the whole reduction
    int inject_timeout;  // test hook: the producer issues no copy, so a bounded wait runs out
    // split-K (single problems only; <= 1 means none): work item t is output tile
    // t / ksplit, k slice t % ksplit (a contiguous range of the nseg * kt k tiles).
    // Every slice's epilogue warp stores its FP32 partial sums to kpart
    // ([tile][slice][epilogue warp][4096]) and counts its arrival in kcnt
    // ([tile][epilogue warp], zero at launch); the last to arrive adds the slices
    // in slice order and runs the epilogue.
    int ksplit;
    float *kpart;
    int *kcnt;
    int bn;  // output tile width chosen at planning (umma_tile_n); 0: derive from epi.M, epi.N
    // stream-K (single non-symmetric problems; 0: off): the tiles x (nseg * kt)
    // k-tile units are split evenly over one CTA per SM. A CTA whose range starts
    // inside a tile stores that segment's FP32 sums in skpart ([CTA][epilogue
    // warp][EPW * 32]) and sets skflag[CTA][epilogue warp] (zero before the
    // launch); the CTA holding the tile's first k tile adds them in k order and
    // runs the epilogue.
    int streamk;
    float *skpart;
    int *skflag;
    // CTA pairs (set by umma_contract / umma_contract_sym for single problems
    // with at least two row tiles): the launch is clusters of two CTAs that
    // compute vertically adjacent output tiles (row tiles 2p and 2p + 1, the
    // same column tile) with tcgen05.mma.cta_group::2: the leader issues M = 256
    // MMAs, each CTA holds its own 128 rows of A and half of the column tile's
    // B, so each SM stages and reads half as much of B.
    short pair;
    // the "stage_beta" knob: a CTA's last 256-wide tile may stage its block of
    // the beta input (D or C) in the stage memory after the mainloop
    short stage_beta;
    // TF32 operands: tcgen05.mma kind::tf32, 32-K tiles. The host sets it with
    // k-tile counts in 64-K blocks; umma_contract doubles them (and halves the
    // term count) before the launch. A packing epilogue writes TF32 blocks.
    // (the flags are short so that the problem keeps the size and layout the
    // epilogue registers were tuned with: a larger struct moved registers into
    // spills in the E/F epilogue)
    short tf32;
    // the "stage_out" knob: a CTA's last 256-wide tile with the packing
    // epilogue builds its packed output in the freed stage memory and writes it
    // with bulk copies
    short stage_out;
    EpiParams epi;
};
// True when LN_FAULT_INJECT=timeout is set in the environment (read per call).
bool inject_timeout_requested();
// Output tile width the engine uses for an M x N output: symmetric problems
// and three split terms use square 128 tiles; otherwise the "tile_n" knob if
// set (128 or 256), else 256 unless 256-wide tiles would fill at most half the
// SMs (then 128: twice the tiles, half the reduction per tile). `nt` of a
// problem counts tiles of this width, and the packed N-side operand must hold
// 128 * (width / 128) * nt rows (zero padded).
int umma_tile_n(int terms, int sym, long long M, long long N);
// Tile width of a symmetric problem with `mt` 128-row tiles and `ktot` k tiles
// (64-K blocks): 256 (tiles of 128 x 256 over the lower triangle) where the
// "sym_wide" knob allows it -- by default where those tiles fill at most half
// the SMs and take stream-K -- else 128. Three split terms always take 128.
int umma_sym_tile_n(int terms, long long mt, int ktot);
// Lower-triangle output tiles of a symmetric problem at tile width bn; 256-wide
// tiles read the packed operand as sym_packed_rt(mt, bn) 128-row tiles (an even
// count, the last one zero).
inline long long sym_tiles(long long mt, int bn) {
    if (bn != 256) return mt * (mt + 1) / 2;
    const long long q = mt / 2;
    return (mt % 2) ? (q + 1) * (q + 1) : q * (q + 1);
}
inline int sym_packed_rt(int mt, int bn) { return bn == 256 ? (mt + 1) / 2 * 2 : mt; }
// Split-K slices for a single problem with `tiles` output tiles and `ktot`
// k tiles (segments x k tiles): enough to fill the SMs, at least four k tiles
// each, none empty; 1 when the tiles already fill the GPU or the "split_k"
// knob is off (its default: the slices' FP32 partials, a burst of fresh
// writes through L2, cost more than the idle SMs save on GB300).
int umma_ksplit(long long tiles, int ktot);
// Workspace of a split: partial sums and arrival counters (bytes, each
// 256-aligned in the plan).
size_t umma_split_part_bytes(long long tiles, int ksplit, int bn);
size_t umma_split_cnt_bytes(long long tiles, int bn);
// Stream-K for a single general contraction of `tiles` output tiles of width bn
// and `ktot` k tiles: 1 when the tiles leave SMs idle (fewer tiles than SMs),
// every CTA gets at least four k tiles and the "stream_k" knob is on.
int umma_streamk(long long tiles, int ktot);
// Workspace of stream-K: the partial sums (one FP32 output tile per CTA) and
// the flags (8 per CTA), which must be zero when the launch starts.
size_t umma_streamk_part_bytes(int bn);
size_t umma_streamk_flag_bytes();
// With `side`, a contraction with the packing epilogue may also pack that
// operand on SMs without an output tile; *side_done says whether it did (if
// not, the caller packs it).
ln_status umma_contract(const UmmaProblem &p, int terms, cudaStream_t st, const PackMulti *side = nullptr,
                        bool *side_done = nullptr);
ln_status umma_contract_sym(const UmmaProblem &p, int terms, cudaStream_t st);  // ln_umma_sym.cu
ln_status umma_read_error_sym(int *value);
// ln_umma_pair.cu: the CTA-pair launches (tcgen05.mma.cta_group::2) of
// umma_contract and umma_contract_sym; `total` counts pair tiles
ln_status umma_contract_pair(int ek, const UmmaProblem &p, int terms, int bn, int total, cudaStream_t st,
                             const PackMulti *side, bool *side_done);
ln_status umma_contract_sym_pair(const UmmaProblem &p, int terms, int total, cudaStream_t st);
ln_status umma_read_error_pair(int *value);
// d_tile_owner[t] = the problem (in d_probs order) that tile t belongs to;
// terms = the split terms of the products (mma_terms); tf32: TF32 operands.
ln_status umma_contract_batched(const UmmaProblem *d_probs, const int *d_tile_prefix, const int *d_tile_owner,
                                int total_tiles, int *d_queue, int terms, int tf32, cudaStream_t st);
// ln_umma_tf32.cu: the TF32 launches (problems already in 32-K tiles, `terms`
// the TF32 term count)
ln_status umma_contract_tf32(int ek, const UmmaProblem &p, int terms, int bn, int total, cudaStream_t st);
ln_status umma_contract_sym_tf32(const UmmaProblem &p, int terms, int bn, int total, cudaStream_t st);
ln_status umma_contract_batched_tf32(const UmmaProblem *d_probs, const int *d_tile_prefix, const int *d_tile_owner,
                                     int total_tiles, int *d_queue, int terms, cudaStream_t st);
ln_status umma_read_error_tf32(int *value);
// ln_umma_tf32_pair.cu: TF32 launches on CTA pairs, 256-wide general tiles
// (`total` counts pair tiles)
ln_status umma_contract_tf32_pair(int ek, const UmmaProblem &p, int terms, int total, cudaStream_t st);
ln_status umma_read_error_tf32_pair(int *value);
ln_status umma_read_error(int *value);
// batched planning on the device
// ln_pack.cu: batched layout. The plan kernel orders instances by decreasing
// work, assigns each its packed-operand offsets, and writes its contraction
// descriptor and tile prefix sums (rank order); the pack kernel then packs
// every instance's operands in one launch.
// terms: 16 KiB pieces per packed block (prec_terms); tf32: TF32 operands
// (the plan then writes problems with 32-K tile counts and the tf32 flag)
ln_status sym_batched_plan(int is_syr2k, int count, const ln_sym_desc *d_descs, int fill, float alpha, float beta,
                           UmmaProblem *d_probs, int *d_tile_prefix, int *d_tile_owner, long long *d_pack_off,
                           int *d_pack_prefix, int *d_order, char *pack_base, int terms, int tf32, cudaStream_t st);
ln_status sym_batched_pack(int is_syr2k, int count, const ln_sym_desc *d_descs, const long long *d_pack_off,
                           const int *d_pack_prefix, const int *d_order, int total_pack_tiles, char *pack_base,
                           int terms, int tf32, cudaStream_t st);
ln_status plain_sym_batched(int is_syr2k, int count, const ln_sym_desc *d_descs, int max_n, int fill, float alpha,
                            float beta, cudaStream_t st);
ln_status simt_sym_batched(int is_syr2k, int count, const ln_sym_desc *d_descs, const int *d_tile_prefix,
                           int total_tiles, int fill, float alpha, float beta, cudaStream_t st);
ln_status simt_sym_batched_prefix(int count, const ln_sym_desc *d_descs, int *d_tile_prefix, cudaStream_t st);
// Lower-triangle tiles of the FP32 tiled batched kernel (its own tile width).
long long simt_sym_batched_tiles(int count, const ln_sym_desc *h);

}  // namespace ln
