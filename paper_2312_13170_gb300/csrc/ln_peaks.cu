// Roofline denominators measured on the device itself: the rate at which one
// SM's tensor core retires tcgen05.mma (BF16 and TF32 operands, M = 128,
// N = 256, both operands resident in shared memory, FP32 accumulation in
// TMEM), the FP32 FFMA rate of the CUDA cores, and a streaming copy through
// HBM. Each probe is one kernel launch on the caller's stream; the caller
// times it with CUDA events and divides the work returned by ln_peak_probe.
//
// The MMA probe runs one CTA per SM (its shared-memory request keeps a second
// one off the SM): warp 0 allocates 256 TMEM columns, one thread issues the
// MMAs back to back on the same operand tiles (four K steps per 128-byte
// swizzled row, as the contraction kernels do), commits them to an mbarrier
// and waits for it with a bound of 2 s on the global timer; a wait that runs
// out sets the caller's error word and the kernel still frees its TMEM.
#include "ln_umma_kernel.cuh"

#include "loopnest.h"

namespace ln {

namespace {

constexpr int PEAK_N = 256;
constexpr int PEAK_A_BYTES = BM * 128;      // 128 rows x 128 bytes
constexpr int PEAK_B_BYTES = PEAK_N * 128;  // 256 rows x 128 bytes
constexpr int PEAK_SMEM = 120 * 1024;       // > half an SM's shared memory: one CTA per SM
constexpr int FFMA_CHAINS = 8;
constexpr int FFMA_UNROLL = 16;

// Finite operand values of either format, from a hash of the element index:
// BF16 halves or TF32 words with exponents near 1 and varied mantissas, so
// the tensor core multiplies data that is neither zero nor constant.
__device__ __forceinline__ uint32_t mix(uint32_t x) {
    x ^= x >> 16;
    x *= 0x7feb352dU;
    x ^= x >> 15;
    x *= 0x846ca68bU;
    x ^= x >> 16;
    return x;
}

template <bool TF>
__global__ void __launch_bounds__(128, 1) k_peak_mma(long long iters, int *err) {
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t *base = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint8_t *a = base, *b = base + PEAK_A_BYTES;
    __shared__ uint64_t done;
    __shared__ uint32_t tmem_base;
    uint32_t *w = reinterpret_cast<uint32_t *>(base);
    for (int i = threadIdx.x; i < (PEAK_A_BYTES + PEAK_B_BYTES) / 4; i += blockDim.x) {
        const uint32_t h = mix(i * 2654435761U + blockIdx.x);
        w[i] = TF ? (0x3F000000U | (h & 0x807FFFFFU))  // +-[0.5, 1)
                  : (0x3F003F00U | (h & 0x807F807FU));  // two +-[0.5, 1)
    }
    if (threadIdx.x == 0) {
        mbar_init(&done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    // the operands were written by the generic proxy; the MMAs read them
    // through the async proxy
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    if (threadIdx.x < 32) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(&tmem_base)),
                     "r"(PEAK_N)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t d = tmem_base;
    if (threadIdx.x == 32) {
        const uint64_t ad = sw128_desc(saddr(a)), bd = sw128_desc(saddr(b));
        for (long long it = 0; it < iters; ++it) {
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {  // 32 bytes of each row per instruction
                if constexpr (TF) umma_tf32<PEAK_N>(d, ad + 2 * kk, bd + 2 * kk, (it | kk) != 0);
                else umma_bf16<PEAK_N>(d, ad + 2 * kk, bd + 2 * kk, (it | kk) != 0);
            }
        }
        umma_commit(&done);
        bool ok = mbar_try_wait(&done, 0);
        const unsigned long long t0 = gtimer();
        for (uint32_t n = 1; !ok; ++n) {
            ok = mbar_try_wait(&done, 0);
            if (!ok && (n & 31) == 0 && gtimer() - t0 > WAIT_NS) {
                atomicExch(err, 1);
                break;
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (threadIdx.x < 32)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(d), "r"(PEAK_N) : "memory");
}

// FFMA_CHAINS independent dependency chains per thread, FFMA_UNROLL steps
// each per iteration; x and y come from the host, so nothing folds.
__global__ void __launch_bounds__(256) k_peak_ffma(long long iters, float x, float y, float *sink) {
    float acc[FFMA_CHAINS];
#pragma unroll
    for (int c = 0; c < FFMA_CHAINS; ++c) acc[c] = (float)(threadIdx.x + c) * 1e-3f;
    for (long long it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < FFMA_UNROLL; ++u) {
#pragma unroll
            for (int c = 0; c < FFMA_CHAINS; ++c) acc[c] = fmaf(acc[c], x, y);
        }
    }
    float s = 0.0f;
#pragma unroll
    for (int c = 0; c < FFMA_CHAINS; ++c) s += acc[c];
    if (s == -1.0f) *sink = s;  // never true for these inputs, unknown to the compiler
}

__global__ void __launch_bounds__(256) k_peak_copy(const float4 *__restrict__ src, float4 *__restrict__ dst,
                                                   long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        dst[i] = src[i];
}

bool g_peak_optin[64][2];

}  // namespace

}  // namespace ln

using namespace ln;

extern "C" ln_status ln_peak_probe(int kind, long long iters, const void *src, void *dst, long long bytes,
                                   double *work, void *stream) {
    clear_error();
    if (!work) return fail(LN_ERR_INVALID_VALUE, "NULL work");
    *work = 0.0;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    switch (kind) {
        case LN_PEAK_MMA_BF16:
        case LN_PEAK_MMA_TF32: {
            if (iters < 1 || iters > (1LL << 20)) return fail(LN_ERR_INVALID_VALUE, "iters %lld out of [1, 2^20]", iters);
            if (!dst || bytes < 4 || (reinterpret_cast<uintptr_t>(dst) & 3))
                return fail(LN_ERR_INVALID_VALUE, "the MMA probe needs a 4-byte-aligned error word in dst");
            const bool tf = kind == LN_PEAK_MMA_TF32;
            const int sms = sm_count();
            int dev = 0;
            LN_CUDA_TRY(cudaGetDevice(&dev));
            if (dev < 0 || dev >= 64) return fail(LN_ERR_UNSUPPORTED, "device ordinal %d out of range", dev);
            auto kern = tf ? k_peak_mma<true> : k_peak_mma<false>;
            if (!g_peak_optin[dev][tf]) {
                LN_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, PEAK_SMEM));
                g_peak_optin[dev][tf] = true;
            }
            LN_CUDA_TRY(cudaMemsetAsync(dst, 0, 4, st));
            {
                LaunchScope ls_(FAM_UMMA, st);
                kern<<<sms, 128, PEAK_SMEM, st>>>(iters, static_cast<int *>(dst));
            }
            if (const ln_status e = check_launch("k_peak_mma"); e != LN_SUCCESS) return e;
            // K = 16 BF16 or 8 TF32 elements per instruction, four per iteration
            *work = 2.0 * BM * PEAK_N * (tf ? 8 : 16) * 4.0 * (double)iters * sms;
            return LN_SUCCESS;
        }
        case LN_PEAK_FFMA: {
            if (iters < 1 || iters > (1LL << 20)) return fail(LN_ERR_INVALID_VALUE, "iters %lld out of [1, 2^20]", iters);
            if (!dst || bytes < 4 || (reinterpret_cast<uintptr_t>(dst) & 3))
                return fail(LN_ERR_INVALID_VALUE, "the FFMA probe needs a 4-byte sink in dst");
            const int blocks = sm_count() * 8;  // 2048 threads per SM: one resident wave
            {
                LaunchScope ls_(FAM_SIMT, st);
                k_peak_ffma<<<blocks, 256, 0, st>>>(iters, 0.999f, 1e-6f, static_cast<float *>(dst));
            }
            if (const ln_status e = check_launch("k_peak_ffma"); e != LN_SUCCESS) return e;
            *work = 2.0 * FFMA_CHAINS * FFMA_UNROLL * (double)iters * blocks * 256.0;
            return LN_SUCCESS;
        }
        case LN_PEAK_COPY: {
            if (!src || !dst || bytes <= 0 || (bytes & 15) || ((reinterpret_cast<uintptr_t>(src) |
                                                                  reinterpret_cast<uintptr_t>(dst)) & 15))
                return fail(LN_ERR_INVALID_VALUE, "the copy probe needs 16-byte-aligned buffers and a size that is a multiple of 16");
            const uintptr_t s0 = reinterpret_cast<uintptr_t>(src), d0 = reinterpret_cast<uintptr_t>(dst);
            if (s0 < d0 + (uintptr_t)bytes && d0 < s0 + (uintptr_t)bytes) return fail(LN_ERR_ALIASING, "src overlaps dst");
            const long long n = bytes / 16;
            const long long want = (n + 255) / 256, wave = sm_count() * 8LL;  // one resident wave
            const int blocks = (int)(want < wave ? want : wave);
            {
                LaunchScope ls_(FAM_STATS, st);
                k_peak_copy<<<blocks, 256, 0, st>>>(static_cast<const float4 *>(src), static_cast<float4 *>(dst), n);
            }
            if (const ln_status e = check_launch("k_peak_copy"); e != LN_SUCCESS) return e;
            *work = 2.0 * (double)bytes;  // read and written
            return LN_SUCCESS;
        }
        default: return fail(LN_ERR_INVALID_VALUE, "unknown probe kind %d", kind);
    }
}
