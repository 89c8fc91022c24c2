// Gram matrix of the whitened orbit matrix on the 5th-generation tensor cores
// (the dense normal-equation contraction of the weight solve, Sec. 2.3):
// C = A A^T with A (K x ldA, BF16, row-major = K-major operands), FP32
// accumulation in tensor memory.  Only tiles on or below the diagonal are
// computed; the Cholesky factorisation reads the lower triangle only.
//
// One CTA per 128 x 128 output tile.  Warp 0 issues TMA loads (128-byte
// swizzle) of the two 128-row operand panels (four with the hi/lo split), 64
// BF16 of the contraction per stage, through a 4-stage (3 with the split)
// mbarrier ring; warp 1 allocates 128 TMEM columns
// and a single thread issues tcgen05.mma (M = 128, N = 128, K = 16) four times
// per stage, committing each stage back to the producer; warps 2-5 read the
// accumulator with tcgen05.ld and store FP32 rows.  Every wait is bounded by
// a wall-clock deadline: on expiry the kernel records an error code, drains
// its own copies, frees TMEM and returns.
#include "sw_linalg.cuh"
#include "sw_tc.cuh"

#include <cuda.h>
#include <cudaTypedefs.h>

namespace sw {

namespace gtc {

using namespace sw::tc;

constexpr int BM = 128, BN = 128, BKC = 64;  // tile rows/cols, BF16 per stage (128 bytes)
constexpr int A_BYTES = BM * BKC * 2, B_BYTES = BN * BKC * 2;
constexpr int THREADS = 192;
// plain: 4 stages of (A, B); split: 3 stages of (A_hi, B_hi, A_lo, B_lo)
template <bool SPLIT> struct Cfg {
    static constexpr int STAGES = SPLIT ? 3 : 4;
    static constexpr int STAGE_BYTES = (SPLIT ? 2 : 1) * (A_BYTES + B_BYTES);
    static constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024 + 256;
};
constexpr uint32_t TMEM_COLS = 128;

// SPLIT: the operand is A = A_hi + A_lo (both BF16, maps hi and lo) and the
// tile accumulates A_hi B_hi^T + A_hi B_lo^T + A_lo B_hi^T (the lo x lo term is
// below FP32 resolution), i.e. a Gram accurate to ~2^-16 relative.
template <bool SPLIT>
__global__ void __launch_bounds__(THREADS, 1) k_gram(const __grid_constant__ CUtensorMap map,
                                                     const __grid_constant__ CUtensorMap map_lo, int64_t K, int nk,
                                                     float* __restrict__ C, int64_t ldc, int* err, int64_t t_off)
{
    constexpr int STAGES = Cfg<SPLIT>::STAGES, STAGE_BYTES = Cfg<SPLIT>::STAGE_BYTES;
    extern __shared__ unsigned char smraw[];
    // 1024-byte aligned stage ring (required by the 128-byte swizzle atoms)
    unsigned char* base = (unsigned char*)(((uintptr_t)smraw + 1023) & ~(uintptr_t)1023);
    uint64_t* full = reinterpret_cast<uint64_t*>(base + STAGES * STAGE_BYTES);
    uint64_t* empty = full + STAGES;
    uint64_t* accum = empty + STAGES;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(accum + 1);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

    // lower-triangular tile (ti >= tj) from the linear block index (tiles before t_off skipped)
    const int64_t t = blockIdx.x + t_off;
    int64_t ti = (int64_t)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
    while ((ti + 1) * (ti + 2) / 2 <= t) ++ti;
    while (ti * (ti + 1) / 2 > t) --ti;
    const int64_t tj = t - ti * (ti + 1) / 2;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(accum, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tmem_slot)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;

    if (warp == 0 && lane == 0) {
        // ---- TMA producer
        int issued = 0;
        for (int kc = 0; kc < nk; ++kc) {
            const int s = kc % STAGES;
            const uint32_t ph = (uint32_t)(kc / STAGES) & 1u;
            if (*abort_flag || !mbar_wait(&empty[s], ph ^ 1u)) {
                *abort_flag = 1;
                break;
            }
            unsigned char* sa = base + s * STAGE_BYTES;
            mbar_expect_tx(&full[s], STAGE_BYTES);
            tma_load_2d(sa, &map, kc * BKC, (int)(ti * BM), &full[s]);
            tma_load_2d(sa + A_BYTES, &map, kc * BKC, (int)(tj * BN), &full[s]);
            if (SPLIT) {
                tma_load_2d(sa + A_BYTES + B_BYTES, &map_lo, kc * BKC, (int)(ti * BM), &full[s]);
                tma_load_2d(sa + 2 * A_BYTES + B_BYTES, &map_lo, kc * BKC, (int)(tj * BN), &full[s]);
            }
            issued = kc + 1;
        }
        if (*abort_flag) {
            // drain this CTA's copies still in flight before leaving
            for (int kc = issued - STAGES < 0 ? 0 : issued - STAGES; kc < issued; ++kc)
                mbar_wait(&full[kc % STAGES], (uint32_t)(kc / STAGES) & 1u);
        }
    } else if (warp == 1 && lane == 0) {
        // ---- MMA issuer
        const uint32_t idesc = idesc_bf16(BM, BN);
        for (int kc = 0; kc < nk; ++kc) {
            const int s = kc % STAGES;
            const uint32_t ph = (uint32_t)(kc / STAGES) & 1u;
            if (*abort_flag || !mbar_wait(&full[s], ph)) {
                *abort_flag = 1;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t sa = su32(base + s * STAGE_BYTES);
            const uint64_t da = smem_desc(sa), db = smem_desc(sa + A_BYTES);
#pragma unroll
            for (int k = 0; k < BKC / 16; ++k)
                umma(tmem, da + (uint64_t)(2 * k), db + (uint64_t)(2 * k), idesc, (kc | k) != 0);
            if (SPLIT) {
                const uint64_t dal = smem_desc(sa + A_BYTES + B_BYTES), dbl = smem_desc(sa + 2 * A_BYTES + B_BYTES);
#pragma unroll
                for (int k = 0; k < BKC / 16; ++k) {
                    umma(tmem, da + (uint64_t)(2 * k), dbl + (uint64_t)(2 * k), idesc, 1u);
                    umma(tmem, dal + (uint64_t)(2 * k), db + (uint64_t)(2 * k), idesc, 1u);
                }
            }
            umma_commit(&empty[s]);
        }
        umma_commit(accum);
    } else if (warp >= 2) {
        // ---- epilogue: TMEM -> registers -> global (lower tiles only)
        const bool ok = mbar_wait(accum, 0);
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (!ok) *abort_flag = 1;
        const int q = warp & 3;  // TMEM lane quarter this warp may access
        const int64_t gi = ti * BM + q * 32 + lane;
        if (ok && !*abort_flag) {
#pragma unroll 1
            for (int c0 = 0; c0 < BN; c0 += 32) {
                uint32_t v[32];
                tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)c0, v);
                const int64_t gj0 = tj * BN + c0;
                if (gi < K) {
                    float* dst = C + (size_t)gi * ldc + gj0;
                    if (gj0 + 32 <= K && (ldc & 3) == 0) {
#pragma unroll
                        for (int j = 0; j < 32; j += 4)
                            *reinterpret_cast<float4*>(dst + j) =
                                make_float4(__uint_as_float(v[j]), __uint_as_float(v[j + 1]),
                                            __uint_as_float(v[j + 2]), __uint_as_float(v[j + 3]));
                    } else {
                        for (int j = 0; j < 32; ++j)
                            if (gj0 + j < K) dst[j] = __uint_as_float(v[j]);
                    }
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (*abort_flag && threadIdx.x == 0) atomicExch(err, 1);
    if (warp == 1) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
    }
}

static PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;

static bool encoder()
{
    if (g_encode) return true;
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn) {
        cudaGetLastError();
        return false;
    }
    g_encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
    return true;
}

}  // namespace gtc

bool gram_tc_available() { return gtc::encoder(); }

static bool make_map(CUtensorMap* map, const __nv_bfloat16* A, int64_t K, int64_t ldA)
{
    using namespace gtc;
    cuuint64_t dims[2] = {(cuuint64_t)ldA, (cuuint64_t)K};
    cuuint64_t strides[1] = {(cuuint64_t)ldA * 2};
    cuuint32_t box[2] = {BKC, BM};
    cuuint32_t estr[2] = {1, 1};
    return g_encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, (void*)A, dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

cudaError_t gram_tc(sw_ctx* ctx, const __nv_bfloat16* A, const __nv_bfloat16* A_lo, int64_t K, int64_t ldA, float* C,
                    int* d_err, int64_t ldc, int64_t row_tile0)
{
    if (ldc <= 0) ldc = K;
    using namespace gtc;
    if (K <= 0) return cudaSuccess;
    if ((ldA % BKC) != 0 || ((uintptr_t)A & 15) != 0 || ((uintptr_t)A_lo & 15) != 0 || !encoder())
        return cudaErrorInvalidValue;
    if (K > 0x7fffff00LL || ldA > 0x7fffff00LL) return cudaErrorInvalidValue;
    CUtensorMap map, map_lo;
    if (!make_map(&map, A, K, ldA)) return cudaErrorInvalidValue;
    if (!make_map(&map_lo, A_lo ? A_lo : A, K, ldA)) return cudaErrorInvalidValue;
    static bool attr[2] = {false, false};
    const bool split = A_lo != nullptr;
    if (!attr[split]) {
        cudaError_t e = split ? cudaFuncSetAttribute(k_gram<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                     Cfg<true>::SMEM_BYTES)
                              : cudaFuncSetAttribute(k_gram<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                     Cfg<false>::SMEM_BYTES);
        if (e != cudaSuccess) return e;
        attr[split] = true;
    }
    const int64_t T = (K + BM - 1) / BM;
    if (row_tile0 < 0 || row_tile0 > T) return cudaErrorInvalidValue;
    const int64_t t_off = row_tile0 * (row_tile0 + 1) / 2;
    const int64_t tiles = T * (T + 1) / 2 - t_off;
    if (tiles <= 0) return cudaSuccess;
    const int nk = (int)(ldA / BKC);
    LaunchTimer lt(ctx, K_GRAM_TC);
    add_work(ctx, K_GRAM_TC, 2.0 * (double)tiles * BM * BM * (double)ldA * (split ? 3.0 : 1.0));
    if (split)
        k_gram<true><<<(unsigned)tiles, THREADS, Cfg<true>::SMEM_BYTES, ctx_stream(ctx)>>>(map, map_lo, K, nk, C, ldc,
                                                                                           d_err, t_off);
    else
        k_gram<false><<<(unsigned)tiles, THREADS, Cfg<false>::SMEM_BYTES, ctx_stream(ctx)>>>(map, map_lo, K, nk, C, ldc,
                                                                                             d_err, t_off);
    return cudaGetLastError();
}

// Retained block of a passive Gram gathered from the previous one (one thread per element of the
// lower triangle, rows over blockIdx.y)
__global__ void k_gather_gram(const float* __restrict__ Gc, int64_t ldc, const int64_t* __restrict__ cidx, int64_t r0,
                              float* __restrict__ G, int64_t ldG)
{
    for (int64_t a = blockIdx.y; a < r0; a += gridDim.y) {
        const int64_t ca = cidx[a];
        for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b <= a; b += (int64_t)gridDim.x * blockDim.x) {
            const int64_t cb = cidx[b];
            G[(size_t)a * ldG + b] = ca >= cb ? Gc[(size_t)ca * ldc + cb] : Gc[(size_t)cb * ldc + ca];
        }
    }
}

cudaError_t gather_gram(sw_ctx* ctx, const float* Gc, int64_t ldc, const int64_t* cidx, int64_t r0, float* G,
                        int64_t ldG)
{
    if (r0 <= 0) return cudaSuccess;
    LaunchTimer lt(ctx, K_MISC);
    add_work(ctx, K_MISC, 8.0 * (double)r0 * (double)r0 / 2.0);
    const unsigned gx = (unsigned)std::min<int64_t>((r0 + 255) / 256, 8);
    const unsigned gy = (unsigned)std::min<int64_t>(r0, 65535);
    k_gather_gram<<<dim3(gx, gy), 256, 0, ctx_stream(ctx)>>>(Gc, ldc, cidx, r0, G, ldG);
    return cudaGetLastError();
}

}  // namespace sw
