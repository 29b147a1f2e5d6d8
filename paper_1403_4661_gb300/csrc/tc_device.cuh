// Device building blocks of the tensor-core contractions: tile constants, PTX wrappers (cp.async,
// mbarrier, tcgen05), exact BF16 slicing of float64 values and the int64 -> float64 conversion.
// Included by the kernels of tc_gemm.cu and chain.cu.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>

#include "sht_internal.cuh"

namespace sht {
namespace {

constexpr int S = kTcSlices;       // 8
constexpr int BETA = kTcSliceBits; // 7
constexpr int MT = 128, NT = 64, KB = 32, CHUNK = 128;
constexpr int REGIONS = 6;                 // diagonals 2..6 exact, 7..9 rounded
constexpr int ACC_SHIFT = 49;              // int64 accumulators hold C * 2^49
constexpr int A_STAGE = S * MT * KB * 2;   // 64 KiB
constexpr int B_STAGE = S * NT * KB * 2;   // 32 KiB
constexpr int STAGE = A_STAGE + B_STAGE;
constexpr int SMEM_BYTES = 2 * STAGE;
constexpr uint32_t TMEM_COLS = 512;        // 6 regions x 64 columns, rounded up to a power of 2

// ---------------------------------------------------------------- PTX wrappers
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src, int src_bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst), "l"(src), "r"(src_bytes)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }
__device__ __forceinline__ void mbar_init(uint32_t a, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(a), "r"(count) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t a, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok) : "r"(a), "r"(parity) : "memory");
    return ok != 0;
}
__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// Waits for phase `parity` of the barrier; false once `limit_ns` have passed (default: the one
// second used for the waits on a CTA's own copies and MMAs before it releases its memory).
constexpr uint64_t kOwnWaitNs = 1000000000ull;
__device__ bool mbar_wait(uint32_t a, uint32_t parity, uint64_t limit_ns = kOwnWaitNs) {
    if (mbar_try_wait(a, parity)) return true;
    const uint64_t t0 = global_ns();
    while (!mbar_try_wait(a, parity))
        if (global_ns() - t0 > limit_ns) return false;
    return true;
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void tmem_alloc(uint32_t dst, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(dst), "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(taddr), "r"(ncols) : "memory");
}
// D[tmem] (+)= A[smem] * B[smem]^T, M = 128, N = 64, K = 16, BF16 in, FP32 accumulate
__device__ __forceinline__ void mma_bf16(uint32_t d, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
        "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
        : "memory");
}
// D[tmem] (+)= A[smem] * B[smem]^T, M = 128, N = 64, K = 8, TF32 in, FP32 accumulate
__device__ __forceinline__ void mma_tf32(uint32_t d, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
        "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
        : "memory");
}
__device__ __forceinline__ void mma_commit(uint32_t mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(mbar)
                 : "memory");
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float v[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}
// v * 2^e as a float64, assembled with integer operations only (round to nearest, ties away from
// zero); the float64 pipe is 1/64 of the integer rate.  Results below the normal range are 0.
__device__ __forceinline__ double i64_scaled(long long v, int e) {
    if (v == 0) return 0.0;
    const unsigned long long sgn = v < 0 ? (1ull << 63) : 0ull;
    unsigned long long a = v < 0 ? (unsigned long long)(-v) : (unsigned long long)v;
    int msb = 63 - __clzll(a);
    unsigned long long m;
    if (msb > 52) {
        const int sh = msb - 52;
        m = (a + (1ull << (sh - 1))) >> sh;
        if (m >> 53) { m >>= 1; ++msb; }
    } else {
        m = a << (52 - msb);
    }
    const int biased = msb + e + 1023;
    if (biased <= 0) return 0.0;
    return __longlong_as_double((long long)(sgn | ((unsigned long long)biased << 52) |
                                            (m & 0xFFFFFFFFFFFFFull)));
}

// Shared-memory matrix descriptor: no swizzle, K-major; lbo = byte step between core matrices
// along K, sbo = byte step between 8-row groups along M (or N).
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;  // descriptor version of tcgen05
    return d;
}
// Descriptor of a K-major tile written by a TMA load with 64-byte swizzling (rows of 64 bytes =
// 32 BF16 along K, 8-row groups 512 bytes apart; the leading offset is unused in this layout).
__device__ __forceinline__ uint64_t sdesc_sw64(uint32_t saddr) {
    uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)1 << 16;
    d |= (uint64_t)(512 >> 4) << 32;
    d |= (uint64_t)1 << 46;   // descriptor version of tcgen05
    d |= (uint64_t)4 << 61;   // 64-byte swizzle
    return d;
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t a, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(a), "r"(bytes) : "memory");
}
// TMA tile load of a 3-D box (x innermost) into shared memory; completes on the mbarrier.
__device__ __forceinline__ void tma_load_3d(uint32_t dst, const void *tmap, int x, int y, int z, uint32_t mbar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];\n"
        ::"r"(dst), "l"(tmap), "r"(x), "r"(y), "r"(z), "r"(mbar)
        : "memory");
}
// TMA tile load of a 2-D box (x innermost) into shared memory; completes on the mbarrier.
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const void *tmap, int x, int y, uint32_t mbar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];\n"
        ::"r"(dst), "l"(tmap), "r"(x), "r"(y), "r"(mbar)
        : "memory");
}
// Instruction descriptor, kind::f16: D = F32, A = B = BF16, both K-major.
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(NT >> 3) << 17) |
                            ((uint32_t)(MT >> 4) << 24);
// The slice-pair MMAs of one 16-K step: A slice s (1..NSL) times B slice t with s + t <= NSL + 1 (the
// pairs of weight 2^-7(s+t) down to the float64 unit).  With EXACT, diagonal d = s + t accumulates in
// TMEM region d - 2 (d <= 6: exact in FP32 over a CHUNK) or 5 (d >= 7: the rounded tail), otherwise
// every pair in region 0.  Fully unrolled: each pair's region and whether it is its region's first
// MMA of the step are compile-time constants, and the shared-memory descriptors advance from ad0 /
// bd0 by constant offsets in 16-byte units (A_SLICE16, B_SLICE16 per slice; the addresses stay below
// 2^18, so the 14-bit address field never carries).  `restart`: the first MMA of every region
// overwrites its accumulator instead of adding to it.
template <int NSL, bool EXACT, uint32_t A_SLICE16, uint32_t B_SLICE16>
__device__ __forceinline__ void mma_slice_pairs(uint32_t tbase, uint64_t ad0, uint64_t bd0, bool restart) {
#pragma unroll
    for (int s = 1; s <= NSL; ++s) {
#pragma unroll
        for (int t = 1; t <= NSL + 1 - s; ++t) {
            const int d = s + t;
            const int reg = EXACT ? (d <= 6 ? d - 2 : 5) : 0;
            const bool lead = s == 1 && (EXACT ? d <= 7 : t == 1);
            mma_bf16(tbase + reg * NT, ad0 + (uint64_t)((s - 1) * A_SLICE16), bd0 + (uint64_t)((t - 1) * B_SLICE16),
                     kIdesc, (lead && restart) ? 0u : 1u);
        }
    }
}

// Instruction descriptor, kind::tf32: D = F32, A = B = TF32 (format code 2), both K-major.
constexpr uint32_t kIdescTf32 = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(NT >> 3) << 17) |
                                ((uint32_t)(MT >> 4) << 24);
// TF32 operand tiles: a 32-K block of the table operand is two TMA boxes of 16 floats (64 bytes,
// 64-byte swizzle) x 128 rows; the right-hand side block is 32 K x 64 columns of floats.
constexpr int TF_A_HALF = MT * 16 * 4;     // 8 KiB
constexpr int TF_A_STAGE = 2 * TF_A_HALF;  // 16 KiB (fits in A_STAGE)
static_assert(TF_A_STAGE <= A_STAGE && NT * KB * 4 <= B_STAGE, "TF32 tiles fit the BF16 stages");

// ---------------------------------------------------------------- slicing
// Integer-only slicing (the float64 pipe is 1/64 of the integer rate): with the biased exponent
// field E of x, |x| < 2^(E - 1022), so the scale exponent of a row or column is the largest field
// minus 1022, exactly floor(log2 max|x|) + 1.  The magnitude of x / 2^e in fixed point with 56
// fraction bits is the 53-bit significand shifted by E - 1075 - e + 56 (truncated: drops below
// 2^-56 of the scale); slice s is bits [56 - 7s, 63 - 7s) of it, with the sign of x.
__device__ __forceinline__ int exp_field(double x) {
    return (int)((__double_as_longlong(x) >> 52) & 0x7FF);
}
__device__ __forceinline__ int scale_from_field(int f) { return f > 0 ? f - 1022 : 0; }
__device__ __forceinline__ void split_value(double x, int e, __nv_bfloat16 out[S]) {
    const long long bits = __double_as_longlong(x);
    const int f = (int)((bits >> 52) & 0x7FF);
    unsigned long long mag = 0;
    if (f > 0) {
        const unsigned long long sig = (unsigned long long)(bits & 0xFFFFFFFFFFFFFll) | (1ull << 52);
        const int sh = f - 1075 - e + 56;                // value * 2^(56 - e) = sig * 2^sh
        if (sh >= 0) mag = sig << sh;                     // sh <= 3 since |x| < 2^e
        else if (sh > -64) mag = sig >> (-sh);
    }
    const float sgn = bits < 0 ? -1.0f : 1.0f;
#pragma unroll
    for (int s = 1; s <= S; ++s) {
        const int a = (int)((mag >> (56 - BETA * s)) & 0x7F);
        // a * 2^-7s, exact in BF16 (7 significant bits)
        out[s - 1] = __float2bfloat16_rn(sgn * __int2float_rn(a) * __int_as_float((127 - BETA * s) << 23));
    }
}

// x * 2^-e rounded to TF32 (10 stored significand bits; nearest, ties away from zero), as the
// bits of a float32 whose 13 low significand bits are zero.  Integer operations only.  |x| < 2^e
// (e a row or column scale of scale_from_field), so the result is at most 1 in magnitude; values
// below the float32 normal range (|x| < 2^(e-126)) become 0.
__device__ __forceinline__ uint32_t tf32_scaled_bits(double x, int e) {
    const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
    const int f = (int)((bits >> 52) & 0x7FF);
    const uint32_t sgn = (uint32_t)(bits >> 63) << 31;
    int fe = f - e - 1023 + 127;                       // float32 exponent field of x * 2^-e
    if (f == 0 || fe <= 0) return sgn;
    unsigned long long m10 = ((bits & 0xFFFFFFFFFFFFFull) + (1ull << 41)) >> 42;   // 10 bits + carry
    if (m10 >> 10) { m10 = 0; ++fe; }
    return sgn | ((uint32_t)fe << 23) | ((uint32_t)m10 << 13);
}

// Slicing of one row x[0..K) with input stride `step` (one warp): scale exponent, S slices, zero
// padding to kp.
__device__ __forceinline__ void slice_row_warp(const double *__restrict__ x, int64_t step, int K,
                                               int kp, __nv_bfloat16 *__restrict__ out,
                                               int64_t sstride, int *__restrict__ expo) {
    const int lane = threadIdx.x & 31;
    int mf = 0;
    for (int k = lane; k < K; k += 32) mf = max(mf, exp_field(x[k * step]));
    for (int o = 16; o > 0; o >>= 1) mf = max(mf, __shfl_xor_sync(0xffffffffu, mf, o));
    const int e = scale_from_field(mf);
    if (lane == 0) *expo = e;
    __nv_bfloat16 sl[S];
    for (int k = lane; k < kp; k += 32) {
        if (k < K) split_value(x[k * step], e, sl);
        else
#pragma unroll
            for (int s = 0; s < S; ++s) sl[s] = __float2bfloat16_rn(0.0f);
#pragma unroll
        for (int s = 0; s < S; ++s) out[s * sstride + k] = sl[s];
    }
}

// Host: a 3-D BF16 TMA map (dims[0] = K innermost, then rows, then slices), 64-byte swizzled
// boxes, zero fill outside the tensor.  The encoder comes from the driver through the runtime.
inline cudaError_t encode_tiled_map(CUtensorMap *map, const __nv_bfloat16 *base, const cuuint64_t dims[3],
                                    const cuuint64_t strides[2], const cuuint32_t box[3]) {
    using Encode = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
    static_assert(sizeof(CUtensorMap) == kTensorMapBytes, "tensor map size");
    void *fn = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess) return e;
    if (q != cudaDriverEntryPointSuccess || fn == nullptr) return cudaErrorNotSupported;
    const cuuint32_t step[3] = {1, 1, 1};
    const CUresult r = reinterpret_cast<Encode>(fn)(
        map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<__nv_bfloat16 *>(base), dims, strides, box, step,
        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// Host: a 2-D float32 TMA map (dims[0] = K innermost, then rows), 64-byte swizzled boxes of
// box[0] x box[1], zero fill outside the tensor.
inline cudaError_t encode_tiled_map_f32(CUtensorMap *map, const float *base, const cuuint64_t dims[2],
                                        cuuint64_t row_stride, const cuuint32_t box[2]) {
    using Encode = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
    void *fn = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess) return e;
    if (q != cudaDriverEntryPointSuccess || fn == nullptr) return cudaErrorNotSupported;
    const cuuint32_t step[2] = {1, 1};
    const cuuint64_t strides[1] = {row_stride};
    const CUresult r = reinterpret_cast<Encode>(fn)(
        map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float *>(base), dims, strides, box, step,
        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

}  // namespace
}  // namespace sht
