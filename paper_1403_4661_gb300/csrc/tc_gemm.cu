// float64-accurate contractions on the 5th-generation tensor cores (tcgen05, BF16 -> FP32 in TMEM).
//
// The contractions of the transforms (synthesis G = P~ X, Eq. (11); the order solves and alias
// products of Procedure 1) need float64 accuracy, and GB300's float64 pipe delivers 1.25 TFLOP/s.
// Each operand is therefore split into S = 8 exact slices of 7 bits with a power-of-two scale per
// row (A) or per column (B):
//     x = 2^e * sum_{s=1..S} a_s 2^{-7 s},   a_s integer, |a_s| < 2^7,
// each slice value a_s 2^{-7s} being exact in BF16.  Then
//     C_ij = 2^{eA_i + eB_j} sum_{s+t <= S+1} sum_k A_s[i,k] B_t[j,k],
// every product A_s B_t being exact in FP32 (14 significant bits).  Products of one diagonal
// d = s + t are multiples of 2^{-7d}; over a K-chunk of 128 the (d-1) pairs of a diagonal d <= 6
// sum to less than 2^{24-7d}, so the tensor core's FP32 accumulation of each such diagonal in its
// own TMEM region is exact (measured: FP32 accumulation of the tensor cores is exact whenever the
// sum is representable).  The diagonals d >= 7 share a sixth region; their sum is below 2^-23 of
// the leading term and its FP32 rounding below 2^-47.  After every chunk each region is read from
// TMEM, converted exactly to an integer at its own scale and added into one int64 per output at
// scale 2^-49.  Dropping the slices beyond S = 8 and the pairs with s + t > 9 leaves an error of
// order 2^-49 max|A_i| max|B_j| per term, comparable with a float64 dot product.
//
// This file: the slicing of the plan tables and of the inverse's coefficients, and the inverse's
// synthesis contraction (k_synthesis below); the forward's order chain is in chain.cu.
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <vector>

#include "epilogue.cuh"
#include "sht_internal.cuh"
#include "tc_device.cuh"

namespace sht {
namespace {

// Plan tables, every order m = blockIdx.y: the P~ block (L rows, K = L - m) or the P_m^{-1} block
// (L - m rows); slices of block m at S * koff[m] rows*kp units.
__global__ void k_slice_rows_orders(const double *__restrict__ tab, int L, bool inverses,
                                    const int64_t *__restrict__ koff, __nv_bfloat16 *__restrict__ out,
                                    int *__restrict__ expo) {
    const int m = blockIdx.y, n = L - m, kp = (n + 7) & ~7;
    const int rows = inverses ? n : L;
    const int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (row >= rows) return;
    const double *blk = tab + (inverses ? pinv_off(L, m) : pt_off(L, m));
    // block m: kTcSlices slices of rows x kp; P~ blocks all have L rows (koff counts kp),
    // inverse blocks have n rows (koff counts n * kp)
    __nv_bfloat16 *ob = out + (int64_t)S * koff[m] * (inverses ? 1 : L);
    int *eb = expo + (inverses ? rows_off(L, m) : (int64_t)m * L);
    slice_row_warp(blk + (int64_t)row * n, 1, n, kp, ob + (int64_t)row * kp, (int64_t)rows * kp, eb + row);
}

// TF32 copies of the plan tables for the TF32 refined forward: row r of block m holds
// P(r, k) * 2^-e_r rounded to TF32 (e_r the row's scale exponent from the BF16 slicing), zero
// padded to kp; same block offsets as the slices without the slice factor.  One warp per row.
__global__ void k_tf32_rows_orders(const double *__restrict__ tab, int L, bool inverses,
                                   const int64_t *__restrict__ koff, const int *__restrict__ expo,
                                   float *__restrict__ out) {
    const int m = blockIdx.y, n = L - m, kp = (n + 7) & ~7;
    const int rows = inverses ? n : L;
    const int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (row >= rows) return;
    const double *x = tab + (inverses ? pinv_off(L, m) : pt_off(L, m)) + (int64_t)row * n;
    const int e = expo[(inverses ? rows_off(L, m) : (int64_t)m * L) + row];
    uint32_t *o = reinterpret_cast<uint32_t *>(out + koff[m] * (inverses ? 1 : L) + (int64_t)row * kp);
    for (int k = threadIdx.x & 31; k < kp; k += 32) o[k] = k < n ? tf32_scaled_bits(x[k], e) : 0u;
}

// Column slicing: X has K rows and `cols` columns (row-major, ld); output row j = column j.
// One block of 256 threads per 32 columns.
__device__ __forceinline__ void slice_cols_block(const double *__restrict__ X, int64_t ld, int K,
                                                 int cols, int kp, __nv_bfloat16 *__restrict__ out,
                                                 int64_t sstride, int *__restrict__ expo, int j0) {
    __shared__ int red[8][32];
    __shared__ int se[32];
    __shared__ __nv_bfloat16 tile[S][32][34];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int j = j0 + lane;
    int mf = 0;
    if (j < cols)
        for (int k = warp; k < K; k += 8) mf = max(mf, exp_field(X[(int64_t)k * ld + j]));
    red[warp][lane] = mf;
    __syncthreads();
    if (warp == 0) {
        for (int w = 1; w < 8; ++w) mf = max(mf, red[w][lane]);
        const int e = scale_from_field(mf);
        se[lane] = e;
        if (j < cols) expo[j] = e;
    }
    __syncthreads();
    for (int k0 = 0; k0 < kp; k0 += 32) {
        // a 32 (k) x 32 (j) tile: lane = j, warp strides k
        for (int kk = warp; kk < 32; kk += 8) {
            const int k = k0 + kk;
            __nv_bfloat16 sl[S];
            if (j < cols && k < K) split_value(X[(int64_t)k * ld + j], se[lane], sl);
            else
#pragma unroll
                for (int s = 0; s < S; ++s) sl[s] = __float2bfloat16_rn(0.0f);
#pragma unroll
            for (int s = 0; s < S; ++s) tile[s][lane][kk] = sl[s];
        }
        __syncthreads();
        // rows j0.. written with lane = k (coalesced along K)
        for (int jj = warp; jj < 32; jj += 8) {
            const int jr = j0 + jj, k = k0 + lane;
            if (jr < cols && k < kp)
#pragma unroll
                for (int s = 0; s < S; ++s) out[s * sstride + (int64_t)jr * kp + k] = tile[s][jj][lane];
        }
        __syncthreads();
    }
}

// Order-major coefficients X (block m: L - m rows of Nc columns), every order m = blockIdx.y.
__global__ void k_slice_cols_orders(const double *__restrict__ X, int L, int Nc,
                                    const int64_t *__restrict__ koff, __nv_bfloat16 *__restrict__ out,
                                    int *__restrict__ expo) {
    const int m = blockIdx.y, n = L - m, kp = (n + 7) & ~7;
    slice_cols_block(X + rows_off(L, m) * Nc, Nc, n, Nc, kp, out + (int64_t)S * Nc * koff[m],
                     (int64_t)Nc * kp, expo + (int64_t)m * Nc, blockIdx.x * 32);
}

// ---------------------------------------------------------------- the synthesis contraction
// Every order m in one launch: G_m (L rings x Nc) = P~_m (L x n) X_m (n x Nc), n = L - m, one CTA
// per 128 x 64 output tile.  Both operands come pre-sliced (plan table, per-call X slices) and are
// staged by TMA, 64-byte swizzled, 32 K per stage, two stages.  Thread 0 is the producer and the
// MMA issuer: it waits for a stage's loads, issues its 36 slice-pair MMAs per 16 K, commits them,
// then refills the other stage once the MMAs that read it are done, so the tensor pipe always has
// the next block queued.  All 8 warps drain the six TMEM regions into int64 accumulators at the
// end of every 128-K chunk (warps w, w + 4: lane quarter w % 4, columns 0..31 / 32..63).
struct SynArgs {
    int L, Nc;
    const int *ptE, *xE;                   // row scales of P~ (m * L + k), column scales of X (m * Nc + j)
    const unsigned char *tmA, *tmB;        // TMA maps: P~ block of order m at (2m + 1), X slices at m
    double *Gt;                            // order-major G: m * L * Nc
    int *status;
    uint64_t wait_ns;                      // limit of the pipeline waits
};

constexpr int kSynThreads = 256;

__global__ void __launch_bounds__(kSynThreads, 1) k_synthesis(SynArgs p) {
    constexpr int kCols = NT / 2;
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ uint64_t mbar[2], full[2];
    __shared__ uint32_t tmem_slot;
    const int tid = threadIdx.x, warp = tid >> 5, half = warp >> 2;
    const int L = p.L, Nc = p.Nc;
    const int tiles_n = (Nc + NT - 1) / NT;
    const int per_m = ((L + MT - 1) / MT) * tiles_n;
    const int m = (int)(blockIdx.x / per_m), tile = (int)(blockIdx.x - (int64_t)m * per_m);
    const int tm = tile / tiles_n, tn = tile - tm * tiles_n;
    const int row0 = tm * MT, col0 = tn * NT;
    const int K = L - m, nkb = (K + KB - 1) / KB;
    const void *tmA = p.tmA + (size_t)(2 * m + 1) * kTensorMapBytes;
    const void *tmB = p.tmB + (size_t)m * kTensorMapBytes;

    if (warp == 0) tmem_alloc(smem_u32(&tmem_slot), TMEM_COLS);
    if (tid == 0) {
        for (int i = 0; i < 2; ++i) {
            mbar_init(smem_u32(&mbar[i]), 1);
            mbar_init(smem_u32(&full[i]), 1);
        }
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tbase = tmem_slot;

    auto load = [&](int kb) {   // thread 0
        const int st = kb & 1;
        const uint32_t sa = smem_u32(smem + st * STAGE), sb = sa + A_STAGE;
        mbar_expect_tx(smem_u32(&full[st]), A_STAGE + B_STAGE);
        tma_load_3d(sa, tmA, kb * KB, row0, 0, smem_u32(&full[st]));
        tma_load_3d(sb, tmB, kb * KB, col0, 0, smem_u32(&full[st]));
    };

    long long acc[kCols];
#pragma unroll
    for (int c = 0; c < kCols; ++c) acc[c] = 0;
    bool ok0 = true, alive = true;   // thread 0's waits; the CTA's vote
    int loads = 0, commits = 0;      // thread 0: issued per CTA (stage = index & 1)
    if (tid == 0) { load(0); ++loads; }
    for (int kb = 0; kb < nkb; ++kb) {
        const int st = kb & 1;
        const uint32_t par = (uint32_t)(kb >> 1) & 1u;   // use kb >> 1 of stage st
        if (tid == 0 && ok0) {
            ok0 = mbar_wait(smem_u32(&full[st]), par, p.wait_ns);
            if (ok0) {
                tc_fence_after();
                const uint32_t sa = smem_u32(smem + st * STAGE), sb = sa + A_STAGE;
                // two 16-K steps; the first of a chunk restarts the accumulator regions
                constexpr uint32_t A16 = (MT * KB * 2) >> 4, B16 = (NT * KB * 2) >> 4;
                const uint64_t ad0 = sdesc_sw64(sa), bd0 = sdesc_sw64(sb);
                mma_slice_pairs<S, true, A16, B16>(tbase, ad0, bd0, (kb * KB) % CHUNK == 0);
                if (kb * KB + 16 < K) mma_slice_pairs<S, true, A16, B16>(tbase, ad0 + (32 >> 4), bd0 + (32 >> 4), false);
                mma_commit(smem_u32(&mbar[st]));
                ++commits;
                // refill the other stage once the MMAs of block kb - 1 (its last reader) are done
                if (kb + 1 < nkb) {
                    if (kb >= 1) ok0 = mbar_wait(smem_u32(&mbar[st ^ 1]), (uint32_t)((kb - 1) >> 1) & 1u, p.wait_ns);
                    if (ok0) { load(kb + 1); ++loads; }
                }
            }
        }
        if (((kb + 1) * KB) % CHUNK == 0 || kb == nkb - 1) {
            // the commit of block kb covers every MMA issued so far
            const bool w = mbar_wait(smem_u32(&mbar[st]), par, p.wait_ns);
            alive = __syncthreads_and(w && (tid != 0 || ok0));
            if (!alive) break;
            tc_fence_after();
            const uint32_t lane_base = tbase + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)(half * kCols);
#pragma unroll
            for (int reg = 0; reg < REGIONS; ++reg) {
                const int d = reg + 2;
                const float up = reg < REGIONS - 1 ? __int_as_float((127 + 7 * d) << 23)
                                                   : __int_as_float((127 + ACC_SHIFT) << 23);
                const int shift = reg < REGIONS - 1 ? ACC_SHIFT - 7 * d : 0;
#pragma unroll
                for (int c0 = 0; c0 < kCols; c0 += 16) {
                    float v[16];
                    tmem_ld16(lane_base + reg * NT + c0, v);
#pragma unroll
                    for (int i = 0; i < 16; ++i) acc[c0 + i] += (long long)__float2int_rn(v[i] * up) << shift;
                }
            }
            tc_fence_before();
            __syncthreads();
        }
    }
    if (!alive && tid == 0) {
        // bounded: let the loads and MMAs in flight finish before the memory is released
        for (int i = max(0, loads - 2); i < loads; ++i) mbar_wait(smem_u32(&full[i & 1]), (uint32_t)(i >> 1) & 1u);
        for (int i = max(0, commits - 2); i < commits; ++i) mbar_wait(smem_u32(&mbar[i & 1]), (uint32_t)(i >> 1) & 1u);
        atomicOr(p.status, 1);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tbase, TMEM_COLS);
    if (!alive) return;

    const int row = row0 + (warp & 3) * 32 + (tid & 31);
    if (row >= L) return;
    const int er = p.ptE[(int64_t)m * L + row];
    const int *eB = p.xE + (int64_t)m * Nc;
    double *C = p.Gt + ((int64_t)m * L + row) * Nc;
#pragma unroll
    for (int g = 0; g < kCols / 4; ++g) {
        const int c0 = col0 + half * kCols + 4 * g;
        if (c0 >= Nc) break;
        double v[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) v[q] = i64_scaled(acc[4 * g + q], er + eB[c0 + q] - ACC_SHIFT);
        *reinterpret_cast<double2 *>(C + c0) = make_double2(v[0], v[1]);
        *reinterpret_cast<double2 *>(C + c0 + 2) = make_double2(v[2], v[3]);
        asm volatile("" ::: "memory");
    }
}

int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

}  // namespace

cudaError_t tc_prepare_kernels() {
    return cudaFuncSetAttribute(k_synthesis, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
}

cudaError_t tc_slice_table(const double *tab, int L, bool inverses, const int64_t *koff,
                           __nv_bfloat16 *out, int *expo, cudaStream_t s) {
    dim3 grid((unsigned)cdiv(L, 8), L);
    k_slice_rows_orders<<<grid, 256, 0, s>>>(tab, L, inverses, koff, out, expo);
    return cudaGetLastError();
}

cudaError_t tc_tf32_table(const double *tab, int L, bool inverses, const int64_t *koff, const int *expo,
                          float *out, cudaStream_t s) {
    dim3 grid((unsigned)cdiv(L, 8), L);
    k_tf32_rows_orders<<<grid, 256, 0, s>>>(tab, L, inverses, koff, expo, out);
    return cudaGetLastError();
}

cudaError_t tc_slice_orders(const double *X, int L, int64_t batch, const int64_t *koff,
                            __nv_bfloat16 *out, int *expo, cudaStream_t s) {
    const int Nc = (int)(4 * batch);
    dim3 grid((unsigned)cdiv(Nc, 32), L);
    k_slice_cols_orders<<<grid, 256, 0, s>>>(X, L, Nc, koff, out, expo);
    return cudaGetLastError();
}

cudaError_t tc_x_tensor_maps(int L, int64_t batch, const __nv_bfloat16 *xS,
                             const std::vector<int64_t> &ptk_off, unsigned char **d_maps) {
    const int Nc = (int)(4 * batch);
    std::vector<CUtensorMap> maps((size_t)L);
    for (int m = 0; m < L; ++m) {
        const cuuint64_t kp = (cuuint64_t)(((L - m) + 7) & ~7);
        const cuuint64_t dims[3] = {kp, (cuuint64_t)Nc, (cuuint64_t)S};
        const cuuint64_t strides[2] = {kp * 2, (cuuint64_t)Nc * kp * 2};
        const cuuint32_t box[3] = {(cuuint32_t)KB, (cuuint32_t)NT, (cuuint32_t)S};
        cudaError_t e = encode_tiled_map(&maps[m], xS + (int64_t)S * Nc * ptk_off[m], dims, strides, box);
        if (e != cudaSuccess) return e;
    }
    const size_t bytes = maps.size() * sizeof(CUtensorMap);
    cudaError_t e = cudaMalloc(d_maps, bytes);
    if (e != cudaSuccess) return e;
    return cudaMemcpy(*d_maps, maps.data(), bytes, cudaMemcpyHostToDevice);
}

cudaError_t tc_synthesis_all_orders(int L, int64_t batch, const int *ptE, const unsigned char *tmA,
                                    const int *xE, const unsigned char *tmB, double *Gt, int *status,
                                    uint64_t wait_ns, cudaStream_t s) {
    SynArgs p{};
    p.wait_ns = wait_ns;
    p.L = L; p.Nc = (int)(4 * batch); p.ptE = ptE; p.xE = xE; p.tmA = tmA; p.tmB = tmB; p.Gt = Gt;
    p.status = status;
    const int64_t grid = (int64_t)L * cdiv(L, MT) * cdiv(p.Nc, NT);
    k_synthesis<<<(unsigned)grid, kSynThreads, SMEM_BYTES, s>>>(p);
    return cudaGetLastError();
}

}  // namespace sht
