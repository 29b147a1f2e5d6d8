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
// Kernel: one CTA of 4 warps per 128 x 64 output tile; operands staged through shared memory in
// the canonical no-swizzle K-major layout (8-row x 16-byte core matrices) by cp.async, two
// stages of 32 K; one thread issues the 36 slice-pair MMAs (M = 128, N = 64, K = 16) per 16 K and
// commits them to an mbarrier per stage; every wait is bounded (1 s) and reports through a
// status word.
#include <cuda_bf16.h>

#include <algorithm>

#include "epilogue.cuh"
#include "sht_internal.cuh"
#include "tc_device.cuh"

namespace sht {
namespace {

// X row-major (rows x K, leading dim ld); one warp per row.
__global__ void k_slice_rows(const double *__restrict__ X, int64_t ld, int rows, int K, int kp,
                             __nv_bfloat16 *__restrict__ out, int64_t sstride, int *__restrict__ expo) {
    const int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (row >= rows) return;
    slice_row_warp(X + (int64_t)row * ld, 1, K, kp, out + (int64_t)row * kp, sstride, expo + row);
}

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

// One warp per column (the order chain's per-step operands: few columns, many warps).
__global__ void k_slice_cols(const double *__restrict__ X, int64_t ld, int K, int cols, int kp,
                             __nv_bfloat16 *__restrict__ out, int64_t sstride, int *__restrict__ expo) {
    const int j = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (j >= cols) return;
    slice_row_warp(X + j, ld, K, kp, out + (int64_t)j * kp, sstride, expo + j);
}

// Order-major coefficients X (block m: L - m rows of Nc columns), every order m = blockIdx.y.
__global__ void k_slice_cols_orders(const double *__restrict__ X, int L, int Nc,
                                    const int64_t *__restrict__ koff, __nv_bfloat16 *__restrict__ out,
                                    int *__restrict__ expo) {
    const int m = blockIdx.y, n = L - m, kp = (n + 7) & ~7;
    slice_cols_block(X + rows_off(L, m) * Nc, Nc, n, Nc, kp, out + (int64_t)S * Nc * koff[m],
                     (int64_t)Nc * kp, expo + (int64_t)m * Nc, blockIdx.x * 32);
}

// ---------------------------------------------------------------- the GEMM
struct TcArgs {
    // single problem
    const __nv_bfloat16 *A; const int *eA; int64_t as; int akp;
    const __nv_bfloat16 *B; const int *eB; int64_t bs; int bkp;
    int M, N, K;
    EpiArgs epi;
    // grouped over orders (synthesis): per m, A = P~ slices, B = X slices
    int L;
    const __nv_bfloat16 *ptS; const int *ptE; const int64_t *kpoff;
    const __nv_bfloat16 *xS; const int *xE;
    double *Gt;
    int *status;
    // split-K: blockIdx.y selects K range [y * kchunk, (y + 1) * kchunk); float64 partials to part
    int kchunk;
    double *part;
};

// NSL = slices used per operand: kTcSlices for float64-accurate products (exact diagonals,
// chunked int64 folding), or 1..2 for the low-precision products of the refinement (every pair in
// one FP32 region over the whole K, converted once at the end).
template <int EPI, bool GROUPED, bool SPLIT, int NSL>
__global__ void __launch_bounds__(128, 1) k_tc_gemm(TcArgs p) {
    constexpr bool EXACT = NSL == S;
    constexpr int NREG = EXACT ? REGIONS : 1;
    constexpr uint32_t NCOLS = EXACT ? TMEM_COLS : 64u;
    constexpr int SHIFT = EXACT ? ACC_SHIFT : 40;
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ uint64_t mbar[2];
    __shared__ uint32_t tmem_slot;
    const int tid = threadIdx.x, warp = tid >> 5;

    const __nv_bfloat16 *A = p.A, *B = p.B;
    const int *eA = p.eA, *eB = p.eB;
    int64_t as = p.as, bs = p.bs;
    int akp = p.akp, bkp = p.bkp, M = p.M, N = p.N, K = p.K;
    EpiArgs epi = p.epi;
    const int tiles_n = (N + NT - 1) / NT;
    int64_t tile = blockIdx.x;
    if (GROUPED) {
        const int L = p.L;
        const int64_t per_m = (int64_t)((L + MT - 1) / MT) * tiles_n;
        const int m = (int)(tile / per_m);
        tile -= (int64_t)m * per_m;
        const int n = L - m, kp = (n + 7) & ~7;
        const int64_t off = p.kpoff[m];
        A = p.ptS + (int64_t)S * L * off; as = (int64_t)L * kp; akp = kp; eA = p.ptE + (int64_t)m * L;
        B = p.xS + (int64_t)S * N * off; bs = (int64_t)N * kp; bkp = kp; eB = p.xE + (int64_t)m * N;
        M = L; K = n;
        epi.C = p.Gt + (int64_t)m * L * N; epi.ldc = N; epi.m = m;
    }
    const int tm = (int)(tile / tiles_n), tn = (int)(tile % tiles_n);
    const int row0 = tm * MT, col0 = tn * NT;
    int kbeg = 0, kend = K;
    if (SPLIT) {
        kbeg = blockIdx.y * p.kchunk;   // a multiple of CHUNK
        kend = min(K, kbeg + p.kchunk);
    }

    if (warp == 0) tmem_alloc(smem_u32(&tmem_slot), NCOLS);
    if (tid == 0) {
        mbar_init(smem_u32(&mbar[0]), 1);
        mbar_init(smem_u32(&mbar[1]), 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tbase = tmem_slot;

    // stage loader: A slices rows row0.., B slices rows col0.., k-block kb
    auto load = [&](int kb, int st) {
        const uint32_t sa = smem_u32(smem + st * STAGE), sb = sa + A_STAGE;
        const int kbase = kb * KB;
        for (int idx = tid; idx < NSL * MT * 4; idx += 128) {
            const int j = idx & 3, r = (idx >> 2) & (MT - 1), s = idx >> 9;
            const int row = row0 + r, kc = kbase + 8 * j;
            const bool ok = row < M && kc < akp;
            const __nv_bfloat16 *src = ok ? A + s * as + (int64_t)row * akp + kc : A;
            cp_async16(sa + s * (MT * KB * 2) + j * (MT * 16) + (r >> 3) * 128 + (r & 7) * 16, src, ok ? 16 : 0);
        }
        for (int idx = tid; idx < NSL * NT * 4; idx += 128) {
            const int j = idx & 3, r = (idx >> 2) & (NT - 1), s = idx >> 8;
            const int row = col0 + r, kc = kbase + 8 * j;
            const bool ok = row < N && kc < bkp;
            const __nv_bfloat16 *src = ok ? B + s * bs + (int64_t)row * bkp + kc : B;
            cp_async16(sb + s * (NT * KB * 2) + j * (NT * 16) + (r >> 3) * 128 + (r & 7) * 16, src, ok ? 16 : 0);
        }
        cp_async_commit();
    };

    long long acc[NT];  // C * 2^-(eA + eB) * 2^49, exact integer accumulation across chunks
#pragma unroll
    for (int c = 0; c < NT; ++c) acc[c] = 0;

    const int kb0 = kbeg / KB, nkb = (kend + KB - 1) / KB;
    uint32_t uses[2] = {0u, 0u};
    bool ok = true;
    if (kb0 < nkb) load(kb0, 0);
    for (int kb = kb0; kb < nkb && ok; ++kb) {
        const int st = (kb - kb0) & 1;
        if (kb + 1 < nkb) {
            const int ns = st ^ 1;
            // the MMAs that read stage ns (k-block kb - 1) must be done before it is refilled;
            // the vote keeps every thread on the same path if the wait gives up
            const bool w = uses[ns] == 0 || mbar_wait(smem_u32(&mbar[ns]), (uses[ns] - 1) & 1u);
            if (!__syncthreads_and(w)) { ok = false; break; }
            load(kb + 1, ns);
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        fence_proxy_async();
        __syncthreads();
        if (tid == 0) {
            tc_fence_after();
            const uint32_t sa = smem_u32(smem + st * STAGE), sb = sa + A_STAGE;
            bool fresh[REGIONS] = {false, false, false, false, false, false};
            for (int h = 0; h < 2; ++h) {
                const int kg = kb * KB + 16 * h;
                if (kg >= kend) break;
                if (EXACT ? (kg % CHUNK == 0) : (kg == kbeg))
                    for (int r = 0; r < REGIONS; ++r) fresh[r] = true;
                for (int s = 1; s <= NSL; ++s)
                    for (int t = 1; s + t <= NSL + 1; ++t) {
                        const int d = s + t, reg = EXACT ? (d <= 6 ? d - 2 : 5) : 0;
                        const uint64_t ad = sdesc(sa + (s - 1) * (MT * KB * 2) + 2 * h * (MT * 16), MT * 16, 128);
                        const uint64_t bd = sdesc(sb + (t - 1) * (NT * KB * 2) + 2 * h * (NT * 16), NT * 16, 128);
                        mma_bf16(tbase + reg * NT, ad, bd, kIdesc, fresh[reg] ? 0u : 1u);
                        fresh[reg] = false;
                    }
            }
            mma_commit(smem_u32(&mbar[st]));
        }
        uses[st] += 1;
        const int kdone = (kb + 1) * KB;
        if ((EXACT && kdone % CHUNK == 0) || kb == nkb - 1) {
            // the commit of this stage covers every MMA issued so far
            const bool w = mbar_wait(smem_u32(&mbar[st]), (uses[st] - 1) & 1u);
            if (!__syncthreads_and(w)) { ok = false; break; }
            tc_fence_after();
            const uint32_t lane_base = tbase + ((uint32_t)(warp * 32) << 16);
            if (EXACT) {
#pragma unroll
                for (int reg = 0; reg < NREG; ++reg) {
                    // region reg holds diagonal d = reg + 2 (multiples of 2^-7d, exact), or the
                    // rounded sum of d >= 7 for the last region
                    const int d = reg + 2;
                    const float up = reg < NREG - 1 ? __int_as_float((127 + 7 * d) << 23)
                                                    : __int_as_float((127 + ACC_SHIFT) << 23);
                    const int shift = reg < NREG - 1 ? ACC_SHIFT - 7 * d : 0;
#pragma unroll
                    for (int c0 = 0; c0 < NT; c0 += 16) {
                        float v[16];
                        tmem_ld16(lane_base + reg * NT + c0, v);
#pragma unroll
                        for (int i = 0; i < 16; ++i)
                            acc[c0 + i] += (long long)__float2int_rn(v[i] * up) << shift;
                    }
                }
            } else {
                // one rounded FP32 sum over the whole K: sum < 2^13, kept at 2^-40 resolution
#pragma unroll
                for (int c0 = 0; c0 < NT; c0 += 16) {
                    float v[16];
                    tmem_ld16(lane_base + c0, v);
#pragma unroll
                    for (int i = 0; i < 16; ++i) acc[c0 + i] = __float2ll_rn(v[i] * 0x1p40f);
                }
            }
            tc_fence_before();
            __syncthreads();
        }
    }
    cp_async_wait<0>();
    if (!ok) {
        // let the MMAs in flight finish (bounded) before the tensor memory is released
        for (int st = 0; st < 2; ++st)
            if (uses[st] > 0) mbar_wait(smem_u32(&mbar[st]), (uses[st] - 1) & 1u);
        if (tid == 0) atomicOr(p.status, 1);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tbase, NCOLS);
    if (!ok) return;

    const int row = row0 + tid;
    if (row >= M) return;
    const int er = eA[row];
#pragma unroll
    for (int g = 0; g < NT / 4; ++g) {
        const int c0 = col0 + 4 * g;
        if (c0 >= N) break;
        double v[4];
#pragma unroll
        for (int q = 0; q < 4; ++q)
            v[q] = (c0 + q < N) ? i64_scaled(acc[4 * g + q], er + eB[c0 + q] - SHIFT) : 0.0;
        if (SPLIT) {
            double *pp = p.part + ((int64_t)blockIdx.y * M + row) * N + c0;
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (c0 + q < N) pp[q] = v[q];
        } else {
            epilogue_row4<EPI>(epi, row, c0, v);
        }
    }
}

// Fixed-order sum of the split-K partials, then the epilogue (deterministic).
template <int EPI>
__global__ void k_tc_reduce(EpiArgs e, const double *__restrict__ part, int splits, int M) {
    const int groups = (e.N + 3) / 4;
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)M * groups) return;
    const int r = (int)(t / groups), c0 = 4 * (int)(t - (int64_t)r * groups);
    double v[4] = {0.0, 0.0, 0.0, 0.0};
    for (int s = 0; s < splits; ++s) {
        const double *pp = part + ((int64_t)s * M + r) * e.N + c0;
#pragma unroll
        for (int q = 0; q < 4; ++q)
            if (c0 + q < e.N) v[q] += pp[q];
    }
    epilogue_row4<EPI>(e, r, c0, v);
}

int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

template <typename Kern>
cudaError_t prepare(Kern k) {
    return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
}

template <int NSL>
cudaError_t prepare_all() {
    cudaError_t e;
    if ((e = prepare(k_tc_gemm<EPI_STORE, false, false, NSL>)) != cudaSuccess) return e;
    if ((e = prepare(k_tc_gemm<EPI_STORE, true, false, NSL>)) != cudaSuccess) return e;
    if ((e = prepare(k_tc_gemm<EPI_SOLVE, false, false, NSL>)) != cudaSuccess) return e;
    if ((e = prepare(k_tc_gemm<EPI_ALIAS, false, false, NSL>)) != cudaSuccess) return e;
    if ((e = prepare(k_tc_gemm<EPI_STORE, false, true, NSL>)) != cudaSuccess) return e;
    if ((e = prepare(k_tc_gemm<EPI_SOLVE, false, true, NSL>)) != cudaSuccess) return e;
    return prepare(k_tc_gemm<EPI_ALIAS, false, true, NSL>);
}

template <bool SPLIT, int NSL>
cudaError_t launch_tc(int epi, dim3 grid, const TcArgs &p, cudaStream_t s) {
    switch (epi) {
        case EPI_STORE: k_tc_gemm<EPI_STORE, false, SPLIT, NSL><<<grid, 128, SMEM_BYTES, s>>>(p); break;
        case EPI_SOLVE: k_tc_gemm<EPI_SOLVE, false, SPLIT, NSL><<<grid, 128, SMEM_BYTES, s>>>(p); break;
        case EPI_ALIAS: k_tc_gemm<EPI_ALIAS, false, SPLIT, NSL><<<grid, 128, SMEM_BYTES, s>>>(p); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <bool SPLIT>
cudaError_t launch_tc_nsl(int nsl, int epi, dim3 grid, const TcArgs &p, cudaStream_t s) {
    if (nsl == S) return launch_tc<SPLIT, S>(epi, grid, p, s);
    if (nsl == 2) return launch_tc<SPLIT, 2>(epi, grid, p, s);
    if (nsl == 1) return launch_tc<SPLIT, 1>(epi, grid, p, s);
    return cudaErrorInvalidValue;
}

}  // namespace

cudaError_t tc_prepare_kernels() {
    cudaError_t e;
    if ((e = prepare_all<S>()) != cudaSuccess) return e;
    if ((e = prepare_all<2>()) != cudaSuccess) return e;
    return prepare_all<1>();
}

cudaError_t tc_slice_rows(const double *X, int64_t ld, int rows, int K, int kp, __nv_bfloat16 *out,
                          int64_t sstride, int *expo, cudaStream_t s) {
    if (rows <= 0) return cudaSuccess;
    k_slice_rows<<<(unsigned)cdiv(rows, 8), 256, 0, s>>>(X, ld, rows, K, kp, out, sstride, expo);
    return cudaGetLastError();
}

cudaError_t tc_slice_cols(const double *X, int64_t ld, int K, int cols, int kp, __nv_bfloat16 *out,
                          int64_t sstride, int *expo, cudaStream_t s) {
    if (cols <= 0) return cudaSuccess;
    k_slice_cols<<<(unsigned)cdiv(cols, 8), 256, 0, s>>>(X, ld, K, cols, kp, out, sstride, expo);
    return cudaGetLastError();
}

cudaError_t tc_slice_table(const double *tab, int L, bool inverses, const int64_t *koff,
                           __nv_bfloat16 *out, int *expo, cudaStream_t s) {
    dim3 grid((unsigned)cdiv(L, 8), L);
    k_slice_rows_orders<<<grid, 256, 0, s>>>(tab, L, inverses, koff, out, expo);
    return cudaGetLastError();
}

cudaError_t tc_slice_orders(const double *X, int L, int64_t batch, const int64_t *koff,
                            __nv_bfloat16 *out, int *expo, cudaStream_t s) {
    const int Nc = (int)(4 * batch);
    dim3 grid((unsigned)cdiv(Nc, 32), L);
    k_slice_cols_orders<<<grid, 256, 0, s>>>(X, L, Nc, koff, out, expo);
    return cudaGetLastError();
}

cudaError_t tc_gemm(const TcOperand &a, const TcOperand &b, int M, int N, int K, int epi,
                    const TcEpilogue &ep, int *status, cudaStream_t s, double *part,
                    int64_t part_cap, int64_t *launches, int nsl) {
    if (M <= 0 || N <= 0) return cudaSuccess;
    TcArgs p{};
    p.A = a.data; p.eA = a.expo; p.as = a.slice_stride; p.akp = a.kp;
    p.B = b.data; p.eB = b.expo; p.bs = b.slice_stride; p.bkp = b.kp;
    p.M = M; p.N = N; p.K = K; p.status = status;
    p.epi = EpiArgs{ep.C, ep.ldc, ep.C0, ep.m, ep.L, N, ep.coeffs, ep.W};
    const int64_t tiles = cdiv(M, MT) * cdiv(N, NT);
    // split K over enough blocks to cover the SMs (chunks of CHUNK keep the exact accumulation)
    int splits = 1;
    if (part && tiles < kNumSMs) {
        splits = (int)std::min<int64_t>(std::min<int64_t>(cdiv(kNumSMs, tiles), cdiv(K, CHUNK)), 16);
        while (splits > 1 && (int64_t)splits * M * N > part_cap) --splits;
    }
    if (splits > 1) {
        p.kchunk = (int)(cdiv(cdiv(K, splits), CHUNK) * CHUNK);
        splits = (int)cdiv(K, p.kchunk);
    }
    if (launches) *launches += splits > 1 ? 2 : 1;
    if (splits <= 1) return launch_tc_nsl<false>(nsl, epi, dim3((unsigned)tiles), p, s);
    p.part = part;
    cudaError_t e = launch_tc_nsl<true>(nsl, epi, dim3((unsigned)tiles, splits), p, s);
    if (e != cudaSuccess) return e;
    const int64_t work = (int64_t)M * cdiv(N, 4);
    const unsigned rg = (unsigned)cdiv(work, 256);
    switch (epi) {
        case EPI_STORE: k_tc_reduce<EPI_STORE><<<rg, 256, 0, s>>>(p.epi, part, splits, M); break;
        case EPI_SOLVE: k_tc_reduce<EPI_SOLVE><<<rg, 256, 0, s>>>(p.epi, part, splits, M); break;
        case EPI_ALIAS: k_tc_reduce<EPI_ALIAS><<<rg, 256, 0, s>>>(p.epi, part, splits, M); break;
    }
    return cudaGetLastError();
}

cudaError_t tc_synthesis_all_orders(int L, int64_t batch, const __nv_bfloat16 *ptS, const int *ptE,
                                    const int64_t *kpoff, const __nv_bfloat16 *xS, const int *xE,
                                    double *Gt, int *status, cudaStream_t s) {
    TcArgs p{};
    p.L = L; p.N = (int)(4 * batch); p.ptS = ptS; p.ptE = ptE; p.kpoff = kpoff; p.xS = xS; p.xE = xE;
    p.Gt = Gt; p.status = status;
    p.epi = EpiArgs{nullptr, p.N, nullptr, 0, L, p.N, nullptr, nullptr};
    const int64_t grid = (int64_t)L * cdiv(L, MT) * cdiv(p.N, NT);
    k_tc_gemm<EPI_STORE, true, false, S><<<(unsigned)grid, 128, SMEM_BYTES, s>>>(p);
    return cudaGetLastError();
}

}  // namespace sht
