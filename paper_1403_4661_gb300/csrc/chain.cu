// The forward's order chain (Procedure 1 in bin space, Eqs. (14)-(16)) on the tensor cores as ONE
// persistent cooperative kernel.
//
// For m = L-1 .. 0 the chain solves F_m = P_m^{-1} g_m (g_m: bins +-m of rings k >= m, already free
// of the orders above m) and subtracts the aliased contribution of orders +-m from the bins of the
// rings k < m.  Each order depends on the one before (order m+1 aliases into ring m), so the
// orders run strictly in sequence; per order the work is two small contractions, n x n and
// m x n by n x 4B.  As separate launches each order costs several kernel starts, tensor-memory
// allocations and mostly idle SMs; here one CTA per SM stays resident for the whole chain, keeps
// its tensor memory and mbarriers, and the steps of an order are phases separated by grid-wide
// barriers:
//     slice g_m (float64 -> 8 exact BF16 slices per column)        | barrier
//     solve tiles x K-splits (tcgen05, as in tc_gemm.cu)           | barrier
//     [sum of the K-split partials in split order; F_m, f_l^{+-m}] | barrier
//     slice F_m                                                    | barrier
//     alias tiles x K-splits                                       | barrier
//     [sum of the partials; subtract from the bins of rings k < m] | barrier
// The cooperative launch guarantees that every CTA is resident, so the barriers cannot wait on a
// CTA that never runs.  Every wait is bounded (one second); a CTA that gives up sets the plan's
// status word and an abort word that every other CTA checks in its barrier waits, so all of them
// leave the chain promptly and release their tensor memory.  Data written by other SMs in an
// earlier phase is read through L2 (cp.async.cg, __ldcg), never through a possibly stale L1 line.
#include <cuda_bf16.h>

#include <algorithm>

#include "epilogue.cuh"
#include "sht_internal.cuh"
#include "tc_device.cuh"

namespace sht {
namespace {

// 8 warps: warps w and w + 4 share TMEM lane quarter w % 4 (rows 32 (w % 4) ..) and take output
// columns 0..31 and 32..63 of the tile, so each thread accumulates 32 int64 values.
constexpr int kThreads = 256;
constexpr int kCols = NT / 2;

struct ChainArgs {
    int L, Nc;                       // Nc = 4 * batch columns
    double *W, *F;                   // order-major bins and solved orders (rows_total x Nc)
    double2 *coeffs;
    const __nv_bfloat16 *piS; const int *piE; const int64_t *pik_off;   // P_m^{-1} slices
    const __nv_bfloat16 *ptS; const int *ptE; const int64_t *ptk_off;   // P~ slices
    __nv_bfloat16 *bS; int *bE;      // slices of the current right-hand sides: [S][Nc][kp], [Nc]
    double *part;                    // K-split partials: splits x M x Nc
    unsigned *bar;                   // [0] arrivals, [32] generation, [64] abort: separate 128-byte
                                     // lines (kChainBarWords, zeroed per launch)
    int *status;
};

// One contraction C (M x Nc) = A (M x K, plan slices) B (K x Nc, slices in bS).
struct Job {
    const __nv_bfloat16 *A; const int *eA; int64_t as; int kp;
    int M, K, tiles_n, tiles, splits, kchunk;
    bool direct;    // epilogue inside the MMA items (no K-splits, no read-modify-write)
};

__device__ __forceinline__ int cdiv_i(int a, int b) { return (a + b - 1) / b; }

__device__ Job make_job(const __nv_bfloat16 *A, const int *eA, int64_t as, int kp, int M, int K, int Nc,
                        bool rmw) {
    Job j;
    j.A = A; j.eA = eA; j.as = as; j.kp = kp; j.M = M; j.K = K;
    j.tiles_n = cdiv_i(Nc, NT);
    j.tiles = cdiv_i(M, MT) * j.tiles_n;
    j.splits = 1;
    j.kchunk = K;
    const int G = (int)gridDim.x;
    if (j.tiles < G) {
        // one round of items over the grid: K-splits of whole 32-row blocks
        int sp = min(min(G / j.tiles, cdiv_i(K, KB)), kSplitCap);
        if (sp > 1) {
            const int kc = cdiv_i(cdiv_i(K, sp), KB) * KB;
            sp = cdiv_i(K, kc);
            if (sp > 1) { j.splits = sp; j.kchunk = kc; }
        }
    }
    // a read-modify-write epilogue (alias bins) always goes through the reduction phase, where
    // one thread per row group keeps many loads in flight
    j.direct = j.splits == 1 && !rmw;
    return j;
}

__device__ __forceinline__ bool aborted(const ChainArgs &p) {
    return *(volatile unsigned *)(p.bar + 64) != 0u;
}
__device__ __forceinline__ void raise_abort(const ChainArgs &p, int bit) {
    atomicOr(p.status, bit);
    atomicExch(p.bar + 64, 1u);
}

// Grid-wide barrier; false (for every thread of the CTA) once any CTA has given up.
__device__ bool grid_barrier(const ChainArgs &p, int *s_flag) {
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        volatile unsigned *gen = p.bar + 32;
        const unsigned g = *gen;
        __threadfence();
        if (atomicAdd(p.bar, 1u) == gridDim.x - 1) {
            atomicExch(p.bar, 0u);
            __threadfence();
            atomicAdd(p.bar + 32, 1u);
        } else {
            const uint64_t t0 = global_ns();
            while (*gen == g) {
                if (aborted(p)) { ok = 0; break; }
                if (global_ns() - t0 > 1000000000ull) { raise_abort(p, 2); ok = 0; break; }
                __nanosleep(32);
            }
        }
        __threadfence();
        if (aborted(p)) ok = 0;
        *s_flag = ok;
    }
    __syncthreads();
    return *s_flag != 0;
}

// Slices of the n x Nc float64 block X (row-major) as right-hand sides: one warp per column,
// scale exponent over the column, zero padding to kp.
__device__ __noinline__ void slice_phase(const ChainArgs &p, const double *X, int n, int kp) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int Nc = p.Nc;
    const int64_t sstride = (int64_t)Nc * kp;
    for (int j = blockIdx.x * (kThreads / 32) + warp; j < Nc; j += (kThreads / 32) * gridDim.x) {
        int mf = 0;
        for (int k0 = lane; k0 < n; k0 += 32 * 8) {
            double x[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int k = k0 + 32 * u;
                x[u] = k < n ? __ldcg(X + (int64_t)k * Nc + j) : 0.0;
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) mf = max(mf, exp_field(x[u]));
        }
        for (int o = 16; o > 0; o >>= 1) mf = max(mf, __shfl_xor_sync(0xffffffffu, mf, o));
        const int e = scale_from_field(mf);
        if (lane == 0) p.bE[j] = e;
        __nv_bfloat16 *out = p.bS + (int64_t)j * kp;
        for (int k0 = lane; k0 < kp; k0 += 32 * 4) {
            double x[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int k = k0 + 32 * u;
                x[u] = k < n ? __ldcg(X + (int64_t)k * Nc + j) : 0.0;   // rows n..kp-1: zero padding
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int k = k0 + 32 * u;
                if (k >= kp) break;
                __nv_bfloat16 sl[S];
                split_value(x[u], e, sl);
#pragma unroll
                for (int s = 0; s < S; ++s) out[s * sstride + k] = sl[s];
            }
        }
    }
}

// The contraction's items (output tile, K-split), one per CTA and round.  Without K-splits the
// epilogue runs here; with them each item stores its float64 partial.  `ok` turns false (for the
// whole CTA) when an mbarrier wait gives up.
template <int EPI, int NSL>
__device__ __forceinline__ void mma_phase(const ChainArgs &p, const Job &jb, const EpiArgs &epi, uint32_t tbase,
                          unsigned char *smem, uint64_t *mbar, uint32_t uses[2], bool &ok) {
    constexpr bool EXACT = NSL == S;
    constexpr int NREG = EXACT ? REGIONS : 1;
    constexpr int SHIFT = EXACT ? ACC_SHIFT : 40;
    const int tid = threadIdx.x, warp = tid >> 5, half = warp >> 2;
    const int Nc = p.Nc, kp = jb.kp, M = jb.M;
    const __nv_bfloat16 *A = jb.A, *B = p.bS;
    const int64_t as = jb.as, bs = (int64_t)Nc * kp;
    const int items = jb.tiles * jb.splits;
    __shared__ int s_eb[NT];   // scale exponents of the tile's B columns
    for (int it = blockIdx.x; it < items && ok; it += gridDim.x) {
        const int tile = it / jb.splits, y = it - tile * jb.splits;
        const int tm = tile / jb.tiles_n, tn = tile - tm * jb.tiles_n;
        const int row0 = tm * MT, col0 = tn * NT;
        const int kbeg = y * jb.kchunk, kend = min(jb.K, kbeg + jb.kchunk);
        __syncthreads();   // the previous item's epilogue is done with s_eb
        if (tid < NT) s_eb[tid] = col0 + tid < Nc ? __ldcg(p.bE + col0 + tid) : 0;

        auto load = [&](int kb, int st) {
            const uint32_t sa = smem_u32(smem + st * STAGE), sb = sa + A_STAGE;
            const int kbase = kb * KB;
            for (int idx = tid; idx < NSL * MT * 4; idx += kThreads) {
                const int j = idx & 3, r = (idx >> 2) & (MT - 1), s = idx >> 9;
                const int row = row0 + r, kc = kbase + 8 * j;
                const bool in = row < M && kc < kp;
                const __nv_bfloat16 *src = in ? A + s * as + (int64_t)row * kp + kc : A;
                cp_async16(sa + s * (MT * KB * 2) + j * (MT * 16) + (r >> 3) * 128 + (r & 7) * 16, src, in ? 16 : 0);
            }
            for (int idx = tid; idx < NSL * NT * 4; idx += kThreads) {
                const int j = idx & 3, r = (idx >> 2) & (NT - 1), s = idx >> 8;
                const int row = col0 + r, kc = kbase + 8 * j;
                const bool in = row < Nc && kc < kp;
                const __nv_bfloat16 *src = in ? B + s * bs + (int64_t)row * kp + kc : B;
                cp_async16(sb + s * (NT * KB * 2) + j * (NT * 16) + (r >> 3) * 128 + (r & 7) * 16, src, in ? 16 : 0);
            }
            cp_async_commit();
        };

        long long acc[kCols];   // columns half * kCols .. of row quarter * 32 + lane
#pragma unroll
        for (int c = 0; c < kCols; ++c) acc[c] = 0;
        const int kb0 = kbeg / KB, nkb = (kend + KB - 1) / KB;
        load(kb0, 0);
        for (int kb = kb0; kb < nkb; ++kb) {
            const int st = (kb - kb0) & 1;
            if (kb + 1 < nkb) {
                const int ns = st ^ 1;
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
                    if (kg == kbeg || (EXACT && kg % CHUNK == 0))
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
                const bool w = mbar_wait(smem_u32(&mbar[st]), (uses[st] - 1) & 1u);
                if (!__syncthreads_and(w)) { ok = false; break; }
                tc_fence_after();
                const uint32_t lane_base = tbase + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)(half * kCols);
                if (EXACT) {
#pragma unroll
                    for (int reg = 0; reg < NREG; ++reg) {
                        const int d = reg + 2;
                        const float up = reg < NREG - 1 ? __int_as_float((127 + 7 * d) << 23)
                                                        : __int_as_float((127 + ACC_SHIFT) << 23);
                        const int shift = reg < NREG - 1 ? ACC_SHIFT - 7 * d : 0;
#pragma unroll
                        for (int c0 = 0; c0 < kCols; c0 += 16) {
                            float v[16];
                            tmem_ld16(lane_base + reg * NT + c0, v);
#pragma unroll
                            for (int i = 0; i < 16; ++i)
                                acc[c0 + i] += (long long)__float2int_rn(v[i] * up) << shift;
                        }
                    }
                } else {
#pragma unroll
                    for (int c0 = 0; c0 < kCols; c0 += 16) {
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
        if (!ok) break;

        const int row = row0 + (warp & 3) * 32 + (tid & 31);
        if (row < M) {
            const int er = jb.eA[row];
#pragma unroll
            for (int g = 0; g < kCols / 4; ++g) {
                const int cl = half * kCols + 4 * g, c0 = col0 + cl;
                if (c0 >= Nc) break;
                double v[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) v[q] = i64_scaled(acc[4 * g + q], er + s_eb[cl + q] - SHIFT);
                if (jb.direct) {
                    epilogue_row4<EPI>(epi, row, c0, v);
                } else {
                    double *pp = p.part + ((int64_t)y * M + row) * Nc + c0;
                    *reinterpret_cast<double2 *>(pp) = make_double2(v[0], v[1]);
                    *reinterpret_cast<double2 *>(pp + 2) = make_double2(v[2], v[3]);
                }
                asm volatile("" ::: "memory");   // one group at a time (register pressure)
            }
        }
    }
}

// Sum of the K-split partials in split order (deterministic), then the epilogue.
template <int EPI>
__device__ __noinline__ void reduce_phase(const ChainArgs &p, const EpiArgs &epi, int M, int splits) {
    const int Nc = p.Nc, groups = Nc / 4;
    const int64_t total = (int64_t)M * groups;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(t / groups), c0 = 4 * (int)(t - (int64_t)r * groups);
        // partials in split order, four loads in flight at a time
        double v[4] = {0.0, 0.0, 0.0, 0.0};
        for (int y0 = 0; y0 < splits; y0 += 4) {
            double2 a[4], b[4];
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (y0 + u < splits) {
                    const double2 *pp =
                        reinterpret_cast<const double2 *>(p.part + ((int64_t)(y0 + u) * M + r) * Nc + c0);
                    a[u] = __ldcg(pp);
                    b[u] = __ldcg(pp + 1);
                }
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (y0 + u < splits) { v[0] += a[u].x; v[1] += a[u].y; v[2] += b[u].x; v[3] += b[u].y; }
        }
        epilogue_row4<EPI>(epi, r, c0, v);
    }
}

template <int NSL>
__global__ void __launch_bounds__(kThreads, 1) k_chain(ChainArgs p) {
    constexpr uint32_t NCOLS = NSL == S ? TMEM_COLS : 64u;
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ uint64_t mbar[2];
    __shared__ uint32_t tmem_slot;
    __shared__ int s_flag;
    const int tid = threadIdx.x, warp = tid >> 5;
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

    uint32_t uses[2] = {0u, 0u};
    bool ok = true, mma_ok = true;
    const int L = p.L, Nc = p.Nc;
    for (int m = L - 1; m >= 0; --m) {
        const int n = L - m, kp = (n + 7) & ~7;
        // Eq. (14): F_m = P_m^{-1} g_m
        slice_phase(p, p.W + rows_off(L, m) * Nc, n, kp);
        if (!(ok = grid_barrier(p, &s_flag))) break;
        const Job js = make_job(p.piS + (int64_t)S * p.pik_off[m], p.piE + rows_off(L, m), (int64_t)n * kp,
                                kp, n, n, Nc, false);
        const EpiArgs es{p.F + rows_off(L, m) * Nc, Nc, nullptr, m, L, Nc, p.coeffs, nullptr};
        mma_phase<EPI_SOLVE, NSL>(p, js, es, tbase, smem, mbar, uses, mma_ok);
        if (!mma_ok) { if (tid == 0) raise_abort(p, 1); ok = false; break; }
        if (!(ok = grid_barrier(p, &s_flag))) break;
        if (!js.direct) {
            reduce_phase<EPI_SOLVE>(p, es, n, js.splits);
            if (!(ok = grid_barrier(p, &s_flag))) break;
        }
        if (m == 0) break;
        // Eqs. (15)-(16): orders +-m out of the bins of rings k < m
        slice_phase(p, p.F + rows_off(L, m) * Nc, n, kp);
        if (!(ok = grid_barrier(p, &s_flag))) break;
        const Job ja = make_job(p.ptS + (int64_t)S * L * p.ptk_off[m], p.ptE + (int64_t)m * L, (int64_t)L * kp,
                                kp, m, n, Nc, true);
        const EpiArgs ea{nullptr, Nc, nullptr, m, L, Nc, nullptr, p.W};
        mma_phase<EPI_ALIAS, NSL>(p, ja, ea, tbase, smem, mbar, uses, mma_ok);
        if (!mma_ok) { if (tid == 0) raise_abort(p, 1); ok = false; break; }
        if (!(ok = grid_barrier(p, &s_flag))) break;
        if (!ja.direct) {
            reduce_phase<EPI_ALIAS>(p, ea, m, ja.splits);
            if (!(ok = grid_barrier(p, &s_flag))) break;
        }
    }
    if (!mma_ok) {
        // let the MMAs in flight finish (bounded) before the tensor memory is released
        for (int st = 0; st < 2; ++st)
            if (uses[st] > 0) mbar_wait(smem_u32(&mbar[st]), (uses[st] - 1) & 1u);
    }
    (void)ok;
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tbase, NCOLS);
}

template <int NSL>
cudaError_t launch_chain(const ChainArgs &p, int grid, cudaStream_t s) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = SMEM_BYTES;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_chain<NSL>, p);
}

}  // namespace

cudaError_t tc_prepare_chain(int *grid) {
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(k_chain<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES)) != cudaSuccess ||
        (e = cudaFuncSetAttribute(k_chain<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES)) != cudaSuccess ||
        (e = cudaFuncSetAttribute(k_chain<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES)) != cudaSuccess)
        return e;
    int dev = 0, sms = 0, per_sm = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_chain<S>, kThreads, SMEM_BYTES)) != cudaSuccess)
        return e;
    // one CTA per SM (the kernel holds the SM's tensor memory); never more than can be resident
    *grid = std::min(sms, sms * per_sm);
    return *grid > 0 ? cudaSuccess : cudaErrorInvalidConfiguration;
}

cudaError_t tc_forward_chain(const ChainTables &t, int L, int64_t batch, double *W, double *F,
                             double2 *coeffs, __nv_bfloat16 *bS, int *bE, double *part,
                             unsigned *bar, int *status, int nsl, int grid, cudaStream_t s) {
    ChainArgs p{};
    p.L = L; p.Nc = (int)(4 * batch);
    p.W = W; p.F = F; p.coeffs = coeffs;
    p.piS = t.piS; p.piE = t.piE; p.pik_off = t.pik_off;
    p.ptS = t.ptS; p.ptE = t.ptE; p.ptk_off = t.ptk_off;
    p.bS = bS; p.bE = bE; p.part = part; p.bar = bar; p.status = status;
    cudaError_t e = cudaMemsetAsync(bar, 0, kChainBarWords * sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    if (nsl == S) return launch_chain<S>(p, grid, s);
    if (nsl == 2) return launch_chain<2>(p, grid, s);
    if (nsl == 1) return launch_chain<1>(p, grid, s);
    return cudaErrorInvalidValue;
}

}  // namespace sht
