// The forward's order chain (Procedure 1 in bin space, Eqs. (14)-(16)) on the tensor cores as ONE
// persistent cooperative kernel.
//
// For m = L-1 .. 0 the chain solves F_m = P_m^{-1} g_m (g_m: bins +-m of rings k >= m, already free
// of the orders above m) and subtracts the aliased contribution of orders +-m from the bins of the
// rings k < m.  Each order depends on the one before (order m+1 aliases into ring m), so the
// orders run strictly in sequence; per order the work is two small contractions, n x n and
// m x n by n x 4B.  As separate launches each order costs several kernel starts, tensor-memory
// allocations and mostly idle SMs; here one CTA per SM stays resident for the whole chain, keeps
// its tensor memory and mbarriers, and the steps of an order are three phases separated by
// grid-wide barriers:
//     solve: tiles x K-splits of P_m^{-1} g_m (tcgen05 on exact BF16 slices)      | barrier
//     sum of the solve's K-split partials -> F_m, f_l^{+-m}, column scales of F_m;
//         order m+1's alias partials subtracted from the bins of rings k < m;
//         column scales of g_{m-1} without its first row (rings >= m, final now)  | barrier
//     alias: tiles x K-splits of P~_m(rings k < m) F_m                             | barrier
// Order m's alias products reach ring m - 1, the first row of g_{m-1}, before they are summed
// into the bins: the items of solve m - 1 add that row's partials up themselves (a few hundred
// values), so no phase waits for the alias subtraction, which runs beside the next reduction.
// The right-hand sides are read in float64 and cut into slices while they are staged in shared
// memory, with the column scales the previous phase gathered; the plan tables (P_m^{-1}, P~) are
// pre-sliced.
//
// The cooperative launch guarantees that every CTA is resident, so the barriers cannot wait on a
// CTA that never runs.  Every wait is bounded (one second); a CTA that gives up sets the plan's
// status word and an abort word that every other CTA checks in its barrier waits, so all of them
// leave the chain promptly and release their tensor memory.  Data written by other SMs in an
// earlier phase is read through L2 (cp.async.cg, __ldcg), never through a possibly stale L1 line.
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <vector>

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
    long long *part_s, *part_a;      // K-split partials of the solves and of the alias products,
                                     // int64 at the scale of the output element (2^-(eA + eB)
                                     // 2^shift): splits x M x Nc
    unsigned *bar;                   // [0] arrivals (monotonic within a launch), [64] abort:
                                     // separate 128-byte lines
    int *eW, *eF;                    // [2][Nc] largest exponent fields of the columns of g_m
                                     // without its first row, and of F_m (slot m & 1)
    int *fS;                         // [Nc] fields of g_m's columns, first row included
                                     // (all of bar, eW, eF, fS zeroed per launch)
    uint64_t wait_ns;                // limit of every wait on other CTAs or on the pipeline
    const unsigned char *tmaps;      // TMA maps of the table slices: order m at 2m (P_m^{-1}) and
                                     // 2m + 1 (P~ block), kTensorMapBytes each
    int *status;
};

// Exact int64 sum of K-split partials, then one conversion: 2^(eA_r + eB_c - shift) * sum.
struct Scales {
    const int *eA;     // row scale exponents
    const int *fB;     // exponent fields of the right-hand side's columns
    int shift;
};
struct Partials {
    const long long *part;
    int M, splits;
    Scales sc;
};

// First row of a solve's right-hand side g_m: ring m, whose bins +-m still hold order m+1's
// alias contribution; `a` is the bin alias_m(m + 1) it was aliased into.
struct FirstRow {
    bool pending;      // m + 1 < L
    Partials alias;    // order m+1's alias partials (row m of them is ring m)
    int a;
};

// One contraction C (M x Nc) = A (M x K, plan slices) B (K x Nc, float64, row-major).
struct Job {
    const void *tmap; const int *eA; int kp;   // A: TMA map {kp, rows, slices}, row scales
    const double *B; const int *eB;  // eB: exponent fields of B's columns (the solve: without the
                                     // first row, which the items complete with `first`)
    long long *part;                 // destination of the partials
    const FirstRow *first;           // solves: completion of the first row (null: alias products)
    int M, K, tiles_n, tiles, splits, kchunk;
};

__device__ __forceinline__ int cdiv_i(int a, int b) { return (a + b - 1) / b; }

__device__ Job make_job(const void *tmap, const int *eA, int kp, const double *B, const int *eB, int M,
                        int K, int Nc) {
    Job j;
    j.tmap = tmap; j.eA = eA; j.kp = kp; j.B = B; j.eB = eB; j.M = M; j.K = K;
    j.part = nullptr; j.first = nullptr;
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
    return j;
}

__device__ __forceinline__ bool aborted(const ChainArgs &p) {
    return *(volatile unsigned *)(p.bar + 64) != 0u;
}
__device__ __forceinline__ void raise_abort(const ChainArgs &p, int bit) {
    atomicOr(p.status, bit);
    atomicExch(p.bar + 64, 1u);
}

// Grid-wide barrier; false (for every thread of the CTA) once any CTA has given up.  The arrival
// counter only grows during a launch: barrier i is passed when it reaches i * G, so there is no
// reset and no second word to publish.
__device__ bool grid_barrier(const ChainArgs &p, int *s_flag, unsigned &target) {
    __syncthreads();
    target += gridDim.x;
    if (threadIdx.x == 0) {
        int ok = 1;
        __threadfence();
        atomicAdd(p.bar, 1u);
        volatile unsigned *cnt = p.bar;
        if (*cnt < target) {
            const uint64_t t0 = global_ns();
            while (*cnt < target) {
                if (aborted(p)) { ok = 0; break; }
                if (global_ns() - t0 > p.wait_ns) { raise_abort(p, 2); ok = 0; break; }
            }
        }
        __threadfence();
        if (aborted(p)) ok = 0;
        *s_flag = ok;
    }
    __syncthreads();
    return *s_flag != 0;
}

// Largest exponent field of each column over `rows` rows of the row-major block X (Nc columns)
// into ef[Nc] (atomicMax).  CTA c takes rows c, c + G, ..; each thread keeps the maximum of its
// column over eight rows in flight at a time, so each column sees at most G atomics.
__device__ void column_fields(const ChainArgs &p, const double *X, int rows, int *ef) {
    const int Nc = p.Nc, C = (int)gridDim.x;
    for (int j = threadIdx.x; j < Nc; j += kThreads) {
        int mf = 0;
        for (int r0 = blockIdx.x; r0 < rows; r0 += 8 * C) {
            double x[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int r = r0 + u * C;
                x[u] = r < rows ? __ldcg(X + (int64_t)r * Nc + j) : 0.0;
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) mf = max(mf, exp_field(x[u]));
        }
        if (mf > 0) atomicMax(ef + j, mf);
    }
}

// Exact int64 sum of the K-split partials of row r, columns c0..c0+3 (all at the scale of the
// output element), then one conversion: 2^(eA_r + eB_c - shift) * sum.
__device__ __forceinline__ void sum_partials(const ChainArgs &p, const Partials &pa, int r, int c0, double v[4]) {
    const int Nc = p.Nc, M = pa.M, splits = pa.splits;
    long long t[4] = {0, 0, 0, 0};
    for (int y0 = 0; y0 < splits; y0 += 8) {
        longlong2 a[8], b[8];
#pragma unroll
        for (int u = 0; u < 8; ++u)
            if (y0 + u < splits) {
                const longlong2 *pp = reinterpret_cast<const longlong2 *>(pa.part + ((int64_t)(y0 + u) * M + r) * Nc + c0);
                a[u] = __ldcg(pp);
                b[u] = __ldcg(pp + 1);
            }
#pragma unroll
        for (int u = 0; u < 8; ++u)
            if (y0 + u < splits) { t[0] += a[u].x; t[1] += a[u].y; t[2] += b[u].x; t[3] += b[u].y; }
    }
    const int er = pa.sc.eA[r] - pa.sc.shift;
#pragma unroll
    for (int q = 0; q < 4; ++q) v[q] = i64_scaled(t[q], er + scale_from_field(__ldcg(pa.sc.fB + c0 + q)));
}

// The contraction's items (output tile, K-split), one per CTA and round; each stores its int64
// partial.  `ok` turns false (for the whole CTA) when an mbarrier wait gives up.
// NSL BF16 slices per operand (kind::f16), or, with TF, one TF32 value per operand (kind::tf32:
// the table rows pre-scaled and rounded at plan time, the right-hand side scaled by its column
// scale and rounded here), accumulated in FP32 as the single-region low-precision path.
template <int NSL, bool TF>
__device__ __noinline__ void mma_phase(const ChainArgs &p, const Job &jb, uint32_t tbase,
                                       unsigned char *smem, uint64_t *mbar, uint64_t *full,
                                       uint32_t uses[2], uint32_t fills[2], bool &ok) {
    constexpr bool EXACT = NSL == S && !TF;
    constexpr int NREG = EXACT ? REGIONS : 1;
    const int tid = threadIdx.x, warp = tid >> 5, half = warp >> 2;
    const int Nc = p.Nc, M = jb.M;
    const int items = jb.tiles * jb.splits;
    __shared__ int s_eb[NT];        // scale exponents of the tile's B columns
    __shared__ double s_row0[NT];   // solve: the tile's part of g_m's first row
    __shared__ double s_v[NT];      // solve: order m+1's alias sums for that row
    for (int it = blockIdx.x; it < items && ok; it += gridDim.x) {
        const int tile = it / jb.splits, y = it - tile * jb.splits;
        const int tm = tile / jb.tiles_n, tn = tile - tm * jb.tiles_n;
        const int row0 = tm * MT, col0 = tn * NT;
        const int kbeg = y * jb.kchunk, kend = min(jb.K, kbeg + jb.kchunk);
        __syncthreads();   // the previous item's epilogue is done with s_eb
        if (jb.first) {
            // ring m of the tile's 16 signals with order m+1's alias contribution removed (every
            // item of a column computes the same values, hence the same column scale): one thread
            // per column sums the alias partials exactly, then applies the bin mapping of EPI_ALIAS
            const FirstRow &fr = *jb.first;
            const int col = col0 + tid;
            if (tid < NT) {
                double v = 0.0;
                if (fr.pending && col < Nc) {
                    const Partials &pa = fr.alias;
                    const int r = pa.M - 1;
                    long long t = 0;
                    for (int y0 = 0; y0 < pa.splits; y0 += 8) {
                        long long a8[8];
#pragma unroll
                        for (int u = 0; u < 8; ++u)
                            a8[u] = y0 + u < pa.splits ? __ldcg(pa.part + ((int64_t)(y0 + u) * pa.M + r) * Nc + col) : 0ll;
#pragma unroll
                        for (int u = 0; u < 8; ++u) t += a8[u];
                    }
                    v = i64_scaled(t, pa.sc.eA[r] - pa.sc.shift + scale_from_field(__ldcg(pa.sc.fB + col)));
                }
                s_v[tid] = v;
            }
            __syncthreads();
            if (tid < NT) {
                double w = col < Nc ? __ldcg(jb.B + col) : 0.0;
                if (fr.pending && col < Nc) {
                    const int q = tid & 3, b0 = tid & ~3;
                    if (fr.a == 0) {
                        if (q < 2) w -= s_v[b0 + q] + s_v[b0 + q + 2];
                    } else {
                        const int sp = fr.a > 0 ? 0 : 2;   // slot of bin a: receives G_{+}
                        w -= (q >> 1) == (sp >> 1) ? s_v[b0 + (q & 1)] : s_v[b0 + 2 + (q & 1)];
                    }
                }
                s_row0[tid] = w;
            }
            __syncthreads();
        }
        if (tid < NT) {
            const int col = col0 + tid;
            int f = col < Nc ? __ldcg(jb.eB + col) : 0;
            if (jb.first && col < Nc) {
                f = max(f, exp_field(s_row0[tid]));
                if (tm == 0 && y == 0) p.fS[col] = f;
            }
            s_eb[tid] = scale_from_field(f);
        }
        __syncthreads();

        // k-block kb into stage st: the A slices (all S of them, 128 rows x 32 K, 64-byte
        // swizzled; zero beyond the table) by one TMA load; B read in float64 (rows >= kend as
        // zero) and sliced here, thread = column j, row pairs (2i, 2i + 1), i = h, h + 4, ..
        auto load = [&](int kb, int st) {
            const uint32_t sa = smem_u32(smem + st * STAGE), sb = sa + A_STAGE;
            const int kbase = kb * KB;
            if (tid == 0) {
                if (TF) {
                    // two boxes of 16 K (64 bytes) x 128 rows
                    mbar_expect_tx(smem_u32(&full[st]), TF_A_STAGE);
                    tma_load_2d(sa, jb.tmap, kbase, row0, smem_u32(&full[st]));
                    tma_load_2d(sa + TF_A_HALF, jb.tmap, kbase + 16, row0, smem_u32(&full[st]));
                } else {
                    mbar_expect_tx(smem_u32(&full[st]), A_STAGE);
                    tma_load_3d(sa, jb.tmap, kbase, row0, 0, smem_u32(&full[st]));
                }
            }
            fills[st] += 1;
            const int j = tid & (NT - 1), h = tid >> 6, col = col0 + j;
            const int e = s_eb[j];
            double x[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int k = kbase + 2 * (h + 4 * (i >> 1)) + (i & 1);
                x[i] = (col < Nc && k < kend) ? __ldcg(jb.B + (int64_t)k * Nc + col) : 0.0;
            }
            if (jb.first && kbase == 0 && h == 0) x[0] = s_row0[j];   // row 0: g_m's completed first row
            const uint32_t cb = sb + (j >> 3) * 128 + (j & 7) * 16;
            if (TF) {
                // canonical K-major layout of 32-bit elements: core matrices of 8 columns x 4 K
                // (16 bytes per column), NT * 16 bytes apart along K; rows kk, kk + 1 side by side
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int kk = 2 * (h + 4 * q);
                    const uint32_t a = cb + (kk >> 2) * (NT * 16) + (kk & 3) * 4;
                    asm volatile("st.shared.v2.u32 [%0], {%1, %2};\n" ::"r"(a), "r"(tf32_scaled_bits(x[2 * q], e)),
                                 "r"(tf32_scaled_bits(x[2 * q + 1], e))
                                 : "memory");
                }
                return;
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int kk = 2 * (h + 4 * q);
                __nv_bfloat16 lo[S], hi[S];
                split_value(x[2 * q], e, lo);
                split_value(x[2 * q + 1], e, hi);
                const uint32_t a = cb + (kk >> 3) * (NT * 16) + (kk & 7) * 2;
#pragma unroll
                for (int s = 0; s < NSL; ++s)
                    asm volatile("st.shared.u32 [%0], %1;\n" ::"r"(a + s * (NT * KB * 2)),
                                 "r"((uint32_t)__bfloat16_as_ushort(lo[s]) |
                                     ((uint32_t)__bfloat16_as_ushort(hi[s]) << 16))
                                 : "memory");
            }
        };

        long long acc[kCols];   // columns half * kCols .. of row quarter * 32 + lane
#pragma unroll
        for (int c = 0; c < kCols; ++c) acc[c] = 0;
        const int kb0 = kbeg / KB, nkb = (kend + KB - 1) / KB;
        load(kb0, 0);
        fence_proxy_async();
        __syncthreads();
        for (int kb = kb0; kb < nkb; ++kb) {
            const int st = (kb - kb0) & 1;
            // stage st holds k-block kb once its TMA load has landed: issue its MMAs, then stage the
            // next block while they run
            {
                const bool w = mbar_wait(smem_u32(&full[st]), (fills[st] - 1) & 1u, p.wait_ns);
                if (!__syncthreads_and(w)) { ok = false; break; }
            }
            if (tid == 0) {
                tc_fence_after();
                const uint32_t sa = smem_u32(smem + st * STAGE), sb = sa + A_STAGE;
                bool fresh[REGIONS] = {false, false, false, false, false, false};
                if (TF)
                    for (int q = 0; q < 4; ++q) {
                        // K = 8 per MMA: 32 bytes along a 64-byte swizzled A row, two core
                        // matrices of B
                        const int kg = kb * KB + 8 * q;
                        if (kg >= kend) break;
                        const uint64_t ad = sdesc_sw64(sa + (q >> 1) * TF_A_HALF + 32 * (q & 1));
                        const uint64_t bd = sdesc(sb + 2 * q * (NT * 16), NT * 16, 128);
                        mma_tf32(tbase, ad, bd, kIdescTf32, kg == kbeg ? 0u : 1u);
                    }
                for (int hh = 0; hh < 2 && !TF; ++hh) {
                    const int kg = kb * KB + 16 * hh;
                    if (kg >= kend) break;
                    if (kg == kbeg || (EXACT && kg % CHUNK == 0))
                        for (int r = 0; r < REGIONS; ++r) fresh[r] = true;
                    for (int s = 1; s <= NSL; ++s)
                        for (int t = 1; s + t <= NSL + 1; ++t) {
                            const int d = s + t, reg = EXACT ? (d <= 6 ? d - 2 : 5) : 0;
                            const uint64_t ad = sdesc_sw64(sa + (s - 1) * (MT * KB * 2) + 32 * hh);
                            const uint64_t bd = sdesc(sb + (t - 1) * (NT * KB * 2) + 2 * hh * (NT * 16), NT * 16, 128);
                            mma_bf16(tbase + reg * NT, ad, bd, kIdesc, fresh[reg] ? 0u : 1u);
                            fresh[reg] = false;
                        }
                }
                mma_commit(smem_u32(&mbar[st]));
            }
            uses[st] += 1;
            if (kb + 1 < nkb) {
                // the MMAs of k-block kb - 1 read stage ns: wait for them before refilling it;
                // the vote keeps every thread on the same path if the wait gives up
                const int ns = st ^ 1;
                const bool w = uses[ns] == 0 || mbar_wait(smem_u32(&mbar[ns]), (uses[ns] - 1) & 1u, p.wait_ns);
                if (!__syncthreads_and(w)) { ok = false; break; }
                load(kb + 1, ns);
                fence_proxy_async();
                __syncthreads();
            }
            const int kdone = (kb + 1) * KB;
            if ((EXACT && kdone % CHUNK == 0) || kb == nkb - 1) {
                // the commit of this stage covers every MMA issued so far
                const bool w = mbar_wait(smem_u32(&mbar[st]), (uses[st] - 1) & 1u, p.wait_ns);
                if (!__syncthreads_and(w)) { ok = false; break; }
                tc_fence_after();
                const uint32_t lane_base = tbase + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)(half * kCols);
                if (EXACT) {
#pragma unroll
                    for (int reg = 0; reg < NREG; ++reg) {
                        // region reg holds diagonal d = reg + 2 (multiples of 2^-7d, exact), or
                        // the rounded sum of d >= 7 for the last region
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
                    // one rounded FP32 sum over the whole K-split: kept at 2^-40 resolution
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
        if (!ok) break;

        const int row = row0 + (warp & 3) * 32 + (tid & 31);
        if (row < M) {
#pragma unroll
            for (int g = 0; g < kCols / 4; ++g) {
                const int cl = half * kCols + 4 * g, c0 = col0 + cl;
                if (c0 >= Nc) break;
                long long *pp = jb.part + ((int64_t)y * M + row) * Nc + c0;
                *reinterpret_cast<longlong2 *>(pp) = make_longlong2(acc[4 * g], acc[4 * g + 1]);
                *reinterpret_cast<longlong2 *>(pp + 2) = make_longlong2(acc[4 * g + 2], acc[4 * g + 3]);
            }
        }
    }
}

// The reduction phase of order m:
//  (a) the solve's partials -> F_m rows and f_l^{+-m}; largest exponent fields of F_m's columns
//      into ef (gathered per CTA in shared memory when the grid's thread count is a multiple of
//      the column groups: every thread then stays on one group and the CTA's groups are a window
//      of kThreads groups; one global atomicMax per CTA and column);
//  (b) order m+1's alias sums subtracted from the bins of rings k < m (ring m, the first row of
//      g_m, was completed by the solve's items and is not needed again);
//  (c) largest exponent fields of g_{m-1}'s columns over its rows 1.. (rings >= m: final, and
//      untouched by (b)) into efw.
__device__ __noinline__ void reduce_phase(const ChainArgs &p, const EpiArgs &es, const Partials &ps, int *ef,
                                          bool prev, const EpiArgs &ea, const Partials &pa,
                                          const double *gnext, int gnext_rows, int *efw) {
    const int groups = p.Nc / 4;
    const int64_t T = (int64_t)gridDim.x * kThreads;
    {
        const int64_t total = (int64_t)ps.M * groups;
        __shared__ int s_ef[4 * kThreads];
        const bool windowed = T % groups == 0;
        const int g0 = (int)(((int64_t)blockIdx.x * kThreads) % groups);
        const int span = min(groups, kThreads);
        for (int i = threadIdx.x; i < 4 * kThreads; i += kThreads) s_ef[i] = 0;
        __syncthreads();
        for (int64_t t = (int64_t)blockIdx.x * kThreads + threadIdx.x; t < total; t += T) {
            const int r = (int)(t / groups), g = (int)(t - (int64_t)r * groups);
            double v[4];
            sum_partials(p, ps, r, 4 * g, v);
            epilogue_row4<EPI_SOLVE>(es, r, 4 * g, v);
            const int w = g - g0 < 0 ? g - g0 + groups : g - g0;   // position in the CTA's window
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int f = exp_field(v[q]);
                if (f == 0) continue;
                if (windowed) atomicMax(&s_ef[4 * w + q], f);
                else atomicMax(ef + 4 * g + q, f);
            }
        }
        __syncthreads();
        if (windowed)
            for (int i = threadIdx.x; i < 4 * span; i += kThreads) {
                const int w = i >> 2, g = g0 + w < groups ? g0 + w : g0 + w - groups;
                if (s_ef[i] > 0) atomicMax(ef + 4 * g + (i & 3), s_ef[i]);
            }
    }
    if (prev) {
        const int64_t total = (int64_t)(pa.M - 1) * groups;
        for (int64_t t = (int64_t)blockIdx.x * kThreads + threadIdx.x; t < total; t += T) {
            const int r = (int)(t / groups), g = (int)(t - (int64_t)r * groups);
            double v[4];
            sum_partials(p, pa, r, 4 * g, v);
            epilogue_row4<EPI_ALIAS>(ea, r, 4 * g, v);
        }
    }
    if (gnext) column_fields(p, gnext, gnext_rows, efw);
}

template <int NSL, bool TF>
__global__ void __launch_bounds__(kThreads, 1) k_chain(ChainArgs p) {
    constexpr uint32_t NCOLS = NSL == S && !TF ? TMEM_COLS : 64u;
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ uint64_t mbar[2];   // MMAs of a stage done
    __shared__ uint64_t full[2];   // TMA load of a stage landed
    __shared__ uint32_t tmem_slot;
    __shared__ int s_flag;
    const int tid = threadIdx.x, warp = tid >> 5;
    if (warp == 0) tmem_alloc(smem_u32(&tmem_slot), NCOLS);
    if (tid == 0) {
        mbar_init(smem_u32(&mbar[0]), 1);
        mbar_init(smem_u32(&mbar[1]), 1);
        mbar_init(smem_u32(&full[0]), 1);
        mbar_init(smem_u32(&full[1]), 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tbase = tmem_slot;

    uint32_t uses[2] = {0u, 0u}, fills[2] = {0u, 0u};
    unsigned target = 0;   // arrivals that complete the next grid barrier
    bool ok = true, mma_ok = true;
    const int L = p.L, Nc = p.Nc;
    constexpr int SHIFT = NSL == S && !TF ? ACC_SHIFT : 40;
    for (int m = L - 1; m >= 0; --m) {
        const int n = L - m, kp = (n + 7) & ~7, sl = m & 1;
        // order m+1's alias products: their partials are still in part_a
        FirstRow first;
        first.pending = m + 1 < L;
        first.a = 0;
        first.alias = Partials{p.part_a, 0, 0, Scales{nullptr, nullptr, SHIFT}};
        if (first.pending) {
            const int n1 = n - 1;
            const Job jp = make_job(nullptr, nullptr, (n1 + 7) & ~7, nullptr, nullptr, m + 1, n1, Nc);
            first.alias = Partials{p.part_a, m + 1, jp.splits,
                                   Scales{p.ptE + (int64_t)(m + 1) * L, p.eF + (sl ^ 1) * Nc, SHIFT}};
            first.a = alias_bin(m + 1, m);
        }
        // Eq. (14): F_m = P_m^{-1} g_m
        Job js = make_job(p.tmaps + (size_t)(2 * m) * kTensorMapBytes, p.piE + rows_off(L, m), kp,
                          p.W + rows_off(L, m) * Nc, p.eW + sl * Nc, n, n, Nc);
        js.part = p.part_s;
        js.first = &first;
        mma_phase<NSL, TF>(p, js, tbase, smem, mbar, full, uses, fills, mma_ok);
        if (!mma_ok) { if (tid == 0) raise_abort(p, 1); ok = false; break; }
        if (!(ok = grid_barrier(p, &s_flag, target))) break;
        {
            const EpiArgs es{p.F + rows_off(L, m) * Nc, Nc, nullptr, m, L, Nc, p.coeffs, nullptr};
            const Partials ps{p.part_s, n, js.splits, Scales{js.eA, p.fS, SHIFT}};
            const EpiArgs ea{nullptr, Nc, nullptr, m + 1, L, Nc, nullptr, p.W};
            const double *gn = m >= 1 ? p.W + (rows_off(L, m - 1) + 1) * Nc : nullptr;
            reduce_phase(p, es, ps, p.eF + sl * Nc, first.pending, ea, first.alias, gn, L - m,
                         p.eW + (sl ^ 1) * Nc);
        }
        if (!(ok = grid_barrier(p, &s_flag, target))) break;
        if (m == 0) break;
        // slots read for the last time: eW of order m, eF of order m + 1 (next written by the
        // reductions of orders m - 1 and m - 1)
        for (int j = blockIdx.x * kThreads + tid; j < Nc; j += gridDim.x * kThreads) {
            p.eW[sl * Nc + j] = 0;
            p.eF[(sl ^ 1) * Nc + j] = 0;
        }
        // Eqs. (15)-(16): orders +-m out of the bins of rings k < m (partials only; summed and
        // subtracted in the next order's phases)
        Job ja = make_job(p.tmaps + (size_t)(2 * m + 1) * kTensorMapBytes, p.ptE + (int64_t)m * L, kp,
                          p.F + rows_off(L, m) * Nc, p.eF + sl * Nc, m, n, Nc);
        ja.part = p.part_a;
        mma_phase<NSL, TF>(p, ja, tbase, smem, mbar, full, uses, fills, mma_ok);
        if (!mma_ok) { if (tid == 0) raise_abort(p, 1); ok = false; break; }
        if (!(ok = grid_barrier(p, &s_flag, target))) break;
    }
    if (!mma_ok) {
        // let the TMA loads and MMAs in flight finish (bounded) before the CTA releases its
        // shared and tensor memory
        for (int st = 0; st < 2; ++st) {
            if (fills[st] > 0) mbar_wait(smem_u32(&full[st]), (fills[st] - 1) & 1u);
            if (uses[st] > 0) mbar_wait(smem_u32(&mbar[st]), (uses[st] - 1) & 1u);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tbase, NCOLS);
}

template <int NSL, bool TF>
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
    return cudaLaunchKernelEx(&cfg, k_chain<NSL, TF>, p);
}

}  // namespace

cudaError_t tc_table_tensor_maps(int L, const __nv_bfloat16 *piS, const std::vector<int64_t> &pik_off,
                                 const __nv_bfloat16 *ptS, const std::vector<int64_t> &ptk_off,
                                 unsigned char **d_maps) {
    std::vector<CUtensorMap> maps((size_t)2 * L);
    for (int m = 0; m < L; ++m) {
        const int n = L - m;
        const cuuint64_t kp = (cuuint64_t)((n + 7) & ~7);
        for (int w = 0; w < 2; ++w) {
            // w = 0: P_m^{-1} block (n rows, slice stride n kp); w = 1: P~ block (L rows)
            const cuuint64_t rows = w == 0 ? (cuuint64_t)n : (cuuint64_t)L;
            const __nv_bfloat16 *base = w == 0 ? piS + (int64_t)S * pik_off[m] : ptS + (int64_t)S * L * ptk_off[m];
            const cuuint64_t dims[3] = {kp, rows, (cuuint64_t)S};
            const cuuint64_t strides[2] = {kp * 2, rows * kp * 2};
            const cuuint32_t box[3] = {(cuuint32_t)KB, (cuuint32_t)MT, (cuuint32_t)S};
            const cudaError_t e = encode_tiled_map(&maps[(size_t)2 * m + w], base, dims, strides, box);
            if (e != cudaSuccess) return e;
        }
    }
    const size_t bytes = maps.size() * sizeof(CUtensorMap);
    const cudaError_t e = cudaMalloc(d_maps, bytes);
    if (e != cudaSuccess) return e;
    return cudaMemcpy(*d_maps, maps.data(), bytes, cudaMemcpyHostToDevice);
}

cudaError_t tc_table_tensor_maps_tf32(int L, const float *piT, const std::vector<int64_t> &pik_off,
                                      const float *ptT, const std::vector<int64_t> &ptk_off,
                                      unsigned char **d_maps) {
    std::vector<CUtensorMap> maps((size_t)2 * L);
    for (int m = 0; m < L; ++m) {
        const int n = L - m;
        const cuuint64_t kp = (cuuint64_t)((n + 7) & ~7);
        for (int w = 0; w < 2; ++w) {
            // w = 0: P_m^{-1} block (n rows); w = 1: P~ block (L rows); rows of kp floats
            const cuuint64_t rows = w == 0 ? (cuuint64_t)n : (cuuint64_t)L;
            const float *base = w == 0 ? piT + pik_off[m] : ptT + (int64_t)L * ptk_off[m];
            const cuuint64_t dims[2] = {kp, rows};
            const cuuint32_t box[2] = {16u, (cuuint32_t)MT};
            const cudaError_t e = encode_tiled_map_f32(&maps[(size_t)2 * m + w], base, dims, kp * 4, box);
            if (e != cudaSuccess) return e;
        }
    }
    const size_t bytes = maps.size() * sizeof(CUtensorMap);
    const cudaError_t e = cudaMalloc(d_maps, bytes);
    if (e != cudaSuccess) return e;
    return cudaMemcpy(*d_maps, maps.data(), bytes, cudaMemcpyHostToDevice);
}

int64_t tc_chain_words(int64_t batch) { return kChainBarWords + 5 * 4 * batch; }

cudaError_t tc_prepare_chain(int *grid) {
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(k_chain<S, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES)) != cudaSuccess ||
        (e = cudaFuncSetAttribute(k_chain<2, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES)) != cudaSuccess ||
        (e = cudaFuncSetAttribute(k_chain<1, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES)) != cudaSuccess ||
        (e = cudaFuncSetAttribute(k_chain<1, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES)) != cudaSuccess)
        return e;
    int dev = 0, sms = 0, per_sm = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_chain<S, false>, kThreads, SMEM_BYTES)) != cudaSuccess)
        return e;
    // one CTA per SM (the kernel holds the SM's tensor memory); never more than can be resident
    *grid = std::min(sms, sms * per_sm);
    return *grid > 0 ? cudaSuccess : cudaErrorInvalidConfiguration;
}

cudaError_t tc_forward_chain(const ChainTables &t, int L, int64_t batch, double *W, double *F,
                             double2 *coeffs, double *part, double *part2, unsigned *words, int *status,
                             int nsl, bool tf32, int grid, uint64_t wait_ns, cudaStream_t s) {
    ChainArgs p{};
    p.L = L; p.Nc = (int)(4 * batch);
    p.W = W; p.F = F; p.coeffs = coeffs;
    p.piS = t.piS; p.piE = t.piE; p.pik_off = t.pik_off;
    p.ptS = t.ptS; p.ptE = t.ptE; p.ptk_off = t.ptk_off;
    p.tmaps = t.tmaps;
    p.part_s = reinterpret_cast<long long *>(part); p.part_a = reinterpret_cast<long long *>(part2);
    p.bar = words; p.status = status; p.wait_ns = wait_ns;
    p.eW = reinterpret_cast<int *>(words + kChainBarWords);
    p.eF = p.eW + 2 * p.Nc;
    p.fS = p.eF + 2 * p.Nc;
    cudaError_t e = cudaMemsetAsync(words, 0, sizeof(unsigned) * tc_chain_words(batch), s);
    if (e != cudaSuccess) return e;
    if (tf32) return launch_chain<1, true>(p, grid, s);
    if (nsl == S) return launch_chain<S, false>(p, grid, s);
    if (nsl == 2) return launch_chain<2, false>(p, grid, s);
    if (nsl == 1) return launch_chain<1, false>(p, grid, s);
    return cudaErrorInvalidValue;
}

}  // namespace sht
