// The forward's order chain (Procedure 1 in bin space, Eqs. (14)-(16)) on the tensor cores as ONE
// persistent cooperative kernel, with the orders taken in blocks of kChainB.
//
// For m = L-1 .. 0 the chain solves F_m = P_m^{-1} g_m (g_m: bins +-m of rings k = m + j >= m) and
// subtracts the aliased contribution G_{+-m}(theta_k) = P~_m(theta_k) F_m of orders +-m from bins
// alias_k(+-m) of the rings k < m.  Row j of g_m (ring m + j, bins +-m) is reached only by orders
// m' = 2(m + j) + 1 - m = m + 2j + 1 and above (m' = +-m mod 2(m+j)+1 with m' > m + j).  So for a
// block of orders [lo, hi] whose orders above hi are done, every row j >= J_m = floor((hi-m+1)/2)
// of every g_m in the block is final already; only the J_m <= kChainB/2 leading rows ("tracked
// entries", rings lo .. hi) still wait for orders of the same block.  Since G_{+-m'}(theta_k) =
// Q_m'[k] g_m' with Q_m' = P~_m' P_m'^{-1} (plan table, rings lo <= k < m'), the tracked entries
// follow from a small recurrence, and the block's heavy products run all at once.  Per block:
//
//   X1  (all CTAs, float64)  the contributions of the block's orders to the tracked entries
//       through their final rows, Q_m'[k, J':] g_m'[J':]                             | barrier
//   X2  (one CTA per signal, float64)  the tracked entries (bins less those contributions), then
//       the recurrence over m' = hi .. lo through the tracked rows, Q_m'[k, :J'] g_m'[:J'], in
//       shared memory; the final entries written back into the bins; column scales of every g_m
//       of the block                                                                 | barrier
//   Y   (tensor cores)  F_m = P_m^{-1} g_m for every order of the block (Eq. (14)); f_l^{+-m},
//       column scales of F_m                                                          | barrier
//   Z   (tensor cores)  G_{+-m'}(theta_k) = P~_m'(theta_k) F_m' for every order of the block and
//       ring k < m' (Eq. (16))                                                        | barrier
//   E   (all CTAs)  G subtracted from bins alias_k(+-m') of every ring (Eq. (15)) that a later
//       block reads (the block's own rows are final and are skipped)                  | barrier
//
// Five grid barriers per block (the last block stops after Y): 5 L / kChainB in all, where one
// phase per order needs three per order.  Y and Z items are (order, 128 x 64 tile) with the whole
// K range, so each item converts its exact int64 accumulators to float64 and stores the result
// itself.  The right-hand sides are read in float64 and cut into BF16 slices while staged in shared
// memory, with the column scales the previous phase gathered; the plan tables (P_m^{-1}, P~) are
// pre-sliced and loaded by TMA.
//
// The cooperative launch guarantees that every CTA is resident, so the barriers cannot wait on a
// CTA that never runs.  Every wait is bounded (the plan's wait limit); a CTA that gives up sets the
// plan's status word and an abort word that every other CTA checks in its barrier waits, so all of
// them leave the chain promptly and release their tensor memory.  Data written by other SMs in an
// earlier phase is read through L2 (cp.async.cg, __ldcg, TMA), never through a possibly stale L1
// line.
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
constexpr int kB = kChainB;

struct ChainArgs {
    int L, Nc, B;                    // Nc = 4 B columns
    double *W, *F;                   // order-major bins and solved orders (rows_total x Nc)
    double2 *coeffs;
    const int *piE, *ptE;            // row scale exponents of the P_m^{-1} and P~ slices
    const double *Q;                 // Q_m = P~_m(rings lo..m-1) P_m^{-1}: kB x n_m at kB rows_off(L, m)
    double *G;                       // Z's output: block order i at i L Nc, row k (ring), Nc columns;
                                     // X1's output (before Z): row (hi - m') kB + (k - lo)
    int *eW, *eF;                    // L x Nc exponent fields of the columns of g_m and of F_m
    unsigned *bar;                   // [0] arrivals (monotonic within a launch), [64] abort
    uint64_t wait_ns;                // limit of every wait on other CTAs or on the pipeline
    const unsigned char *tmaps;      // TMA maps of the table slices: order m at 2m (P_m^{-1}) and
                                     // 2m + 1 (P~ block), kTensorMapBytes each
    int *status;
};

// Block geometry.  Block b covers orders hi = L-1-b kB down to lo = max(0, hi-kB+1); its order
// m = hi - i has J(i) = floor((i+1)/2) tracked rows (rings m .. m+J-1), stored from row offH(i) of H.
__host__ __device__ __forceinline__ int blk_J(int i) { return (i + 1) >> 1; }
__host__ __device__ __forceinline__ int blk_offH(int i) { const int p = i >> 1; return p * p + (i & 1) * p; }

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

// Subtract the contributions (G+ = g[0..1] re/im, G- = g[2..3] re/im) of an order m' from the four
// columns of one signal in row (o, ring k) of the bins, where a = alias_k(m') is the bin of G+
// (o = |a|): bin a gets G+, bin -a gets G-; slot 0 holds bin +o, slot 2 bin -o (zero for o = 0).
__device__ __forceinline__ void sub_alias(double w[4], int a, const double g[4]) {
    if (a == 0) {
        w[0] -= g[0] + g[2];
        w[1] -= g[1] + g[3];
    } else if (a > 0) {
        w[0] -= g[0]; w[1] -= g[1]; w[2] -= g[2]; w[3] -= g[3];
    } else {
        w[0] -= g[2]; w[1] -= g[3]; w[2] -= g[0]; w[3] -= g[1];
    }
}

// The same contributions as they land in the row's four columns (what sub_alias subtracts).
__device__ __forceinline__ void alias_map(int a, const double g[4], double out[4]) {
    if (a == 0) {
        out[0] = g[0] + g[2]; out[1] = g[1] + g[3]; out[2] = 0.0; out[3] = 0.0;
    } else if (a > 0) {
        out[0] = g[0]; out[1] = g[1]; out[2] = g[2]; out[3] = g[3];
    } else {
        out[0] = g[2]; out[1] = g[3]; out[2] = g[0]; out[3] = g[1];
    }
}

// One contraction of a phase: C (M x Nc) = A (M x K, plan slices) B (K x Nc, float64, row-major).
struct Job {
    const void *tmap; const int *eA; int kp;   // A: TMA map {kp, rows, slices}, row scales
    const double *B; const int *eB;            // eB: exponent fields of B's columns
    int M, K, tiles_n, tiles;
    int mode;                                  // 0: solve (Y), 1: alias values (Z)
    int m;                                     // the order
    double *out;                               // Y: F block m; Z: G rows of the order
    int *ef;                                   // Y: exponent fields of F_m's columns
};

__device__ __forceinline__ int cdiv_i(int a, int b) { return (a + b - 1) / b; }

// Job of block order i (m = hi - i) in phase Y (solve) or Z (alias).
__device__ Job make_job(const ChainArgs &p, bool solve, int hi, int i) {
    const int L = p.L, Nc = p.Nc, m = hi - i, n = L - m;
    Job j;
    j.tiles_n = cdiv_i(Nc, NT);
    j.m = m;
    j.K = n;
    j.kp = (n + 7) & ~7;
    if (solve) {
        j.tmap = p.tmaps + (size_t)(2 * m) * kTensorMapBytes;
        j.eA = p.piE + rows_off(L, m);
        j.B = p.W + rows_off(L, m) * Nc;
        j.eB = p.eW + (int64_t)m * Nc;
        j.M = n;
        j.mode = 0;
        j.out = p.F + rows_off(L, m) * Nc;
        j.ef = p.eF + (int64_t)m * Nc;
    } else {
        j.tmap = p.tmaps + (size_t)(2 * m + 1) * kTensorMapBytes;
        j.eA = p.ptE + (int64_t)m * L;
        j.B = p.F + rows_off(L, m) * Nc;
        j.eB = p.eF + (int64_t)m * Nc;
        j.M = m;   // rings 0 .. m-1
        j.mode = 1;
        j.out = p.G + (int64_t)i * L * Nc;
        j.ef = nullptr;
    }
    j.tiles = j.M > 0 ? cdiv_i(j.M, MT) * j.tiles_n : 0;
    return j;
}

// The items (block order, output tile) of phase Y or Z, one per CTA and round, each over the whole
// K range; each stores its float64 result.  `ok` turns false (for the whole CTA) when an mbarrier
// wait gives up.  NSL BF16 slices per operand (kind::f16), or, with TF, one TF32 value per operand
// (kind::tf32: the table rows pre-scaled and rounded at plan time, the right-hand side scaled by its
// column scale and rounded here), accumulated in FP32 as the single-region low-precision path.
template <int NSL, bool TF>
__device__ __noinline__ void mma_phase(const ChainArgs &p, bool solve, int hi, int lo, uint32_t tbase,
                                       unsigned char *smem, uint64_t *mbar, uint64_t *full,
                                       uint32_t uses[2], uint32_t fills[2], bool &ok) {
    constexpr bool EXACT = NSL == S && !TF;
    constexpr int NREG = EXACT ? REGIONS : 1;
    constexpr int SHIFT = EXACT ? ACC_SHIFT : 40;
    const int tid = threadIdx.x, warp = tid >> 5, half = warp >> 2, lane = tid & 31;
    const int Nc = p.Nc, nb = hi - lo + 1;
    __shared__ int s_eb[NT];           // scale exponents of the tile's B columns
    __shared__ int s_start[kB + 1];    // first item of each block order
    __syncthreads();
    if (tid == 0) {
        s_start[0] = 0;
        for (int i = 0; i < nb; ++i) s_start[i + 1] = s_start[i] + make_job(p, solve, hi, i).tiles;
    }
    __syncthreads();
    const int items = s_start[nb];
    for (int it = blockIdx.x; it < items && ok; it += gridDim.x) {
        int i = 0;
        while (s_start[i + 1] <= it) ++i;
        const Job jb = make_job(p, solve, hi, i);
        const int tile = it - s_start[i];
        const int tm = tile / jb.tiles_n, tn = tile - tm * jb.tiles_n;
        const int row0 = tm * MT, col0 = tn * NT;
        const int kend = jb.K;
        __syncthreads();   // the previous item's epilogue is done with s_eb
        if (tid < NT) {
            const int col = col0 + tid;
            const int f = col < Nc ? __ldcg(jb.eB + col) : 0;
            s_eb[tid] = scale_from_field(f);
        }
        __syncthreads();

        // k-block kb into stage st: the A slices (all S of them, 128 rows x 32 K, 64-byte
        // swizzled; zero beyond the table) by one TMA load; B read in float64 (rows >= kend as
        // zero) and sliced here, thread = column j, row pairs (2i, 2i + 1), i = h, h + 4, ..
        // B values of a k-block (thread = column j, rows 2(h + 4i) + {0, 1}), fetched one k-block
        // ahead of their slicing so that the loads' latency hides behind a whole iteration
        auto fetch = [&](int kb, double x[8]) {
            const int j = tid & (NT - 1), h = tid >> 6, col = col0 + j, kbase = kb * KB;
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int k = kbase + 2 * (h + 4 * (q >> 1)) + (q & 1);
                x[q] = (col < Nc && k < kend) ? __ldcg(jb.B + (int64_t)k * Nc + col) : 0.0;
            }
        };
        auto load = [&](int kb, int st, const double *x) {
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
            const int j = tid & (NT - 1), h = tid >> 6;
            const int e = s_eb[j];
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
                __nv_bfloat16 lo_s[S], hi_s[S];
                split_value(x[2 * q], e, lo_s);
                split_value(x[2 * q + 1], e, hi_s);
                const uint32_t a = cb + (kk >> 3) * (NT * 16) + (kk & 7) * 2;
#pragma unroll
                for (int s = 0; s < NSL; ++s)
                    asm volatile("st.shared.u32 [%0], %1;\n" ::"r"(a + s * (NT * KB * 2)),
                                 "r"((uint32_t)__bfloat16_as_ushort(lo_s[s]) |
                                     ((uint32_t)__bfloat16_as_ushort(hi_s[s]) << 16))
                                 : "memory");
            }
        };

        long long acc[kCols];   // columns half * kCols .. of row quarter * 32 + lane
#pragma unroll
        for (int c = 0; c < kCols; ++c) acc[c] = 0;
        const int nkb = (kend + KB - 1) / KB;
        double xn[8];   // the next k-block's B values
        fetch(0, xn);
        load(0, 0, xn);
        if (nkb > 1) fetch(1, xn);
        fence_proxy_async();
        __syncthreads();
        for (int kb = 0; kb < nkb; ++kb) {
            const int st = kb & 1;
            // stage st holds k-block kb once its TMA load has landed: issue its MMAs, then stage the
            // next block while they run
            {
                const bool w = mbar_wait(smem_u32(&full[st]), (fills[st] - 1) & 1u, p.wait_ns);
                if (!__syncthreads_and(w)) { ok = false; break; }
            }
            if (tid == 0) {
                tc_fence_after();
                const uint32_t sa = smem_u32(smem + st * STAGE), sb = sa + A_STAGE;
                if (TF) {
                    for (int q = 0; q < 4; ++q) {
                        // K = 8 per MMA: 32 bytes along a 64-byte swizzled A row, two core
                        // matrices of B
                        const int kg = kb * KB + 8 * q;
                        if (kg >= kend) break;
                        const uint64_t ad = sdesc_sw64(sa + (q >> 1) * TF_A_HALF + 32 * (q & 1));
                        const uint64_t bd = sdesc(sb + 2 * q * (NT * 16), NT * 16, 128);
                        mma_tf32(tbase, ad, bd, kIdescTf32, kg == 0 ? 0u : 1u);
                    }
                } else {
                    // two 16-K steps; the first of a chunk (or of the item) restarts the regions
                    constexpr uint32_t A16 = (MT * KB * 2) >> 4, B16 = (NT * KB * 2) >> 4;
                    const uint64_t ad0 = sdesc_sw64(sa), bd0 = sdesc(sb, NT * 16, 128);
                    const bool restart = kb == 0 || (EXACT && (kb * KB) % CHUNK == 0);
                    mma_slice_pairs<NSL, EXACT, A16, B16>(tbase, ad0, bd0, restart);
                    if (kb * KB + 16 < kend)
                        mma_slice_pairs<NSL, EXACT, A16, B16>(tbase, ad0 + (32 >> 4), bd0 + ((2 * NT * 16) >> 4), false);
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
                double xc[8];
#pragma unroll
                for (int q = 0; q < 8; ++q) xc[q] = xn[q];
                if (kb + 2 < nkb) fetch(kb + 2, xn);
                load(kb + 1, ns, xc);
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
                            for (int q = 0; q < 16; ++q)
                                acc[c0 + q] += (long long)__float2int_rn(v[q] * up) << shift;
                        }
                    }
                } else {
                    // one rounded FP32 sum over the whole K range: kept at 2^-40 resolution
#pragma unroll
                    for (int c0 = 0; c0 < kCols; c0 += 16) {
                        float v[16];
                        tmem_ld16(lane_base + c0, v);
#pragma unroll
                        for (int q = 0; q < 16; ++q) acc[c0 + q] = __float2ll_rn(v[q] * 0x1p40f);
                    }
                }
                tc_fence_before();
                __syncthreads();
            }
        }
        if (!ok) break;

        // epilogue: one conversion per element, 2^(eA_row + eB_col - SHIFT) * acc
        const int row = row0 + (warp & 3) * 32 + lane;
        const bool live = row < jb.M;
        const int er = live ? __ldg(jb.eA + row) - SHIFT : 0;
        double v[kCols];
#pragma unroll
        for (int c = 0; c < kCols; ++c) v[c] = live ? i64_scaled(acc[c], er + s_eb[half * kCols + c]) : 0.0;
        if (jb.mode == 0) {
            const EpiArgs es{jb.out, Nc, nullptr, jb.m, p.L, Nc, p.coeffs, nullptr};
#pragma unroll
            for (int g = 0; g < kCols / 4; ++g) {
                const int c0 = col0 + half * kCols + 4 * g;
                if (live && c0 < Nc) epilogue_row4<EPI_SOLVE>(es, row, c0, v + 4 * g);
            }
            // largest exponent field of each column over the tile's rows: warp maximum, one
            // atomic per warp and column
#pragma unroll
            for (int c = 0; c < kCols; ++c) {
                const unsigned f = __reduce_max_sync(0xffffffffu, (unsigned)exp_field(v[c]));
                const int col = col0 + half * kCols + c;
                if (lane == 0 && f > 0u && col < Nc) atomicMax(jb.ef + col, (int)f);
            }
        } else if (live) {
            double *o = jb.out + (int64_t)row * Nc + col0 + half * kCols;
#pragma unroll
            for (int c = 0; c < kCols; c += 2)
                if (col0 + half * kCols + c < Nc) *reinterpret_cast<double2 *>(o + c) = make_double2(v[c], v[c + 1]);
        }
    }
}

// X1: for every order m' of block [lo, hi] and ring k (lo <= k < m') whose alias bin is a tracked
// entry, the contribution of m' through its final rows, Q_m'[k, J':] g_m'[J':] (the four columns
// G+ re/im, G- re/im of each signal), into the scratch rows (hi - m') kB + (k - lo) of p.G.  One
// warp per (order, ring, signal), lanes along the row, so that every warp does one row's work
// whatever the number of orders that reach an entry (X2 adds them up per entry).
__device__ void phase_x1(const ChainArgs &p, int hi, int lo) {
    const int L = p.L, Nc = p.Nc, B = p.B, nb = hi - lo + 1;
    const int lane = threadIdx.x & 31;
    const int64_t nw = ((int64_t)gridDim.x * kThreads) >> 5;
    const int64_t total = (int64_t)nb * kB * B;
    for (int64_t w = ((int64_t)blockIdx.x * kThreads + threadIdx.x) >> 5; w < total; w += nw) {
        const int pr = (int)(w / B), s = (int)(w - (int64_t)pr * B);
        const int ip = pr / kB, kk = pr - ip * kB, mp = hi - ip, k = lo + kk;
        if (k >= mp) continue;                                   // rings below m' only
        const int a = alias_bin(mp, k), o = a < 0 ? -a : a;
        if (o < lo || k - o >= blk_J(hi - o)) continue;          // not a tracked entry
        const int Jp = blk_J(ip), np = L - mp;
        const double *q = p.Q + (int64_t)kB * rows_off(L, mp) + (int64_t)kk * np;
        const double *g = p.W + rows_off(L, mp) * Nc + 4 * s;
        double gs[4] = {0.0, 0.0, 0.0, 0.0};
        for (int c = Jp + lane; c < np; c += 32) {
            const double qv = __ldg(q + c);
            const double2 g01 = __ldcg(reinterpret_cast<const double2 *>(g + (int64_t)c * Nc));
            const double2 g23 = __ldcg(reinterpret_cast<const double2 *>(g + (int64_t)c * Nc + 2));
            gs[0] = fma(qv, g01.x, gs[0]);
            gs[1] = fma(qv, g01.y, gs[1]);
            gs[2] = fma(qv, g23.x, gs[2]);
            gs[3] = fma(qv, g23.y, gs[3]);
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1)
#pragma unroll
            for (int q4 = 0; q4 < 4; ++q4) gs[q4] += __shfl_xor_sync(0xffffffffu, gs[q4], off);
        if (lane < 4) p.G[(int64_t)pr * Nc + 4 * s + lane] = gs[lane];
    }
}

// X2: per signal (one CTA each), the recurrence of the tracked entries over the block's orders
// m' = hi .. lo: once every order above m' is applied, rows 0..J'-1 of g_m' are final, and its
// contribution Q_m'[k, :J'] g_m'[:J'] is subtracted from the tracked entries it reaches (rings
// lo <= k < m').  The entries and Q's leading columns live in shared memory.  Then the final
// entries go back into the bins, the exponent fields of every g_m of the block (all its rows) are
// gathered for Y, and F_m's fields are cleared for Y's atomics.
__device__ void phase_x2(const ChainArgs &p, int hi, int lo, double *sm) {
    const int L = p.L, Nc = p.Nc, nb = hi - lo + 1, nE = blk_offH(nb), tid = threadIdx.x;
    __shared__ int s_qoff[kB + 1];    // order i's Q block: (m - lo) rings x J(i) columns
    __shared__ int s_f[kB * 4];       // exponent fields of the block's g_m, four columns
    if ((int)blockIdx.x < p.B) {
        if (tid == 0) {
            s_qoff[0] = 0;
            for (int i = 0; i < nb; ++i) s_qoff[i + 1] = s_qoff[i] + (hi - i - lo) * blk_J(i);
        }
        __syncthreads();
        double *qs = sm, *hs = sm + s_qoff[nb];
        for (int t = tid; t < s_qoff[nb]; t += kThreads) {
            int i = 0;
            while (s_qoff[i + 1] <= t) ++i;
            const int J = blk_J(i), r = t - s_qoff[i], kk = r / J, c = r - kk * J, m = hi - i;
            qs[t] = __ldg(p.Q + (int64_t)kB * rows_off(L, m) + (int64_t)kk * (L - m) + c);
        }
        for (int s = blockIdx.x; s < p.B; s += gridDim.x) {
            __syncthreads();
            // tracked entries: the bins less X1's contributions of the orders that reach them
            for (int t = tid; t < 4 * nE; t += kThreads) {
                const int e = t >> 2, q4 = t & 3;
                int i = 0;
                while (blk_offH(i + 1) <= e) ++i;
                const int m = hi - i, j = e - blk_offH(i), k = m + j;
                double v = __ldcg(p.W + (rows_off(L, m) + j) * Nc + 4 * s + q4);
                // every order above ring k: its scratch row exists, so the loads carry no branch
                // and several are in flight; orders that do not reach this entry add nothing
#pragma unroll 4
                for (int mp = hi; mp > k; --mp) {
                    const int a = alias_bin(mp, k);
                    const bool hit = (a < 0 ? -a : a) == m && !(a == 0 && q4 >= 2);   // bin 0: slots 2, 3 stay zero
                    const double *gp = p.G + ((int64_t)(hi - mp) * kB + (k - lo)) * Nc + 4 * s;
                    const double g1 = __ldcg(gp + (a >= 0 ? q4 : (q4 ^ 2)));
                    const double g2 = a == 0 ? __ldcg(gp + (q4 & 1) + 2) : 0.0;
                    v -= hit ? g1 + g2 : 0.0;
                }
                hs[t] = v;
            }
            for (int t = tid; t < 4 * nb; t += kThreads) s_f[t] = 0;
            __syncthreads();
            for (int ip = 0; ip < nb; ++ip) {
                const int mp = hi - ip, Jp = blk_J(ip);
                if (Jp > 0) {
                    const double *h = hs + 4 * blk_offH(ip);      // rows 0..Jp-1 of g_m' (final)
                    for (int t = tid; t < 4 * (mp - lo); t += kThreads) {
                        const int kk = t >> 2, q4 = t & 3, k = lo + kk;
                        const int a = alias_bin(mp, k), o = a < 0 ? -a : a;
                        if (o < lo || k - o >= blk_J(hi - o)) continue;   // not a tracked entry
                        if (a == 0 && q4 >= 2) continue;                 // bin 0: slots 2, 3 stay zero
                        const int c1 = a >= 0 ? q4 : (q4 ^ 2);            // source column (alias_map)
                        const double *qr = qs + s_qoff[ip] + kk * Jp;
                        double g = 0.0;
                        for (int c = 0; c < Jp; ++c) {
                            const double hv = a == 0 ? h[4 * c + q4] + h[4 * c + q4 + 2] : h[4 * c + c1];
                            g = fma(qr[c], hv, g);
                        }
                        hs[4 * (blk_offH(hi - o) + (k - o)) + q4] -= g;
                    }
                }
                __syncthreads();
            }
            // the final entries back into the bins
            for (int t = tid; t < 4 * nE; t += kThreads) {
                const int e = t >> 2;
                int i = 0;
                while (blk_offH(i + 1) <= e) ++i;
                const int m = hi - i, j = e - blk_offH(i);
                p.W[(rows_off(L, m) + j) * Nc + 4 * s + (t & 3)] = hs[t];
            }
            __syncthreads();
            // exponent fields of the columns of g_m (every row), for the slicing in Y
            for (int i = 0; i < nb; ++i) {
                const int m = hi - i, n = L - m;
                const double *g = p.W + rows_off(L, m) * Nc + 4 * s;
                int f = 0;
                for (int r = tid >> 2; r < n; r += kThreads >> 2) f = max(f, exp_field(__ldcg(g + (int64_t)r * Nc + (tid & 3))));
                if (f > 0) atomicMax(&s_f[4 * i + (tid & 3)], f);
            }
            __syncthreads();
            for (int t = tid; t < 4 * nb; t += kThreads) {
                const int m = hi - (t >> 2);
                p.eW[(int64_t)m * Nc + 4 * s + (t & 3)] = s_f[t];
                p.eF[(int64_t)m * Nc + 4 * s + (t & 3)] = 0;
            }
        }
    }
    // the shared buffer is the MMA stages' next: order these generic accesses before the TMA writes
    fence_proxy_async();
}

// E: the block's alias values subtracted from the bins that a later block reads.  Thread = (ring k,
// signal), orders m' = hi .. max(lo, k+1) in turn (several may reach the same bin: fixed order).
__device__ void phase_e(const ChainArgs &p, int hi, int lo) {
    const int L = p.L, Nc = p.Nc, B = p.B;
    const int64_t T = (int64_t)gridDim.x * kThreads;
    for (int64_t t = (int64_t)blockIdx.x * kThreads + threadIdx.x; t < (int64_t)hi * B; t += T) {
        const int k = (int)(t / B), s = (int)(t - (int64_t)k * B);
        for (int mp = hi; mp >= lo && mp > k; --mp) {
            const int a = alias_bin(mp, k), o = a < 0 ? -a : a;
            if (o >= lo) continue;   // a row of the block's own orders: final, not read again
            const double *gp = p.G + ((int64_t)(hi - mp) * L + k) * Nc + 4 * s;
            const double2 g01 = __ldcg(reinterpret_cast<const double2 *>(gp));
            const double2 g23 = __ldcg(reinterpret_cast<const double2 *>(gp + 2));
            const double g[4] = {g01.x, g01.y, g23.x, g23.y};
            double2 *wp = reinterpret_cast<double2 *>(p.W + (rows_off(L, o) + (k - o)) * Nc + 4 * s);
            const double2 w01 = __ldcg(wp), w23 = __ldcg(wp + 1);
            double w[4] = {w01.x, w01.y, w23.x, w23.y};
            sub_alias(w, a, g);
            wp[0] = make_double2(w[0], w[1]);
            wp[1] = make_double2(w[2], w[3]);
        }
    }
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
    bool mma_ok = true;
    for (int hi = p.L - 1; hi >= 0; hi -= kB) {
        const int lo = max(0, hi - kB + 1);
        phase_x1(p, hi, lo);
        if (!grid_barrier(p, &s_flag, target)) break;
        phase_x2(p, hi, lo, reinterpret_cast<double *>(smem));
        if (!grid_barrier(p, &s_flag, target)) break;
        mma_phase<NSL, TF>(p, true, hi, lo, tbase, smem, mbar, full, uses, fills, mma_ok);
        if (!mma_ok) { if (tid == 0) raise_abort(p, 1); break; }
        if (!grid_barrier(p, &s_flag, target)) break;
        if (lo == 0) break;   // no order below: the chain is done
        mma_phase<NSL, TF>(p, false, hi, lo, tbase, smem, mbar, full, uses, fills, mma_ok);
        if (!mma_ok) { if (tid == 0) raise_abort(p, 1); break; }
        if (!grid_barrier(p, &s_flag, target)) break;
        phase_e(p, hi, lo);
        if (!grid_barrier(p, &s_flag, target)) break;
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

// Q_m = P~_m(rings lo..m-1) P_m^{-1} for every order m (lo the first order of m's block): CTA
// (m, y) takes rings lo + y, lo + y + gridDim.y, ..; thread = column c of Q (coalesced reads of
// P_m^{-1}'s rows), float64.
__global__ void k_chain_q(int L, const double *__restrict__ pt, const double *__restrict__ pinv, double *__restrict__ Q) {
    const int m = blockIdx.x, n = L - m;
    const int hi = L - 1 - ((L - 1 - m) / kB) * kB, lo = max(0, hi - kB + 1);
    const double *pi = pinv + pinv_off(L, m);
    double *q = Q + (int64_t)kB * rows_off(L, m);
    for (int r = blockIdx.y; r < m - lo; r += gridDim.y) {
        const double *prow = pt + pt_off(L, m) + (int64_t)(lo + r) * n;
        for (int c = threadIdx.x; c < n; c += blockDim.x) {
            double acc = 0.0;
            for (int l = 0; l < n; ++l) acc = fma(__ldg(prow + l), __ldg(pi + (int64_t)l * n + c), acc);
            q[(int64_t)r * n + c] = acc;
        }
    }
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

int64_t tc_chain_words(int L, int64_t batch) { return kChainBarWords + 2 * (int64_t)L * 4 * batch; }

cudaError_t tc_chain_q_table(int L, const double *pt, const double *pinv, double *Q, cudaStream_t s) {
    if (L <= 1) return cudaSuccess;
    k_chain_q<<<dim3((unsigned)L, (unsigned)std::min(L, kB)), 128, 0, s>>>(L, pt, pinv, Q);
    return cudaGetLastError();
}

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
                             double2 *coeffs, double *G, unsigned *words, int *status,
                             int nsl, bool tf32, int grid, uint64_t wait_ns, cudaStream_t s) {
    ChainArgs p{};
    p.L = L; p.B = (int)batch; p.Nc = (int)(4 * batch);
    p.W = W; p.F = F; p.coeffs = coeffs;
    p.piE = t.piE; p.ptE = t.ptE; p.Q = t.Q;
    p.tmaps = t.tmaps;
    p.G = G;
    p.bar = words; p.status = status; p.wait_ns = wait_ns;
    p.eW = reinterpret_cast<int *>(words + kChainBarWords);
    p.eF = p.eW + (int64_t)L * p.Nc;
    // the barrier words only: the kernel writes every field it reads before reading it
    cudaError_t e = cudaMemsetAsync(words, 0, sizeof(unsigned) * kChainBarWords, s);
    if (e != cudaSuccess) return e;
    if (tf32) return launch_chain<1, true>(p, grid, s);
    if (nsl == S) return launch_chain<S, false>(p, grid, s);
    if (nsl == 2) return launch_chain<2, false>(p, grid, s);
    if (nsl == 1) return launch_chain<1, false>(p, grid, s);
    return cudaErrorInvalidValue;
}

}  // namespace sht
