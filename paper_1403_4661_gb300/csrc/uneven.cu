// Uneven batches (signals of different band-limits L_i) in ONE persistent launch per direction.
//
// The per-signal transform is the paper's (Procedure 1 in bin space, Eqs. (14)-(16); Procedure 2,
// Eqs. (11), (18)); batching signals of uneven L is this library's.  The batch is described once
// (sht_uneven_create: every signal's plan and offset, copied to the device), then each call is one
// cooperative launch of a grid that stays resident and walks the batch's work items:
//
//   inverse  phase 1: items (signal i, order m), L_i per signal: G_{+-m}(theta_k) for every ring k
//                     of signal i (Eq. (11)), from its coefficients and its plan's P~ block m;
//            grid barrier;
//            phase 2: items (signal i, ring k): fold of the orders into the ring's 2k+1 bins and
//                     the inverse ring DFT (Eq. (18)), with the plan's chirp-z tables;
//   forward  phase 1: items (signal i, ring k): ring DFT into the signal's order-major bins;
//            grid barrier;
//            phase 2: each signal's order chain, m = L-1..0, solve (plan's P_m^{-1}) and alias
//                     subtraction (plan's P~ block m, or P~ regenerated): the signals whose chain
//                     is a large share of the batch on teams of up to 16 CTAs (rows and rings
//                     split, two team barriers per order), the rest one CTA each, largest L
//                     first, from a queue.
//
// All arithmetic is float64 on the SIMT pipes, on the plans' float64 tables (every complex128
// scalar plan keeps them).  Items of one phase are independent; the waits on other CTAs are the
// grid barrier between the phases and the team barriers, all bounded (the plan wait limit of the
// first plan): a CTA that gives up sets the batch's status word and an abort word, and every CTA
// leaves.  The cooperative launch guarantees that all CTAs are resident, so no barrier can wait on
// a CTA that never runs.  Scratch (bins or synthesis table per signal) is allocated by
// sht_uneven_create; a call allocates nothing and synchronises nothing.
#include <algorithm>
#include <cstring>
#include <numeric>
#include <vector>

#include "fft_device.cuh"
#include "uneven_schedule.h"

namespace sht {
namespace {

using namespace fft;

constexpr int kUThreads = 256;

struct UPlan {
    int L, Mtab;
    const double *pt, *pinv;                    // P~ table (null: regenerated), per-order inverses
    const double *theta;                        // ring co-latitudes
    const double *sect_mant; const int *sect_expo;   // P~_m^m(theta_k) = mant * 2^expo, [m][k]
    const double *rec_a, *rec_b;                // recursion coefficients, block m at rows_off(L, m)
    const double2 *chirp, *filt, *tw;           // ring DFT tables
    const int *ring_M;                          // per ring: chirp-z length (0: direct)
    const int64_t *ring_foff;                   // per ring: filter offset
};

struct USig {
    int plan, L;
    int64_t off;      // complex-element offset of the signal in the caller's arrays
    int64_t ws;       // double offset of the signal's scratch (4 columns per row)
    int64_t item0;    // first item of the signal in the per-(signal, order / ring) phases
};

struct UArgs {
    const UPlan *plans;
    const USig *sigs;
    const UTask *tasks;      // team tasks, CTA c: tasks[task_start[c] .. task_start[c+1])
    const int *task_start;   // gridDim.x + 1 entries
    const int *small;        // signals chained by one CTA, descending L
    int nsmall;
    unsigned *team_bar;      // team t's barrier counter at 32 t (zeroed per launch)
    int nsig;
    int64_t items;    // sum of L_i
    double *ws;
    unsigned *bar;    // [0] arrivals, [32] abort (separate 128-byte lines)
    int *status;
    uint64_t wait_ns;
    const double2 *in;
    double2 *out;
};

__device__ __forceinline__ uint64_t now_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Signal of work item `it` (sigs ordered by item0).
__device__ __forceinline__ int item_signal(const UArgs &a, int64_t it) {
    int lo = 0, hi = a.nsig - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (a.sigs[mid].item0 <= it) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// One grid-wide barrier (the only one of a launch); false once any CTA has given up.
__device__ bool grid_barrier_once(const UArgs &a, int *flag) {
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        __threadfence();
        atomicAdd(a.bar, 1u);
        volatile unsigned *cnt = a.bar, *abort_w = a.bar + 32;
        const uint64_t t0 = now_ns();
        while (*cnt < gridDim.x) {
            if (*abort_w) { ok = 0; break; }
            if (now_ns() - t0 > a.wait_ns) {
                atomicOr(a.status, 2);
                atomicExch(a.bar + 32, 1u);
                ok = 0;
                break;
            }
        }
        __threadfence();
        *flag = ok;
    }
    __syncthreads();
    return *flag != 0;
}

// sum_{l = m..L-1} P~_l^m(theta_k) v[l - m][0..3] with P~ regenerated by its recursion (Sec. III-G)
// instead of read from a table: the sectoral start value is carried as mantissa * 2^e while it is
// below the float64 range (values below 2^-960 contribute nothing and are skipped), then the
// recursion continues on plain values (they only grow from there).  v: 4 doubles per degree.
__device__ __forceinline__ void recur_dot(const UPlan &pl, int L, int m, int k, double xk, const double *v,
                                          double &s0, double &s1, double &s2, double &s3) {
    const int n = L - m;
    double p = __ldg(pl.sect_mant + (int64_t)m * L + k), pp = 0.0;
    int e = __ldg(pl.sect_expo + (int64_t)m * L + k);
    const double *ra = pl.rec_a + rows_off(L, m), *rb = pl.rec_b + rows_off(L, m);
    bool live = false;
    s0 = s1 = s2 = s3 = 0.0;
    for (int j = 0; j < n; ++j) {
        if (j > 0) {
            const double nx = __ldg(ra + j) * fma(xk, p, -__ldg(rb + j) * pp);
            pp = p;
            p = nx;
        }
        if (!live) {
            const int be = (int)((__double_as_longlong(p) >> 52) & 0x7ff) - 1023;   // exponent of p
            if (p != 0.0 && be + e >= -960) {
                p = scalbn(p, e);
                pp = scalbn(pp, e);
                live = true;
            } else if (e < 0 && be > 512) {   // keep the mantissa in range while e < 0
                p = scalbn(p, -512);
                pp = scalbn(pp, -512);
                e += 512;
            }
        }
        if (live) {
            s0 = fma(p, v[4 * j], s0);
            s1 = fma(p, v[4 * j + 1], s1);
            s2 = fma(p, v[4 * j + 2], s2);
            s3 = fma(p, v[4 * j + 3], s3);
        }
    }
}

__device__ __forceinline__ void warp_sum4(double &s0, double &s1, double &s2, double &s3) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        s0 += __shfl_xor_sync(0xffffffffu, s0, o);
        s1 += __shfl_xor_sync(0xffffffffu, s1, o);
        s2 += __shfl_xor_sync(0xffffffffu, s2, o);
        s3 += __shfl_xor_sync(0xffffffffu, s3, o);
    }
}

// sum_c row[c] v[4c .. 4c+3], c < n, by one warp (lanes over c, coalesced row reads), summed
// across the warp: every lane returns the four sums.
__device__ __forceinline__ void warp_dot4(const double *__restrict__ row, const double *v, int n, int lane,
                                          double &s0, double &s1, double &s2, double &s3) {
    s0 = s1 = s2 = s3 = 0.0;
    for (int c = lane; c < n; c += 32) {
        const double pv = __ldg(row + c);
        s0 = fma(pv, v[4 * c], s0);
        s1 = fma(pv, v[4 * c + 1], s1);
        s2 = fma(pv, v[4 * c + 2], s2);
        s3 = fma(pv, v[4 * c + 3], s3);
    }
    warp_sum4(s0, s1, s2, s3);
}

// ---- inverse ----------------------------------------------------------------------------------

// Bin t of ring k (2k+1 bins) folded from the signal's synthesis table G (rows (|m|, k), 4
// columns): sum over m = q mod N, |m| < L; threads of `group` (g = 0..G-1) split the orders.
__device__ __forceinline__ double2 fold_part(const double *__restrict__ G, int L, int k, int t, int g, int Gn) {
    const int N = 2 * k + 1, q = t <= k ? t : t - N;
    double ax = 0.0, ay = 0.0;
    for (int m = q - ((q + L - 1) / N) * N + g * N; m <= L - 1; m += Gn * N) {
        const int o = m < 0 ? -m : m;
        const double *p = G + ((int64_t)o * L + k) * 4 + (m < 0 ? 2 : 0);
        ax += __ldcg(p);       // written by other CTAs before the grid barrier: read through L2
        ay += __ldcg(p + 1);
    }
    return make_double2(ax, ay);
}

__global__ void __launch_bounds__(kUThreads) k_uneven_inverse(UArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double *xs = reinterpret_cast<double *>(smem_raw);
    double2 *sm = reinterpret_cast<double2 *>(smem_raw);
    __shared__ int s_flag;
    const int tid = threadIdx.x;
    // phase 1: G_{+-m}(theta_k) = sum_l P~_l^m(theta_k) (f_l^m, (-1)^m f_l^{-m}) for all k
    for (int64_t it = blockIdx.x; it < a.items; it += gridDim.x) {
        const USig sg = a.sigs[item_signal(a, it)];
        const UPlan pl = a.plans[sg.plan];
        const int L = sg.L, m = (int)(it - sg.item0), n = L - m;
        const double2 *c = a.in + sg.off;
        __syncthreads();   // the previous item is done with xs
        for (int r = tid; r < n; r += blockDim.x) {
            const int l = m + r;
            const double2 p = c[(int64_t)l * l + l + m];
            double2 q = make_double2(0.0, 0.0);
            if (m > 0) {
                q = c[(int64_t)l * l + l - m];
                if (m & 1) { q.x = -q.x; q.y = -q.y; }
            }
            xs[4 * r] = p.x; xs[4 * r + 1] = p.y; xs[4 * r + 2] = q.x; xs[4 * r + 3] = q.y;
        }
        __syncthreads();
        double *G = a.ws + sg.ws + (int64_t)m * L * 4;
        if (pl.pt && n >= 64) {
            // one ring per warp, lanes along the table row (coalesced)
            const int lane = tid & 31;
            for (int k = tid >> 5; k < L; k += (int)blockDim.x >> 5) {
                double s0, s1, s2, s3;
                warp_dot4(pl.pt + pt_off(L, m) + (int64_t)k * n, xs, n, lane, s0, s1, s2, s3);
                if (lane == 0) {
                    double *g = G + 4 * (int64_t)k;
                    g[0] = s0; g[1] = s1; g[2] = s2; g[3] = s3;
                }
            }
            continue;
        }
        for (int k = tid; k < L; k += blockDim.x) {
            double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
            if (pl.pt) {
                const double *row = pl.pt + pt_off(L, m) + (int64_t)k * n;
                for (int r = 0; r < n; ++r) {
                    const double pv = __ldg(row + r);
                    s0 = fma(pv, xs[4 * r], s0);
                    s1 = fma(pv, xs[4 * r + 1], s1);
                    s2 = fma(pv, xs[4 * r + 2], s2);
                    s3 = fma(pv, xs[4 * r + 3], s3);
                }
            } else {
                recur_dot(pl, L, m, k, cos(__ldg(pl.theta + k)), xs, s0, s1, s2, s3);
            }
            double *g = G + 4 * (int64_t)k;
            g[0] = s0; g[1] = s1; g[2] = s2; g[3] = s3;
        }
    }
    if (!grid_barrier_once(a, &s_flag)) return;
    // phase 2: fold + inverse ring DFT per (signal, ring)
    for (int64_t it = blockIdx.x; it < a.items; it += gridDim.x) {
        const USig sg = a.sigs[item_signal(a, it)];
        const UPlan pl = a.plans[sg.plan];
        const int L = sg.L, k = (int)(it - sg.item0), N = 2 * k + 1;
        const double *G = a.ws + sg.ws;
        double2 *y = a.out + sg.off + (int64_t)k * k;
        const int M = __ldg(pl.ring_M + k);
        __syncthreads();   // the previous item is done with the shared buffer
        if (M == 0) {
            // direct ring: bins by groups of threads, then the direct sum with a root table
            double2 *B = sm, *roots = sm + N, *part = sm + 2 * N;
            const int Gn = max(1, (int)blockDim.x / N);
            for (int t = tid; t < N * Gn; t += blockDim.x) part[t] = fold_part(G, L, k, t % N, t / N, Gn);
            for (int t = tid; t < N; t += blockDim.x) {
                double s, cc;
                sincospi(2.0 * (double)t / (double)N, &s, &cc);
                roots[t] = make_double2(cc, s);   // e^{+2 pi i t / N}
            }
            __syncthreads();
            for (int j = tid; j < N; j += blockDim.x) {
                double2 acc = part[j];
                for (int g = 1; g < Gn; ++g) acc = cadd(acc, part[g * N + j]);
                B[j] = acc;
            }
            __syncthreads();
            for (int nn = tid; nn < N; nn += blockDim.x) {
                double2 acc = make_double2(0.0, 0.0);
                int idx = 0;
                for (int j = 0; j < N; ++j) {
                    acc = cadd(acc, cmul(B[j], roots[idx]));
                    idx += nn; if (idx >= N) idx -= N;
                }
                y[nn] = acc;
            }
            continue;
        }
        const Stages st = stages_of(M);
        const double2 *cz = pl.chirp + (int64_t)k * k;
        const double2 *f = pl.filt + __ldg(pl.ring_foff + k);
        bluestein(sm, N, M, st, pl.tw, pl.Mtab, cz, f,
                  [&](int t) { return conjd(fold_part(G, L, k, t, 0, 1)); },
                  [&](int t, double2 v) { y[t] = conjd(v); });
    }
}

// ---- forward ----------------------------------------------------------------------------------

// Bin t of ring k into the signal's order-major bins W (rows rows_off(L, |q|) + k - |q|, 4
// columns), scaled 1/N.
__device__ __forceinline__ void store_bin_u(double *W, int L, int k, int t, double2 v) {
    const int N = 2 * k + 1, q = t <= k ? t : t - N;
    const double sc = 1.0 / (double)N;
    const int o = q < 0 ? -q : q;
    double *w = W + (rows_off(L, o) + (k - o)) * 4;
    if (q >= 0) { w[0] = v.x * sc; w[1] = v.y * sc; }
    else        { w[2] = v.x * sc; w[3] = v.y * sc; }
    if (q == 0) { w[2] = 0.0; w[3] = 0.0; }
}

// Barrier of the T CTAs of one team (counter `bar`, growing within a launch; the j-th barrier is
// passed at j T arrivals); false once any CTA of the launch has given up.  T = 1: the CTA alone.
__device__ bool team_barrier(const UArgs &a, unsigned *bar, int T, unsigned &target, int *flag) {
    __syncthreads();
    if (T == 1) return true;
    target += (unsigned)T;
    if (threadIdx.x == 0) {
        int ok = 1;
        __threadfence();
        atomicAdd(bar, 1u);
        volatile unsigned *cnt = bar, *abort_w = a.bar + 32;
        if (*cnt < target) {
            const uint64_t t0 = now_ns();
            while (*cnt < target) {
                if (*abort_w) { ok = 0; break; }
                if (now_ns() - t0 > a.wait_ns) {
                    atomicOr(a.status, 2);
                    atomicExch(a.bar + 32, 1u);
                    ok = 0;
                    break;
                }
            }
        }
        __threadfence();
        *flag = ok;
    }
    __syncthreads();
    return *flag != 0;
}

// Order chain of signal `sig` (Eqs. (14)-(16), m = L-1..0) as member `rank` of a team of T CTAs:
// the member solves rows [rank n / T, (rank+1) n / T) of F_m = P_m^{-1} g_m and subtracts the
// aliases of rings [rank m / T, (rank+1) m / T); F_m passes between members through global
// scratch (the signal's scratch beyond its bins), with a team barrier after the solve and one
// after the alias subtraction.  T = 1 keeps everything in the CTA.  Rows and rings of n >= 64
// go one per warp (lanes along the row: coalesced table reads), shorter ones one per thread.
__device__ bool chain_signal(const UArgs &a, int sig, int rank, int T, unsigned *bar, double *ds, int *flag) {
    const USig sg = a.sigs[sig];
    const UPlan pl = a.plans[sg.plan];
    const int L = sg.L, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = (int)blockDim.x >> 5;
    double *W = a.ws + sg.ws;
    double *Fg = W + 4 * rows_total(L);   // F_m of the team (4 L doubles; the scratch holds 4 L^2)
    double2 *co = a.out + sg.off;
    double *g = ds, *fm = ds + 4 * L;
    unsigned target = 0;
    for (int m = L - 1; m >= 0; --m) {
        const int n = L - m;
        __syncthreads();
        // g_m: bins +-m of rings k >= m (Eq. (11)), free of the orders above m by now
        const double *Wm = W + rows_off(L, m) * 4;
        for (int i = tid; i < 4 * n; i += blockDim.x) g[i] = __ldcg(Wm + i);   // written by other CTAs
        __syncthreads();
        // Eq. (14): rows r0..r1 of F_m = P_m^{-1} g_m; f_l^{+m} and f_l^{-m} = (-1)^m F^{-}
        const double *Pi = pl.pinv + pinv_off(L, m);
        const int r0 = (int)((int64_t)rank * n / T), r1 = (int)((int64_t)(rank + 1) * n / T);
        double *F = T > 1 ? Fg : fm;
        auto emit = [&](int r, double s0, double s1, double s2, double s3) {
            F[4 * r] = s0; F[4 * r + 1] = s1; F[4 * r + 2] = s2; F[4 * r + 3] = s3;
            const int l = m + r;
            double2 *cl = co + (int64_t)l * l + l;
            cl[m] = make_double2(s0, s1);
            if (m > 0) cl[-m] = (m & 1) ? make_double2(-s2, -s3) : make_double2(s2, s3);
        };
        if (n >= 64) {
            for (int r = r0 + warp; r < r1; r += nw) {
                double s0, s1, s2, s3;
                warp_dot4(Pi + (int64_t)r * n, g, n, lane, s0, s1, s2, s3);
                if (lane == 0) emit(r, s0, s1, s2, s3);
            }
        } else {
            for (int r = r0 + tid; r < r1; r += blockDim.x) {
                const double *row = Pi + (int64_t)r * n;
                double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
                for (int c = 0; c < n; ++c) {
                    const double pv = __ldg(row + c);
                    s0 = fma(pv, g[4 * c], s0);
                    s1 = fma(pv, g[4 * c + 1], s1);
                    s2 = fma(pv, g[4 * c + 2], s2);
                    s3 = fma(pv, g[4 * c + 3], s3);
                }
                emit(r, s0, s1, s2, s3);
            }
        }
        if (m == 0) break;
        if (!team_barrier(a, bar, T, target, flag)) return false;
        if (T > 1)
            for (int i = tid; i < 4 * n; i += blockDim.x) fm[i] = __ldcg(Fg + i);
        __syncthreads();
        // Eqs. (15)-(16): G_{+-m}(theta_k), k < m, out of bins alias_k(+-m) of ring k
        const int k0 = (int)((int64_t)rank * m / T), k1 = (int)((int64_t)(rank + 1) * m / T);
        auto subtract = [&](int k, double s0, double s1, double s2, double s3) {
            const int aa = alias_bin(m, k), o = aa < 0 ? -aa : aa;
            double *w = W + (rows_off(L, o) + (k - o)) * 4;
            if (aa == 0) {
                w[0] = __ldcg(w) - (s0 + s2);
                w[1] = __ldcg(w + 1) - (s1 + s3);
            } else {
                const int sp = aa > 0 ? 0 : 2, sq = 2 - sp;   // slots of bins aa and -aa
                w[sp] = __ldcg(w + sp) - s0; w[sp + 1] = __ldcg(w + sp + 1) - s1;
                w[sq] = __ldcg(w + sq) - s2; w[sq + 1] = __ldcg(w + sq + 1) - s3;
            }
        };
        if (pl.pt && n >= 64) {
            for (int k = k0 + warp; k < k1; k += nw) {
                double s0, s1, s2, s3;
                warp_dot4(pl.pt + pt_off(L, m) + (int64_t)k * n, fm, n, lane, s0, s1, s2, s3);
                if (lane == 0) subtract(k, s0, s1, s2, s3);
            }
        } else {
            for (int k = k0 + tid; k < k1; k += blockDim.x) {
                double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
                if (pl.pt) {
                    const double *row = pl.pt + pt_off(L, m) + (int64_t)k * n;
                    for (int r = 0; r < n; ++r) {
                        const double pv = __ldg(row + r);
                        s0 = fma(pv, fm[4 * r], s0);
                        s1 = fma(pv, fm[4 * r + 1], s1);
                        s2 = fma(pv, fm[4 * r + 2], s2);
                        s3 = fma(pv, fm[4 * r + 3], s3);
                    }
                } else {
                    recur_dot(pl, L, m, k, cos(__ldg(pl.theta + k)), fm, s0, s1, s2, s3);
                }
                subtract(k, s0, s1, s2, s3);
            }
        }
        if (!team_barrier(a, bar, T, target, flag)) return false;
    }
    return true;
}

__global__ void __launch_bounds__(kUThreads) k_uneven_forward(UArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double2 *sm = reinterpret_cast<double2 *>(smem_raw);
    double *ds = reinterpret_cast<double *>(smem_raw);
    __shared__ int s_flag;
    const int tid = threadIdx.x;
    // phase 1: ring DFTs into bins
    for (int64_t it = blockIdx.x; it < a.items; it += gridDim.x) {
        const USig sg = a.sigs[item_signal(a, it)];
        const UPlan pl = a.plans[sg.plan];
        const int L = sg.L, k = (int)(it - sg.item0), N = 2 * k + 1;
        double *W = a.ws + sg.ws;
        const double2 *x = a.in + sg.off + (int64_t)k * k;
        const int M = __ldg(pl.ring_M + k);
        __syncthreads();
        if (M == 0) {
            double2 *xs = sm, *roots = sm + N;
            for (int t = tid; t < N; t += blockDim.x) {
                xs[t] = x[t];
                double s, cc;
                sincospi(2.0 * (double)t / (double)N, &s, &cc);
                roots[t] = make_double2(cc, -s);   // e^{-2 pi i t / N}
            }
            __syncthreads();
            for (int j = tid; j < N; j += blockDim.x) {
                double2 acc = make_double2(0.0, 0.0);
                int idx = 0;
                for (int nn = 0; nn < N; ++nn) {
                    acc = cadd(acc, cmul(xs[nn], roots[idx]));
                    idx += j; if (idx >= N) idx -= N;
                }
                store_bin_u(W, L, k, j, acc);
            }
            continue;
        }
        const Stages st = stages_of(M);
        const double2 *cz = pl.chirp + (int64_t)k * k;
        const double2 *f = pl.filt + __ldg(pl.ring_foff + k);
        bluestein(sm, N, M, st, pl.tw, pl.Mtab, cz, f,
                  [&](int t) { return x[t]; },
                  [&](int t, double2 v) { store_bin_u(W, L, k, t, v); });
    }
    if (!grid_barrier_once(a, &s_flag)) return;
    // phase 2a: the large signals' chains, each on a team of CTAs (static lists, in one global
    // order, so that a team only ever waits for members busy with earlier teams)
    for (int t = a.task_start[blockIdx.x]; t < a.task_start[blockIdx.x + 1]; ++t) {
        const UTask tk = a.tasks[t];
        if (!chain_signal(a, tk.sig, tk.rank, tk.T, a.team_bar + 32 * tk.team, ds, &s_flag)) return;
    }
    // phase 2b: the other signals, one CTA each, largest L first from a shared queue
    __shared__ int s_next;
    for (;;) {
        __syncthreads();
        if (tid == 0) s_next = (int)atomicAdd(a.bar + 64, 1u);
        __syncthreads();
        if (s_next >= a.nsmall) break;
        chain_signal(a, a.small[s_next], 0, 1, nullptr, ds, &s_flag);
    }
}

}  // namespace
}  // namespace sht

using namespace sht;

struct sht_uneven_s {
    int device = 0;
    int nsig = 0;
    int64_t items = 0;
    int64_t span = 0;              // complex elements covered: max(offset + L^2)
    std::vector<sht_plan_t> plans;
    UPlan *d_plans = nullptr;
    USig *d_sigs = nullptr;
    UTask *d_tasks = nullptr;      // forward team tasks and their per-CTA ranges
    int *d_task_start = nullptr;
    int *d_small = nullptr;        // signals chained by one CTA, descending L
    int nsmall = 0, nteams = 0;
    unsigned *team_bar = nullptr;  // 32 words per team
    double *ws = nullptr;
    unsigned *bar = nullptr;       // kBarWords words: arrival counter [0], abort word [32], queue [64]
    int *status = nullptr;
    size_t smem = 0;
    int grid_inv = 0, grid_fwd = 0;
    uint64_t wait_ns = 1000000000ull;
    uint64_t bytes = 0;
};

namespace {

void uneven_free(sht_uneven_t u) {
    if (!u) return;
    cudaFree(u->d_plans); cudaFree(u->d_sigs); cudaFree(u->d_tasks); cudaFree(u->d_task_start);
    cudaFree(u->d_small); cudaFree(u->team_bar); cudaFree(u->ws);
    cudaFree(u->bar); cudaFree(u->status);
    delete u;
}

constexpr int kBarWords = 96;   // arrival counter [0], abort word [32], small-signal queue [64]

template <typename K>
cudaError_t coop_grid(K kernel, size_t smem, int *grid) {
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, per_sm = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kUThreads, smem)) != cudaSuccess) return e;
    *grid = sms * per_sm;
    return *grid > 0 ? cudaSuccess : cudaErrorInvalidConfiguration;
}

sht_status uneven_launch(sht_uneven_t u, bool forward, const void *d_in, void *d_out, void *stream) {
    if (!u) return set_error(SHT_ERR_INVALID_ARG, "uneven batch is NULL");
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_check(e, "cudaGetDevice");
    if (dev != u->device) return set_error(SHT_ERR_INVALID_ARG, "current device is not the batch's device");
    if (u->nsig == 0) return SHT_OK;
    if (!d_in || !d_out) return set_error(SHT_ERR_INVALID_ARG, "NULL buffer");
    if (((uintptr_t)d_in & 15u) || ((uintptr_t)d_out & 15u))
        return set_error(SHT_ERR_INVALID_ARG, "buffers must be 16-byte aligned");
    const uintptr_t bytes = (uintptr_t)16 * (uintptr_t)u->span, a = (uintptr_t)d_in, b = (uintptr_t)d_out;
    if (a < b + bytes && b < a + bytes) return set_error(SHT_ERR_INVALID_ARG, "input and output overlap");
    cudaStream_t s = (cudaStream_t)stream;
    UArgs args{u->d_plans, u->d_sigs, u->d_tasks, u->d_task_start, u->d_small, u->nsmall, u->team_bar,
               u->nsig, u->items, u->ws, u->bar, u->status, u->wait_ns,
               (const double2 *)d_in, (double2 *)d_out};
    if ((e = cudaMemsetAsync(u->bar, 0, kBarWords * sizeof(unsigned), s)) != cudaSuccess ||
        (u->nteams && (e = cudaMemsetAsync(u->team_bar, 0, 32 * sizeof(unsigned) * (size_t)u->nteams, s)) != cudaSuccess))
        return cuda_check(e, "uneven barrier");
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(forward ? u->grid_fwd : u->grid_inv));
    cfg.blockDim = dim3(kUThreads);
    cfg.dynamicSmemBytes = u->smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    e = forward ? cudaLaunchKernelEx(&cfg, k_uneven_forward, args) : cudaLaunchKernelEx(&cfg, k_uneven_inverse, args);
    return cuda_check(e, forward ? "sht_uneven_forward" : "sht_uneven_inverse");
}

}  // namespace

extern "C" {

sht_status sht_uneven_create(const sht_plan_t *plans, int nplans, int64_t nsig, const int *plan_index,
                             const int64_t *offsets, sht_uneven_t *out) {
    if (!out) return set_error(SHT_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (nsig < 0 || nplans < 0) return set_error(SHT_ERR_INVALID_ARG, "negative count");
    if (nsig > 0 && (!plans || !plan_index || !offsets || nplans == 0))
        return set_error(SHT_ERR_INVALID_ARG, "NULL plan, index or offset array");
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_check(e, "cudaGetDevice");
    int Lmax = 1, Mmax = 16;
    for (int g = 0; g < nplans; ++g) {
        sht_status st = check_plan(plans[g]);
        if (st != SHT_OK) return st;
        if (plans[g]->dtype == SHT_F32)
            return set_error(SHT_ERR_UNSUPPORTED, "uneven batches take complex128 plans (not SHT_F32)");
        if (plans[g]->spin != 0) return set_error(SHT_ERR_UNSUPPORTED, "uneven batches take scalar (spin-0) plans");
        Lmax = std::max(Lmax, plans[g]->L);
        Mmax = std::max(Mmax, plans[g]->dft.Mmax);
    }
    // signals as intervals [offset, offset + L^2) of complex elements: in range, disjoint
    std::vector<std::pair<int64_t, int64_t>> iv((size_t)nsig);
    for (int64_t i = 0; i < nsig; ++i) {
        const int g = plan_index[i];
        if (g < 0 || g >= nplans) return set_error(SHT_ERR_INVALID_ARG, "plan index out of range");
        if (offsets[i] < 0) return set_error(SHT_ERR_INVALID_ARG, "negative offset");
        const int64_t L = plans[g]->L;
        iv[(size_t)i] = {offsets[i], offsets[i] + L * L};
    }
    std::vector<std::pair<int64_t, int64_t>> sorted = iv;
    std::sort(sorted.begin(), sorted.end());
    for (size_t i = 1; i < sorted.size(); ++i)
        if (sorted[i].first < sorted[i - 1].second) return set_error(SHT_ERR_INVALID_ARG, "signals overlap");

    sht_uneven_t u = new sht_uneven_s;
    u->device = dev;
    u->nsig = (int)nsig;
    u->plans.assign(plans, plans + nplans);
    std::vector<UPlan> hp((size_t)nplans);
    for (int g = 0; g < nplans; ++g) {
        const sht_plan_t p = plans[g];
        hp[(size_t)g] = UPlan{p->L, p->dft.Mtab, p->pt, p->pinv, p->d_theta, p->sect_mant, p->sect_expo,
                              p->rec_a, p->rec_b, p->dft.chirp, p->dft.filt, p->dft.twiddle,
                              p->dft.d_ring_M, p->dft.d_ring_foff};
    }
    std::vector<USig> hs((size_t)nsig);
    int64_t ws = 0, items = 0;
    for (int64_t i = 0; i < nsig; ++i) {
        const int g = plan_index[i], L = plans[g]->L;
        hs[(size_t)i] = USig{g, L, offsets[i], ws, items};
        ws += 4 * std::max<int64_t>(rows_total(L), (int64_t)L * L);   // bins (forward) or G (inverse)
        items += L;
        u->span = std::max(u->span, iv[(size_t)i].second);
    }
    u->items = items;
    std::vector<int> lpt((size_t)nsig);
    std::iota(lpt.begin(), lpt.end(), 0);
    std::stable_sort(lpt.begin(), lpt.end(), [&](int x, int y) { return hs[(size_t)x].L > hs[(size_t)y].L; });
    // shared memory: the largest chirp-z ring, the chain's two order vectors, the synthesis input
    u->smem = std::max({sizeof(double2) * (size_t)Mmax, sizeof(double) * 8 * (size_t)Lmax,
                        sizeof(double2) * (size_t)(2 * (2 * 31 + 1) + kUThreads + 2 * 63)});
    u->wait_ns = nplans > 0 ? plans[0]->wait_ns : 1000000000ull;
    if ((e = coop_grid(k_uneven_inverse, u->smem, &u->grid_inv)) != cudaSuccess ||
        (e = coop_grid(k_uneven_forward, u->smem, &u->grid_fwd)) != cudaSuccess) {
        uneven_free(u);
        return cuda_check(e, "uneven batch set-up");
    }
    std::vector<UTask> tasks;
    std::vector<int> task_start, small;
    std::vector<int> Ls((size_t)nsig);
    for (int64_t i = 0; i < nsig; ++i) Ls[(size_t)i] = hs[(size_t)i].L;
    plan_teams(Ls, lpt, u->grid_fwd, tasks, task_start, small, u->nteams);
    u->nsmall = (int)small.size();
    const size_t b_ws = sizeof(double) * (size_t)std::max<int64_t>(ws, 1);
    if ((e = cudaMalloc(&u->d_plans, sizeof(UPlan) * std::max<size_t>(hp.size(), 1))) != cudaSuccess ||
        (e = cudaMalloc(&u->d_sigs, sizeof(USig) * std::max<size_t>(hs.size(), 1))) != cudaSuccess ||
        (e = cudaMalloc(&u->d_tasks, sizeof(UTask) * std::max<size_t>(tasks.size(), 1))) != cudaSuccess ||
        (e = cudaMalloc(&u->d_task_start, sizeof(int) * task_start.size())) != cudaSuccess ||
        (e = cudaMalloc(&u->d_small, sizeof(int) * std::max<size_t>(small.size(), 1))) != cudaSuccess ||
        (e = cudaMalloc(&u->team_bar, 32 * sizeof(unsigned) * (size_t)std::max(u->nteams, 1))) != cudaSuccess ||
        (e = cudaMalloc(&u->ws, b_ws)) != cudaSuccess ||
        (e = cudaMalloc(&u->bar, kBarWords * sizeof(unsigned))) != cudaSuccess ||
        (e = cudaMalloc(&u->status, sizeof(int))) != cudaSuccess) {
        uneven_free(u);
        return cuda_check(e, "uneven batch allocation");
    }
    u->bytes = b_ws + sizeof(UPlan) * hp.size() + sizeof(USig) * hs.size() + sizeof(UTask) * tasks.size() +
               sizeof(int) * (task_start.size() + small.size()) + 128 * (size_t)u->nteams;
    if ((nplans && (e = cudaMemcpy(u->d_plans, hp.data(), sizeof(UPlan) * hp.size(), cudaMemcpyHostToDevice)) != cudaSuccess) ||
        (nsig && (e = cudaMemcpy(u->d_sigs, hs.data(), sizeof(USig) * hs.size(), cudaMemcpyHostToDevice)) != cudaSuccess) ||
        (!tasks.empty() && (e = cudaMemcpy(u->d_tasks, tasks.data(), sizeof(UTask) * tasks.size(), cudaMemcpyHostToDevice)) != cudaSuccess) ||
        (e = cudaMemcpy(u->d_task_start, task_start.data(), sizeof(int) * task_start.size(), cudaMemcpyHostToDevice)) != cudaSuccess ||
        (!small.empty() && (e = cudaMemcpy(u->d_small, small.data(), sizeof(int) * small.size(), cudaMemcpyHostToDevice)) != cudaSuccess) ||
        (e = cudaMemset(u->status, 0, sizeof(int))) != cudaSuccess) {
        uneven_free(u);
        return cuda_check(e, "uneven batch set-up");
    }
    *out = u;
    return SHT_OK;
}

sht_status sht_uneven_forward(sht_uneven_t u, const void *d_samples, void *d_coeffs, void *stream) {
    return uneven_launch(u, true, d_samples, d_coeffs, stream);
}

sht_status sht_uneven_inverse(sht_uneven_t u, const void *d_coeffs, void *d_samples, void *stream) {
    return uneven_launch(u, false, d_coeffs, d_samples, stream);
}

sht_status sht_uneven_check(sht_uneven_t u) {
    if (!u) return set_error(SHT_ERR_INVALID_ARG, "uneven batch is NULL");
    int h = 0;
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(&h, u->status, sizeof(int), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && h) e = cudaMemset(u->status, 0, sizeof(int));
    if (e != cudaSuccess) return cuda_check(e, "sht_uneven_check");
    if (h) return set_error(SHT_ERR_TIMEOUT, "the grid barrier of an uneven-batch launch gave up");
    return SHT_OK;
}

sht_status sht_uneven_set_wait_limit(sht_uneven_t u, double seconds) {
    if (!u) return set_error(SHT_ERR_INVALID_ARG, "uneven batch is NULL");
    if (!(seconds >= 1e-9 && seconds <= 60.0))
        return set_error(SHT_ERR_INVALID_ARG, "wait limit must be in [1e-9, 60] seconds");
    u->wait_ns = (uint64_t)(seconds * 1e9);
    return SHT_OK;
}

sht_status sht_uneven_destroy(sht_uneven_t u) {
    if (!u) return SHT_OK;
    cudaDeviceSynchronize();
    uneven_free(u);
    return SHT_OK;
}

}  // extern "C"
