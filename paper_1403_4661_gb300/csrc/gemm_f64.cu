// Float64 contractions of the transforms: register-tiled SIMT GEMM (FFMA64), row-major operands,
// with the epilogues the order chain needs.  On GB300 float64 runs at ~1/64 of the float32 rate,
// so a tile keeps the FP64 pipe busy with few warps; what matters is filling all 152 SMs, which
// the launcher does by picking the tile shape from the problem size.  The same kernels,
// instantiated for float, are the contractions of SHT_F32 plans (FFMA32).
//
// Contractions served (N = 4 * batch real columns: signal b, +m / -m, re / im):
//  synthesis  G_{+-m}(theta_k) = sum_l P~_l^m(theta_k) X_m[l]  for every m and ring k   (Eq. (11))
//  analysis   the transposed contraction (adjoint of synthesis)
//  solve      F_m = P_m^{-1} W_m  (Eq. (14)), writing f_l^{+-m} to the coefficient output
//  alias      G_{+-m}(theta_k), k < m, subtracted from bin alias_k(+-m) of ring k (Eqs. (15)-(16))
#include <algorithm>

#include "epilogue.cuh"
#include "sht_internal.cuh"

namespace sht {
namespace {

constexpr int BK = 16;
constexpr int kMaxSplit = 16;

// Streaming multiprocessors of the current device (looked up once per device; 152 on GB300).
int sm_count() {
    static int cached[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 152;
    if (!cached[dev]) {
        int n = 0;
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 152;
        cached[dev] = n;
    }
    return cached[dev];
}

enum Mode : int { MODE_SINGLE = 0, MODE_SYNTH = 1, MODE_ANALYSIS = 2 };

template <typename T>
struct Params {
    const T *A; int64_t lda;
    const T *B; int64_t ldb;
    T *C; int64_t ldc;
    const T *C0;
    int M, K, N;
    int m;              // order (single-problem epilogues)
    int L;
    cplx_t<T> *coeffs;  // EPI_SOLVE
    T *W;               // EPI_ALIAS
    const T *pt; const T *X; T *Y;  // grouped modes
    T *part;            // split-K partial sums [split][M][N]
    int splits, kchunk;
    int slots;          // epilogue column pairs (bit 0: +m, bit 1: -m)
};

// sum_{j=1..x} ceil(j / bm)
__host__ __device__ __forceinline__ int64_t ceil_sum(int64_t x, int64_t bm) {
    int64_t q = x / bm, r = x % bm;
    return bm * q * (q + 1) / 2 + r * (q + 1);
}

template <int EPI, typename T>
__device__ __forceinline__ void epilogue(const Params<T> &p, T *C, int64_t ldc, int m, int N,
                                         int r, int c0, const T v[4]) {
    EpiArgsT<T> e{C, ldc, p.C0, m, p.L, N, p.coeffs, p.W, p.slots};
    epilogue_row4<EPI>(e, r, c0, v);
}

// Tile BM x BN, each thread TM rows x 4 columns (one signal), K in steps of BK through shared
// memory.  SPLIT: blockIdx.y selects a K chunk and the raw partial sums go to p.part.
template <typename T, int BM, int BN, int TM, bool TA, int EPI, int MODE, bool SPLIT>
__global__ void __launch_bounds__((BM / TM) * (BN / 4)) k_gemm(Params<T> p) {
    using C2 = cplx_t<T>;
    constexpr int NT = (BM / TM) * (BN / 4);
    __shared__ __align__(16) T As[BK][BM + 2];
    __shared__ __align__(16) T Bs[BK][BN + 2];

    const T *A = p.A, *B = p.B;
    T *C = p.C;
    int64_t lda = p.lda, ldb = p.ldb, ldc = p.ldc;
    int M = p.M, K = p.K, m = p.m;
    const int N = p.N;
    const int tiles_n = (N + BN - 1) / BN;
    int64_t tile = blockIdx.x;

    if (MODE == MODE_SYNTH) {
        // every order has M = L rows, so every order has the same tile count
        const int64_t per_m = (int64_t)((p.L + BM - 1) / BM) * tiles_n;
        m = (int)(tile / per_m);
        tile -= (int64_t)m * per_m;
        const int n = p.L - m;
        A = p.pt + pt_off(p.L, m); lda = n;
        B = p.X + rows_off(p.L, m) * N; ldb = N;
        C = p.Y + (int64_t)m * p.L * N; ldc = N;
        M = p.L; K = n;
    } else if (MODE == MODE_ANALYSIS) {
        // order m has M = L - m rows: tiles before m = tiles_n * (S(L) - S(L - m))
        const int64_t SL = ceil_sum(p.L, BM);
        int lo = 0, hi = p.L - 1;
        while (lo < hi) {
            int mid = (lo + hi + 1) >> 1;
            int64_t before = (int64_t)tiles_n * (SL - ceil_sum(p.L - mid, BM));
            if (before <= tile) lo = mid; else hi = mid - 1;
        }
        m = lo;
        tile -= (int64_t)tiles_n * (SL - ceil_sum(p.L - m, BM));
        const int n = p.L - m;
        A = p.pt + pt_off(p.L, m); lda = n;            // stored L x n, used transposed
        B = p.X + (int64_t)m * p.L * N; ldb = N;       // U[m][k][:]
        C = p.Y + rows_off(p.L, m) * N; ldc = N;
        M = n; K = p.L;
    }
    int kbeg = 0, kend = K;
    if (SPLIT) {
        kbeg = blockIdx.y * p.kchunk;
        kend = min(K, kbeg + p.kchunk);
    }
    const int tm = (int)(tile / tiles_n), tn = (int)(tile % tiles_n);
    const int row0 = tm * BM, col0 = tn * BN;
    const int tx = threadIdx.x % (BN / 4), ty = threadIdx.x / (BN / 4);

    T acc[TM][4];
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0;

    for (int k0 = kbeg; k0 < kend; k0 += BK) {
        for (int idx = threadIdx.x; idx < BM * BK; idx += NT) {
            int i, kk;
            if (!TA) { i = idx / BK; kk = idx % BK; } else { kk = idx / BM; i = idx % BM; }
            int r = row0 + i, k = k0 + kk;
            T v = 0;
            if (r < M && k < kend) v = TA ? A[(int64_t)k * lda + r] : A[(int64_t)r * lda + k];
            As[kk][i] = v;
        }
        for (int idx = threadIdx.x; idx < BN * BK; idx += NT) {
            int kk = idx / BN, j = idx % BN;
            int k = k0 + kk, c = col0 + j;
            Bs[kk][j] = (k < kend && c < N) ? B[(int64_t)k * ldb + c] : (T)0;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            T a[TM];
            if (TM == 1) {
                a[0] = As[kk][ty];
            } else {
#pragma unroll
                for (int i = 0; i < TM; i += 2) {
                    C2 t = *reinterpret_cast<const C2 *>(&As[kk][ty * TM + i]);
                    a[i] = t.x; a[i + 1] = t.y;
                }
            }
            C2 b01 = *reinterpret_cast<const C2 *>(&Bs[kk][tx * 4]);
            C2 b23 = *reinterpret_cast<const C2 *>(&Bs[kk][tx * 4 + 2]);
            T b[4] = {b01.x, b01.y, b23.x, b23.y};
#pragma unroll
            for (int i = 0; i < TM; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }

    const int c0 = col0 + tx * 4;
    if (c0 >= N) return;
#pragma unroll
    for (int i = 0; i < TM; ++i) {
        const int r = row0 + ty * TM + i;
        if (r >= M) break;
        if (SPLIT) {
            T *pp = p.part + ((int64_t)blockIdx.y * M + r) * N + c0;
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if (c0 + j < N) pp[j] = acc[i][j];
        } else {
            epilogue<EPI>(p, C, ldc, m, N, r, c0, acc[i]);
        }
    }
}

// Sum of the split-K partials in a fixed order (deterministic), then the epilogue.
template <typename T, int EPI>
__global__ void k_split_reduce(Params<T> p) {
    const int groups = (p.N + 3) / 4;
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)p.M * groups) return;
    const int r = (int)(t / groups), c0 = 4 * (int)(t - (int64_t)r * groups);
    T v[4] = {0, 0, 0, 0};
    for (int s = 0; s < p.splits; ++s) {
        const T *pp = p.part + ((int64_t)s * p.M + r) * p.N + c0;
#pragma unroll
        for (int j = 0; j < 4; ++j)
            if (c0 + j < p.N) v[j] += pp[j];
    }
    epilogue<EPI>(p, p.C, p.ldc, p.m, p.N, r, c0, v);
}

inline int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

struct Cfg { int bm, bn; };

// Tile choice: enough blocks for >= 2 per SM when the problem allows, each block 8 warps so
// that all four FP64 units of an SM are fed.
template <typename T, bool TA, int EPI, int MODE, bool SPLIT>
cudaError_t launch_cfg(const Params<T> &p, Cfg c, dim3 grid, cudaStream_t s) {
    if (c.bn == 64) {
        if (c.bm == 64) k_gemm<T, 64, 64, 4, TA, EPI, MODE, SPLIT><<<grid, 256, 0, s>>>(p);
        else if (c.bm == 32) k_gemm<T, 32, 64, 2, TA, EPI, MODE, SPLIT><<<grid, 256, 0, s>>>(p);
        else k_gemm<T, 16, 64, 1, TA, EPI, MODE, SPLIT><<<grid, 256, 0, s>>>(p);
    } else {
        k_gemm<T, 16, 16, 1, TA, EPI, MODE, SPLIT><<<grid, 64, 0, s>>>(p);
    }
    return cudaGetLastError();
}

int64_t tiles_of(int M, int N, Cfg c) { return cdiv(M, c.bm) * cdiv(N, c.bn); }

template <typename T, bool TA, int EPI>
cudaError_t launch_single(Params<T> p, cudaStream_t s, T *part, int64_t part_cap, int64_t *count,
                          int split_cap) {
    const int cap = split_cap > 0 ? std::min(split_cap, kMaxSplit) : kMaxSplit;
    const int kSMs = sm_count();
    Cfg c{64, 64};
    if (p.N <= 32) {
        c = Cfg{16, 16};
    } else {
        for (int bm : {64, 32, 16}) {
            c = Cfg{bm, 64};
            if (tiles_of(p.M, p.N, c) >= 2 * kSMs) break;
        }
    }
    const int64_t tiles = tiles_of(p.M, p.N, c);
    int splits = 1;
    if (part && tiles < 2 * kSMs && p.K >= 128) {
        splits = (int)std::min<int64_t>(std::min<int64_t>(cdiv(2 * kSMs, tiles), p.K / 64), cap);
        while (splits > 1 && (int64_t)splits * p.M * p.N > part_cap) --splits;
    }
    if (count) *count += splits <= 1 ? 1 : 2;
    if (splits <= 1) return launch_cfg<T, TA, EPI, MODE_SINGLE, false>(p, c, dim3((unsigned)tiles), s);
    p.splits = splits;
    p.kchunk = (int)(cdiv(cdiv(p.K, splits), BK) * BK);
    p.splits = (int)cdiv(p.K, p.kchunk);
    p.part = part;
    cudaError_t e = launch_cfg<T, TA, EPI, MODE_SINGLE, true>(p, c, dim3((unsigned)tiles, p.splits), s);
    if (e != cudaSuccess) return e;
    const int64_t work = (int64_t)p.M * cdiv(p.N, 4);
    k_split_reduce<T, EPI><<<(unsigned)cdiv(work, 256), 256, 0, s>>>(p);
    return cudaGetLastError();
}

template <typename T>
cudaError_t gemm_t(bool transA, int M, int K, int N, const T *A, int64_t lda, const T *B, int64_t ldb,
                   T *C, int64_t ldc, int epi, const GemmArgsT<T> &ga, cudaStream_t s, const T *C0) {
    if (M <= 0 || N <= 0) return cudaSuccess;
    Params<T> p{};
    p.A = A; p.lda = lda; p.B = B; p.ldb = ldb; p.C = C; p.ldc = ldc; p.C0 = C0;
    p.M = M; p.K = K; p.N = N; p.m = ga.m; p.L = ga.L; p.coeffs = ga.coeffs; p.W = ga.W;
    p.slots = ga.slots;
#define SHT_GEMM_CASE(E)                                                                        \
    if (epi == E) return transA ? launch_single<T, true, E>(p, s, ga.part, ga.part_cap, ga.launches, ga.split_cap) \
                                : launch_single<T, false, E>(p, s, ga.part, ga.part_cap, ga.launches, ga.split_cap);
    SHT_GEMM_CASE(EPI_STORE)
    SHT_GEMM_CASE(EPI_SOLVE)
    SHT_GEMM_CASE(EPI_ALIAS)
    SHT_GEMM_CASE(EPI_SUB)
#undef SHT_GEMM_CASE
    return cudaErrorInvalidValue;
}

template <typename T>
cudaError_t synthesis_t(int L, int64_t batch, const T *pt, const T *X, T *Gt, cudaStream_t s, int slots = 3) {
    Params<T> p{};
    p.L = L; p.N = (int)(4 * batch); p.pt = pt; p.X = X; p.Y = Gt; p.slots = slots;
    Cfg c = p.N <= 32 ? Cfg{16, 16} : Cfg{64, 64};
    const int64_t tiles = (int64_t)L * cdiv(L, c.bm) * cdiv(p.N, c.bn);
    return launch_cfg<T, false, EPI_STORE, MODE_SYNTH, false>(p, c, dim3((unsigned)tiles), s);
}

template <typename T>
cudaError_t analysis_t(int L, int64_t batch, const T *pt, const T *U, T *X, cudaStream_t s, int slots = 3) {
    Params<T> p{};
    p.L = L; p.N = (int)(4 * batch); p.pt = pt; p.X = U; p.Y = X; p.slots = slots;
    Cfg c = p.N <= 32 ? Cfg{16, 16} : Cfg{64, 64};
    const int64_t tiles = cdiv(p.N, c.bn) * ceil_sum(L, c.bm);
    return launch_cfg<T, true, EPI_STORE, MODE_ANALYSIS, false>(p, c, dim3((unsigned)tiles), s);
}

}  // namespace

cudaError_t gemm_f64(bool transA, int M, int K, int N, const double *A, int64_t lda,
                     const double *B, int64_t ldb, double *C, int64_t ldc, int epi,
                     const GemmArgs &ga, cudaStream_t s, const double *C0) {
    return gemm_t<double>(transA, M, K, N, A, lda, B, ldb, C, ldc, epi, ga, s, C0);
}
cudaError_t gemm_f32(bool transA, int M, int K, int N, const float *A, int64_t lda,
                     const float *B, int64_t ldb, float *C, int64_t ldc, int epi,
                     const GemmArgsT<float> &ga, cudaStream_t s, const float *C0) {
    return gemm_t<float>(transA, M, K, N, A, lda, B, ldb, C, ldc, epi, ga, s, C0);
}
cudaError_t synthesis_all_orders(int L, int64_t batch, const double *pt, const double *X,
                                 double *Gt, cudaStream_t s) {
    return synthesis_t<double>(L, batch, pt, X, Gt, s);
}
cudaError_t synthesis_all_orders(int L, int64_t batch, const float *pt, const float *X,
                                 float *Gt, cudaStream_t s) {
    return synthesis_t<float>(L, batch, pt, X, Gt, s);
}
cudaError_t analysis_all_orders(int L, int64_t batch, const double *pt, const double *U,
                                double *X, cudaStream_t s) {
    return analysis_t<double>(L, batch, pt, U, X, s);
}
cudaError_t analysis_all_orders(int L, int64_t batch, const float *pt, const float *U,
                                float *X, cudaStream_t s) {
    return analysis_t<float>(L, batch, pt, U, X, s);
}
cudaError_t synthesis_all_orders_slots(int L, int64_t batch, const double *pt, const double *X,
                                       double *Gt, int slots, cudaStream_t s) {
    return synthesis_t<double>(L, batch, pt, X, Gt, s, slots);
}
cudaError_t analysis_all_orders_slots(int L, int64_t batch, const double *pt, const double *U,
                                      double *X, int slots, cudaStream_t s) {
    return analysis_t<double>(L, batch, pt, U, X, s, slots);
}

}  // namespace sht
