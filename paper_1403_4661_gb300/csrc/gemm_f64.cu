// Float64 contractions of the transforms: register-tiled SIMT GEMM (FFMA64), row-major operands,
// with the epilogues the order chain needs.  On GB300 float64 runs at ~1/64 of the float32 rate,
// so a tile keeps the FP64 pipe busy with few warps; what matters is filling all 152 SMs, which
// the launcher does by picking the tile shape from the problem size.
//
// Contractions served (N = 4 * batch real columns: signal b, +m / -m, re / im):
//  synthesis  G_{+-m}(theta_k) = sum_l P~_l^m(theta_k) X_m[l]  for every m and ring k   (Eq. (11))
//  analysis   the transposed contraction (adjoint of synthesis)
//  solve      F_m = P_m^{-1} W_m  (Eq. (14)), writing f_l^{+-m} to the coefficient output
//  alias      G_{+-m}(theta_k), k < m, subtracted from bin alias_k(+-m) of ring k (Eqs. (15)-(16))
#include "sht_internal.cuh"

namespace sht {
namespace {

constexpr int BK = 16;

enum Mode : int { MODE_SINGLE = 0, MODE_SYNTH = 1, MODE_ANALYSIS = 2 };

struct Params {
    const double *A; int64_t lda;
    const double *B; int64_t ldb;
    double *C; int64_t ldc;
    const double *C0;
    int M, K, N;
    int m;           // order (single-problem epilogues)
    int L;
    double2 *coeffs; // EPI_SOLVE
    double *W;       // EPI_ALIAS
    const double *pt; const double *X; double *Y;  // grouped modes
};

// sum_{j=1..x} ceil(j / bm)
__device__ __forceinline__ int64_t ceil_sum(int64_t x, int64_t bm) {
    int64_t q = x / bm, r = x % bm;
    return bm * q * (q + 1) / 2 + r * (q + 1);
}

template <int BM, int BN, bool TA, int EPI, int MODE>
__global__ void __launch_bounds__((BM / 4) * (BN / 4)) k_gemm(Params p) {
    constexpr int NT = (BM / 4) * (BN / 4);
    __shared__ __align__(16) double As[BK][BM + 2];
    __shared__ __align__(16) double Bs[BK][BN + 2];

    const double *A = p.A, *B = p.B;
    double *C = p.C;
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
    const int tm = (int)(tile / tiles_n), tn = (int)(tile % tiles_n);
    const int row0 = tm * BM, col0 = tn * BN;
    const int tx = threadIdx.x % (BN / 4), ty = threadIdx.x / (BN / 4);

    double acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;

    for (int k0 = 0; k0 < K; k0 += BK) {
        for (int idx = threadIdx.x; idx < BM * BK; idx += NT) {
            int i, kk;
            if (!TA) { i = idx / BK; kk = idx % BK; } else { kk = idx / BM; i = idx % BM; }
            int r = row0 + i, k = k0 + kk;
            double v = 0.0;
            if (r < M && k < K) v = TA ? A[(int64_t)k * lda + r] : A[(int64_t)r * lda + k];
            As[kk][i] = v;
        }
        for (int idx = threadIdx.x; idx < BN * BK; idx += NT) {
            int kk = idx / BN, j = idx % BN;
            int k = k0 + kk, c = col0 + j;
            Bs[kk][j] = (k < K && c < N) ? B[(int64_t)k * ldb + c] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            double2 a01 = *reinterpret_cast<const double2 *>(&As[kk][ty * 4]);
            double2 a23 = *reinterpret_cast<const double2 *>(&As[kk][ty * 4 + 2]);
            double2 b01 = *reinterpret_cast<const double2 *>(&Bs[kk][tx * 4]);
            double2 b23 = *reinterpret_cast<const double2 *>(&Bs[kk][tx * 4 + 2]);
            double a[4] = {a01.x, a01.y, a23.x, a23.y};
            double b[4] = {b01.x, b01.y, b23.x, b23.y};
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }

    const int c0 = col0 + tx * 4;
    if (c0 >= N) return;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int r = row0 + ty * 4 + i;
        if (r >= M) break;
        if (EPI == EPI_STORE || EPI == EPI_SOLVE) {
            double *cr = C + (int64_t)r * ldc + c0;
            if (c0 + 4 <= N && (ldc & 1) == 0) {
                *reinterpret_cast<double2 *>(cr) = make_double2(acc[i][0], acc[i][1]);
                *reinterpret_cast<double2 *>(cr + 2) = make_double2(acc[i][2], acc[i][3]);
            } else {
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    if (c0 + j < N) cr[j] = acc[i][j];
            }
        }
        if (EPI == EPI_SUB) {
            const double *c0r = p.C0 + (int64_t)r * ldc + c0;
            double *cr = C + (int64_t)r * ldc + c0;
#pragma unroll
            for (int j = 0; j < 4; ++j) cr[j] = c0r[j] - acc[i][j];
        }
        if (EPI == EPI_SOLVE) {
            // row r is degree l = m + r; columns (b, +m re/im, -m re/im)
            const int64_t L2 = (int64_t)p.L * p.L;
            const int l = m + r, b = c0 >> 2;
            double2 *cb = p.coeffs + (int64_t)b * L2 + (int64_t)l * l + l;
            cb[m] = make_double2(acc[i][0], acc[i][1]);
            if (m > 0) {
                const double sg = (m & 1) ? -1.0 : 1.0;   // f_l^{-m} = (-1)^m F_l^{-}
                cb[-m] = make_double2(sg * acc[i][2], sg * acc[i][3]);
            }
        }
        if (EPI == EPI_ALIAS) {
            // row r is ring k = r < m; subtract G_{+m}, G_{-m} from bins a, -a of ring k
            const int k = r, b = c0 >> 2;
            const int a = alias_bin(m, k);
            const int o = a < 0 ? -a : a;
            double *w = p.W + (rows_off(p.L, o) + (k - o)) * (int64_t)N + 4 * b;
            if (a == 0) {
                w[0] -= acc[i][0] + acc[i][2];
                w[1] -= acc[i][1] + acc[i][3];
            } else {
                const int sp = a > 0 ? 0 : 2;   // slot of bin a  (+o or -o)
                const int sm = 2 - sp;          // slot of bin -a
                w[sp] -= acc[i][0];
                w[sp + 1] -= acc[i][1];
                w[sm] -= acc[i][2];
                w[sm + 1] -= acc[i][3];
            }
        }
    }
}

constexpr int kSMs = 152;

template <bool TA, int EPI, int MODE>
cudaError_t launch(const Params &p, int64_t tiles64, int64_t tiles32, cudaStream_t s) {
    // 64x64 tiles (256 threads) when they alone give >= 2 waves of 152 SMs, else 32x32 (64 threads)
    if (tiles64 >= 2 * kSMs) {
        k_gemm<64, 64, TA, EPI, MODE><<<(unsigned)tiles64, 256, 0, s>>>(p);
    } else {
        k_gemm<32, 32, TA, EPI, MODE><<<(unsigned)tiles32, 64, 0, s>>>(p);
    }
    return cudaGetLastError();
}

inline int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

}  // namespace

cudaError_t gemm_f64(bool transA, int M, int K, int N, const double *A, int64_t lda,
                     const double *B, int64_t ldb, double *C, int64_t ldc, int epi,
                     const GemmArgs &ga, cudaStream_t s, const double *C0) {
    if (M <= 0 || N <= 0) return cudaSuccess;
    Params p{};
    p.A = A; p.lda = lda; p.B = B; p.ldb = ldb; p.C = C; p.ldc = ldc; p.C0 = C0;
    p.M = M; p.K = K; p.N = N; p.m = ga.m; p.L = ga.L; p.coeffs = ga.coeffs; p.W = ga.W;
    int64_t t64 = cdiv(M, 64) * cdiv(N, 64), t32 = cdiv(M, 32) * cdiv(N, 32);
#define SHT_GEMM_CASE(E)                                                                  \
    if (epi == E) return transA ? launch<true, E, MODE_SINGLE>(p, t64, t32, s)            \
                                : launch<false, E, MODE_SINGLE>(p, t64, t32, s);
    SHT_GEMM_CASE(EPI_STORE)
    SHT_GEMM_CASE(EPI_SOLVE)
    SHT_GEMM_CASE(EPI_ALIAS)
    SHT_GEMM_CASE(EPI_SUB)
#undef SHT_GEMM_CASE
    return cudaErrorInvalidValue;
}

cudaError_t synthesis_all_orders(int L, int64_t batch, const double *pt, const double *X,
                                 double *Gt, cudaStream_t s) {
    Params p{};
    p.L = L; p.N = (int)(4 * batch); p.pt = pt; p.X = X; p.Y = Gt;
    int64_t t64 = (int64_t)L * cdiv(L, 64) * cdiv(p.N, 64);
    int64_t t32 = (int64_t)L * cdiv(L, 32) * cdiv(p.N, 32);
    return launch<false, EPI_STORE, MODE_SYNTH>(p, t64, t32, s);
}

cudaError_t analysis_all_orders(int L, int64_t batch, const double *pt, const double *U,
                                double *X, cudaStream_t s) {
    Params p{};
    p.L = L; p.N = (int)(4 * batch); p.pt = pt; p.X = U; p.Y = X;
    auto csum = [](int64_t x, int64_t bm) {
        int64_t q = x / bm, r = x % bm;
        return bm * q * (q + 1) / 2 + r * (q + 1);
    };
    int64_t t64 = cdiv(p.N, 64) * csum(L, 64);
    int64_t t32 = cdiv(p.N, 32) * csum(L, 32);
    return launch<true, EPI_STORE, MODE_ANALYSIS>(p, t64, t32, s);
}

}  // namespace sht
