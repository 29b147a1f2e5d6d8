// K2: scaled associated Legendre functions P~_l^m(theta) = Y_l^m(theta, 0), float64.
//
// Definition: Sec. III-B (after Eq. (11)) and Appendix A, Eq. (29) (orthonormal, Condon-Shortley
// phase).  Evaluation: Sec. III-G, three-term recursion in increasing l at fixed m, started from
// the sectoral value, with adaptive rescaling.  The printed recursion coefficients and base
// (Eqs. (21), (22)) do not satisfy the definition; the recursion used here is the one that does:
//   P~_m^m     = -sqrt((2m+1)/(2m)) sin(theta) P~_{m-1}^{m-1},   P~_0^0 = 1/sqrt(4 pi)
//   P~_{m+1}^m = sqrt(2m+3) cos(theta) P~_m^m
//   P~_l^m     = a_lm (cos(theta) P~_{l-1}^m - b_lm P~_{l-2}^m)
//   a_lm = sqrt((4l^2-1)/(l^2-m^2)),  b_lm = sqrt(((l-1)^2-m^2)/(4(l-1)^2-1)).
//
// The sectoral value underflows float64 near the poles for large m (sin^m theta), yet the
// recursion can grow it back to O(1) before l reaches L.  Each value is therefore carried as
// mantissa * 2^e: pass 1 forms the sectoral values with their exponents, pass 2 runs the
// recursion on mantissas and moves 2^kShiftBits from the mantissa into e whenever the mantissa
// exceeds 2^kShiftBits while e < 0.  Values below 2^-1022 are written as 0.
#include "sht_internal.cuh"

namespace sht {
namespace {

constexpr int kShiftBits = 512;

// Pass 1: one thread per row (co-latitude); sectoral mantissa/exponent for every order.
__global__ void k_sectoral(int L, const double *__restrict__ theta, int nrows,
                           double *__restrict__ mant, int *__restrict__ expo) {
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nrows) return;
    double s = sin(theta[r]);
    int e;
    double v = frexp(0.28209479177387814347403972578038629292202531466450, &e);  // 1/sqrt(4 pi)
    mant[r] = v;
    expo[r] = e;
    for (int m = 1; m < L; ++m) {
        double f = -sqrt((2.0 * m + 1.0) / (2.0 * m)) * s;
        int de;
        v = frexp(v * f, &de);
        e = (v == 0.0) ? 0 : e + de;
        mant[(int64_t)m * nrows + r] = v;
        expo[(int64_t)m * nrows + r] = e;
    }
}

__device__ __forceinline__ double emit_value(double p, int e) {
    if (p == 0.0 || e < -1200) return 0.0;
    double v = scalbn(p, e);
    return (fabs(v) < 2.2250738585072014e-308) ? 0.0 : v;
}

// Pass 2: block = 4 warps; each warp owns 32 consecutive rows of one order m (blockIdx.y) and
// walks l in chunks of 32, staging a 32x32 tile in shared memory so that the row-major table
// is written with coalesced 256-byte row segments.
__global__ void __launch_bounds__(128) k_table(int L, const double *__restrict__ theta, int nrows,
                                               const double *__restrict__ mant,
                                               const int *__restrict__ expo,
                                               double *__restrict__ table) {
    __shared__ double tile[4][32][33];
    __shared__ double ca[4][32], cb[4][32];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m = blockIdx.y;
    const int row0 = (blockIdx.x * 4 + warp) * 32;
    if (row0 >= nrows) return;
    const int r = row0 + lane;
    const bool live = r < nrows;
    const int n = L - m;
    double *blk = table + (int64_t)nrows * rows_off(L, m);

    double x = live ? cos(theta[r]) : 0.0;
    double p = live ? mant[(int64_t)m * nrows + r] : 0.0;
    int e = live ? expo[(int64_t)m * nrows + r] : 0;
    double pp = 0.0;  // P~_{l-2}
    const double md = (double)m;

    for (int l0 = m; l0 < L; l0 += 32) {
        {   // recursion coefficients for l = l0 + lane
            int l = l0 + lane;
            double a = 0.0, b = 0.0;
            if (l >= m + 2 && l < L) {
                double ld = (double)l, l1 = ld - 1.0;
                a = sqrt((4.0 * ld * ld - 1.0) / (ld * ld - md * md));
                b = sqrt((l1 * l1 - md * md) / (4.0 * l1 * l1 - 1.0));
            }
            ca[warp][lane] = a;
            cb[warp][lane] = b;
        }
        __syncwarp();
        const int cnt = min(32, L - l0);
        for (int j = 0; j < cnt; ++j) {
            int l = l0 + j;
            if (l == m + 1) {
                double nx = sqrt(2.0 * md + 3.0) * x * p;
                pp = p;
                p = nx;
            } else if (l >= m + 2) {
                double nx = ca[warp][j] * (x * p - cb[warp][j] * pp);
                pp = p;
                p = nx;
            }
            if (e < 0 && fabs(p) > 0x1p512) {
                p = scalbn(p, -kShiftBits);
                pp = scalbn(pp, -kShiftBits);
                e += kShiftBits;
            }
            tile[warp][lane][j] = emit_value(p, e);
        }
        __syncwarp();
        for (int rr = 0; rr < 32; ++rr) {
            int row = row0 + rr;
            if (row < nrows && lane < cnt) blk[(int64_t)row * n + (l0 - m) + lane] = tile[warp][rr][lane];
        }
        __syncwarp();
    }
}

// Recursion coefficients of every order, block m at rows_off(L, m), entry l - m for the step that
// produces degree l (l >= m + 1): a = sqrt(2m+3), b = 0 for l = m + 1, else a_lm, b_lm above.
__global__ void k_recursion_coeffs(int L, double *__restrict__ ra, double *__restrict__ rb) {
    const int m = blockIdx.x;
    const int n = L - m;
    double *a = ra + rows_off(L, m), *b = rb + rows_off(L, m);
    const double md = (double)m;
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        const int l = m + j;
        double av = 0.0, bv = 0.0;
        if (l == m + 1) {
            av = sqrt(2.0 * md + 3.0);
        } else if (l >= m + 2) {
            const double ld = (double)l, l1 = ld - 1.0;
            av = sqrt((4.0 * ld * ld - 1.0) / (ld * ld - md * md));
            bv = sqrt((l1 * l1 - md * md) / (4.0 * l1 * l1 - 1.0));
        }
        a[j] = av;
        b[j] = bv;
    }
}

}  // namespace

cudaError_t recursion_coeffs(int L, double *ra, double *rb, cudaStream_t s) {
    k_recursion_coeffs<<<L, 128, 0, s>>>(L, ra, rb);
    return cudaGetLastError();
}

cudaError_t sectoral_values(int L, const double *d_theta_rows, int nrows, double *mant, int *expo,
                            cudaStream_t s) {
    k_sectoral<<<(nrows + 127) / 128, 128, 0, s>>>(L, d_theta_rows, nrows, mant, expo);
    return cudaGetLastError();
}

cudaError_t build_ptilde_table(int L, const double *d_theta_rows, int nrows, double *d_table,
                               cudaStream_t s) {
    double *mant = nullptr;
    int *expo = nullptr;
    cudaError_t e = cudaMallocAsync((void **)&mant, sizeof(double) * (size_t)L * nrows, s);
    if (e != cudaSuccess) return e;
    e = cudaMallocAsync((void **)&expo, sizeof(int) * (size_t)L * nrows, s);
    if (e != cudaSuccess) { cudaFreeAsync(mant, s); return e; }
    k_sectoral<<<(nrows + 127) / 128, 128, 0, s>>>(L, d_theta_rows, nrows, mant, expo);
    dim3 grid((nrows + 127) / 128, L);
    k_table<<<grid, 128, 0, s>>>(L, d_theta_rows, nrows, mant, expo, d_table);
    e = cudaGetLastError();
    cudaFreeAsync(mant, s);
    cudaFreeAsync(expo, s);
    return e;
}

}  // namespace sht
