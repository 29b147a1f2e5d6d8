// Spin-s transforms (Sec. III-H; Appendix A): the tables sP~_l^m(theta_k) = sY_l^m(theta_k, 0), the
// per-order (pseudo-)inverses, and the forward, inverse and inverse-adjoint flows on the float64
// SIMT kernels.
//
// Definition (Appendix A): sY_l^m(theta, phi) = (-1)^s sqrt((2l+1)/(4 pi)) e^{i m phi} d^l_{m,-s}(theta),
// |s| <= l, d^l the Wigner small-d function (rotation e^{-i beta J_y}).  Evaluation as Appendix A
// prescribes: a three-term recursion in increasing l at fixed (m, s), with a = m, b = -s,
//     l D_l d^{l+1} = (2l+1)(l(l+1) cos(theta) - a b) d^l - (l+1) sqrt((l^2-a^2)(l^2-b^2)) d^{l-1},
//     D_l = sqrt(((l+1)^2 - a^2)((l+1)^2 - b^2)),
// written here on the normalised values y_l = (-1)^s sqrt((2l+1)/(4 pi)) d^l, started at
// l0 = max(|m|, |s|).  The printed start value has the powers of cos(theta/2) and sin(theta/2)
// exchanged relative to the definition; the definition governs.  For |m| >= |s| the start value
// is the scalar sectoral value P~_m^m (carried as mantissa * 2^e, legendre.cu) times
//     sqrt(m!^2 / ((m-|s|)! (m+|s|)!)) tan(theta/2)^(+-s)
// (the ratio of the single terms of the explicit sum for d^m_{+-m,-s} and d^m_{m,0}); for |m| < |s|
// it is the single term at j = |s|, evaluated directly (|s| is small).
//
// Layouts: two tables in the scalar P~ layout (block m: L rings x (L - m) degrees l = m..L-1):
// `pt` holds sP~_l^{+m}, `pt2` holds (-1)^m sP~_l^{-m} (the sign matches the order-major data, whose
// -m slot carries (-1)^m f_l^{-m}); degrees l < |s| are 0.  The inverses likewise: `pinv` and
// `pinv2`, block m of n x n (row l - m, column k - m).  For m >= |s| they are the inverses of the
// square matrices; for m < |s| the matrices have more rings (L - m) than degrees (L - |s|), and
// the blocks hold their least-squares pseudo-inverses (rows of l < |s| zero), computed on the host.
// There is no P_{-m} = (-1)^m P_m relation for s != 0, so every contraction runs once per sign of m,
// each with its table, keeping only that sign's columns.
#include <cmath>
#include <vector>

#include "sht_internal.cuh"

namespace sht {
namespace {

constexpr int kShiftBits = 512;

__device__ __forceinline__ double emit_value(double p, int e) {
    if (p == 0.0 || e < -1200) return 0.0;
    double v = scalbn(p, e);
    return (fabs(v) < 2.2250738585072014e-308) ? 0.0 : v;
}

__device__ double factorial_d(int n) {
    double f = 1.0;
    for (int i = 2; i <= n; ++i) f *= (double)i;
    return f;
}

// d^j_{a,b}(theta) at j = max(|a|, |b|) by the single term of the explicit sum (small j only).
__device__ double small_start(int j, int a, int b, double theta) {
    const int t = max(0, b - a);
    const double num = factorial_d(j + a) * factorial_d(j - a) * factorial_d(j + b) * factorial_d(j - b);
    const double den = factorial_d(j + b - t) * factorial_d(t) * factorial_d(a - b + t) * factorial_d(j - a - t);
    const int p = 2 * j + b - a - 2 * t, q = a - b + 2 * t;
    double c, s;
    sincos(0.5 * theta, &s, &c);
    double v = sqrt(num) / den;
    for (int i = 0; i < p; ++i) v *= c;
    for (int i = 0; i < q; ++i) v *= s;
    return ((a - b + t) & 1) ? -v : v;
}

// One block: 4 warps x 32 rows of one order m (blockIdx.y) and sign (blockIdx.z: 0 -> +m,
// 1 -> -m); each warp walks l in chunks of 32 and writes its 32 x 32 tile row-major, coalesced.
__global__ void __launch_bounds__(128) k_spin_table(int L, int spin, const double *__restrict__ theta,
                                                    const double *__restrict__ mant, const int *__restrict__ expo,
                                                    double *__restrict__ tab_p, double *__restrict__ tab_m) {
    __shared__ double tile[4][32][33];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m = blockIdx.y, neg = blockIdx.z;
    if (neg && m == 0) return;                 // order -0 is order 0
    const int row0 = (blockIdx.x * 4 + warp) * 32;
    if (row0 >= L) return;
    const int r = row0 + lane;
    const bool live = r < L;
    const int n = L - m, as = spin < 0 ? -spin : spin;
    const int a = neg ? -m : m, b = -spin;
    const int l0 = max(m, as);
    double *blk = (neg ? tab_m : tab_p) + (int64_t)L * rows_off(L, m);
    const double th = live ? theta[r] : 0.5;
    const double x = cos(th);

    // start value y_{l0} = mant * 2^e (for the -m table times (-1)^m)
    double p = 0.0;
    int e = 0;
    if (live) {
        if (m >= as) {
            p = mant[(int64_t)m * L + r];
            e = expo[(int64_t)m * L + r];
            double ratio = 1.0;
            for (int i = 1; i <= as; ++i) ratio *= (double)(m - as + i) / (double)(m + i);
            int de;
            p = frexp(p * sqrt(ratio), &de);
            e += de;
            double sh, ch;
            sincos(0.5 * th, &sh, &ch);
            const int pw = neg ? -spin : spin;   // power of tan(theta/2)
            const double f = pw > 0 ? sh / ch : ch / sh;
            for (int i = 0; i < (pw < 0 ? -pw : pw); ++i) {
                p = frexp(p * f, &de);
                e += de;
            }
            if (neg && (as & 1)) p = -p;         // (-1)^s of the -m start
        } else {
            p = small_start(as, a, b, th) * sqrt((2.0 * as + 1.0) / (4.0 * M_PI));
            if (spin & 1) p = -p;                // (-1)^s of the definition
            if (neg && (m & 1)) p = -p;          // (-1)^m of the -m table
            int de;
            p = frexp(p, &de);
            e = de;
        }
        if (p == 0.0) e = 0;
    }
    double pp = 0.0;   // y_{l-1}
    const double ad = (double)a, bd = (double)b;
    for (int c0 = 0; c0 < n; c0 += 32) {
        const int cnt = min(32, n - c0);
        for (int j = 0; j < cnt; ++j) {
            const int l = m + c0 + j;
            if (l > l0) {
                const double lp = (double)(l - 1);   // advance from l - 1 to l
                const double D = sqrt(((lp + 1) * (lp + 1) - ad * ad) * ((lp + 1) * (lp + 1) - bd * bd));
                const double A = sqrt((2 * lp + 3) * (2 * lp + 1)) / (lp * D);
                const double B = (lp + 1) * sqrt((2 * lp + 3) / (2 * lp - 1)) *
                                 sqrt(fmax(0.0, (lp * lp - ad * ad) * (lp * lp - bd * bd))) / (lp * D);
                const double nx = A * (lp * (lp + 1) * x - ad * bd) * p - B * pp;
                pp = p;
                p = nx;
                if (e < 0 && fabs(p) > 0x1p512) {
                    p = scalbn(p, -kShiftBits);
                    pp = scalbn(pp, -kShiftBits);
                    e += kShiftBits;
                }
            }
            tile[warp][lane][j] = (live && l >= l0) ? emit_value(p, e) : 0.0;
        }
        __syncwarp();
        for (int rr = 0; rr < 32; ++rr) {
            const int row = row0 + rr;
            if (row < L && lane < cnt) blk[(int64_t)row * n + c0 + lane] = tile[warp][rr][lane];
        }
        __syncwarp();
    }
}

// Least-squares pseudo-inverse (A^T A)^{-1} A^T = R^{-1} Q^T of a full-column-rank A (n x c,
// row-major), by classical Gram-Schmidt with one reorthogonalisation (as accurate as Householder
// for full-rank A); out is c x n row-major.
void ls_pseudo_inverse(const std::vector<double> &A, int n, int c, std::vector<double> &out) {
    std::vector<double> Q((size_t)n * c, 0.0), R((size_t)c * c, 0.0), v((size_t)n);
    for (int j = 0; j < c; ++j) {
        for (int i = 0; i < n; ++i) v[i] = A[(size_t)i * c + j];
        for (int pass = 0; pass < 2; ++pass)
            for (int q = 0; q < j; ++q) {
                double d = 0.0;
                for (int i = 0; i < n; ++i) d += Q[(size_t)i * c + q] * v[i];
                R[(size_t)q * c + j] += d;
                for (int i = 0; i < n; ++i) v[i] -= d * Q[(size_t)i * c + q];
            }
        double nrm = 0.0;
        for (int i = 0; i < n; ++i) nrm += v[i] * v[i];
        nrm = std::sqrt(nrm);
        R[(size_t)j * c + j] = nrm;
        for (int i = 0; i < n; ++i) Q[(size_t)i * c + j] = nrm > 0.0 ? v[i] / nrm : 0.0;
    }
    // out = R^{-1} Q^T: back substitution, one column of Q^T (= row i of Q) at a time
    out.assign((size_t)c * n, 0.0);
    for (int i = 0; i < n; ++i)
        for (int j = c - 1; j >= 0; --j) {
            double t = Q[(size_t)i * c + j];
            for (int q = j + 1; q < c; ++q) t -= R[(size_t)j * c + q] * out[(size_t)q * n + i];
            out[(size_t)j * n + i] = R[(size_t)j * c + j] != 0.0 ? t / R[(size_t)j * c + j] : 0.0;
        }
}

}  // namespace

cudaError_t build_spin_tables(int L, int spin, const double *d_theta, double *pt, double *pt2,
                              double *pinv, double *pinv2, bool &singular, cudaStream_t s) {
    singular = false;
    const int as = spin < 0 ? -spin : spin;
    double *mant = nullptr;
    int *expo = nullptr;
    cudaError_t e = cudaMallocAsync((void **)&mant, sizeof(double) * (size_t)L * L, s);
    if (e != cudaSuccess) return e;
    e = cudaMallocAsync((void **)&expo, sizeof(int) * (size_t)L * L, s);
    if (e != cudaSuccess) { cudaFreeAsync(mant, s); return e; }
    const size_t tb = sizeof(double) * (size_t)pt_off(L, L);
    if ((e = cudaMemsetAsync(pt2, 0, tb, s)) == cudaSuccess &&
        (e = sectoral_values(L, d_theta, L, mant, expo, s)) == cudaSuccess) {
        k_spin_table<<<dim3((L + 127) / 128, L, 2), 128, 0, s>>>(L, spin, d_theta, mant, expo, pt, pt2);
        e = cudaGetLastError();
    }
    cudaFreeAsync(mant, s);
    cudaFreeAsync(expo, s);
    if (e != cudaSuccess) return e;
    // square orders m >= |s|: Gauss-Jordan inverses of both tables
    e = build_inverses(L, pt, pinv, s, as);
    if (e == cudaSuccess) e = build_inverses(L, pt2, pinv2, s, as);
    if (e == cudaErrorInvalidValue) { singular = true; return e; }
    if (e != cudaSuccess) return e;
    // orders m < |s|: least-squares pseudo-inverses on the host (a few orders, |s| small)
    for (int m = 0; m < as && m < L; ++m)
        for (int sg = 0; sg < 2; ++sg) {
            if (sg == 1 && m == 0) continue;
            const int n = L - m, c = L - as;
            std::vector<double> blk((size_t)n * n), A((size_t)n * c), out;
            // rows k = m..L-1 of block m (L x n, columns l - m); keep the degrees l >= |s|
            e = cudaMemcpyAsync(blk.data(), (sg ? pt2 : pt) + pt_off(L, m) + (int64_t)m * n,
                                sizeof(double) * blk.size(), cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) return e;
            for (int i = 0; i < n; ++i)
                for (int j = 0; j < c; ++j) A[(size_t)i * c + j] = blk[(size_t)i * n + (as - m) + j];
            ls_pseudo_inverse(A, n, c, out);
            std::vector<double> pad((size_t)n * n, 0.0);   // row l - m; rows of l < |s| zero
            for (int j = 0; j < c; ++j)
                for (int i = 0; i < n; ++i) pad[(size_t)(as - m + j) * n + i] = out[(size_t)j * n + i];
            e = cudaMemcpyAsync((sg ? pinv2 : pinv) + pinv_off(L, m), pad.data(), sizeof(double) * pad.size(),
                                cudaMemcpyHostToDevice, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) return e;
        }
    return cudaSuccess;
}

// Inverse (Procedure 2 with sY): both signs' synthesis into the order table, then the fold and
// inverse ring DFTs of the scalar path.
cudaError_t spin_inverse(sht_plan_t p, const double2 *d_coeffs, double2 *d_samples, int64_t batch, cudaStream_t s) {
    const int L = p->L;
    cudaError_t e = coeffs_to_orders(L, batch, d_coeffs, p->ws.a, s);
    if (e == cudaSuccess) e = synthesis_all_orders_slots(L, batch, p->pt, p->ws.a, p->ws.g, 1, s);
    if (e == cudaSuccess) e = synthesis_all_orders_slots(L, batch, p->pt2, p->ws.a, p->ws.g, 2, s);
    if (e == cudaSuccess) e = fold_ring_idft(L, p->dft, p->ws.g, d_samples, batch, s);
    p->launches += 3;
    return e;
}

// Adjoint of the inverse: ring DFTs unfolded to every order, both signs' transposed contraction.
cudaError_t spin_inverse_adjoint(sht_plan_t p, const double2 *d_samples, double2 *d_coeffs, int64_t batch,
                                 cudaStream_t s) {
    const int L = p->L;
    cudaError_t e = ring_dft_unfold(L, p->dft, d_samples, p->ws.g, batch, s);
    if (e == cudaSuccess) e = analysis_all_orders_slots(L, batch, p->pt, p->ws.g, p->ws.a, 1, s);
    if (e == cudaSuccess) e = analysis_all_orders_slots(L, batch, p->pt2, p->ws.g, p->ws.a, 2, s);
    if (e == cudaSuccess) e = orders_to_coeffs(L, batch, p->ws.a, d_coeffs, s);
    p->launches += 3;
    return e;
}

// Forward (Procedure 1 with sY, in bin space): ring DFTs into bins, then for m = L-1..0 each
// sign's solve (Eq. (14); least squares for m < |s|) and alias subtraction (Eqs. (15)-(16)).
cudaError_t spin_forward(sht_plan_t p, const double2 *d_samples, double2 *d_coeffs, int64_t batch, cudaStream_t s) {
    const int L = p->L;
    const int64_t Nc = 4 * batch;
    double *W = p->ws.a, *F = p->ws.b;
    cudaError_t e = ring_dft_to_bins(L, p->dft, d_samples, W, batch, true, s);
    GemmArgs ga{};
    ga.L = L; ga.batch = batch; ga.coeffs = d_coeffs; ga.W = W;
    ga.part = p->ws.part; ga.part_cap = (int64_t)kSplitCap * L * Nc;
    ga.launches = &p->launches;
    for (int m = L - 1; m >= 0 && e == cudaSuccess; --m) {
        const int n = L - m;
        ga.m = m;
        for (int sg = 0; sg < 2 && e == cudaSuccess; ++sg) {
            if (sg == 1 && m == 0) break;
            ga.slots = sg ? 2 : 1;
            e = gemm_f64(false, n, n, (int)Nc, (sg ? p->pinv2 : p->pinv) + pinv_off(L, m), n,
                         W + rows_off(L, m) * Nc, Nc, F + rows_off(L, m) * Nc, Nc, EPI_SOLVE, ga, s);
        }
        for (int sg = 0; sg < 2 && m > 0 && e == cudaSuccess; ++sg) {
            ga.slots = sg ? 2 : 1;
            e = gemm_f64(false, m, n, (int)Nc, (sg ? p->pt2 : p->pt) + pt_off(L, m), n, F + rows_off(L, m) * Nc,
                         Nc, nullptr, Nc, EPI_ALIAS, ga, s);
        }
    }
    return e;
}

}  // namespace sht
